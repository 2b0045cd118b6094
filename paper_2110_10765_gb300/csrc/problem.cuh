// Internal state of a CI problem: species lists, basis, staged interaction
// tables, species connectivity and the CSR matrix.
#pragma once

#include <memory>

#include "common.cuh"

namespace ci {

// ------------------------------------------------------------------ species

// One species determinant list, sorted by (2M, q, value of the bit string),
// split into blocks of equal 2M (block b has 2M = m2min + 2b).
struct SpeciesList {
    int A = 0, W = 1;
    int64_t n = 0;
    std::vector<uint64_t> bits;     // [n][W]
    std::vector<int32_t> q, twoM;   // [n]
    std::vector<uint8_t> occ;       // [n][A] occupied states, ascending
    std::vector<int32_t> local;     // [n] index inside its 2M block
    int m2min = 0, nblk = 0;
    int nq = 1;                     // stored q caps 0..nq-1 (1 when no Nmax cut)
    std::vector<int64_t> blk_start; // [nblk+1]
    std::vector<int64_t> blk_qend;  // [nblk][nq] end of (q' <= q) inside the block

    DevBuf<uint64_t> d_bits;
    DevBuf<int64_t> d_blk_start;
    DevBuf<int32_t> d_q, d_twoM, d_local;
    DevBuf<uint8_t> d_occ;

    int block_of(int twoM_) const {
        int t = twoM_ - m2min;
        if (t < 0 || (t & 1)) return -1;
        t >>= 1;
        return t < nblk ? t : -1;
    }
};

// ------------------------------------------------------------------ tables

// Interaction tables of one precision, staged from the flat TBMEs.
//   C*  : compact like-pair blocks, V_cdab = C[row[c*S+d] + col[a*S+b]] (c<d, a<b)
//   Tpn : proton-transition x neutron-transition blocks,
//         V^pn_{c c', a a'} = Tpn[tr_base[c*S+a] + tr_idx[c'*S+a']]
//         (rows: proton moves a -> c, columns: neutron moves a' -> c', grouped
//         by the change of 2m, which the two moves must cancel)
//   U*  : one-move spectator tables, U[(c*S+a)*S+k] = V_{ck,ak}
//   Wpn : neutron-move pn spectators, Wpn[(d*S+b)*S+k] = V^pn_{kd,kb}
//   D*  : pair diagonals, D[a*S+b] = V_abab
template <class T>
struct Tables {
    DevBuf<T> eps;
    DevBuf<T> Cpp, Cnn, Tpn;
    DevBuf<T> Upp, Unn, Upn, Wpn;
    DevBuf<T> Dpp, Dnn, Dpn;
    bool ready = false;
};

// One entry of a species connectivity list (row determinant s = bra,
// partner s' = ket).  info: bits 0-1 difference code (0: d=0, 1: d=2,
// 2: d=4), bit 2 sign (1: negative), bits 3-10 state a (in s' only), bits
// 11-18 state c (in s only).  Neutron lists: bits 19-31 of d=2 entries hold
// the column index of the move a -> c in the pn transition table (< 8192).
// Proton list: bits 19-23 hold q(s') (capped at 31; only read under an
// Nmax cut, which is <= 31), bits 24-31 (2M(s') - 2M(s))/2 + 128.
// tgt: neutron lists, the partner s'; proton list, the first basis row of
// s' (p_row_base[s']), the partner index itself being kept in ConnList::tgt.
// local: neutron lists, index of s' inside its 2M block; proton list, for
// d=2 entries the row offset tr_base of the move a -> c in that table.
// val: d=0 like-particle diagonal energy (one-body + pairs); d=2 unsigned
// like-particle spectator sum; d=4 signed V.
template <class T>
struct ConnEntry {
    int32_t tgt;
    int32_t local;
    uint32_t info;
    T val;
};

constexpr int kMaxTcol = 1 << 13;   // pn transition-table columns an entry can address

__host__ __device__ inline int info_dcode(uint32_t i) { return (int)(i & 3u); }
__host__ __device__ inline int info_neg(uint32_t i) { return (int)((i >> 2) & 1u); }
__host__ __device__ inline int info_a(uint32_t i) { return (int)((i >> 3) & 255u); }
__host__ __device__ inline int info_c(uint32_t i) { return (int)((i >> 11) & 255u); }
__host__ __device__ inline int info_tcol(uint32_t i) { return (int)(i >> 19); }
__host__ __device__ inline int info_q(uint32_t i) { return (int)((i >> 19) & 31u); }
__host__ __device__ inline int info_dslot(uint32_t i) { return (int)(i >> 24) - 128; }
__host__ __device__ inline uint32_t make_info(int dcode, int neg, int a, int c) {
    return (uint32_t)dcode | ((uint32_t)neg << 2) | ((uint32_t)a << 3) | ((uint32_t)c << 11);
}
__host__ __device__ inline uint32_t info_with_tcol(uint32_t i, int tcol) { return i | ((uint32_t)tcol << 19); }
__host__ __device__ inline uint32_t info_with_partner(uint32_t i, int q, int dslot) {
    return (i & 0x7FFFFu) | ((uint32_t)(q < 31 ? q : 31) << 19) | ((uint32_t)(dslot + 128) << 24);
}

// A species list inside a group allocation: ptr [n+1] holds absolute
// positions into ent (the buffers are shared by every list built in the
// same batched launch).
template <class T>
struct ConnList {
    std::shared_ptr<DevBuf<int64_t>> ptr_buf;
    std::shared_ptr<DevBuf<ConnEntry<T>>> ent_buf;
    std::shared_ptr<DevBuf<int32_t>> tgt_buf, xr_buf;
    const int64_t *ptr = nullptr;
    ConnEntry<T> *ent = nullptr;
    const int32_t *tgt = nullptr;   // partner index per entry (absolute positions, as ent)
    // proton lists: for a same-2M entry, the number of same-2M entries of
    // the other proton list (O2 <-> O4) of its row with a smaller partner
    const int32_t *xr = nullptr;
    int64_t n = 0;      // determinants (rows of the list)
    int64_t first = 0;  // ptr[0]
    int64_t total = 0;  // ptr[n] - ptr[0]
};

// Which species pairs a list keeps (see ci_species_filter).  The proton
// pairs are split by their difference: O2 (d <= 2, any M) and O4 (d = 4,
// same M); ci_get_species_conn merges them back into one list.
enum ConnMode { CONN_OUTER = 0, CONN_L2 = 1, CONN_L4 = 2, CONN_O4 = 3 };
constexpr int kModes = 4;

template <class T>
struct Connectivity {
    ConnList<T> outer;   // protons: d <= 2 (any M)
    ConnList<T> outer4;  // protons: d = 4 (same M)
    ConnList<T> l2;      // neutrons: d <= 2 (any M)
    ConnList<T> l4;      // neutrons: d <= 4, same M
    DevBuf<int32_t> seg2;  // [nN][nds][nq] end of L2 entries with slot<s or (slot==s, q<=c), relative
    DevBuf<int32_t> seg4;  // [nN][nq] end of L4 entries with q <= c, relative
    DevBuf<int32_t> oseg2; // [nP][nds][nq] the same for the O2 list (slot of 2M(p') - 2M(p))
    DevBuf<int32_t> oseg4; // [nP][nq] end of O4 entries with q(p') <= c, relative
    DevBuf<int32_t> qmin2; // [nN][nds] smallest q of the L2 entries in a 2M slot (nq if none)
    bool ready = false;
};

// ------------------------------------------------------------------ problem

struct Problem {
    int S = 0;
    std::vector<int32_t> sp_N, sp_twom;
    std::vector<double> sp_energy;
    int Z = 0, N = 0, nmax = -1, twoM = 0;
    int K = 0;      // max |2m| over the s.p. states
    int nds = 1;    // 2K+1 slots of 2M change in one move

    // flat TBMEs kept on the device only until the tables are staged
    int tbme_source = CI_TBME_TABLES;
    uint64_t tbme_seed = 0;
    int tbme_dtype = CI_F32;
    DevBuf<unsigned char> flat[3];   // pp, nn, pn (tbme_dtype elements)

    // like pairs a<b grouped by m_a + m_b; one-particle moves a -> c grouped
    // by 2m_c - 2m_a (tr_base: row offset as a proton move, tr_idx: column
    // index as a neutron move)
    DevBuf<int32_t> like_row, like_col, tr_base, tr_idx;
    int64_t like_size = 0, tr_size = 0;   // entries of the compact tables
    // group layouts of the compact tables (kept for staging)
    int like_G = 0, tr_G = 0;
    DevBuf<int64_t> lg_off, tg_off;
    DevBuf<int32_t> lg_ncol, lg_rows, lg_cols, lg_items, tg_ncol, tg_rows, tg_cols, tg_items;
    DevBuf<int32_t> d_twom;
    DevBuf<double> d_eps;

    Tables<float> t32;
    Tables<double> t64;

    bool enumerated = false;
    SpeciesList sp[2];
    int64_t dim = 0;
    std::vector<int64_t> p_row_base;   // [nP+1]
    std::vector<int64_t> p_nstart;     // [nP] first neutron index of each proton's rows
    DevBuf<int64_t> d_p_row_base, d_p_nstart;
    DevBuf<int32_t> d_row_p, d_row_n;  // [dim]

    Connectivity<float> c32;
    Connectivity<double> c64;
    int conn_prec = -1;                // precision of the last species filter

    DevBuf<int64_t> scan_scratch;      // block sums of the exclusive scan

    template <class T> Tables<T> &tables();
    template <class T> Connectivity<T> &conn();
};

template <> inline Tables<float> &Problem::tables<float>() { return t32; }
template <> inline Tables<double> &Problem::tables<double>() { return t64; }
template <> inline Connectivity<float> &Problem::conn<float>() { return c32; }
template <> inline Connectivity<double> &Problem::conn<double>() { return c64; }

// ------------------------------------------------------------------ matrix

struct Matrix {
    int64_t dim = 0, nnz = 0;
    int vtype = CI_F32;
    DevBuf<int64_t> row_ptr;
    DevBuf<int32_t> col;
    DevBuf<unsigned char> val;       // float, double or bf16 bits
    DevBuf<float> row_scale;         // BF16 only
    bool upper = false;              // only the upper triangle (col >= row) is stored
    // row ranges of balanced work for the 8-vector SpMM (spmm_prepare):
    // range b is rows [spmm_bnd[b], spmm_bnd[b+1]), b < spmm_nb
    DevBuf<int64_t> spmm_bnd;
    int64_t spmm_nb = 0;
};

// Block-diagonal preconditioner over many-body basis orbitals: sub-blocks of
// at most kSubMax rows, their shifted inverses in FP32 (precond.cu).
constexpr int kSubMax = 128;
struct BlockPrecond {
    int64_t dim = 0, nsub = 0;
    int smax = 0;                    // rows of the largest sub-block
    DevBuf<int32_t> rows;            // [dim] rows grouped by sub-block, ascending inside
    DevBuf<int32_t> sub_of, loc_of;  // [dim] sub-block of a row, index inside it
    DevBuf<int64_t> sub_start;       // [nsub+1] into rows
    DevBuf<int64_t> inv_off;         // [nsub+1] into inv
    DevBuf<float> inv;               // row-major inverses of the shifted sub-blocks
    DevBuf<double> shift;            // [nsub] shift used by each sub-block
    // sub-blocks of <= 32, <= 64 and <= kSubMax rows (largest first in each
    // bin): one inversion launch per bin, its shared memory sized to the bin
    DevBuf<int32_t> bin_ids;         // [nsub]
    int64_t bin_off[4] = {0, 0, 0, 0};
    int bin_max[3] = {0, 0, 0};
    DevBuf<int32_t> status;          // [1] set when a sub-block could not be inverted
};
void orbital_blocks(Problem *p, const int32_t *sp_orbital, int32_t *block, int64_t *nblocks, cudaStream_t s);
void precond_setup(BlockPrecond &bp, const Matrix *H, const int32_t *row_block, int64_t nblocks, cudaStream_t s);
void precond_factor(BlockPrecond &bp, const Matrix *H, double sigma, cudaStream_t s);
void precond_apply(const BlockPrecond &bp, const double *R, int nv, double *W, cudaStream_t s);
void precond_row_shift(const BlockPrecond &bp, double *out, cudaStream_t s);

// ------------------------------------------------------------------ steps

// Rows of a group of problems built together (one launch per step for the
// whole group): problem g owns rows [row_off[g], row_off[g+1]) of the
// group's counts, offsets, col and val.
struct GroupCSR {
    std::vector<int64_t> row_off;    // [G+1]
    DevBuf<int32_t> row_cnt;         // [rows]
    DevBuf<int64_t> row_ptr;         // [rows+1] absolute positions
    DevBuf<int32_t> col;             // [nnz] problem-local columns
    DevBuf<unsigned char> val;       // [nnz] float or double
    int64_t nnz = 0;
    int prec = 0;                    // 0 float, 1 double
    std::vector<int64_t> nnz_of;     // [G]
};

void problem_create(const ci_problem_desc *d, Problem *p);
void enumerate_basis(Problem *p, cudaStream_t s);
template <class T> void stage_tables_group(const std::vector<Problem *> &ps, cudaStream_t s);
// Tables of a two-body operator drawn by the seeded recipe (no one-body
// part; zero_eps: S zero doubles on the device).
template <class T>
void stage_operator_tables(Problem *p, uint64_t seed, Tables<T> &t, const double *zero_eps, cudaStream_t s);
// Slater-Condon entries of every connectivity list with the tables t into
// ents (the layout of the lists' shared entry array).
template <class T>
void operator_entries(Problem *p, const Tables<T> &t, ConnEntry<T> *ents, cudaStream_t s);
// sum_i X[i][q] (O X)[i][q] for q < 8 of the operator with tables t and
// entries ents; X [dim][8] FP64 on the device; one partial per block in
// part (nblk x 8, device); returns nblk.
template <class T>
int observable_apply(Problem *p, const Tables<T> &t, const ConnEntry<T> *ents, const double *L8, const double *R8,
                     double *part, cudaStream_t s);
template <class T> void species_filter_group(const std::vector<Problem *> &ps, cudaStream_t s);
template <class T> void species_filter(Problem *p, cudaStream_t s) { species_filter_group<T>({p}, s); }
// count (and optionally fill) the rows of every problem of ps in one launch each
void count_group(const std::vector<Problem *> &ps, int prec, GroupCSR *g, cudaStream_t s);
void fill_group(const std::vector<Problem *> &ps, GroupCSR *g, cudaStream_t s);
void exclusive_scan_i32(const int32_t *counts, int64_t n, int64_t *offsets,
                        DevBuf<int64_t> &scratch, cudaStream_t s);
// src[idx[i]] for every i, copied to the host (synchronises s)
std::vector<int64_t> gather_i64(const int64_t *src, const std::vector<int64_t> &idx, cudaStream_t s);
void build_matrix(Problem *p, int vtype, Matrix *m, cudaStream_t s);
void upper_matrix(const Matrix *full, Matrix *out, cudaStream_t s);
// Y = H X for 16 FP32 vectors [dim][16] (FP32 or BF16 values, full storage)
void apply_matrix16(const Matrix *m, const float *X, float *Y, cudaStream_t s);
// Y8 = H R8 ([dim][8]) in FP64 with every element evaluated on the fly
void h64_apply(Problem *p, const double *R8, double *Y8, cudaStream_t s);
void apply_matrix(const Matrix *m, const void *X, void *Y, int nvec, cudaStream_t s);
// The row ranges of a full-storage matrix's 8-vector SpMM (after its CSR is final).
void spmm_prepare(Matrix *m, cudaStream_t s);
// W = H X for 8 FP32 vectors with the result in FP64 ([dim][8]) of a
// full-storage FP32 or BF16 matrix; false (nothing launched) for other
// matrices.
bool apply_matrix8_f64out(const Matrix *m, const float *X, double *W, cudaStream_t s);
// FP64-exact products on the tensor cores (ozaki.cu) for a basis A of
// na <= 64 orthonormal columns (|A| < 1.99), read in its fixed-point
// shadow form Y (oz_fix; even ldy, so rows are 16-byte aligned; A may start
// at an odd column).
//   oz_tn: part[blk][na][8] = A[rows of blk]^T B over nblk row blocks (B
//          8-byte aligned, ldb even)
//   oz_nn: W = beta W + alpha A C, C [na][8]
// An entry outside the digits' range sets bit 0 of *flag, a tensor-core
// wait that ran out bit 1.
bool oz_supported(int na);
// x32: nullable [dim][nc], the entries rounded to FP32
void oz_fix(int64_t dim, int nc, const double *A, int lda, unsigned long long *Y, int ldy, int *flag,
            cudaStream_t s, float *x32 = nullptr);
// x32: nullable [dim][nc], the copied columns rounded to FP32; skip:
// nullable, when set on the device nothing is copied
void oz_copy_fix(int64_t dim, int nc, const double *src, int lds, double *dst, int ldd, unsigned long long *Y, int ldy,
                 float *x32, int *flag, cudaStream_t s, const int *skip = nullptr);
void oz_tn(int64_t dim, const unsigned long long *Y, int ldy, int na, const double *B, int ldb, double *part,
           int nblk, int *flag, cudaStream_t s);
// skip: nullable, when set on the device the product is not formed
void oz_nn(int64_t dim, const unsigned long long *Y, int ldy, int na, const double *C, double *W, int ldw,
           double alpha, double beta, int *flag, cudaStream_t s, const int *skip = nullptr);
int oz_tn_blocks(int64_t dim);
void lowest_eigs(const Matrix *H, const ci_eig_opts *opts, double *evals, double *evecs, ci_eig_info *info,
                 cudaStream_t s);

}  // namespace ci

struct ci_problem { ci::Problem impl; };
struct ci_matrix { ci::Matrix impl; };
