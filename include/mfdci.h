/*
 * mfdci.h -- C ABI of the GB300 (sm_103a) library for the hot path of
 * MFDn-style nuclear configuration interaction (CI):
 *
 *   enumerate the proton x neutron Slater-determinant basis as bit strings,
 *   filter determinant pairs by XOR + popcount, count -> scan -> fill the
 *   sparse Hamiltonian H, apply it to a block of vectors (SpMM), and find
 *   its lowest eigenpairs by block Lanczos; plus a batched form and a
 *   submit/poll solve queue.
 *
 * Paper: B. Cook, P. J. Fasano, P. Maris, C. Yang, D. Oryspayev,
 * "Accelerating quantum many-body configuration interaction with
 * directives" (2021): Fig. 1 (the matrix-construction and eigensolve
 * pipeline), Sec. 2.1 (bit representation, popcount filter, Listing 2),
 * Sec. 2.2 (counts -> offsets, Eq. 1), Sec. 2.3 (filling shared arrays,
 * Listing 7), Sec. 2 (SpMV/SpMM and LOBPCG/Lanczos eigensolvers).
 *
 * Conventions (every function):
 *   - returns ci_status; CI_OK is 0.  On error, ci_last_error() gives a
 *     message for the calling thread.  No exception crosses the ABI and the
 *     library never aborts the process.
 *   - handles (ci_problem, ci_matrix, ci_batch, ci_queue) are owned by the
 *     library and freed by their *_destroy call.  Buffers passed in are
 *     owned by the caller; the library copies what it keeps.
 *   - "device" pointers are CUDA global-memory pointers of the current
 *     device (e.g. torch.Tensor.data_ptr()); "host" pointers are ordinary
 *     process memory.  Where a parameter says "host or device" the library
 *     tells them apart with cudaPointerGetAttributes.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Calls that return host results synchronise the
 *     stream before returning.
 *   - all matrices and vectors are row-major; indices are 0-based.
 *
 * Single-particle (s.p.) states: the caller lists them (S <= 256 per
 * species) with their HO shell N and 2m.  A species determinant is a bit
 * string with bit a set when state a is occupied (Sec. 2.1), stored as
 * W = ceil(S/64) little-endian 64-bit words.  A basis state is a pair (p, n)
 * of a proton and a neutron determinant, |p;n> = (prod_{a in p, ascending}
 * a+_{a,p}) (prod_{b in n, ascending} a+_{b,n}) |0>.
 *
 * Hamiltonian:  H = sum_a eps_a a+_a a_a  (both species)
 *   + 1/4 sum V^pp_abcd a+_a a+_b a_d a_c  + (the same for nn)
 *   + sum V^pn_abcd a+_{a,p} a+_{b,n} a_{d,n} a_{c,p},
 * V^pp and V^nn antisymmetrised, all three real, Hermitian and conserving m.
 */
#ifndef MFDCI_H
#define MFDCI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CI_OK = 0,
    CI_ERR_INVALID_ARG = 1,  /* a bad argument; nothing was changed        */
    CI_ERR_OOM = 2,          /* a device or host allocation failed         */
    CI_ERR_CUDA = 3,         /* a CUDA call failed (message names it)      */
    CI_ERR_CAPACITY = 4,     /* a size beyond a documented limit           */
    CI_ERR_TIMEOUT = 5,      /* a bounded wait gave up                     */
    CI_NOT_READY = 6,        /* ci_poll: the request is still running      */
    CI_ERR_CANCELLED = 7,    /* the request was cancelled                  */
    CI_ERR_INTERNAL = 8,     /* an internal consistency check failed      */
    CI_ERR_NOT_CONVERGED = 9,/* eigensolver hit its iteration limit        */
    CI_ERR_STATE = 10        /* call order violated (e.g. no basis yet)    */
} ci_status;

/* Precision of the stored H values (and of the arithmetic that makes them).
 * CI_F32: float values, FP32 accumulation of matrix-element terms.
 * CI_F64: double values, FP64 accumulation (the plain FP64 form).
 * CI_BF16_ROWSCALE: bf16 values times a per-row float scale (FP32 compute):
 *   the row is built in FP32, scale_r = max_j |H_rj| (1 for a zero row) and
 *   the stored value is H_rj / scale_r rounded to the nearest bf16; the SpMM
 *   multiplies each row's sum by scale_r (6 bytes per nonzero, values to
 *   about 2^-9 of the row's largest). */
typedef enum { CI_F32 = 0, CI_F64 = 1, CI_BF16_ROWSCALE = 2 } ci_value_type;

/* Where the two-body matrix elements come from. */
typedef enum {
    CI_TBME_TABLES = 0,  /* caller's flat tables v_pp, v_nn, v_pn            */
    CI_TBME_SEED = 1     /* counter-based generator from tbme_seed (below)   */
} ci_tbme_source;

typedef struct ci_problem ci_problem;
typedef struct ci_matrix ci_matrix;
typedef struct ci_batch ci_batch;
typedef struct ci_queue ci_queue;

/* Problem description (Sec. 2: many-body basis of A = Z + N nucleons).
 *
 * n_sp        S, s.p. states per species, 1..256 (|2m| <= 63).
 * sp_N        host [S]: HO shell N of each state (>= 0).
 * sp_twom     host [S]: 2m of each state (odd).
 * sp_energy   host [S]: one-body energies eps_a (both species).
 * Z, N        protons and neutrons, 0..min(S, 16).
 * nmax        Nmax cut on the total excess HO quanta q_p + q_n (q = sum of
 *             shells minus the lowest possible sum); -1 for no cut, else
 *             0..31.
 * twoM        total 2M of the basis.
 * tbme_source CI_TBME_TABLES or CI_TBME_SEED.
 * tbme_dtype  CI_F32 or CI_F64: element type of v_pp / v_nn / v_pn.
 * v_pp, v_nn, v_pn  flat tables V[((a*S+b)*S+c)*S+d], S^4 entries each, host
 *             or device memory, read during ci_problem_create only.
 * tbme_seed   with CI_TBME_SEED: V is drawn from SplitMix64 as follows.
 *             Like pairs a<b have index P = b(b-1)/2 + a, pn pairs (a,b)
 *             P = a*S + b; for pair indices P <= Q of pairs with equal
 *             m_a+m_b, counter c = (ch<<32)|(P<<16)|Q with ch = 0 (pp),
 *             1 (nn), 2 (pn); g = sum_{k=0..11} (mix(seed + (12c+k+1)*
 *             0x9E3779B97F4A7C15) >> 32) * 2^-32 - 6 (exact in binary64);
 *             V_abcd = V_cdab = g, completed by antisymmetry for pp, nn;
 *             an FP64 build uses g itself, an FP32 build g rounded to the
 *             nearest float (the float32 table of the same recipe). */
typedef struct {
    int32_t n_sp;
    const int32_t *sp_N;
    const int32_t *sp_twom;
    const double *sp_energy;
    int32_t Z, N;
    int32_t nmax;
    int32_t twoM;
    int32_t tbme_source;
    int32_t tbme_dtype;
    const void *v_pp, *v_nn, *v_pn;
    uint64_t tbme_seed;
} ci_problem_desc;

/* ---------------------------------------------------------------- errors */

/* Message of the last failed call on this thread ("" if none).  The
 * pointer stays valid until the next call on this thread. */
const char *ci_last_error(void);
/* Static name of a status code. */
const char *ci_status_string(ci_status s);
/* Library version string. */
const char *ci_version(void);

/* ---------------------------------------------------------------- problem */

/* Validate desc, copy the s.p. table, and stage the interaction on the
 * current device as compact m-blocked tables.  Errors: INVALID_ARG (bad
 * sizes, S > 256, Z or N > 16 or > S, missing tables), CAPACITY (nmax > 31,
 * |2m| > 63, more than 8192 one-particle moves with one change of 2m), OOM,
 * CUDA. */
ci_status ci_problem_create(const ci_problem_desc *desc, ci_problem **out);
void ci_problem_destroy(ci_problem *p);

/* Step 1 of Fig. 1: enumerate the species determinant lists and the
 * product basis (Sec. 2.1).  Each species list holds every A-particle
 * determinant with q <= nmax, sorted by (2M, q, value of the bit string).
 * The basis is p-major: for each proton determinant p (list order), every
 * neutron determinant n with 2M_p + 2M_n = twoM and q_p + q_n <= nmax, in
 * list order.  *dim receives the basis dimension.  Idempotent. */
ci_status ci_enumerate_basis(ci_problem *p, int64_t *dim, void *stream);

/* Size of a species list (species 0 = protons, 1 = neutrons) and its words
 * per bit string. Needs ci_enumerate_basis. */
ci_status ci_species_size(const ci_problem *p, int32_t species, int64_t *n, int32_t *words);
/* Copy a species list to host arrays of cap >= n entries: bits [n][words],
 * q [n], twoM [n]; any pointer may be NULL. */
ci_status ci_get_species(const ci_problem *p, int32_t species, uint64_t *bits,
                         int32_t *q, int32_t *twoM, int64_t cap);
/* Copy the basis to host arrays [dim]: the proton and neutron list index of
 * every basis state.  cap must be >= dim. */
ci_status ci_get_basis(const ci_problem *p, int32_t *p_idx, int32_t *n_idx, int64_t cap);

/* Fig. 1, tile filter (tiles) at the species level: for every determinant s of
 * a species, the determinants s' it can connect to through H, found by
 * popcount(BIN(s) XOR BIN(s')) (Sec. 2.1, Listing 2).  Kept: all s' with
 * 0 or 2 differing states, and s' with 4 differing states and 2M_s' =
 * 2M_s (a two-particle move of one species leaves the other species fixed,
 * so only equal-M partners can pair up in the basis).  Idempotent; called
 * by ci_count_nnz if needed. */
ci_status ci_species_filter(ci_problem *p, void *stream);
/* Copy species `species`' connectivity to host arrays: ptr [n+1] (int64),
 * idx [total] and d [total] (number of differing s.p. states: 0, 2, 4),
 * each row in ascending s'.  *total receives the entry count; with idx ==
 * NULL only *total and ptr are written. */
ci_status ci_get_species_conn(const ci_problem *p, int32_t species, int64_t *ptr,
                              int32_t *idx, int8_t *d, int64_t cap, int64_t *total);

/* Fig. 1, count step: number of structurally nonzero entries of every row,
 * i.e. basis states (p', n') within 4 differing s.p. states of the row
 * state (Listing 2's test, p and n bits side by side).  *nnz receives the
 * total; row_cnt (nullable, host or device, int32 [dim]) the per-row counts. */
ci_status ci_count_nnz(ci_problem *p, int64_t *nnz, int32_t *row_cnt, void *stream);

/* ---- Observables (Fig. 1, observables step, Sec. 2.4, Eq. 2) ------------------ */

/* Expectation values and transition elements
 *   a[k][v] = sum_ij X[i][v] (O_k)_ij Y[j][v]
 * of m two-body operators O_k over the problem's basis, for n vector pairs
 * (Y = NULL means Y = X: the expectation values of Eq. 2).  O_k has the pp,
 * nn and pn TBMEs of the CI_TBME_SEED recipe with seed op_seeds[k] and no
 * one-body part; its elements are evaluated on the fly by the Slater-Condon
 * rules of the Hamiltonian build (FP64 tables) and never stored.
 *   op_seeds  host, m seeds; m in 1..4096.
 *   X, Y      device, double [dim][n] in basis order, n in 1..16; Y may be
 *             NULL.  Both are only read.
 *   a         host, double [m][n] (written; the stream is synchronised).
 * The row kernel takes the vectors eight at a time, so n in 9..16 costs two
 * element evaluations per operator.  The problem's basis and FP64 species
 * connectivity are built on first use.
 * Errors: CI_ERR_INVALID_ARG (sizes, NULL or host X, host Y). */
ci_status ci_observables(ci_problem *p, const uint64_t *op_seeds, int32_t m, const double *X, const double *Y,
                         int32_t n, double *a, void *stream);

/* ---- Nonzero-count benchmark (Sec. 2.1, Listings 1-2, Figs. 3-4) ------- */

/* Forms of the pair test of ci_count_pairs; all give the same counts. */
typedef enum {
    CI_COUNT_HYBRID = 0,  /* popcount over the lowest 64 s.p. states, then the
                             MBS comparison for pairs that pass (Listing 2) */
    CI_COUNT_MBS = 1,     /* MBS comparison for every pair (no prefilter) */
    CI_COUNT_BITS = 2     /* full bit representation, popcount only; S <= 128 */
} ci_count_variant;

/* For n independent N-particle states, the number of states j (all n,
 * j = i included) whose occupations differ from state i in at most
 * max_diff single-particle states, both sides counted (Sec. 2.1: 2d = 4 for
 * a two-body operator, 6 for three-body).
 *   mbs         device, uint16 [n][N]: each state's occupied s.p. indices,
 *               strictly ascending, all < S (the MBS form of Sec. 2.1).
 *               Other inputs give unspecified counts but no fault.
 *   N           1..32; S: N..65535 (<= 128 for CI_COUNT_BITS).
 *   total       host int64: sum of the counts (the stream is synchronised).
 *   row_counts  device int64 [n] or NULL: the per-state counts.
 * Errors: CI_ERR_INVALID_ARG for bad sizes, host pointers or an unknown
 * variant; CI_ERR_CAPACITY when the launch grid would be too large. */
ci_status ci_count_pairs(const uint16_t *mbs, int64_t n, int32_t N, int32_t S, int32_t variant,
                         int32_t max_diff, int64_t *total, int64_t *row_counts, void *stream);

/* Eq. 1 / Alg. 1 (Sec. 2.2): exclusive prefix sum of n int32 counts into
 * n+1 int64 offsets, offsets[0] = 0 and offsets[n] = total.  counts and
 * offsets are device pointers; n >= 0 (n = 0 writes offsets[0] = 0).
 * Uses a library-owned scratch buffer, grown on demand. */
ci_status ci_exclusive_scan(const int32_t *counts, int64_t n, int64_t *offsets, void *stream);

/* The same exclusive scan without any device allocation, for callers that
 * cannot allocate: code whose device memory is owned by another caching
 * allocator or a fixed reservation, and latency-critical threads on which
 * cudaMalloc / cudaFree would stall by synchronising the device.  The
 * paper has no counterpart.  Its tile sums live in one static device array
 * (512 KB, held by every GPU that loads the library until the process
 * exits), so n is limited to 2^28 counts; larger n returns CI_ERR_CAPACITY.
 * The first call on a device looks up the array's device address (make it
 * before any stream capture) and keeps it for the life of the process: after
 * cudaDeviceReset on that device the kept address is stale, and later calls
 * on that device are invalid.  All calls share the array: calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Outputs are identical to ci_exclusive_scan. */
ci_status ci_exclusive_scan_noalloc(const int32_t *counts, int64_t n, int64_t *offsets, void *stream);

/* Fig. 1, offsets and fill (Sec. 2.3, Listing 7): build H in CSR form on the
 * device.  Row i holds every column j with at most 4 differing s.p. states
 * (stored even when its value is 0), columns ascending.  H_ij = <Phi_i|H|Phi_j>
 * by the Slater-Condon rules, the phase from masked popcounts.  The matrix
 * is library-owned (int64 row_ptr [dim+1], int32 col [nnz], values of vtype;
 * CI_BF16_ROWSCALE adds float row_scale [dim]). */
ci_status ci_build_H(ci_problem *p, int32_t vtype, ci_matrix **out, void *stream);
void ci_matrix_destroy(ci_matrix *m);

/* Half storage of the symmetric H (Fig. 2, optional FMA: a stored H_ij also
 * updates the j-th output with the i-th input): a new matrix holding the
 * upper triangle (col >= row, diagonal included) of m, same value type and
 * row scales, nnz = (nnz(m) + dim) / 2 for H's symmetric pattern.
 * ci_apply_H on it zeroes Y and adds H_ij X_j to Y_i and H_ij X_i to Y_j with
 * atomic adds (run-to-run differences in the last bits of Y); the
 * eigensolvers and the block preconditioner accept it (the preconditioner
 * mirrors the stored elements).  ci_matrix_export returns the stored
 * triangle.  Errors: CI_ERR_INVALID_ARG (NULL, m already half-stored). */
ci_status ci_matrix_upper(const ci_matrix *m, ci_matrix **out, void *stream);
ci_status ci_matrix_info(const ci_matrix *m, int64_t *dim, int64_t *nnz, int32_t *vtype);
/* Copy H out to caller buffers (each host or device, each nullable):
 * row_ptr [dim+1] int64, col [nnz] int32, val [nnz] (float, double or
 * uint16 bf16 bits by vtype), row_scale [dim] float (BF16 only). */
ci_status ci_matrix_export(const ci_matrix *m, int64_t *row_ptr, int32_t *col,
                           void *val, float *row_scale, void *stream);

/* Fig. 2, optional FMA (Sec. 2): Y = H X for a block of nvec vectors (1..8, or
 * 16), X and Y device arrays [dim][nvec] (float for CI_F32 / CI_BF16_ROWSCALE,
 * double for CI_F64), not overlapping.  Each row is accumulated in the value
 * precision in ascending column order within each of 32 lanes.  nvec = 16
 * (full-storage CI_F32 or CI_BF16_ROWSCALE only, 16-byte aligned X and Y) is
 * the product LOBPCG uses for [X P]: one gather of a 64-byte X row per
 * nonzero, each row's sum split over 8 lane groups instead of 16, so its
 * results differ from two 8-vector products in the last FP32 bits.
 * Errors: CI_ERR_INVALID_ARG (other nvec, misaligned X or Y, nvec = 16 on
 * a half-stored or FP64 matrix). */
ci_status ci_apply_H(const ci_matrix *m, const void *X, void *Y, int32_t nvec, void *stream);

/* ---------------------------------------------------------------- eigensolver */

/* Sec. 2, Fig. 1 eigensolve: the products of the block Lanczos solver's
 * full FP64 reorthogonalisation against its basis A (n rows, columns
 * orthonormal, |A_iu| <= 1), exposed for tests and for callers with a basis
 * of their own.  Device pointers, row-major, caller-owned:
 *   op CI_PRODUCT_TN: C [na][nb] = A^T B   (A [n][lda], B [n][ldb])
 *   op CI_PRODUCT_NN: B = beta B + alpha A C   (C [na][nb], B [n][ldb];
 *                     beta = 0 does not read B)
 * method CI_PRODUCT_FP64: FP64 FMAs on the CUDA cores (1 <= na <= 256,
 * 1 <= nb <= 8).  method CI_PRODUCT_TC: on the tensor cores (tcgen05.mma,
 * FP16 inputs, FP32 accumulation): each operand is cut into eight balanced
 * 8-bit digit planes relative to a power-of-two scale (A: 2^0, so
 * |A| < 1.99 is required; B and C: per vector, above its largest entry),
 * every plane product is exact, and the planes are recombined in 64- and
 * 128-bit integers with one or two roundings to FP64 per output.  The result
 * differs from the exact product by at most about 2^-52 |result| +
 * 2^-60 n max|B| (TN) or 2^-52 |result| + 2^-60 na max|C| (NN) -- FP64
 * accuracy -- and needs nb = 8 and na <= 64.
 * Synchronises the stream.
 * Errors: CI_ERR_INVALID_ARG (shapes, an entry of A with |a| >= 1.99 or a
 * non-finite operand for CI_PRODUCT_TC), CI_ERR_TIMEOUT (a tensor-core wait
 * ran out; the context stays usable). */
enum { CI_PRODUCT_TN = 0, CI_PRODUCT_NN = 1 };
enum { CI_PRODUCT_FP64 = 0, CI_PRODUCT_TC = 1 };
ci_status ci_basis_product(int32_t op, int32_t method, int64_t n, const double *A, int32_t lda, int32_t na,
                           double *B, int32_t ldb, int32_t nb, double *C, double alpha, double beta, void *stream);

/* Options of ci_lowest_eigs; zero fields take the defaults in brackets. */
typedef struct {
    int32_t k;            /* eigenpairs wanted, 1..32                      [5]  */
    int32_t block;        /* block size b, 1..8                            [8]  */
    int32_t max_basis;    /* Krylov vectors kept before a thick restart   [64] */
    int32_t max_iter;     /* block steps in total                       [2000] */
    double tol;           /* converged when the Ritz residual estimate is
                             <= tol*||H|| [1e-6 for FP32 H, 1e-10 for FP64 H];
                             the eigenvalue error is then ~ residual^2/gap */
    uint64_t seed;        /* seed of the start block                      [1]  */
    int32_t reorth_passes;/* full Gram-Schmidt passes per step after the
                             projection on the two newest blocks, 1..2    [1]  */
    int32_t check_every;  /* block steps between convergence checks       [1]  */
    int32_t fp64_products;/* 1: the reorthogonalisation products on the FP64
                             CUDA cores; 0: on the tensor cores as exact
                             products of 8-bit digit planes (FP64 accuracy,
                             see ci_basis_product)                          [0] */
} ci_eig_opts;

typedef struct {
    int32_t iterations;   /* block steps taken                                  */
    int32_t restarts;     /* thick restarts                                     */
    int32_t converged;    /* number of converged pairs among the k              */
    int32_t basis_size;   /* Krylov vectors at the end                          */
    double hnorm_est;     /* estimate of ||H||_2 (largest |Ritz value| seen)    */
    double residual[32];  /* ||H x_i - theta_i x_i||_2, FP64, with the stored H */
    double seconds;       /* wall time of the call                              */
    int32_t host_qr;      /* block Lanczos: block steps whose block QR fell back
                             from the device (Cholesky) path to the host's
                             rank-revealing one (deflation, random completion) */
    int32_t qr_one_pass;  /* block Lanczos: block steps whose first (device)
                             block-QR pass already left the block orthonormal
                             to 1e-13, so the second pass formed no product */
} ci_eig_info;

/* Fig. 1, eigensolve (Sec. 2): lowest k eigenvalues of H by block Lanczos with
 * full FP64 reorthogonalisation (classical Gram-Schmidt against the two
 * newest blocks, then reorth_passes passes over the whole basis) and thick
 * restart.  SpMM in the matrix's precision, everything else in FP64.  Each
 * new block is orthonormalised on the device (Cholesky QR, then a
 * Newton-Schulz pass, whose product is skipped when the block's Gram matrix
 * is already the identity to 1e-13) without a host sync; a numerically
 * rank-deficient
 * block is redone by the host's rank-revealing QR (info->host_qr counts
 * those).  The host reads the projection coefficients and the coupling
 * while the next product runs.  evals: host [k], ascending.  evecs:
 * nullable device double [dim][k], unit norm.  info: nullable.  Returns
 * CI_ERR_NOT_CONVERGED (with the best estimates written) if max_iter is hit. */
ci_status ci_lowest_eigs(const ci_matrix *m, const ci_eig_opts *opts, double *evals,
                         double *evecs, ci_eig_info *info, void *stream);

/* Fig. 1, eigensolve (Sec. 2): the same lowest k eigenpairs by LOBPCG (block
 * size opts->block >= k, search space [X, W, P] of three blocks), W = T R
 * the preconditioned residuals, Rayleigh-Ritz through the FP64 Gram
 * matrices of the three blocks (Cholesky of the overlap; P is dropped for an
 * iteration when the overlap loses rank).  SpMM in the matrix's precision,
 * everything else in FP64.
 *   row_block, nblocks  NULL / 0: the diagonal (Jacobi) preconditioner
 *             T = (diag(H) - theta_v)^-1 per vector.  Otherwise a device
 *             int32 [dim] group index in 0..nblocks-1 of every row (e.g.
 *             from ci_orbital_blocks) and the block-diagonal preconditioner
 *             of ci_block_precond_apply over those groups, its shift sigma =
 *             theta_1 - |r_1| taken from the Rayleigh-Ritz of iterations
 *             0, 2, 6, 14, 30, ... (the blocks are re-inverted then).
 * Options and outputs as ci_lowest_eigs; max_basis, reorth_passes and
 * check_every are ignored, max_iter counts iterations [1000].  The default
 * tol is 4e-3 for a CI_BF16_ROWSCALE matrix: its per-row scales round H_ij
 * and H_ji differently, and the true residuals of the nearly symmetric
 * operator stop near that rounding (2^-9).  Dimensions up to 4*block use the
 * dense path of ci_lowest_eigs.  Errors as
 * ci_lowest_eigs, plus CI_ERR_INVALID_ARG for a row_block entry outside
 * 0..nblocks-1 or a host row_block. */
ci_status ci_lowest_eigs_lobpcg(const ci_matrix *m, const ci_eig_opts *opts, const int32_t *row_block,
                                int64_t nblocks, double *evals, double *evecs, ci_eig_info *info, void *stream);

/* Refinement of Ritz pairs found with a reduced-precision H (an FP32 or
 * BF16 build): the FP64 Hamiltonian of the problem, its elements evaluated
 * on the fly by the Slater-Condon rules of the build (nothing stored), is
 * applied to the k vectors; Rayleigh-Ritz in FP64 on their span, then
 * `iters` Rayleigh-Ritz steps on span[X, R] with the FP64 residuals
 * R = H X - X Theta.  The Ritz values then carry the FP64 operator's
 * rounding instead of the FP32 matrix's.
 *   k          1..16 vectors; iters 0..16 (each costs one FP64 application
 *              of H to k vectors, eight per pass).
 *   evecs      device double [dim][k], the approximate eigenvectors in basis
 *              order; overwritten with the refined, orthonormal vectors.
 *   evals      host [k]: refined Ritz values, ascending.
 *   residuals  host [k] or NULL: ||H x - theta x|| with the FP64 H.
 * Errors: CI_ERR_INVALID_ARG (sizes, host evecs, dependent vectors). */
ci_status ci_refine_eigs(ci_problem *p, int32_t k, int32_t iters, double *evecs, double *evals,
                         double *residuals, void *stream);

/* Many-body basis orbitals (Sec. 2): the basis states that put the
 * nucleons of each species into the same single-particle orbitals, i.e.
 * differ only in the orbitals' magnetic substates, form one group; a
 * group of the product basis is a pair (proton group, neutron group).
 *   sp_orbital  host int32 [S]: orbital label (>= 0) of every s.p. state;
 *               states with equal labels belong to one orbital (n, l, j).
 *   block       device int32 [dim] or NULL: group of every basis state,
 *               numbered 0, 1, ... in order of first appearance by row.
 *   nblocks     host int64: number of groups.
 * Errors: CI_ERR_INVALID_ARG (NULL or negative labels, host block). */
ci_status ci_orbital_blocks(ci_problem *p, const int32_t *sp_orbital, int32_t *block, int64_t *nblocks,
                            void *stream);

/* The block-diagonal preconditioner of LOBPCG (Sec. 2: the diagonal blocks
 * of H over many-body orbitals), applied once:
 *   W = T R,  T = blockdiag_b (H_bb - sigma_b I)^-1.
 * The blocks are the groups of row_block, each cut into consecutive
 * sub-blocks of at most 128 rows (member rows ascending, split into
 * ceil(c/128) parts whose sizes differ by at most one, the larger first).
 * sigma_b = sigma when H_bb - sigma I is positive definite (every pivot of
 * the Gauss-Jordan inversion > 1e-12 (||H_bb||_inf + |sigma|)), else
 * min(sigma, g_b) - 1e-3 max(||H_bb||_inf, |sigma|) with g_b the Gershgorin
 * lower bound min_i (H_ii - sum_{j != i} |H_ij|) over the sub-block.
 * Inverses are formed in FP64, stored and applied in FP32.
 *   row_block, nblocks  as ci_lowest_eigs_lobpcg (device, required).
 *   R, W        device double [dim][nvec], nvec 1..8.
 *   row_shift   device double [dim] or NULL: sigma_b of each row's sub-block.
 * The stream is synchronised.  Errors: CI_ERR_INVALID_ARG (pointers, sizes,
 * group indices, non-finite sigma). */
ci_status ci_block_precond_apply(const ci_matrix *m, const int32_t *row_block, int64_t nblocks, double sigma,
                                 const double *R, double *W, int32_t nvec, double *row_shift, void *stream);

/* ---------------------------------------------------------------- batched solves */

/* Many independent problems built and solved together (Fig. 1, basis through eigensolve
 * for each): every build step runs as one launch over all problems (the
 * matrices form one block-diagonal CSR, FP32 values), and the solve is a
 * block Lanczos whose per-problem control (basis size, thick restart,
 * FP64 Ritz solve by Jacobi, convergence) runs in kernels, so one step of
 * every unfinished problem is a CUDA graph replay.
 *
 * probs: n problem handles (borrowed; they must outlive the batch).
 * k: per-problem eigenpair counts (1..16), or NULL to use opts->k.
 * opts: block must be 0 or 8; max_basis (default 64) a multiple of 8 in
 * 32..96 with 2(k+8) <= max_basis; tol default 1e-7 (relative to ||H||);
 * max_iter default 400 steps; check_every default 4 steps.
 * Problems need dimension > max_basis + 16. */
ci_status ci_batch_create(ci_problem *const *probs, int32_t n, const int32_t *k, const ci_eig_opts *opts,
                          ci_batch **out);
/* Build every H and solve.  Synchronous. */
ci_status ci_batch_run(ci_batch *b, void *stream);
/* Eigenvalues of problem i (host [k], ascending) and, in info, the steps
 * taken and the FP64 residuals ||H x - theta x|| (H applied in FP32).
 * Returns CI_ERR_NOT_CONVERGED (with the values written) if the problem
 * stopped at max_iter. */
ci_status ci_batch_result(const ci_batch *b, int32_t i, double *evals, ci_eig_info *info);
/* Wall time of the build and of the solve, engine steps, total nonzeros. */
ci_status ci_batch_stats(const ci_batch *b, double *build_s, double *solve_s, int32_t *steps, int64_t *nnz);

/* The launch shape the autotuner picked for the batch's persistent kernels
 * (CTAs per SM of the row-tile kernels and of the SpMM; every tile is
 * handled by one CTA and every row by one warp, so results do not depend
 * on it), and the best step time it measured (0 when the choice came from
 * its cache).  ci_batch_run times two real Lanczos steps per candidate
 * (tile kernels 2, 4, 8, 16 CTAs per SM, then SpMM 4, 8, 16) and caches the
 * choice per device, slot count and row count (to a power of two).
 * Errors: CI_ERR_STATE before ci_batch_run. */
ci_status ci_batch_tuning(const ci_batch *b, int32_t *tile_ctas_per_sm, int32_t *spmm_ctas_per_sm,
                          double *best_step_ms);
void ci_batch_destroy(ci_batch *b);

/* ---------------------------------------------------------------- serving */

/* A solve queue with continuous batching.  A worker thread owns the GPU:
 * between two steps of the batched block Lanczos (see ci_batch_create) it
 * returns finished problems and admits waiting ones, first come first
 * served, into free slots while their device memory (CSR, Krylov basis,
 * connectivity lists, tables) fits mem_budget.  Admitted problems are built
 * together and join the running ones at the next step, so requests that
 * arrive while others run overlap with them; each keeps H and its Krylov
 * vectors on the device until it finishes.  A problem's result does not
 * depend on what else runs beside it (per-problem start block and
 * reductions).  A request whose basis has at most max_basis + 16 states is
 * too small for the engine's blocks: the worker builds its FP32 H alone and
 * solves it at admission with ci_lowest_eigs' whole-space Rayleigh-Ritz
 * (k must not exceed the dimension; an empty basis fails with
 * CI_ERR_INVALID_ARG).  The paper has no counterpart. */
typedef struct {
    size_t mem_budget;    /* device bytes the queue may hold; 0 = 70 % of free memory */
    int32_t max_slots;    /* problems running at once, 1..4096                  [256] */
    int32_t max_basis;    /* Krylov vectors per problem (multiple of 8, 32..96)  [64] */
    int32_t max_iter;     /* block steps per problem                             [400] */
    int32_t max_tiles;    /* 256-row tiles over all running problems           [65536] */
    double tol;           /* residual tolerance relative to ||H||              [1e-7] */
} ci_queue_desc;

typedef struct {
    ci_problem_desc desc; /* copied at submission (tables too) */
    int32_t k;            /* eigenpairs, 1..16 with 2(k+8) <= max_basis */
} ci_request;

typedef struct {
    int32_t status;       /* CI_OK, CI_NOT_READY, or the request's error */
    int32_t k;
    int32_t iterations;
    int64_t dim, nnz;
    double evals[16];     /* ascending */
    double residual[16];  /* ||H x - theta x||, FP64 */
    double t_submit, t_admit, t_done;  /* seconds on the queue's steady clock */
    double latency_s;     /* t_done - t_submit */
} ci_result;

ci_status ci_queue_create(const ci_queue_desc *desc, ci_queue **out);
/* Queue a request; returns at once with a ticket. */
ci_status ci_submit(ci_queue *q, const ci_request *req, uint64_t *ticket);
/* CI_NOT_READY while the request waits or runs; then its final status
 * (CI_OK, CI_ERR_NOT_CONVERGED, CI_ERR_CAPACITY, CI_ERR_CANCELLED, ...),
 * with res filled either way. */
ci_status ci_poll(ci_queue *q, uint64_t ticket, ci_result *res);
/* Cancel a waiting or running request (it finishes as CI_ERR_CANCELLED). */
ci_status ci_cancel(ci_queue *q, uint64_t ticket);
ci_status ci_queue_stats(ci_queue *q, int64_t *submitted, int64_t *admitted, int64_t *completed, int64_t *steps,
                         size_t *mem_used);
/* Cancels what is left, waits for the worker and frees everything. */
void ci_queue_destroy(ci_queue *q);

/* ---------------------------------------------------------------- motifs */

/* The paper's motif benchmarks (Sec. 2.2-2.4), as measured primitives.
 *
 * Listing 5 / Fig. 5: the serial prefix sum on the device, one thread:
 * offsets[0] = 0, offsets[i+1] = offsets[i] + counts[i].  The control for
 * the parallel ci_exclusive_scan (same inputs and outputs, device
 * pointers).  The stream is synchronised. */
ci_status ci_scan_serial(const int32_t *counts, int64_t n, int64_t *offsets, void *stream);

/* Listing 7 / Fig. 6: fill a shared array from per-row offsets.  Row i
 * (0..n-1) stores the values j in 1..m with j mod p == 0, ascending, at
 * arr[offset[i] + r], r = 0, 1, ... (the rank replaces the listing's
 * atomic counter, so the result is deterministic).  offset: device int64
 * [n] (e.g. the exclusive scan of m/p per row); arr: device int32, large
 * enough for every row.  m >= 0, p >= 1.  The stream is synchronised. */
ci_status ci_fill_shared(const int64_t *offset, int64_t n, int32_t m, int32_t p, int32_t *arr, void *stream);

/* Eq. 2 / Listings 8-9 / Fig. 7: the small-array reduction
 *   a[k] = sum_{i,j < n} x[k + m i] * y[k + m j],   k < m,
 * over all n^2 pairs (x, y: device float, column-major m x n, as the
 * listings' x(k,i)).  FP32 products and per-lane FP32 sums; the block and
 * grid partials are added in a fixed order in FP64; a: device float [m].
 * m in {8, 16, 32, 64, 128, 256}.  The stream is synchronised. */
ci_status ci_array_reduction(const float *x, const float *y, int64_t n, int32_t m, float *a, void *stream);

/* ---------------------------------------------------------------- tracing */

/* Kernel tracing.  While on, every kernel the library launches is counted
 * per name and bracketed by two CUDA events on its launch stream: every
 * launch (on = 1) or, sampled, the first of every `on` launches of each
 * kernel (on >= 2; total_ms is then the timed launches' mean times the
 * launch count).  Each timed launch costs two event records on the host.
 * on = 0 turns tracing off.  No paper counterpart beyond timing regions
 * (Listing 10). */
typedef struct {
    char name[48];       /* kernel name                                  */
    int64_t launches;    /* launches recorded since the last reset       */
    double total_ms;     /* their event-measured durations (ms), summed;
                            sampled: mean of the timed ones x launches  */
} ci_trace_entry;

ci_status ci_trace_enable(int32_t on);
/* Synchronise the recorded events and copy up to cap entries (sorted by
 * name) to out; *n receives the number of kernel names.  reset != 0 clears
 * the statistics after reading. */
ci_status ci_trace_read(ci_trace_entry *out, int32_t cap, int32_t *n, int32_t reset);

#ifdef __cplusplus
}
#endif
#endif /* MFDCI_H */
