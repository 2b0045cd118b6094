/*
 * FP64 CPU oracle of the configuration-interaction (CI) hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load or run this file.  It shares no code
 * with the CUDA library and it is deliberately plain and slow.
 *
 * What it computes (paper, Sec. 2 and Sec. 2.1; Fig. 1):
 *   - the species determinant lists (one list per species), each determinant
 *     stored as its ascending tuple of occupied s.p. states (the MBS form of
 *     Sec. 2.1);
 *   - the product basis Phi = (p, n) with total 2M fixed and the Nmax cut;
 *   - the number of differently occupied s.p. states of two determinants
 *     (Sec. 2.1: always even, at most 2d = 4 for a two-body H);
 *   - the matrix element <Phi_i|H|Phi_j> by the textbook Slater-Condon rules
 *     (the paper leaves matrix elements to "separate subroutine calls",
 *     Sec. 2.1), with the fermion phase found by applying the creation and
 *     annihilation operators one at a time to the ket's occupation list;
 *   - rows of H in ascending column order, visiting every column j as in the
 *     dense count of Listing 2, and the full CSR matrix;
 *   - the count benchmark of Sec. 2.1 (Listing 2 over independent random
 *     states in MBS form): per state, the number of states that differ from
 *     it in at most max_diff single-particle states.
 *
 * Hamiltonian:  H = sum_a eps_a a+_a a_a   (both species)
 *                 + 1/4 sum V^pp_abcd a+_a a+_b a_d a_c   (same for nn)
 *                 + sum V^pn_abcd a+_{a,p} a+_{b,n} a_{d,n} a_{c,p}
 * with antisymmetrised V^pp, V^nn and flat tables V[((a*S+b)*S+c)*S+d], or,
 * without tables, the seeded counter-based draws described at V_seeded.
 * Determinant convention: |p;n> = (prod_{i in p, ascending} a+_{i,p})
 *                                 (prod_{j in n, ascending} a+_{j,n}) |0>.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXA 32

typedef struct {
    int S;                 /* s.p. states per species                     */
    const int *sp_N;       /* [S] HO shell of each s.p. state             */
    const int *sp_twom;    /* [S] 2m of each s.p. state                   */
    const double *eps;     /* [S] one-body energies                       */
    const double *Vpp, *Vnn, *Vpn;   /* [S^4] each, or all NULL: drawn     */
    int A[2];              /* particles: [0] protons, [1] neutrons         */
    int nmax;              /* -1: no Nmax cut                              */
    int twoM;              /* total 2M                                     */
    uint64_t seed;         /* with NULL tables: seed of the drawn TBMEs    */
    int round_f32;         /* with NULL tables: round each draw to float32 */
} orc_problem;

/* ---------------------------------------------------------------------- */
/* Species determinants                                                    */
/* ---------------------------------------------------------------------- */

typedef struct {
    int A;
    int64_t n;
    uint8_t *occ;   /* [n][A] ascending occupied s.p. states */
    int *q;         /* [n] excess HO quanta above the lowest filling */
    int *twoM;      /* [n] total 2M of the species determinant      */
} orc_species;

/* Smallest possible sum of N over A particles: fill the lowest N first. */
static int min_quanta(const orc_problem *pr, int A)
{
    int *Ns = (int *)malloc(sizeof(int) * (size_t)pr->S);
    for (int i = 0; i < pr->S; ++i) Ns[i] = pr->sp_N[i];
    /* plain selection of the A smallest values */
    int total = 0;
    for (int k = 0; k < A; ++k) {
        int best = k;
        for (int i = k + 1; i < pr->S; ++i) if (Ns[i] < Ns[best]) best = i;
        int t = Ns[k]; Ns[k] = Ns[best]; Ns[best] = t;
        total += Ns[k];
    }
    free(Ns);
    return total;
}

typedef struct { uint8_t *buf; int64_t n, cap; int A; } occ_list;

static void occ_push(occ_list *L, const uint8_t *occ)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->buf = (uint8_t *)realloc(L->buf, (size_t)(L->cap * (L->A ? L->A : 1)));
    }
    if (L->A) memcpy(L->buf + L->n * L->A, occ, (size_t)L->A);
    L->n++;
}

/* All ascending A-tuples of states 0..S-1 (every Slater determinant of A
 * fermions), keeping those with excess quanta q <= nmax. */
static void enumerate_rec(const orc_problem *pr, int A, int nmin, int start,
                          int depth, int Nsum, uint8_t *occ, occ_list *L)
{
    if (depth == A) {
        if (pr->nmax < 0 || Nsum - nmin <= pr->nmax) occ_push(L, occ);
        return;
    }
    for (int o = start; o < pr->S; ++o) {
        occ[depth] = (uint8_t)o;
        enumerate_rec(pr, A, nmin, o + 1, depth + 1, Nsum + pr->sp_N[o], occ, L);
    }
}

/* Order of a species list: by 2M, then by q, then by the numeric value of
 * the bit string BIN = sum_i 2^(occupied state i).  Two bit strings with the
 * same number of ones compare like their highest differing bit, i.e. like
 * the occupied tuples read from the top down. */
static const orc_species *g_sort_sp;
static int species_cmp(const void *x, const void *y)
{
    int64_t i = *(const int64_t *)x, j = *(const int64_t *)y;
    const orc_species *s = g_sort_sp;
    if (s->twoM[i] != s->twoM[j]) return s->twoM[i] < s->twoM[j] ? -1 : 1;
    if (s->q[i] != s->q[j]) return s->q[i] < s->q[j] ? -1 : 1;
    for (int k = s->A - 1; k >= 0; --k) {
        int a = s->occ[i * s->A + k], b = s->occ[j * s->A + k];
        if (a != b) return a < b ? -1 : 1;
    }
    return 0;
}

int orc_species_build(const orc_problem *pr, int species, orc_species *out)
{
    int A = pr->A[species];
    if (A < 0 || A > ORC_MAXA || A > pr->S) return -1;
    int nmin = min_quanta(pr, A);
    occ_list L = {0};
    L.A = A;
    uint8_t occ[ORC_MAXA];
    enumerate_rec(pr, A, nmin, 0, 0, 0, occ, &L);
    orc_species raw;
    raw.A = A; raw.n = L.n; raw.occ = L.buf;
    raw.q = (int *)malloc(sizeof(int) * (size_t)(L.n ? L.n : 1));
    raw.twoM = (int *)malloc(sizeof(int) * (size_t)(L.n ? L.n : 1));
    for (int64_t i = 0; i < L.n; ++i) {
        int Nsum = 0, m = 0;
        for (int k = 0; k < A; ++k) {
            Nsum += pr->sp_N[L.buf[i * A + k]];
            m += pr->sp_twom[L.buf[i * A + k]];
        }
        raw.q[i] = Nsum - nmin;
        raw.twoM[i] = m;
    }
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L.n ? L.n : 1));
    for (int64_t i = 0; i < L.n; ++i) perm[i] = i;
    g_sort_sp = &raw;
    qsort(perm, (size_t)L.n, sizeof(int64_t), species_cmp);
    out->A = A; out->n = L.n;
    out->occ = (uint8_t *)malloc((size_t)(L.n * (A ? A : 1)));
    out->q = (int *)malloc(sizeof(int) * (size_t)(L.n ? L.n : 1));
    out->twoM = (int *)malloc(sizeof(int) * (size_t)(L.n ? L.n : 1));
    for (int64_t i = 0; i < L.n; ++i) {
        if (A) memcpy(out->occ + i * A, raw.occ + perm[i] * A, (size_t)A);
        out->q[i] = raw.q[perm[i]];
        out->twoM[i] = raw.twoM[perm[i]];
    }
    free(perm); free(raw.occ); free(raw.q); free(raw.twoM);
    return 0;
}

void orc_species_free(orc_species *s)
{
    free(s->occ); free(s->q); free(s->twoM);
    memset(s, 0, sizeof(*s));
}

/* ---------------------------------------------------------------------- */
/* Product basis (Sec. 2: many-body states Phi = proton x neutron)         */
/* ---------------------------------------------------------------------- */

/* Basis states (p, n): p-major over the proton list, and for each p every
 * n of the neutron list (in list order) with 2M_p + 2M_n = 2M and, when
 * nmax >= 0, q_p + q_n <= nmax.  With p_idx == NULL only counts. */
int64_t orc_basis(const orc_problem *pr, const orc_species *P,
                  const orc_species *Nn, int32_t *p_idx, int32_t *n_idx)
{
    int64_t dim = 0;
    for (int64_t p = 0; p < P->n; ++p) {
        for (int64_t n = 0; n < Nn->n; ++n) {
            if (P->twoM[p] + Nn->twoM[n] != pr->twoM) continue;
            if (pr->nmax >= 0 && P->q[p] + Nn->q[n] > pr->nmax) continue;
            if (p_idx) { p_idx[dim] = (int32_t)p; n_idx[dim] = (int32_t)n; }
            ++dim;
        }
    }
    return dim;
}

/* ---------------------------------------------------------------------- */
/* Differences and fermion phases (Sec. 2.1)                               */
/* ---------------------------------------------------------------------- */

/* Number of s.p. states occupied in exactly one of two A-particle
 * determinants given as ascending tuples (a merge walk over both). */
int orc_count_difference(const uint8_t *s1, const uint8_t *s2, int A)
{
    int i = 0, j = 0, d = 0;
    while (i < A && j < A) {
        if (s1[i] < s2[j]) { ++d; ++i; }
        else if (s1[i] > s2[j]) { ++d; ++j; }
        else { ++i; ++j; }
    }
    return d + (A - i) + (A - j);
}

/* Annihilate state o in the ascending list occ[0..*n).  Returns 0 if o is
 * empty, else (-1)^(number of occupied states below o), and removes o. */
static int apply_annihilate(uint8_t *occ, int *n, int o)
{
    int pos = -1;
    for (int k = 0; k < *n; ++k) if (occ[k] == o) { pos = k; break; }
    if (pos < 0) return 0;
    for (int k = pos; k < *n - 1; ++k) occ[k] = occ[k + 1];
    --*n;
    return (pos % 2) ? -1 : 1;
}

/* Create state o in the ascending list occ[0..*n).  Returns 0 if o is
 * occupied, else (-1)^(number of occupied states below o), and inserts o. */
static int apply_create(uint8_t *occ, int *n, int o)
{
    int pos = 0;
    for (int k = 0; k < *n; ++k) {
        if (occ[k] == o) return 0;
        if (occ[k] < o) pos = k + 1;
    }
    for (int k = *n; k > pos; --k) occ[k] = occ[k - 1];
    occ[pos] = (uint8_t)o;
    ++*n;
    return (pos % 2) ? -1 : 1;
}

/* States occupied in x but not in y (ascending), returns how many. */
static int set_minus(const uint8_t *x, const uint8_t *y, int A, int *out)
{
    int c = 0;
    for (int i = 0; i < A; ++i) {
        int found = 0;
        for (int j = 0; j < A; ++j) if (x[i] == y[j]) { found = 1; break; }
        if (!found) out[c++] = x[i];
    }
    return c;
}

static double absd(double x) { return x < 0 ? -x : x; }

/* SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014). */
static uint64_t splitmix_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* One seeded TBME draw for pair indices P <= Q of channel ch: twelve
 * SplitMix64 outputs at stream positions 12c+1 .. 12c+12 of the counter
 * c = (ch << 32) | (P << 16) | Q, each taken as a uniform (z >> 32) 2^-32,
 * summed, minus 6 (Irwin-Hall).  The partial sums are exact in binary64. */
static double seeded_draw(uint64_t seed, int ch, uint64_t P, uint64_t Q)
{
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    uint64_t c = ((uint64_t)ch << 32) | (P << 16) | Q;
    double g = 0.0;
    for (int k = 1; k <= 12; ++k)
        g += (double)(splitmix_mix(seed + (12 * c + (uint64_t)k) * gamma) >> 32) * 0x1p-32;
    return g - 6.0;
}

/* V_abcd of channel ch (0 pp, 1 nn, 2 pn) when no tables are given: zero
 * unless m_a + m_b = m_c + m_d; like-particle elements are antisymmetric in
 * (a, b) and in (c, d) and vanish for a == b or c == d, with a < b pairs
 * numbered P = b(b-1)/2 + a; pn pairs are numbered P = a S + b; the element
 * of the unordered pair of pair indices is one draw (V_abcd = V_cdab). */
static double V_seeded(const orc_problem *pr, int ch, int a, int b, int c, int d)
{
    const int *m = pr->sp_twom;
    if (m[a] + m[b] != m[c] + m[d]) return 0.0;
    double sign = 1.0;
    uint64_t P, Q;
    if (ch < 2) {
        if (a == b || c == d) return 0.0;
        if (a > b) { int t = a; a = b; b = t; sign = -sign; }
        if (c > d) { int t = c; c = d; d = t; sign = -sign; }
        P = (uint64_t)b * (uint64_t)(b - 1) / 2 + (uint64_t)a;
        Q = (uint64_t)d * (uint64_t)(d - 1) / 2 + (uint64_t)c;
    } else {
        P = (uint64_t)a * (uint64_t)pr->S + (uint64_t)b;
        Q = (uint64_t)c * (uint64_t)pr->S + (uint64_t)d;
    }
    double g = P <= Q ? seeded_draw(pr->seed, ch, P, Q) : seeded_draw(pr->seed, ch, Q, P);
    if (pr->round_f32) g = (double)(float)g;
    return sign * g;
}

/* V_abcd of channel ch from the flat table V[((a*S+b)*S+c)*S+d], or drawn. */
static double Vch(const orc_problem *pr, int ch, int a, int b, int c, int d)
{
    const double *V = ch == 0 ? pr->Vpp : ch == 1 ? pr->Vnn : pr->Vpn;
    if (!V) return V_seeded(pr, ch, a, b, c, d);
    const int64_t S = pr->S;
    return V[(((int64_t)a * S + b) * S + c) * S + d];
}

/* Phase of the operator string applied right to left to the ket tuple, and
 * check that it lands on the bra tuple. ops[k] = +o (create o) or -(o+1)
 * (annihilate o), applied ops[0] first. */
static int phase_of(const uint8_t *ket, const uint8_t *bra, int A,
                    const int *ops, int nops)
{
    uint8_t w[ORC_MAXA + 4];
    int n = A, s = 1;
    memcpy(w, ket, (size_t)A);
    for (int k = 0; k < nops; ++k) {
        int f = ops[k] >= 0 ? apply_create(w, &n, ops[k])
                            : apply_annihilate(w, &n, -ops[k] - 1);
        if (f == 0) return 0;
        s *= f;
    }
    if (n != A || memcmp(w, bra, (size_t)A) != 0) return 0;
    return s;
}

/* <bra|H|ket> by the Slater-Condon rules.  bra = (pb, nb), ket = (pk, nk).
 * *absum receives the sum of |terms| (for the rounding bound of a float32
 * evaluation).  Returns 0 with *absum = 0 when the pair differs in more
 * than 4 s.p. states. */
double orc_element(const orc_problem *pr, const uint8_t *pb, const uint8_t *nb,
                   const uint8_t *pk, const uint8_t *nk, double *absum)
{
    const int Ap = pr->A[0], An = pr->A[1];
    int ap[2], cp[2], an_[2], cn[2];   /* annihilated (ket only), created (bra only) */
    int dp = orc_count_difference(pb, pk, Ap);
    int dn = orc_count_difference(nb, nk, An);
    double v = 0.0, ab = 0.0;
    *absum = 0.0;
    if (dp + dn > 4) return 0.0;
    if (dp == 0 && dn == 0) {
        /* diagonal: one-body energies + pair energies of every occupied pair */
        for (int i = 0; i < Ap; ++i) { v += pr->eps[pk[i]]; ab += absd(pr->eps[pk[i]]); }
        for (int i = 0; i < An; ++i) { v += pr->eps[nk[i]]; ab += absd(pr->eps[nk[i]]); }
        for (int i = 0; i < Ap; ++i)
            for (int j = i + 1; j < Ap; ++j) {
                double t = Vch(pr, 0, pk[i], pk[j], pk[i], pk[j]);
                v += t; ab += absd(t);
            }
        for (int i = 0; i < An; ++i)
            for (int j = i + 1; j < An; ++j) {
                double t = Vch(pr, 1, nk[i], nk[j], nk[i], nk[j]);
                v += t; ab += absd(t);
            }
        for (int i = 0; i < Ap; ++i)
            for (int j = 0; j < An; ++j) {
                double t = Vch(pr, 2, pk[i], nk[j], pk[i], nk[j]);
                v += t; ab += absd(t);
            }
        *absum = ab;
        return v;
    }
    set_minus(pk, pb, Ap, ap); set_minus(pb, pk, Ap, cp);
    set_minus(nk, nb, An, an_); set_minus(nb, nk, An, cn);
    if (dp == 2 && dn == 0) {
        /* one proton moved a -> c; spectators: the other protons, all neutrons */
        int a = ap[0], c = cp[0];
        int ops[2] = { -(a + 1), c };
        int s = phase_of(pk, pb, Ap, ops, 2);
        for (int i = 0; i < Ap; ++i) {
            if (pk[i] == a) continue;
            double t = Vch(pr, 0, c, pk[i], a, pk[i]);
            v += t; ab += absd(t);
        }
        for (int j = 0; j < An; ++j) {
            double t = Vch(pr, 2, c, nk[j], a, nk[j]);
            v += t; ab += absd(t);
        }
        *absum = ab;
        return s * v;
    }
    if (dp == 0 && dn == 2) {
        /* one neutron moved b -> d; spectators: the other neutrons, all protons */
        int b = an_[0], d = cn[0];
        int ops[2] = { -(b + 1), d };
        int s = phase_of(nk, nb, An, ops, 2);
        for (int j = 0; j < An; ++j) {
            if (nk[j] == b) continue;
            double t = Vch(pr, 1, d, nk[j], b, nk[j]);
            v += t; ab += absd(t);
        }
        for (int i = 0; i < Ap; ++i) {
            double t = Vch(pr, 2, pk[i], d, pk[i], b);
            v += t; ab += absd(t);
        }
        *absum = ab;
        return s * v;
    }
    if (dp == 4) {
        /* two protons moved (a<b) -> (c<d): term V_cdab a+_c a+_d a_b a_a */
        int a = ap[0], b = ap[1], c = cp[0], d = cp[1];
        int ops[4] = { -(a + 1), -(b + 1), d, c };
        int s = phase_of(pk, pb, Ap, ops, 4);
        double t = Vch(pr, 0, c, d, a, b);
        *absum = absd(t);
        return s * t;
    }
    if (dn == 4) {
        int a = an_[0], b = an_[1], c = cn[0], d = cn[1];
        int ops[4] = { -(a + 1), -(b + 1), d, c };
        int s = phase_of(nk, nb, An, ops, 4);
        double t = Vch(pr, 1, c, d, a, b);
        *absum = absd(t);
        return s * t;
    }
    {
        /* one proton a -> c and one neutron b -> d: term V^pn_cdab
         * a+_{c,p} a+_{d,n} a_{b,n} a_{a,p} = (a+_c a_a)_p (a+_d a_b)_n */
        int a = ap[0], c = cp[0], b = an_[0], d = cn[0];
        int opp[2] = { -(a + 1), c }, opn[2] = { -(b + 1), d };
        int s = phase_of(pk, pb, Ap, opp, 2) * phase_of(nk, nb, An, opn, 2);
        double t = Vch(pr, 2, c, d, a, b);
        *absum = absd(t);
        return s * t;
    }
}

/* ---------------------------------------------------------------------- */
/* Rows of H (Fig. 1, count and fill, Listing 2: every column of the row)       */
/* ---------------------------------------------------------------------- */

typedef struct {
    const orc_problem *pr;
    const orc_species *sp[2];
    int64_t dim;
    const int32_t *p_idx, *n_idx;
} orc_basis_view;

/* Differences of the row's species determinants against every determinant
 * of the same species; the difference count of a product state is the sum
 * of its two species' counts (bit strings of both species side by side). */
static void species_diffs(const orc_species *s, int64_t row_s, uint8_t *out)
{
    for (int64_t t = 0; t < s->n; ++t)
        out[t] = (uint8_t)orc_count_difference(s->occ + row_s * s->A,
                                               s->occ + t * s->A, s->A);
}

/* Row i: every column j (ascending) whose determinant differs from row i's
 * in at most 4 s.p. states.  Writes up to cap entries; returns the count.
 * cols/vals/absums/dtot may be NULL (count only). dtot receives the total
 * difference count of each stored pair (0, 2 or 4). */
int64_t orc_row(const orc_basis_view *B, int64_t i, int64_t cap, int64_t *cols,
                double *vals, double *absums, int8_t *dtot,
                uint8_t *scratch_p, uint8_t *scratch_n)
{
    const orc_species *P = B->sp[0], *Nn = B->sp[1];
    int32_t pi = B->p_idx[i], ni = B->n_idx[i];
    species_diffs(P, pi, scratch_p);
    species_diffs(Nn, ni, scratch_n);
    int64_t c = 0;
    for (int64_t j = 0; j < B->dim; ++j) {
        int d = scratch_p[B->p_idx[j]] + scratch_n[B->n_idx[j]];
        if (d > 4) continue;
        if (c < cap) {
            if (cols) cols[c] = j;
            if (vals) {
                double ab;
                vals[c] = orc_element(B->pr, P->occ + (int64_t)pi * P->A,
                                      Nn->occ + (int64_t)ni * Nn->A,
                                      P->occ + (int64_t)B->p_idx[j] * P->A,
                                      Nn->occ + (int64_t)B->n_idx[j] * Nn->A, &ab);
                if (absums) absums[c] = ab;
            }
            if (dtot) dtot[c] = (int8_t)d;
        }
        ++c;
    }
    return c;
}

/* Number of stored entries of rows i0 <= i < i1 (Fig. 1, count step) into
 * counts[i - i0].  Rows that share a proton determinant reuse its
 * difference list (same result as recomputing it per row). */
void orc_row_counts_range(const orc_basis_view *B, int64_t i0, int64_t i1, int64_t *counts)
{
    const orc_species *P = B->sp[0], *Nn = B->sp[1];
    #pragma omp parallel
    {
        uint8_t *dp = (uint8_t *)malloc((size_t)(P->n ? P->n : 1));
        uint8_t *dn = (uint8_t *)malloc((size_t)(Nn->n ? Nn->n : 1));
        int64_t last_p = -1;
        #pragma omp for schedule(dynamic, 64)
        for (int64_t i = i0; i < i1; ++i) {
            if (B->p_idx[i] != last_p) { species_diffs(P, B->p_idx[i], dp); last_p = B->p_idx[i]; }
            species_diffs(Nn, B->n_idx[i], dn);
            int64_t c = 0;
            for (int64_t j = 0; j < B->dim; ++j)
                if (dp[B->p_idx[j]] + dn[B->n_idx[j]] <= 4) ++c;
            counts[i - i0] = c;
        }
        free(dp); free(dn);
    }
}

/* Number of stored entries of every row. */
void orc_row_counts(const orc_basis_view *B, int64_t *counts)
{
    orc_row_counts_range(B, 0, B->dim, counts);
}

/* Fill rows i0 <= i < i1 of a CSR whose offsets the caller has made from
 * orc_row_counts_range and the scan (Fig. 1, fill step): row i goes to
 * positions [row_ptr[i - i0], row_ptr[i - i0 + 1]).  absums may be NULL. */
void orc_fill_range(const orc_basis_view *B, int64_t i0, int64_t i1, const int64_t *row_ptr,
                    int64_t *cols, double *vals, double *absums)
{
    const orc_species *P = B->sp[0], *Nn = B->sp[1];
    #pragma omp parallel
    {
        uint8_t *dp = (uint8_t *)malloc((size_t)(P->n ? P->n : 1));
        uint8_t *dn = (uint8_t *)malloc((size_t)(Nn->n ? Nn->n : 1));
        #pragma omp for schedule(dynamic, 64)
        for (int64_t i = i0; i < i1; ++i) {
            int64_t o = row_ptr[i - i0];
            orc_row(B, i, row_ptr[i - i0 + 1] - o, cols + o, vals + o,
                    absums ? absums + o : NULL, NULL, dp, dn);
        }
        free(dp); free(dn);
    }
}

/* Fill the whole CSR. */
void orc_fill(const orc_basis_view *B, const int64_t *row_ptr, int64_t *cols,
              double *vals, double *absums)
{
    orc_fill_range(B, 0, B->dim, row_ptr, cols, vals, absums);
}

/* Threads of the OpenMP loops above (n <= 0: leave the default); returns
 * the number the next parallel region will use. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Y = H X in FP64 over a CSR (Fig. 2, optional FMA: H_ij with the j-th
 * vector element), X and Y row-major [dim][nvec]. */
void orc_spmm(int64_t dim, const int64_t *row_ptr, const int64_t *cols,
              const double *vals, const double *X, double *Y, int nvec)
{
    for (int64_t i = 0; i < dim; ++i) {
        for (int v = 0; v < nvec; ++v) Y[i * nvec + v] = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            for (int v = 0; v < nvec; ++v)
                Y[i * nvec + v] += vals[e] * X[cols[e] * nvec + v];
    }
}

/* Exclusive prefix sum with the total in the last slot (Eq. 1):
 * y[0] = 0, y[i+1] = y[i] + x[i], for i = 0..n-1. */
void orc_exclusive_scan(const int64_t *x, int64_t n, int64_t *y)
{
    y[0] = 0;
    for (int64_t i = 0; i < n; ++i) y[i + 1] = y[i] + x[i];
}

/* Count benchmark (Sec. 2.1, Listing 2).  mbs holds n states of N
 * particles, each the ascending list of its occupied s.p. states.  For each
 * of the nrows states rows[r], out[r] = the number of states j (all n,
 * j = rows[r] included) whose occupations differ from it in at most
 * max_diff s.p. states, both sides counted (Sec. 2.1).  The difference of
 * two states is found by walking both sorted lists, as in Listing 1. */
static int diff_u16(const uint16_t *a, const uint16_t *b, int N)
{
    int i = 0, j = 0, d = 0;
    while (i < N && j < N) {
        if (a[i] < b[j]) { ++d; ++i; }
        else if (a[i] > b[j]) { ++d; ++j; }
        else { ++i; ++j; }
    }
    return d + (N - i) + (N - j);
}

void orc_count_pairs(const uint16_t *mbs, int64_t n, int N, int max_diff, const int64_t *rows, int64_t nrows,
                     int64_t *out)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrows; ++r) {
        const uint16_t *a = mbs + rows[r] * N;
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j)
            if (diff_u16(a, mbs + j * N, N) <= max_diff) ++c;
        out[r] = c;
    }
}
