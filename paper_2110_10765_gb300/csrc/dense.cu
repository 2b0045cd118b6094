// Host symmetric eigensolver: Householder tridiagonalisation + implicit
// symmetric QR with Wilkinson shift (Golub & Van Loan, Sec. 8.3).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "dense.h"

namespace ci {

namespace {

// Rotation coefficients with [c s; -s c]^T [x; z] = [r; 0].
void givens(double x, double z, double &c, double &s) {
    if (z == 0.0) { c = 1.0; s = 0.0; return; }
    double r = std::hypot(x, z);
    c = x / r;
    s = -z / r;
}

// T is tridiagonal: a[i] = T(i,i), b[i] = T(i+1,i).  One implicit QR step
// with Wilkinson shift on the unreduced block l..h, chasing the bulge with
// rotations in planes (k, k+1); each rotation G is applied as T <- G^T T G
// on a 4 x 4 window and Z <- Z G.
void qr_step(int n, std::vector<double> &a, std::vector<double> &b, int l, int h, std::vector<double> &Z) {
    double d = 0.5 * (a[h - 1] - a[h]);
    double bb = b[h - 1];
    double den = d + (d >= 0 ? 1.0 : -1.0) * std::hypot(d, bb);
    double mu = a[h] - (den != 0.0 ? bb * bb / den : 0.0);
    double x = a[l] - mu, z = b[l];
    double bulge = 0.0;
    for (int k = l; k < h; ++k) {
        double c, s;
        if (k > l) { x = b[k - 1]; z = bulge; }
        givens(x, z, c, s);
        // window rows/cols k-1 .. k+2 (local 0..3), clipped to l..h
        double M[4][4] = {{0}};
        int g0 = k - 1;
        auto in = [&](int g) { return g >= l && g <= h; };
        for (int i = 0; i < 4; ++i) {
            int gi = g0 + i;
            if (!in(gi)) continue;
            M[i][i] = a[gi];
            if (i + 1 < 4 && in(gi + 1)) M[i + 1][i] = M[i][i + 1] = b[gi];
        }
        if (k > l) M[2][0] = M[0][2] = bulge;
        // M <- G^T M G on local indices 1, 2
        for (int j = 0; j < 4; ++j) {  // rows: G^T M
            double r1 = M[1][j], r2 = M[2][j];
            M[1][j] = c * r1 - s * r2;
            M[2][j] = s * r1 + c * r2;
        }
        for (int i = 0; i < 4; ++i) {  // cols: (G^T M) G
            double c1 = M[i][1], c2 = M[i][2];
            M[i][1] = c * c1 - s * c2;
            M[i][2] = s * c1 + c * c2;
        }
        for (int i = 0; i < 4; ++i) {
            int gi = g0 + i;
            if (!in(gi)) continue;
            a[gi] = M[i][i];
            if (i + 1 < 4 && in(gi + 1)) b[gi] = M[i + 1][i];
        }
        bulge = (k + 2 <= h) ? M[3][1] : 0.0;  // new entry (k+2, k)
        for (int r = 0; r < n; ++r) {
            double z1 = Z[(size_t)r * n + k], z2 = Z[(size_t)r * n + k + 1];
            Z[(size_t)r * n + k] = c * z1 - s * z2;
            Z[(size_t)r * n + k + 1] = s * z1 + c * z2;
        }
    }
}

}  // namespace

bool sym_eig(int n, const std::vector<double> &A0, std::vector<double> &w, std::vector<double> &Zout) {
    w.assign(n, 0.0);
    Zout.assign((size_t)n * n, 0.0);
    if (n == 0) return true;
    std::vector<double> A(A0.begin(), A0.begin() + (size_t)n * n);
    std::vector<double> Z((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
    std::vector<double> v(n), p(n), wv(n);
    // Householder reduction: zero A[k+2.., k] with H = I - 2 v v^T on k+1..
    for (int k = 0; k + 2 < n; ++k) {
        int m = n - k - 1;
        double nx = 0.0;
        for (int i = 0; i < m; ++i) nx += A[(size_t)(k + 1 + i) * n + k] * A[(size_t)(k + 1 + i) * n + k];
        nx = std::sqrt(nx);
        if (nx == 0.0) continue;
        double x0 = A[(size_t)(k + 1) * n + k];
        double alpha = x0 > 0 ? -nx : nx;
        for (int i = 0; i < m; ++i) v[i] = A[(size_t)(k + 1 + i) * n + k];
        v[0] -= alpha;
        double nv = 0.0;
        for (int i = 0; i < m; ++i) nv += v[i] * v[i];
        nv = std::sqrt(nv);
        if (nv == 0.0) continue;
        for (int i = 0; i < m; ++i) v[i] /= nv;
        // p = A22 v, K = v.p, w = 2p - 2K v, A22 -= v w^T + w v^T
        double K = 0.0;
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            const double *row = &A[(size_t)(k + 1 + i) * n + k + 1];
            for (int j = 0; j < m; ++j) s += row[j] * v[j];
            p[i] = s;
            K += v[i] * s;
        }
        for (int i = 0; i < m; ++i) wv[i] = 2.0 * p[i] - 2.0 * K * v[i];
        for (int i = 0; i < m; ++i) {
            double *row = &A[(size_t)(k + 1 + i) * n + k + 1];
            for (int j = 0; j < m; ++j) row[j] -= v[i] * wv[j] + wv[i] * v[j];
        }
        A[(size_t)(k + 1) * n + k] = A[(size_t)k * n + k + 1] = alpha;
        for (int i = 1; i < m; ++i) A[(size_t)(k + 1 + i) * n + k] = A[(size_t)k * n + k + 1 + i] = 0.0;
        // Z <- Z H on columns k+1..
        for (int r = 0; r < n; ++r) {
            double *zr = &Z[(size_t)r * n + k + 1];
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += zr[j] * v[j];
            for (int j = 0; j < m; ++j) zr[j] -= 2.0 * s * v[j];
        }
    }
    std::vector<double> a(n), b(n > 1 ? n - 1 : 1, 0.0);
    for (int i = 0; i < n; ++i) a[i] = A[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) b[i] = A[(size_t)(i + 1) * n + i];
    const double eps = 2.220446049250313e-16;
    int h = n - 1, iter = 0;
    bool ok = true;
    while (h > 0) {
        for (int i = 0; i < h; ++i)
            if (std::fabs(b[i]) <= eps * (std::fabs(a[i]) + std::fabs(a[i + 1]))) b[i] = 0.0;
        if (b[h - 1] == 0.0) { --h; continue; }
        int l = h - 1;
        while (l > 0 && b[l - 1] != 0.0) --l;
        qr_step(n, a, b, l, h, Z);
        if (++iter > 60 * n) { ok = false; break; }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return a[x] < a[y]; });
    for (int i = 0; i < n; ++i) {
        w[i] = a[idx[i]];
        for (int r = 0; r < n; ++r) Zout[(size_t)r * n + i] = Z[(size_t)r * n + idx[i]];
    }
    return ok;
}

}  // namespace ci
