// mr3_adjoint.cu -- the eigenvector part of the backward pass one eigenvector at a time,
// in O(n) work per eigenpair.
//
// For a simple eigenvalue, dz_k = -(T - lambda_k I)^+ dT z_k, so the eigenvector part of
// Tbar is  -sum_k w_k z_k^T  with  w_k = (T - lambda_k I)^+ G_k  (G_k = dL/dz_k), the same
// matrix as the dense Z (F o (Z^T G)) Z^T of mr3_backward.  w_k solves (T - lambda_k I) x = b
// with b = G_k projected off z_k, by tridiagonal Gaussian elimination with partial pivoting
// (backward stable; the one-sided pivots of a twisted factorization grow too large for a
// general right-hand side when lambda_k is interior), and x is projected off z_k: the
// near-singular direction carries only rounding.  The solve amplifies rounding errors by
// ||T|| / gap, so eigenvalues closer than kTight ||T|| to each other form a group that is
// projected out of b and x together, and the pairs inside a group get the dense formula
// z_i F_ik (z_i^T G_k), F_ik = D / (D^2 + delta^2), D = lambda_k - lambda_i (the
// regularisation of mr3_backward).  Eigenvalues outside the computed range are not seen:
// with a subset, the result is the gradient of a loss of the computed eigenpairs as long as
// no other eigenvalue lies within kTight ||T|| of a computed one.
#include "mr3_kernels.h"

namespace mr3 {
namespace {

constexpr double kTight = 1e-6;  // group threshold, relative to ||T||
constexpr int kMaxGroup = 64;    // longest group projected and treated densely
constexpr int kWarps = 4;        // warps per block (one eigenpair each)

// One warp per eigenpair c.  Scratch: the three diagonals of U (3 n doubles per
// eigenpair).  Y column c receives -w_c plus the dense in-group terms (Y Z^T is the
// eigenvector part of Tbar).
__global__ void __launch_bounds__(32 * kWarps) k_adjoint(
    int n, int k, const double *__restrict__ d, const double *__restrict__ e,
    const double *__restrict__ w, const double *__restrict__ Z, int ldz,
    const double *__restrict__ G, int ldg, double tnorm, double *scratch, double *Y) {
    __shared__ double s_s[kWarps][kMaxGroup], t_s[kWarps][kMaxGroup];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kWarps + wib;
    if (c >= k) return; // whole warps only
    const double lam = w[c];
    const double thr = kTight * tnorm;
    const double delta = n * kEps * tnorm;
    // the tight group [g0, g1] around c (at most kMaxGroup members)
    int g0 = c, g1 = c;
    while (g0 > 0 && c - g0 + 1 < kMaxGroup / 2 && w[g0] - w[g0 - 1] < thr) --g0;
    while (g1 < k - 1 && g1 - g0 + 1 < kMaxGroup && w[g1 + 1] - w[g1] < thr) ++g1;
    const int m = g1 - g0 + 1;
    const double *gc = G + (size_t)c * ldg;
    double *y = Y + (size_t)c * n;
    // s_j = z_j^T G_c for the group; b = G_c - sum_j s_j z_j
    for (int q = 0; q < m; ++q) {
        const double *zq = Z + (size_t)(g0 + q) * ldz;
        double a = 0.0;
        for (int i = lane; i < n; i += 32) a = fma(zq[i], gc[i], a);
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s_s[wib][q] = a;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        double b = gc[i];
        for (int q = 0; q < m; ++q) b = fma(-s_s[wib][q], Z[(size_t)(g0 + q) * ldz + i], b);
        y[i] = b;
    }
    // x = (T - lam I)^{-1} b by Gaussian elimination with partial pivoting (row i or row
    // i+1 as the pivot of column i), the forward substitution done alongside: U is upper
    // triangular with two superdiagonals (U0, U1, U2 in scratch), y overwrites b, then back
    // substitution.  A pivot below pm = eps ||T|| in magnitude (the matrix is singular up to
    // rounding at an eigenvalue) is replaced by pm with its sign: the null direction then
    // carries |z^T b| / pm ~ ||b|| / ||T||, which the projection removes, instead of an
    // amplitude that would swamp the solution.
    const double pm = kEps * tnorm;
    double *U0 = scratch + (size_t)c * 3 * n, *U1 = U0 + n, *U2 = U1 + n;
    if (lane == 0) {
        double u0 = d[0] - lam, u1 = (n > 1) ? e[0] : 0.0, u2 = 0.0; // current row, cols i..i+2
        double beta = y[0];                                          // its right-hand side
        for (int i = 0; i < n - 1; ++i) {
            const double s = e[i], t = d[i + 1] - lam, v = (i + 2 < n) ? e[i + 1] : 0.0;
            const double bn = y[i + 1];
            if (fabs(u0) >= fabs(s)) {
                if (fabs(u0) < pm) u0 = u0 < 0.0 ? -pm : pm;
                const double mlt = s / u0;
                U0[i] = u0; U1[i] = u1; U2[i] = u2;
                y[i] = beta;
                beta = fma(-mlt, beta, bn);
                u0 = fma(-mlt, u1, t);
                u1 = fma(-mlt, u2, v);
            } else {
                const double mlt = u0 / s;
                U0[i] = s; U1[i] = t; U2[i] = v;
                y[i] = bn;
                beta = fma(-mlt, bn, beta);
                const double nu0 = fma(-mlt, t, u1);
                u1 = fma(-mlt, v, u2);
                u0 = nu0;
            }
            u2 = 0.0;
        }
        if (fabs(u0) < pm) u0 = u0 < 0.0 ? -pm : pm;
        U0[n - 1] = u0;
        U1[n - 1] = 0.0;
        U2[n - 1] = 0.0;
        y[n - 1] = beta;
        double x1 = 0.0, x2 = 0.0; // x_{i+1}, x_{i+2}
        for (int i = n - 1; i >= 0; --i) {
            const double x = (y[i] - U1[i] * x1 - U2[i] * x2) / U0[i];
            y[i] = x;
            x2 = x1;
            x1 = x;
        }
    }
    __syncwarp();
    // x projected off the group: t_j = z_j^T x
    for (int q = 0; q < m; ++q) {
        const double *zq = Z + (size_t)(g0 + q) * ldz;
        double a = 0.0;
        for (int i = lane; i < n; i += 32) a = fma(zq[i], y[i], a);
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) t_s[wib][q] = a;
    }
    __syncwarp();
    // Y_c = -(x - sum_j t_j z_j) + sum_{j in group, j != c} z_j F_jc s_j
    for (int i = lane; i < n; i += 32) {
        double v = -y[i];
        for (int q = 0; q < m; ++q) {
            const int j = g0 + q;
            double f = t_s[wib][q];
            if (j != c) {
                const double D = lam - w[j];
                f += (D / fma(D, D, delta * delta)) * s_s[wib][q];
            }
            v = fma(f, Z[(size_t)j * ldz + i], v);
        }
        y[i] = v;
    }
}

} // namespace

void launch_adjoint(int n, int k, const double *d, const double *e, const double *w,
                    const double *Z, int ldz, const double *G, int ldg, double tnorm,
                    double *scratch, double *Y, cudaStream_t s) {
    if (n <= 0 || k <= 0) return;
    k_adjoint<<<(k + kWarps - 1) / kWarps, 32 * kWarps, 0, s>>>(n, k, d, e, w, Z, ldz, G, ldg,
                                                                tnorm, scratch, Y);
}

} // namespace mr3
