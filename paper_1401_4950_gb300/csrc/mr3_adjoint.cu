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
//
// Three launches.  The projections are inner products over n, one warp per eigenpair
// (k_adjoint_rhs, k_adjoint_fin); the elimination and back substitution are serial
// recurrences over n, one lane per eigenpair (k_adjoint_solve): a binary64 warp
// instruction costs the same whatever the number of active lanes, so 32 chains share each.
#include "mr3_kernels.h"

namespace mr3 {
namespace {

#define FULL_MASK 0xffffffffu

constexpr double kTight = 1e-6;  // group threshold, relative to ||T||
constexpr int kMaxGroup = 64;    // longest group projected and treated densely
constexpr int kWarps = 4;        // warps per block in the warp-per-eigenpair launches

// The tight group [g0, g0 + m) around eigenpair c (at most kMaxGroup members).
__device__ __forceinline__ void tight_group(int c, int k, const double *__restrict__ w, double thr,
                                            int &g0, int &m) {
    int a = c, b = c;
    while (a > 0 && c - a + 1 < kMaxGroup / 2 && w[a] - w[a - 1] < thr) --a;
    while (b < k - 1 && b - a + 1 < kMaxGroup && w[b + 1] - w[b] < thr) ++b;
    g0 = a;
    m = b - a + 1;
}

// One warp per eigenpair c: s_j = z_j^T G_c for the group (kept in S[c kMaxGroup + q]) and
// the right-hand side b = G_c - sum_j s_j z_j in Y column c.
__global__ void __launch_bounds__(32 * kWarps) k_adjoint_rhs(
    int n, int k, const double *__restrict__ w, const double *__restrict__ Z, int ldz,
    const double *__restrict__ G, int ldg, double thr, double *S, double *Y) {
    __shared__ double s_s[kWarps][kMaxGroup];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kWarps + wib;
    if (c >= k) return; // whole warps only
    int g0, m;
    tight_group(c, k, w, thr, g0, m);
    const double *gc = G + (size_t)c * ldg;
    double *y = Y + (size_t)c * n;
    for (int q = 0; q < m; ++q) {
        const double *zq = Z + (size_t)(g0 + q) * ldz;
        double a = 0.0;
        for (int i = lane; i < n; i += 32) a = fma(zq[i], gc[i], a);
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(FULL_MASK, a, o);
        if (lane == 0) {
            s_s[wib][q] = a;
            S[(size_t)c * kMaxGroup + q] = a;
        }
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        double b = gc[i];
        for (int q = 0; q < m; ++q) b = fma(-s_s[wib][q], Z[(size_t)(g0 + q) * ldz + i], b);
        y[i] = b;
    }
}

// One lane per eigenpair c: x = (T - lambda_c I)^{-1} b in place in Y column c, by Gaussian
// elimination with partial pivoting (row i or row i+1 as the pivot of column i) with the
// forward substitution done alongside, then back substitution.  U is upper triangular with
// two superdiagonals, stored interleaved by lane (U0, U1, U2 of index i for the 32
// eigenpairs of a warp are adjacent).  A pivot below pm = eps ||T|| in magnitude (the
// matrix is singular up to rounding at an eigenvalue) is replaced by pm with its sign: the
// null direction then carries |z^T b| / pm ~ ||b|| / ||T||, which the projection removes,
// instead of an amplitude that would swamp the solution.  The pivot choice is a select, not
// a branch, so the lanes of a warp stay together; the operands of step i + 1 are loaded
// during step i.
__global__ void __launch_bounds__(128) k_adjoint_solve(int n, int k, const double *__restrict__ d,
                                                       const double *__restrict__ e,
                                                       const double *__restrict__ w, double pm,
                                                       double *scratch, double *Y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    const long long kpad = ((long long)k + 31) / 32 * 32;
    const int gw = c >> 5, l = c & 31;
    double *U0 = scratch + (size_t)gw * n * 32 + l;
    double *U1 = U0 + (size_t)kpad * n, *U2 = U1 + (size_t)kpad * n;
    double *y = Y + (size_t)c * n;
    const double lam = w[c];
    double u0 = d[0] - lam, u1 = (n > 1) ? e[0] : 0.0; // current row, columns i, i+1 (i+2 is 0)
    double beta = y[0];                                // its right-hand side
    // operands of step i: e_i, d_{i+1} - lam, e_{i+1}, b_{i+1}
    double sn = 0.0, tn = 0.0, vn = 0.0, bn = 0.0;
    if (n > 1) {
        sn = e[0];
        tn = d[1] - lam;
        vn = (n > 2) ? e[1] : 0.0;
        bn = y[1];
    }
    for (int i = 0; i < n - 1; ++i) {
        const double s = sn, t = tn, v = vn, b = bn;
        if (i + 1 < n - 1) {
            sn = e[i + 1];
            tn = d[i + 2] - lam;
            vn = (i + 3 < n) ? e[i + 2] : 0.0;
            bn = y[i + 2];
        }
        const bool piv = fabs(u0) >= fabs(s);
        const double u0f = (piv && fabs(u0) < pm) ? (u0 < 0.0 ? -pm : pm) : u0;
        const double mlt = (piv ? s : u0) / (piv ? u0f : s);
        const double o0 = piv ? u0f : s, o1 = piv ? u1 : t, o2 = piv ? 0.0 : v;
        const double oy = piv ? beta : b;
        U0[(size_t)i * 32] = o0;
        U1[(size_t)i * 32] = o1;
        U2[(size_t)i * 32] = o2;
        y[i] = oy;
        beta = fma(-mlt, oy, piv ? b : beta);
        const double nu0 = fma(-mlt, o1, piv ? t : u1);
        u1 = fma(-mlt, o2, piv ? v : 0.0);
        u0 = nu0;
    }
    if (fabs(u0) < pm) u0 = u0 < 0.0 ? -pm : pm;
    U0[(size_t)(n - 1) * 32] = u0;
    U1[(size_t)(n - 1) * 32] = 0.0;
    U2[(size_t)(n - 1) * 32] = 0.0;
    y[n - 1] = beta;
    // back substitution (the reciprocal of the next pivot is formed off the chain)
    double x1 = 0.0, x2 = 0.0; // x_{i+1}, x_{i+2}
    double yn = y[n - 1], an = U1[(size_t)(n - 1) * 32], cn = U2[(size_t)(n - 1) * 32];
    double rn = 1.0 / U0[(size_t)(n - 1) * 32];
    for (int i = n - 1; i >= 0; --i) {
        const double yy = yn, aa = an, cc = cn, rr = rn;
        if (i > 0) {
            yn = y[i - 1];
            an = U1[(size_t)(i - 1) * 32];
            cn = U2[(size_t)(i - 1) * 32];
            rn = 1.0 / U0[(size_t)(i - 1) * 32];
        }
        const double x = (yy - aa * x1 - cc * x2) * rr;
        y[i] = x;
        x2 = x1;
        x1 = x;
    }
}

// One warp per eigenpair c: x projected off the group (t_j = z_j^T x) and the column
// Y_c = -(x - sum_j t_j z_j) + sum_{j in group, j != c} z_j F_jc s_j  (Y Z^T is the
// eigenvector part of Tbar).
__global__ void __launch_bounds__(32 * kWarps) k_adjoint_fin(
    int n, int k, const double *__restrict__ w, const double *__restrict__ Z, int ldz,
    double thr, double delta, const double *__restrict__ S, double *Y) {
    __shared__ double t_s[kWarps][kMaxGroup];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kWarps + wib;
    if (c >= k) return; // whole warps only
    int g0, m;
    tight_group(c, k, w, thr, g0, m);
    const double lam = w[c];
    double *y = Y + (size_t)c * n;
    for (int q = 0; q < m; ++q) {
        const double *zq = Z + (size_t)(g0 + q) * ldz;
        double a = 0.0;
        for (int i = lane; i < n; i += 32) a = fma(zq[i], y[i], a);
        for (int o = 16; o; o >>= 1) a += __shfl_xor_sync(FULL_MASK, a, o);
        if (lane == 0) t_s[wib][q] = a;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        double v = -y[i];
        for (int q = 0; q < m; ++q) {
            const int j = g0 + q;
            double f = t_s[wib][q];
            if (j != c) {
                const double D = lam - w[j];
                f += (D / fma(D, D, delta * delta)) * S[(size_t)c * kMaxGroup + q];
            }
            v = fma(f, Z[(size_t)j * ldz + i], v);
        }
        y[i] = v;
    }
}

} // namespace

size_t adjoint_scratch_doubles(int n, int k) {
    const size_t kpad = ((size_t)std::max(k, 0) + 31) / 32 * 32;
    return 3 * kpad * (size_t)std::max(n, 1) + (size_t)kMaxGroup * std::max(k, 1);
}

void launch_adjoint(int n, int k, const double *d, const double *e, const double *w,
                    const double *Z, int ldz, const double *G, int ldg, double tnorm,
                    double *scratch, double *Y, cudaStream_t s) {
    if (n <= 0 || k <= 0) return;
    const double thr = kTight * tnorm, delta = n * kEps * tnorm, pm = kEps * tnorm;
    const size_t kpad = ((size_t)k + 31) / 32 * 32;
    double *S = scratch + 3 * kpad * (size_t)n;
    const unsigned wblocks = (unsigned)((k + kWarps - 1) / kWarps);
    k_adjoint_rhs<<<wblocks, 32 * kWarps, 0, s>>>(n, k, w, Z, ldz, G, ldg, thr, S, Y);
    // small launches in 32-thread blocks, so that the warps spread over the SMs
    const int bs = k >= 152 * 128 ? 128 : 32;
    k_adjoint_solve<<<(unsigned)((k + bs - 1) / bs), bs, 0, s>>>(n, k, d, e, w, pm, scratch, Y);
    k_adjoint_fin<<<wblocks, 32 * kWarps, 0, s>>>(n, k, w, Z, ldz, thr, delta, S, Y);
}

} // namespace mr3
