// mr3_backward.cu -- gradient of a scalar loss L(lambda, Z) of the eigenpairs of the
// tridiagonal T = tridiag(e, d, e) with respect to d and e.
//
// The thesis has no backward pass; the formulas are the first-order perturbation theory
// of a symmetric eigen-decomposition T = Z diag(lambda) Z^T:
//   d lambda_i = z_i^T dT z_i,   dz_i = sum_{k != i} z_k (z_k^T dT z_i) / (lambda_i - lambda_k),
// which give  Tbar = Z (diag(g) + F o (Z^T G)) Z^T,  F_ik = 1/(lambda_k - lambda_i), F_ii = 0,
// and, because d_j sits at (j, j) and e_j at (j, j+1) and (j+1, j):
//   dbar_j = Tbar_jj,   ebar_j = Tbar_{j,j+1} + Tbar_{j+1,j}.
// The eigenvalue part reduces to dbar_j = sum_i g_i z_ji^2, ebar_j = 2 sum_i g_i z_ji z_{j+1,i}.
// Pairs closer than the solver resolves are regularised: F_ik = D/(D^2 + delta^2),
// D = lambda_k - lambda_i, delta = n eps ||T||.
#include <algorithm>
#include <cstring>
#include "mr3.h"
#include "mr3_internal.cuh"

namespace mr3 {
namespace {

// dbar_j = sum_i g_i z_ji^2 ; ebar_j = 2 sum_i g_i z_ji z_{j+1,i}  (one thread per row j,
// columns visited in order so that a warp reads 32 consecutive rows of a column).
__global__ void k_bwd_eigvals(int n, int k, const double *__restrict__ Z, int ldz,
                              const double *__restrict__ gw, double *dd, double *de) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sd = 0.0, se = 0.0;
    if (gw) {
        for (int i = 0; i < k; ++i) {
            const double g = __ldg(gw + i);
            const double a = __ldg(Z + (size_t)i * ldz + j);
            sd = fma(g * a, a, sd);
            if (j < n - 1) se = fma(g * a, __ldg(Z + (size_t)i * ldz + j + 1), se);
        }
    }
    dd[j] = sd;
    if (j < n - 1) de[j] = 2.0 * se;
}

// C (m x n, column-major, ldc) = op(A) * B with op(A) = A^T (transA) or A; A, B
// column-major.  64 x 64 tile per CTA, 256 threads with a 4 x 4 register tile each,
// k in steps of 16 through shared memory.
template <bool TRANS_A>
__global__ void __launch_bounds__(256) k_gemm_f64(int m, int n, int kdim, const double *__restrict__ A,
                                                  int lda, const double *__restrict__ B, int ldb,
                                                  double *C, int ldc) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.x * 64, col0 = blockIdx.y * 64;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < kdim; k0 += 16) {
        // load A tile: rows row0..row0+63 of op(A), k0..k0+15
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int kk = t / 64, r = t % 64;
            const int gr = row0 + r, gk = k0 + kk;
            double v = 0.0;
            if (gr < m && gk < kdim) v = TRANS_A ? A[(size_t)gr * lda + gk] : A[(size_t)gk * lda + gr];
            As[kk][r] = v;
        }
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int c = t / 16, kk = t % 16;
            const int gc = col0 + c, gk = k0 + kk;
            double v = 0.0;
            if (gc < n && gk < kdim) v = B[(size_t)gc * ldb + gk];
            Bs[kk][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty * 4 + q]; b[q] = Bs[kk][tx * 4 + q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gr = row0 + ty * 4 + x, gc = col0 + tx * 4 + y;
            if (gr < m && gc < n) C[(size_t)gc * ldc + gr] = acc[x][y];
        }
}

// B_ik = F_ik C_ik in place (C column-major n x n).
__global__ void k_apply_F(int n, const double *__restrict__ w, double delta, double *C) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int kcol = (int)(idx / n), i = (int)(idx % n);
    if (i == kcol) { C[idx] = 0.0; return; }
    const double D = w[kcol] - w[i];
    C[idx] = C[idx] * (D / (D * D + delta * delta));
}

// dbar_j += sum_b Y_jb Z_jb ; ebar_j += sum_b (Y_jb Z_{j+1,b} + Y_{j+1,b} Z_jb).
__global__ void k_bwd_vec_reduce(int n, const double *__restrict__ Y, const double *__restrict__ Z,
                                 int ldz, double *dd, double *de) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double sd = 0.0, se = 0.0;
    for (int b = 0; b < n; ++b) {
        const double y = Y[(size_t)b * n + j], z = Z[(size_t)b * ldz + j];
        sd = fma(y, z, sd);
        if (j < n - 1) {
            const double y1 = Y[(size_t)b * n + j + 1], z1 = Z[(size_t)b * ldz + j + 1];
            se = fma(y, z1, fma(y1, z, se));
        }
    }
    dd[j] += sd;
    if (j < n - 1) de[j] += se;
}

} // namespace
} // namespace mr3

using namespace mr3;

extern "C" int mr3_backward(int n, int k, const double *w, const double *Z, int ldz,
                            const double *gw, const double *gZ, int ldgz, double *dd, double *de,
                            const mr3_opts *opts, void *stream) {
    (void)opts;
    if (n < 0) return -1;
    if (k < 0 || k > n || (gZ && k != n)) return -2;
    if (k > 0 && !w) return -3;
    if (k > 0 && !Z) return -4;
    if (ldz < std::max(1, n)) return -5;
    if (gZ && ldgz < std::max(1, n)) return -8;
    if (n > 0 && !dd) return -9;
    if (n > 1 && !de) return -10;
    if (n == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    k_bwd_eigvals<<<(n + 127) / 128, 128, 0, s>>>(n, k, Z, ldz, gw, dd, de);
    if (gZ && n > 1) {
        double *C = nullptr, *Y = nullptr;
        if (cudaMallocAsync((void **)&C, sizeof(double) * (size_t)n * n, s) != cudaSuccess ||
            cudaMallocAsync((void **)&Y, sizeof(double) * (size_t)n * n, s) != cudaSuccess) {
            cudaGetLastError();
            if (C) cudaFreeAsync(C, s);
            return MR3_EOOM;
        }
        // ||T|| from the eigenvalues (ascending): max(|lambda_1|, |lambda_n|)
        double w0, wn;
        cudaMemcpyAsync(&w0, w, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&wn, w + n - 1, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        const double tnorm = std::max(std::fabs(w0), std::fabs(wn));
        const double delta = n * kEps * (tnorm > 0 ? tnorm : 1.0);
        dim3 g((n + 63) / 64, (n + 63) / 64);
        k_gemm_f64<true><<<g, 256, 0, s>>>(n, n, n, Z, ldz, gZ, ldgz, C, n);
        k_apply_F<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(n, w, delta, C);
        k_gemm_f64<false><<<g, 256, 0, s>>>(n, n, n, Z, ldz, C, n, Y, n);
        k_bwd_vec_reduce<<<(n + 127) / 128, 128, 0, s>>>(n, Y, Z, ldz, dd, de);
        cudaFreeAsync(C, s);
        cudaFreeAsync(Y, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return MR3_ECUDA; }
    return 0;
}
