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
//
// The two n x n x n products (C = Z^T G and Y = Z (F o C)) are the whole cost.  GB300 runs
// binary64 at about 1.2 TFLOP/s, so for n >= kOzakiMinN they are computed as exact sums of
// bf16 tensor-core products (the error-free splitting of Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59 (2012)): every row of the left factor and every column of the
// right one is scaled by a power of two into (-1, 1) and cut into s slices of beta bits,
// each an integer held exactly in bf16; a slice-by-slice product summed over a chunk of at
// most 2^(24 - 2 beta) terms is an integer below 2^24 and comes out of an FP32-accumulating
// GEMM exactly; the slice products whose weight 2^(-beta (p + q)) is below 2^(-beta (s+1))
// are dropped (their sum is below 2^-54 of the scale), and the rest is summed in binary64.
// The slice GEMMs are plain cuBLAS bf16 GEMMs.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <cublas_v2.h>
#include <cuda_bf16.h>
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

// ---- Ozaki splitting

constexpr int kOzakiMinN = 256;   // below this the binary64 tile GEMM is as fast
constexpr int kOzakiChunk = 4096; // longest contraction summed inside one GEMM

struct OzakiPlan {
    int beta;  // bits per slice
    int s;     // slices per operand
    int chunk; // contraction length per GEMM
};

OzakiPlan ozaki_plan(int K) {
    OzakiPlan p;
    p.chunk = std::min(K, kOzakiChunk);
    int lg = 0;
    while ((1 << lg) < p.chunk) ++lg;
    // |slice 1| <= 2^beta, |slice p>1| <= 2^(beta-1): a chunk sum is at most 2^(2 beta + lg)
    p.beta = std::min(8, (24 - lg) / 2); // bf16 holds integers up to 2^8 exactly
    p.s = (54 + p.beta - 1) / p.beta;
    return p;
}

// Scale exponents: ex[r] = the least e with max_c |X(r, c)| < 2^e (0 for a zero line).
// by_row: r indexes rows (max over columns); else r indexes columns (max over rows).
__global__ void k_line_exponent(int n, const double *__restrict__ X, int ldx, bool by_row,
                                int *ex) {
    if (by_row) {
        const int r = blockIdx.x * blockDim.x + threadIdx.x;
        if (r >= n) return;
        double m = 0.0;
        for (int c = 0; c < n; ++c) m = fmax(m, fabs(X[(size_t)c * ldx + r]));
        ex[r] = m > 0.0 ? ilogb(m) + 1 : 0;
    } else {
        // one warp per column
        const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int lane = threadIdx.x & 31;
        if (c >= n) return;
        double m = 0.0;
        for (int r = lane; r < n; r += 32) m = fmax(m, fabs(X[(size_t)c * ldx + r]));
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) ex[c] = m > 0.0 ? ilogb(m) + 1 : 0;
    }
}

// Slices of X (n x n, column-major): x 2^-e = sum_p a_p 2^(-beta (p+1)) + rest, a_p integers,
// written as bf16 planes S[p] (column-major, leading dimension n).  e per row or column.
__global__ void k_slice(int n, const double *__restrict__ X, int ldx, const int *__restrict__ ex,
                        bool by_row, int beta, int s, __nv_bfloat16 *S) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int c = (int)(idx / n), r = (int)(idx % n);
    double x = ldexp(X[(size_t)c * ldx + r], -(by_row ? ex[r] : ex[c]));
    const size_t plane = (size_t)n * n;
    for (int p = 0; p < s; ++p) {
        const double y = ldexp(x, beta);
        const double a = rint(y);
        S[p * plane + idx] = __double2bfloat16(a);
        x = y - a;
    }
}

// acc(i, k) += sum_{q < nq} 2^(-beta (p + q + 2)) Cp(i, q n + k)  (Cp: n x nq n, FP32, ld n).
__global__ void k_ozaki_accumulate(int n, int nq, int p, int beta, const float *__restrict__ Cp,
                                   double *acc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const size_t plane = (size_t)n * n;
    double t = 0.0;
    for (int q = nq - 1; q >= 0; --q) t += ldexp((double)Cp[q * plane + idx], -beta * (p + q + 2));
    acc[idx] += t;
}

// B = F o (2^(ea_i + eb_k) acc) in place, F as in the header comment (C = Z^T G stage).
__global__ void k_ozaki_finish_F(int n, const int *__restrict__ ea, const int *__restrict__ eb,
                                 const double *__restrict__ w, double delta, double *acc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int k = (int)(idx / n), i = (int)(idx % n);
    if (i == k) { acc[idx] = 0.0; return; }
    const double D = w[k] - w[i];
    acc[idx] = ldexp(acc[idx], ea[i] + eb[k]) * (D / (D * D + delta * delta));
}

// Y = 2^(ea_j + eb_k) acc in place (Y = Z B stage).
__global__ void k_ozaki_finish_scale(int n, const int *__restrict__ ea, const int *__restrict__ eb,
                                     double *acc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int k = (int)(idx / n), j = (int)(idx % n);
    acc[idx] = ldexp(acc[idx], ea[j] + eb[k]);
}

// One cuBLAS handle per device, created on first use; the mutex serialises its users.
std::mutex g_blas_mutex;
cublasHandle_t g_blas[64] = {};

cublasHandle_t blas_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!g_blas[dev] && cublasCreate(&g_blas[dev]) != CUBLAS_STATUS_SUCCESS) g_blas[dev] = nullptr;
    return g_blas[dev];
}

// acc = op(A) * B summed exactly slice by slice; transA: op(A) = A^T with A's columns
// scaled (ea), else op(A) = A with A's rows scaled (ea); B's columns scaled (eb).
// SA, SB: s planes of n x n bf16 each; Cbuf: n x s n floats.
int ozaki_product(cublasHandle_t h, int n, const OzakiPlan &pl, bool transA,
                  const __nv_bfloat16 *SA, const __nv_bfloat16 *SB, float *Cbuf, double *acc,
                  cudaStream_t st) {
    const size_t plane = (size_t)n * n;
    const unsigned nblk = (unsigned)((plane + 255) / 256);
    const float one = 1.f, zero = 0.f;
    cudaMemsetAsync(acc, 0, sizeof(double) * plane, st);
    for (int c0 = 0; c0 < n; c0 += pl.chunk) {
        const int kc = std::min(pl.chunk, n - c0);
        for (int p = pl.s - 1; p >= 0; --p) {
            const int nq = pl.s - p; // slices q with p + q <= s - 1
            const __nv_bfloat16 *A = SA + p * plane + (transA ? (size_t)c0 : (size_t)c0 * n);
            const __nv_bfloat16 *B = SB + c0;
            const cublasStatus_t rc = cublasGemmEx(
                h, transA ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, n, nq * n, kc, &one, A,
                CUDA_R_16BF, n, B, CUDA_R_16BF, n, &zero, Cbuf, CUDA_R_32F, n,
                CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
            if (rc != CUBLAS_STATUS_SUCCESS) return MR3_ECUDA;
            k_ozaki_accumulate<<<nblk, 256, 0, st>>>(n, nq, p, pl.beta, Cbuf, acc);
        }
    }
    return 0;
}

// Vector part of the backward for n >= kOzakiMinN: dd, de += diag terms of Z (F o Z^T G) Z^T.
int backward_vectors_ozaki(int n, const double *w, const double *Z, int ldz, const double *gZ,
                           int ldgz, double delta, double *dd, double *de, cudaStream_t st) {
    const OzakiPlan pl = ozaki_plan(n);
    const size_t plane = (size_t)n * n;
    __nv_bfloat16 *SA = nullptr, *SB = nullptr;
    float *Cbuf = nullptr;
    double *acc = nullptr, *Y = nullptr;
    int *ex = nullptr;
    auto fail = [&](int code) {
        if (SA) cudaFreeAsync(SA, st);
        if (SB) cudaFreeAsync(SB, st);
        if (Cbuf) cudaFreeAsync(Cbuf, st);
        if (acc) cudaFreeAsync(acc, st);
        if (Y) cudaFreeAsync(Y, st);
        if (ex) cudaFreeAsync(ex, st);
        return code;
    };
    if (cudaMallocAsync((void **)&SA, sizeof(__nv_bfloat16) * plane * pl.s, st) != cudaSuccess ||
        cudaMallocAsync((void **)&SB, sizeof(__nv_bfloat16) * plane * pl.s, st) != cudaSuccess ||
        cudaMallocAsync((void **)&Cbuf, sizeof(float) * plane * pl.s, st) != cudaSuccess ||
        cudaMallocAsync((void **)&acc, sizeof(double) * plane, st) != cudaSuccess ||
        cudaMallocAsync((void **)&Y, sizeof(double) * plane, st) != cudaSuccess ||
        cudaMallocAsync((void **)&ex, sizeof(int) * 4 * n, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(MR3_EOOM);
    }
    int *ea = ex, *eb = ex + n, *ea2 = ex + 2 * n, *eb2 = ex + 3 * n;
    const unsigned nblk = (unsigned)((plane + 255) / 256);
    const unsigned wblk = (unsigned)((32ll * n + 255) / 256);
    const unsigned rblk = (unsigned)((n + 127) / 128);
    std::lock_guard<std::mutex> lock(g_blas_mutex);
    cublasHandle_t h = blas_for_current_device();
    if (!h || cublasSetStream(h, st) != CUBLAS_STATUS_SUCCESS) return fail(MR3_ECUDA);
    // C = Z^T G: columns of Z and of G scaled
    k_line_exponent<<<wblk, 256, 0, st>>>(n, Z, ldz, false, ea);
    k_line_exponent<<<wblk, 256, 0, st>>>(n, gZ, ldgz, false, eb);
    k_slice<<<nblk, 256, 0, st>>>(n, Z, ldz, ea, false, pl.beta, pl.s, SA);
    k_slice<<<nblk, 256, 0, st>>>(n, gZ, ldgz, eb, false, pl.beta, pl.s, SB);
    int rc = ozaki_product(h, n, pl, true, SA, SB, Cbuf, acc, st);
    if (rc) return fail(rc);
    k_ozaki_finish_F<<<nblk, 256, 0, st>>>(n, ea, eb, w, delta, acc);
    // Y = Z B: rows of Z and columns of B scaled
    k_line_exponent<<<rblk, 128, 0, st>>>(n, Z, ldz, true, ea2);
    k_line_exponent<<<wblk, 256, 0, st>>>(n, acc, n, false, eb2);
    k_slice<<<nblk, 256, 0, st>>>(n, Z, ldz, ea2, true, pl.beta, pl.s, SA);
    k_slice<<<nblk, 256, 0, st>>>(n, acc, n, eb2, false, pl.beta, pl.s, SB);
    rc = ozaki_product(h, n, pl, false, SA, SB, Cbuf, Y, st);
    if (rc) return fail(rc);
    k_ozaki_finish_scale<<<nblk, 256, 0, st>>>(n, ea2, eb2, Y);
    k_bwd_vec_reduce<<<rblk, 128, 0, st>>>(n, Y, Z, ldz, dd, de);
    return fail(0);
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
    if (gZ && n >= kOzakiMinN) {
        double w0, wn;
        cudaMemcpyAsync(&w0, w, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&wn, w + n - 1, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        const double tnorm = std::max(std::fabs(w0), std::fabs(wn));
        const double delta = n * kEps * (tnorm > 0 ? tnorm : 1.0);
        const int rc = backward_vectors_ozaki(n, w, Z, ldz, gZ, ldgz, delta, dd, de, s);
        if (rc) return rc;
    } else if (gZ && n > 1) {
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
