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
// right one is scaled by a power of two into (-1, 1) and cut into s slices of beta bits
// (consecutive bit fields of its fixed-point fraction), each an integer held exactly in
// bf16; a slice-by-slice product summed over a chunk of at
// most 2^(24 - 2 beta) terms is an integer below 2^24 and comes out of an FP32-accumulating
// GEMM exactly; the slice products whose weight 2^(-beta (p + q)) is below 2^(-beta (s+1))
// are dropped (their sum is below 2^-54 of the scale), and the rest is summed in binary64.
// The slice GEMMs run on the library's own tcgen05 kernel (mr3_tc_gemm.cu): slice planes
// are stored K-major with a leading dimension padded to a multiple of 64 elements (the
// left operand of Y = Z B written transposed), so both operands load by TMA.
#include <algorithm>
#include <cstring>
#include <mutex>
#include "mr3.h"
#include "mr3_kernels.h"

namespace mr3 {
namespace {

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

// ||T|| = max(|lambda_1|, |lambda_n|) of T itself (the norm the regularisation delta of
// mr3_backward is relative to), one warp: lanes 0-15 and 16-31 bracket lambda_1 and
// lambda_n by 16-point multisection from the Gershgorin interval with binary64 Sturm
// counts on T (App. B, NegCount on T; a pivot below pivmin counts as -pivmin).
// Number of eigenvalues of T below x: the signs of the leading principal minors
// c_i = (d_i - x) c_{i-1} - e_{i-1}^2 c_{i-2} change once per negative pivot of T - x I
// (Sturm sequence), with no division on the chain.  The data enter scaled by rs = 1 / s
// (s the Gershgorin magnitude of T), so that |c_i| grows by at most a factor 3 per step;
// the pair (c_i, c_{i-1}) is brought back near 1 by a power of two every 8 steps, and an
// exact zero counts as a negative pivot.
__device__ int sturm_T(int n, const double *__restrict__ d, const double *__restrict__ e,
                       double x, double rs) {
    int cnt = 0;
    double c1 = 1.0, c0 = 0.0;
    int i = 0;
    for (; i + 8 <= n; i += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = i + u;
            const double a = (__ldg(d + j) - x) * rs;
            const double eu = j > 0 ? __ldg(e + j - 1) * rs : 0.0;
            double c = fma(a, c1, -(eu * eu) * c0);
            c = (c == 0.0) ? -c1 * 0x1p-80 : c;
            cnt += (c < 0.0) != (c1 < 0.0);
            c0 = c1;
            c1 = c;
        }
        const int ex = biased_exp(c1);
        const double sc = (ex > 0 && ex < 0x7ff) ? pow2i(1023 - ex) : 1.0;
        c1 *= sc;
        c0 *= sc;
    }
    for (; i < n; ++i) {
        const double a = (__ldg(d + i) - x) * rs;
        const double eu = i > 0 ? __ldg(e + i - 1) * rs : 0.0;
        double c = fma(a, c1, -(eu * eu) * c0);
        c = (c == 0.0) ? -c1 * 0x1p-80 : c;
        cnt += (c < 0.0) != (c1 < 0.0);
        c0 = c1;
        c1 = c;
    }
    return cnt;
}

// ||T|| = max(|lambda_1|, |lambda_n|) by multisection of both extreme eigenvalues, spread
// over many blocks: st holds {L, H} of each end and the scale; a sweep counts at P points of
// each bracket (k_tnorm_count) and one thread moves the brackets (k_tnorm_update).
constexpr int kTnormPoints = 2048; // points per end and sweep (64 single-warp blocks)
constexpr int kTnormSweeps = 4;    // 11 bits per sweep: 2^-44 of the Gershgorin width

__global__ void k_tnorm_init(int n, const double *__restrict__ d, const double *__restrict__ e,
                             double *st, int *tcnt) {
    __shared__ double s_lo[256], s_hi[256];
    double gl = INFINITY, gu = -INFINITY;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j < n - 1 ? fabs(e[j]) : 0.0);
        gl = fmin(gl, d[j] - r);
        gu = fmax(gu, d[j] + r);
    }
    s_lo[threadIdx.x] = gl;
    s_hi[threadIdx.x] = gu;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_lo[threadIdx.x] = fmin(s_lo[threadIdx.x], s_lo[threadIdx.x + o]);
            s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st[0] = st[2] = s_lo[0];
        st[1] = st[3] = s_hi[0];
        const double gs = fmax(fabs(s_lo[0]), fabs(s_hi[0]));
        st[4] = gs > 0.0 ? 1.0 / gs : 1.0;
        tcnt[0] = tcnt[1] = 0;
    }
}

__device__ __forceinline__ double tnorm_point(double L, double H, int p) {
    return L + (double)(p + 1) * ((H - L) / (double)(kTnormPoints + 1));
}

// blockIdx.y = 0: the lowest eigenvalue (count < 1 below it), 1: the highest (count < n)
__global__ void k_tnorm_count(int n, const double *__restrict__ d, const double *__restrict__ e,
                              const double *__restrict__ st, int *tcnt) {
    const int end = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const double L = st[2 * end], H = st[2 * end + 1];
    bool below = false;
    if (p < kTnormPoints) below = sturm_T(n, d, e, tnorm_point(L, H, p), st[4]) < (end ? n : 1);
    const unsigned b = __ballot_sync(0xffffffffu, below);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(tcnt + end, __popc(b));
}

__global__ void k_tnorm_update(double *st, int *tcnt, double *out, int last) {
    if (threadIdx.x != 0) return;
    double mid[2];
    for (int end = 0; end < 2; ++end) {
        const double L = st[2 * end], H = st[2 * end + 1];
        const int t = tcnt[end]; // points below the eigenvalue
        const double nl = t > 0 ? tnorm_point(L, H, t - 1) : L;
        const double nh = t < kTnormPoints ? tnorm_point(L, H, t) : H;
        st[2 * end] = nl;
        st[2 * end + 1] = nh;
        tcnt[end] = 0;
        mid[end] = 0.5 * (nl + nh);
    }
    if (last) *out = fmax(fabs(mid[0]), fabs(mid[1]));
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
    // every slice is an integer of magnitude < 2^beta, so a chunk sum of slice products
    // stays below 2^(2 beta + lg) <= 2^24; bf16 holds integers below 2^8 exactly
    p.beta = std::min(8, (24 - lg) / 2);
    p.s = (54 + p.beta - 1) / p.beta; // beta s <= 56 < 64: the slices fit one 64-bit word
    return p;
}

// x 2^e exactly (up to the rounding of a subnormal result) by two power-of-two factors.
__device__ __forceinline__ double scale2(double x, int e) {
    e = max(-2044, min(2046, e));
    const int e1 = e / 2, e2 = e - e1;
    return x * pow2i(e1) * pow2i(e2);
}

// Largest |X| per row (by_row) or per column, as the bit pattern of the binary64 value
// (for non-negative doubles the integer order is the numeric order).  Blocks of 32 rows x 8
// column lanes, each block over 256 columns; mx must start at zero.
__global__ void k_line_max(int n, const double *__restrict__ X, int ldx, bool by_row,
                           unsigned long long *mx) {
    const int r = blockIdx.x * 32 + (threadIdx.x & 31);
    const int cl = threadIdx.x >> 5;
    const int c0 = blockIdx.y * 256;
    unsigned long long m = 0;
    for (int t = 0; t < 32; ++t) {
        const int c = c0 + t * 8 + cl;
        unsigned long long v = 0;
        if (r < n && c < n) v = (unsigned long long)__double_as_longlong(X[(size_t)c * ldx + r]) & 0x7fffffffffffffffull;
        if (by_row) {
            m = v > m ? v : m;
        } else {
            for (int o = 16; o; o >>= 1) {
                const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
                v = u > v ? u : v;
            }
            if ((threadIdx.x & 31) == 0 && c < n && v) atomicMax(mx + c, v);
        }
    }
    if (by_row && r < n && m) atomicMax(mx + r, m);
}

// ex[r] = the least e with max |X(line r)| < 2^e (0 for a zero line; a non-finite maximum
// gives 0 too, and its slices carry the NaN).
__global__ void k_line_exponent(int n, const unsigned long long *__restrict__ mx, int *ex) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const unsigned long long b = mx[r];
    const int eb = (int)(b >> 52);
    int e = 0;
    if (b == 0 || eb == 0x7ff) e = 0;
    else if (eb == 0) e = (63 - __clzll((long long)b)) - 1073; // subnormal maximum
    else e = eb - 1022;
    ex[r] = e;
}

// Slices of X (n x n, column-major) by integer arithmetic: |x| 2^-e < 1 is read as the
// 64-bit fixed-point fraction F (its bits below 2^-64 truncated), slice p is bits
// [64 - beta (p+1), 64 - beta p) of F with the sign of x, an integer of magnitude < 2^beta,
// written as bf16 to plane S[p] (n x ldp elements): entry (r, c) at c ldp + r, or at
// r ldp + c with trans_out.  Hence x 2^-e = sum_p a_p 2^(-beta (p+1)) + r with
// |r| < 2^(-beta s).
__global__ void k_slice(int n, const double *__restrict__ X, int ldx, const int *__restrict__ ex,
                        bool by_row, int beta, int s, int ldp, bool trans_out, unsigned short *S) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int c = (int)(idx / n), r = (int)(idx % n);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(X[(size_t)c * ldx + r]);
    const unsigned sgn = (unsigned)(bits >> 63) << 15;
    const int eb = (int)((bits >> 52) & 0x7ff);
    const size_t plane = (size_t)n * ldp;
    const size_t o = trans_out ? (size_t)r * ldp + c : (size_t)c * ldp + r;
    if (eb == 0x7ff) { // NaN or infinity: propagate a NaN through the products
        for (int p = 0; p < s; ++p) S[p * plane + o] = (unsigned short)0x7fc0;
        return;
    }
    const unsigned long long m = eb ? ((bits & 0xfffffffffffffull) | (1ull << 52)) : (bits & 0xfffffffffffffull);
    const int E = eb ? eb - 1075 : -1074;
    const int sh = E + 64 - (by_row ? ex[r] : ex[c]);
    const unsigned long long F = sh >= 0 ? (m << sh) : (-sh >= 64 ? 0ull : (m >> -sh));
    const unsigned mask = (1u << beta) - 1u;
    for (int p = 0; p < s; ++p) {
        const unsigned v = (unsigned)(F >> (64 - beta * (p + 1))) & mask;
        unsigned short h = 0;
        if (v) {
            const int e2 = 31 - __clz((int)v);
            h = (unsigned short)(sgn | ((unsigned)(e2 + 127) << 7) | ((v << (7 - e2)) & 0x7fu));
        }
        S[p * plane + o] = h;
    }
}

// acc(i, k) += sum_{q < nq} 2^(-beta (p + q + 2)) Cp(i, q n + k)  (Cp: n x nq n, FP32, ld n;
// each Cp entry an exact integer of magnitude < 2^24).  Up to G consecutive terms are first
// combined exactly in a 64-bit integer (Horner in powers of 2^beta: below 2^(25 + beta (G-1))
// <= 2^62), so the binary64 pipe sees one conversion and one FMA per group; groups are added
// from the smallest weight up.
__global__ void k_ozaki_accumulate(int n, int nq, int p, int beta, const float *__restrict__ Cp,
                                   double *acc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const size_t plane = (size_t)n * n;
    const int G = 1 + 37 / beta;
    double t = 0.0;
    for (int q1 = nq; q1 > 0; q1 -= G) {
        const int q0 = max(0, q1 - G);
        long long S = 0;
        for (int q = q0; q < q1; ++q) S = S * (1ll << beta) + (long long)__float2int_rn(__ldg(Cp + q * plane + idx));
        t = fma((double)S, pow2i(-beta * (p + q1 + 1)), t);
    }
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
    acc[idx] = scale2(acc[idx], ea[i] + eb[k]) * (D / fma(D, D, delta * delta));
}

// Y = 2^(ea_j + eb_k) acc in place (Y = Z B stage).
__global__ void k_ozaki_finish_scale(int n, const int *__restrict__ ea, const int *__restrict__ eb,
                                     double *acc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int k = (int)(idx / n), j = (int)(idx % n);
    acc[idx] = scale2(acc[idx], ea[j] + eb[k]);
}

// acc = op(A) * B summed exactly slice by slice: A_p (s planes, K-major, leading dimension
// ldp: row m of op(A) at A_p + m ldp), B (s planes of n columns side by side, column j of
// the wide operand at B + j ldp); Cbuf: n x s n floats.  Slice p of A meets slices
// q < s - p of B in one tensor-core product per contraction chunk.
int ozaki_product(int n, int ldp, const OzakiPlan &pl, const unsigned short *SA,
                  const unsigned short *SB, float *Cbuf, double *acc, int *err, cudaStream_t st) {
    const size_t plane = (size_t)n * ldp;
    const unsigned nblk = (unsigned)(((size_t)n * n + 255) / 256);
    if (cudaMemsetAsync(acc, 0, sizeof(double) * n * n, st) != cudaSuccess) return MR3_ECUDA;
    for (int c0 = 0; c0 < n; c0 += pl.chunk) {
        const int kc = std::min(pl.chunk, n - c0);
        for (int p = pl.s - 1; p >= 0; --p) {
            const int nq = pl.s - p; // slices q with p + q <= s - 1
            if (tc_gemm_bf16(n, nq * n, n, c0, c0 + kc, SA + p * plane, ldp, SB, ldp, Cbuf, n,
                             err, st))
                return MR3_ECUDA;
            k_ozaki_accumulate<<<nblk, 256, 0, st>>>(n, nq, p, pl.beta, Cbuf, acc);
        }
    }
    return 0;
}

// Row reductions onto d and e, in two passes with a fixed summation order: blocks of 32
// rows x 8 column lanes write one partial sum per row and column chunk, then
// k_rows_finish adds the chunks.
//   kind 0 (eigenvalue part): sd_j = sum_i g_i Z_ji^2,  se_j = 2 sum_i g_i Z_ji Z_j+1,i
//   kind 1 (vector part):     sd_j = sum_b Y_jb Z_jb,   se_j = sum_b Y_jb Z_j+1,b + Y_j+1,b Z_jb
constexpr int kRowChunks = 32;

template <int KIND>
__global__ void __launch_bounds__(256) k_row_dots(int n, int ncols, const double *__restrict__ Y,
                                                  int ldy, const double *__restrict__ Z, int ldz,
                                                  const double *__restrict__ g, double *pd,
                                                  double *pe) {
    __shared__ double sd_s[8][33], se_s[8][33];
    const int tr = threadIdx.x & 31, cl = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + tr;
    const int per = (ncols + kRowChunks - 1) / kRowChunks;
    const int b0 = blockIdx.y * per, b1 = min(ncols, b0 + per);
    double sd = 0.0, se = 0.0;
    if (j < n) {
        for (int b = b0 + cl; b < b1; b += 8) {
            const double *zc = Z + (size_t)b * ldz;
            const double z = zc[j];
            const double z1 = (j + 1 < n) ? zc[j + 1] : 0.0;
            if (KIND == 0) {
                const double gz = __ldg(g + b) * z;
                sd = fma(gz, z, sd);
                se = fma(gz, z1, se);
            } else {
                const double *yc = Y + (size_t)b * ldy;
                const double y = yc[j];
                const double y1 = (j + 1 < n) ? yc[j + 1] : 0.0;
                sd = fma(y, z, sd);
                se = fma(y, z1, fma(y1, z, se));
            }
        }
    }
    sd_s[cl][tr] = sd;
    se_s[cl][tr] = se;
    __syncthreads();
    if (cl == 0 && j < n) {
        double a = 0.0, c = 0.0;
        for (int q = 0; q < 8; ++q) { a += sd_s[q][tr]; c += se_s[q][tr]; }
        pd[(size_t)blockIdx.y * n + j] = a;
        pe[(size_t)blockIdx.y * n + j] = c;
    }
}

// dd_j (=|+=) sum of the chunks' partial sums; de_j likewise with factor fe.
__global__ void k_rows_finish(int n, const double *__restrict__ pd, const double *__restrict__ pe,
                              double fe, bool add, double *dd, double *de) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double a = 0.0, c = 0.0;
    for (int q = 0; q < kRowChunks; ++q) { a += pd[(size_t)q * n + j]; c += pe[(size_t)q * n + j]; }
    if (add) {
        dd[j] += a;
        if (j < n - 1) de[j] += fe * c;
    } else {
        dd[j] = a;
        if (j < n - 1) de[j] = fe * c;
    }
}

// Y = Z (F o (Z^T G)) for n >= kOzakiMinN through the slice products (Y: n x n, ld n).
int vector_part_ozaki(int n, const double *w, const double *Z, int ldz, const double *gZ,
                      int ldgz, double delta, double *Y, cudaStream_t st) {
    const OzakiPlan pl = ozaki_plan(n);
    const size_t plane = (size_t)n * n;
    const int ldp = (n + 63) / 64 * 64; // slice planes: leading dimension a multiple of 64
    const size_t splane = (size_t)n * ldp;
    unsigned short *SA = nullptr, *SB = nullptr;
    float *Cbuf = nullptr;
    double *acc = nullptr;
    int *ex = nullptr;
    unsigned long long *mx = nullptr;
    int *err = nullptr;
    auto done = [&](int code) {
        if (err) cudaFreeAsync(err, st);
        if (SA) cudaFreeAsync(SA, st);
        if (SB) cudaFreeAsync(SB, st);
        if (Cbuf) cudaFreeAsync(Cbuf, st);
        if (acc) cudaFreeAsync(acc, st);
        if (ex) cudaFreeAsync(ex, st);
        if (mx) cudaFreeAsync(mx, st);
        return code;
    };
    if (lib_malloc_async((void **)&SA, sizeof(unsigned short) * splane * pl.s, st) != cudaSuccess ||
        lib_malloc_async((void **)&SB, sizeof(unsigned short) * splane * pl.s, st) != cudaSuccess ||
        lib_malloc_async((void **)&err, sizeof(int), st) != cudaSuccess ||
        lib_malloc_async((void **)&Cbuf, sizeof(float) * plane * pl.s, st) != cudaSuccess ||
        lib_malloc_async((void **)&acc, sizeof(double) * plane, st) != cudaSuccess ||
        lib_malloc_async((void **)&ex, sizeof(int) * 4 * n, st) != cudaSuccess ||
        lib_malloc_async((void **)&mx, sizeof(unsigned long long) * 4 * n, st) != cudaSuccess) {
        cudaGetLastError();
        return done(MR3_EOOM);
    }
    int *ea = ex, *eb = ex + n, *ea2 = ex + 2 * n, *eb2 = ex + 3 * n;
    unsigned long long *ma = mx, *mb = mx + n, *ma2 = mx + 2 * n, *mb2 = mx + 3 * n;
    const unsigned nblk = (unsigned)((plane + 255) / 256);
    const unsigned rblk = (unsigned)((n + 127) / 128);
    const dim3 mgrid((n + 31) / 32, (n + 255) / 256);
    if (cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 4 * n, st) != cudaSuccess ||
        cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
        return done(MR3_ECUDA);
    // C = Z^T G: columns of Z and of G scaled
    k_line_max<<<mgrid, 256, 0, st>>>(n, Z, ldz, false, ma);
    k_line_max<<<mgrid, 256, 0, st>>>(n, gZ, ldgz, false, mb);
    k_line_exponent<<<rblk, 128, 0, st>>>(n, ma, ea);
    k_line_exponent<<<rblk, 128, 0, st>>>(n, mb, eb);
    // op(A) = Z^T: row m of Z^T is column m of Z (K-major as stored)
    k_slice<<<nblk, 256, 0, st>>>(n, Z, ldz, ea, false, pl.beta, pl.s, ldp, false, SA);
    k_slice<<<nblk, 256, 0, st>>>(n, gZ, ldgz, eb, false, pl.beta, pl.s, ldp, false, SB);
    int rc = ozaki_product(n, ldp, pl, SA, SB, Cbuf, acc, err, st);
    if (rc) return done(rc);
    k_ozaki_finish_F<<<nblk, 256, 0, st>>>(n, ea, eb, w, delta, acc);
    // Y = Z B: rows of Z and columns of B scaled
    k_line_max<<<mgrid, 256, 0, st>>>(n, Z, ldz, true, ma2);
    k_line_max<<<mgrid, 256, 0, st>>>(n, acc, n, false, mb2);
    k_line_exponent<<<rblk, 128, 0, st>>>(n, ma2, ea2);
    k_line_exponent<<<rblk, 128, 0, st>>>(n, mb2, eb2);
    // op(A) = Z: its slices written transposed so that row m of Z is contiguous
    k_slice<<<nblk, 256, 0, st>>>(n, Z, ldz, ea2, true, pl.beta, pl.s, ldp, true, SA);
    k_slice<<<nblk, 256, 0, st>>>(n, acc, n, eb2, false, pl.beta, pl.s, ldp, false, SB);
    rc = ozaki_product(n, ldp, pl, SA, SB, Cbuf, Y, err, st);
    if (rc) return done(rc);
    k_ozaki_finish_scale<<<nblk, 256, 0, st>>>(n, ea2, eb2, Y);
    // a tensor-core product whose pipeline gave up leaves the error flag set
    int herr = 0;
    if (read_back(&herr, err, sizeof(int), st) != cudaSuccess || herr) return done(MR3_ECUDA);
    return done(0);
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
    double *part = nullptr, *C = nullptr, *Y = nullptr;
    const bool vec = gZ && n > 1;
    auto done = [&](int code) {
        if (part) cudaFreeAsync(part, s);
        if (C) cudaFreeAsync(C, s);
        if (Y) cudaFreeAsync(Y, s);
        if (code == 0 && cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return (int)MR3_ECUDA; }
        return code;
    };
    if (lib_malloc_async((void **)&part, sizeof(double) * 2 * kRowChunks * (size_t)n, s) != cudaSuccess ||
        (vec && lib_malloc_async((void **)&Y, sizeof(double) * (size_t)n * n, s) != cudaSuccess) ||
        (vec && n < kOzakiMinN && lib_malloc_async((void **)&C, sizeof(double) * (size_t)n * n, s) != cudaSuccess)) {
        cudaGetLastError();
        return done(MR3_EOOM);
    }
    double *pd = part, *pe = part + (size_t)kRowChunks * n;
    const dim3 rgrid((n + 31) / 32, kRowChunks);
    const unsigned fblk = (unsigned)((n + 127) / 128);
    // eigenvalue part: dbar_j = sum_i g_i z_ji^2, ebar_j = 2 sum_i g_i z_ji z_j+1,i
    if (gw && k > 0) {
        k_row_dots<0><<<rgrid, 256, 0, s>>>(n, k, nullptr, 1, Z, ldz, gw, pd, pe);
        k_rows_finish<<<fblk, 128, 0, s>>>(n, pd, pe, 2.0, false, dd, de);
    } else {
        if (cudaMemsetAsync(dd, 0, sizeof(double) * n, s) != cudaSuccess ||
            (n > 1 && cudaMemsetAsync(de, 0, sizeof(double) * (n - 1), s) != cudaSuccess))
            return done(MR3_ECUDA);
    }
    if (vec) {
        // ||T|| from the eigenvalues (ascending): max(|lambda_1|, |lambda_n|)
        double w0, wn;
        if (cudaMemcpyAsync(&w0, w, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&wn, w + n - 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return done(MR3_ECUDA);
        }
        const double tnorm = std::max(std::fabs(w0), std::fabs(wn));
        const double delta = n * kEps * (tnorm > 0 ? tnorm : 1.0);
        if (n >= kOzakiMinN) {
            const int rc = vector_part_ozaki(n, w, Z, ldz, gZ, ldgz, delta, Y, s);
            if (rc) return done(rc);
        } else {
            dim3 g((n + 63) / 64, (n + 63) / 64);
            k_gemm_f64<true><<<g, 256, 0, s>>>(n, n, n, Z, ldz, gZ, ldgz, C, n);
            k_apply_F<<<(unsigned)(((long long)n * n + 255) / 256), 256, 0, s>>>(n, w, delta, C);
            k_gemm_f64<false><<<g, 256, 0, s>>>(n, n, n, Z, ldz, C, n, Y, n);
        }
        k_row_dots<1><<<rgrid, 256, 0, s>>>(n, n, Y, n, Z, ldz, nullptr, pd, pe);
        k_rows_finish<<<fblk, 128, 0, s>>>(n, pd, pe, 1.0, true, dd, de);
    }
    return done(0);
}

extern "C" int mr3_backward_solve(int n, int k, const double *d, const double *e, const double *w,
                                  const double *Z, int ldz, const double *gw, const double *gZ,
                                  int ldgz, double *dd, double *de, const mr3_opts *opts,
                                  void *stream) {
    (void)opts;
    if (n < 0) return -1;
    if (k < 0 || k > n) return -2;
    if (n > 0 && !d) return -3;
    if (n > 1 && !e) return -4;
    if (k > 0 && !w) return -5;
    if (k > 0 && !Z) return -6;
    if (ldz < std::max(1, n)) return -7;
    if (gZ && ldgz < std::max(1, n)) return -10;
    if (n > 0 && !dd) return -11;
    if (n > 1 && !de) return -12;
    if (n == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    double *part = nullptr, *Y = nullptr, *scr = nullptr;
    const bool vec = gZ && n > 1 && k > 0;
    auto done = [&](int code) {
        if (part) cudaFreeAsync(part, s);
        if (Y) cudaFreeAsync(Y, s);
        if (scr) cudaFreeAsync(scr, s);
        if (code == 0 && cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); return (int)MR3_ECUDA; }
        return code;
    };
    if (lib_malloc_async((void **)&part, sizeof(double) * 2 * kRowChunks * (size_t)n, s) != cudaSuccess ||
        (vec && lib_malloc_async((void **)&Y, sizeof(double) * (size_t)n * k, s) != cudaSuccess) ||
        (vec && lib_malloc_async((void **)&scr, sizeof(double) * adjoint_scratch_doubles(n, k), s) != cudaSuccess)) {
        cudaGetLastError();
        return done(MR3_EOOM);
    }
    double *pd = part, *pe = part + (size_t)kRowChunks * n;
    const dim3 rgrid((n + 31) / 32, kRowChunks);
    const unsigned fblk = (unsigned)((n + 127) / 128);
    if (gw && k > 0) {
        k_row_dots<0><<<rgrid, 256, 0, s>>>(n, k, nullptr, 1, Z, ldz, gw, pd, pe);
        k_rows_finish<<<fblk, 128, 0, s>>>(n, pd, pe, 2.0, false, dd, de);
    } else {
        if (cudaMemsetAsync(dd, 0, sizeof(double) * n, s) != cudaSuccess ||
            (n > 1 && cudaMemsetAsync(de, 0, sizeof(double) * (n - 1), s) != cudaSuccess))
            return done(MR3_ECUDA);
    }
    if (vec) {
        // ||T|| = max |lambda| of T: the ends of w when all eigenpairs are given (as the
        // dense path takes it), else by bisection of T's extreme eigenvalues
        double hd[2] = {0.0, 0.0};
        int rc = 0;
        if (k == n) {
            if (read_back(hd, w, sizeof(double), s) != cudaSuccess ||
                read_back(hd + 1, w + (k - 1), sizeof(double), s) != cudaSuccess)
                return done(MR3_ECUDA);
            hd[0] = std::max(std::fabs(hd[0]), std::fabs(hd[1]));
        } else {
            double *gmax = nullptr;
            if (lib_malloc_async((void **)&gmax, sizeof(double) * 8, s) != cudaSuccess) { cudaGetLastError(); return done(MR3_EOOM); }
            double *st = gmax + 1;
            int *tcnt = (int *)(gmax + 6);
            k_tnorm_init<<<1, 256, 0, s>>>(n, d, e, st, tcnt);
            for (int sw = 0; sw < kTnormSweeps; ++sw) {
                // one warp per block: the counts' binary64 instructions spread over the SMs
                k_tnorm_count<<<dim3(kTnormPoints / 32, 2), 32, 0, s>>>(n, d, e, st, tcnt);
                k_tnorm_update<<<1, 32, 0, s>>>(st, tcnt, gmax, sw == kTnormSweeps - 1);
            }
            if (read_back(hd, gmax, sizeof(double), s) != cudaSuccess) rc = MR3_ECUDA;
            cudaFreeAsync(gmax, s);
            if (rc) return done(rc);
        }
        const double tnorm = hd[0] > 0.0 ? hd[0] : 1.0;
        launch_adjoint(n, k, d, e, w, Z, ldz, gZ, ldgz, tnorm, scr, Y, s);
        k_row_dots<1><<<rgrid, 256, 0, s>>>(n, k, Y, n, Z, ldz, nullptr, pd, pe);
        k_rows_finish<<<fblk, 128, 0, s>>>(n, pd, pe, 1.0, true, dd, de);
    }
    return done(0);
}
