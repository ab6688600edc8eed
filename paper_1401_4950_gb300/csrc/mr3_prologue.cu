// mr3_prologue.cu -- everything before the representation tree is traversed:
// splitting into irreducible blocks (Sec. 3.2.1), Gershgorin intervals (App. B,
// Alg. Gershgorin), selection of the requested eigenpairs (App. A ranges), and the root
// representation M_root = T - mu I with its random perturbation (Alg. MRRR).
#include <float.h>
#include "mr3_kernels.h"
#include "mr3_df.cuh"

namespace mr3 {

#define FULL_MASK 0xffffffffu

// ------------------------------------------------------------------ helpers

// Index of the matrix that owns packed row `row` (mats sorted by offset).
__device__ __forceinline__ int find_mat(int nmat, const MatDesc *mats, long long row) {
    int lo = 0, hi = nmat - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (mats[mid].off <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}

// Number of eigenvalues of sgn*T strictly below sgn*x (FP64, homogeneous three-term form
// of App. B Alg. NegCount on T).  sgn = -1 gives #(eigenvalues of T > x).
__device__ int negcount_T_f64(int n, const double *__restrict__ d, const double *__restrict__ e,
                              double x, int neg) {
    double pm2 = 0.0, pm1 = 1.0;
    int sp = 0, cnt = 0;
    for (int i = 0; i < n; ++i) {
        const double ai = neg ? (x - __ldg(d + i)) : (__ldg(d + i) - x);
        double q = 0.0;
        if (i > 0) { const double b = __ldg(e + i - 1); q = (b * b) * pm2; }
        double p = fma(ai, pm1, -q);
        // zero pivot: negative (the limit x -> x+), p_i = 0 kept; the next step then gives
        // p_{i+1} = -beta_i^2 p_{i-1}, the pivot +infinity
        const bool z = is_zero(p);
        const int sc = z ? (sp ^ 1) : sign_bit(p);
        cnt += sc ^ sp;
        const int ex = biased_exp(p);
        if ((unsigned)(ex - (1023 - 200)) > 400u && !z) {
            const double s = pow2i(1023 - ex);
            p *= s;
            pm1 *= s;
        }
        pm2 = pm1;
        pm1 = p;
        sp = sc;
    }
    return cnt;
}

// #(eigenvalues of T <= x) = n - #(eigenvalues of -T < -x).
__device__ __forceinline__ int count_le_T(int n, const double *d, const double *e, double x) {
    return n - negcount_T_f64(n, d, e, x, 1);
}

// ------------------------------------------------------------------ matrix norms

__global__ void k_mat_norm(int nmat, MatDesc *mats, const double *__restrict__ d,
                           const double *__restrict__ e, int *bad_input) {
    const int b = blockIdx.x;
    if (b >= nmat) return;
    const int n = mats[b].n;
    const long long off = mats[b].off;
    double lo = DBL_MAX, hi = -DBL_MAX;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double di = d[off + i];
        double r = 0.0;
        if (i > 0) r += fabs(e[off + i - 1]);
        if (i < n - 1) { const double ei = e[off + i]; r += fabs(ei); if (!is_finite(ei)) bad = 1; }
        if (!is_finite(di)) bad = 1;
        lo = fmin(lo, di - r);
        hi = fmax(hi, di + r);
    }
    __shared__ double slo[32], shi[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) atomicOr(&sbad, 1);
    lo = warp_min(lo);
    hi = warp_max(hi);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { slo[w] = lo; shi[w] = hi; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        lo = (l < nw) ? slo[l] : DBL_MAX;
        hi = (l < nw) ? shi[l] : -DBL_MAX;
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (l == 0) {
            mats[b].tnorm = (n > 0) ? fmax(fabs(lo), fabs(hi)) : 0.0;
            if (sbad) atomicOr(bad_input, 1);
        }
    }
}

void launch_mat_norm(int nmat, MatDesc *mats, const double *d, const double *e, int *bad_input,
                     cudaStream_t s) {
    if (nmat > 0) k_mat_norm<<<nmat, 256, 0, s>>>(nmat, mats, d, e, bad_input);
}

// ------------------------------------------------------------------ splitting

// Row i starts a block when it starts its matrix or |beta_{i-1}| <= eps sqrt(n) ||T||
// (Sec. 3.2.1, tol_split = eps sqrt(n)).
__global__ void k_split_flags(int nmat, const MatDesc *__restrict__ mats, long long nrows,
                              const double *__restrict__ e, int *flags) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    const int b = find_mat(nmat, mats, i);
    const MatDesc M = mats[b];
    int f;
    if (i == M.off) {
        f = 1;
    } else {
        const double tol = kEps * sqrt((double)M.n) * M.tnorm;
        f = (fabs(e[i - 1]) <= tol) ? 1 : 0;
    }
    flags[i] = f;
}

void launch_split_flags(int nmat, const MatDesc *mats, long long nrows, const double *d,
                        const double *e, int *flags, cudaStream_t s) {
    (void)d;
    if (nrows <= 0) return;
    const int bs = 256;
    k_split_flags<<<(unsigned)((nrows + bs - 1) / bs), bs, 0, s>>>(nmat, mats, nrows, e, flags);
}

// ------------------------------------------------------------------ exclusive scan
// Three-pass scan: tiles of 2048 ints scanned per CTA, tile sums scanned by one CTA,
// then offsets added.
#define SCAN_TILE 2048

__device__ __forceinline__ int block_excl_scan_1024(int v, int *sh, int &total) {
    // v: this thread's value; returns exclusive prefix within the CTA of 1024 threads.
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = sh[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL_MASK, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s; // inclusive over warps
    }
    __syncthreads();
    const int warp_off = (w > 0) ? sh[w - 1] : 0;
    total = sh[31];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const int *in, int *out, long long n, int *tile_sums) {
    __shared__ int sh[32];
    const long long base = (long long)blockIdx.x * SCAN_TILE;
    const long long i0 = base + 2 * threadIdx.x;
    const int a = (i0 < n) ? in[i0] : 0;
    const int b = (i0 + 1 < n) ? in[i0 + 1] : 0;
    int total;
    const int ex = block_excl_scan_1024(a + b, sh, total);
    if (i0 < n) out[i0] = ex;
    if (i0 + 1 < n) out[i0 + 1] = ex + a;
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int *tile_sums, long long ntiles, int *total_out) {
    __shared__ int sh[32];
    int carry = 0;
    for (long long base = 0; base < ntiles; base += 1024) {
        const long long i = base + threadIdx.x;
        const int v = (i < ntiles) ? tile_sums[i] : 0;
        int total;
        const int ex = block_excl_scan_1024(v, sh, total);
        if (i < ntiles) tile_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int *out, long long n, const int *tile_sums) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sums[i / SCAN_TILE];
}

size_t scan_tmp_ints(long long n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 1; }

void launch_exclusive_scan(const int *in, int *out, long long n, int *total, int *tmp,
                           cudaStream_t s) {
    if (n <= 0) { cudaMemsetAsync(total, 0, sizeof(int), s); return; }
    const long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_tiles<<<(unsigned)ntiles, 1024, 0, s>>>(in, out, n, tmp);
    k_scan_sums<<<1, 1024, 0, s>>>(tmp, ntiles, total);
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, tmp);
}

// ------------------------------------------------------------------ blocks

__global__ void k_blocks_from_flags(long long nrows, const int *flags, const int *scanned,
                                    int nmat, const MatDesc *mats, BlkDesc *blks) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows || !flags[i]) return;
    const int id = scanned[i];
    const int b = find_mat(nmat, mats, i);
    BlkDesc B;
    B.off = i;
    B.mat = b;
    B.roff = (int)(i - mats[b].off);
    B.n = 0;
    B.rep = (long long)kRepStride * i + (long long)kRepPad * id;
    B.dfok = 0;
    B.dfexp = 0;
    B.j0 = 1;
    B.j1 = 0;
    B.col0 = 0;
    B.gl = B.gu = B.mu = B.spdiam = 0.0;
    blks[id] = B;
}

__global__ void k_blocks_finish(int nblk_total, const int *nblk_dev, BlkDesc *blks, int nmat,
                                MatDesc *mats) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int nblk = *nblk_dev;
    if (id >= nblk || id >= nblk_total) return;
    const BlkDesc B = blks[id];
    const MatDesc M = mats[B.mat];
    long long end = M.off + M.n;
    if (id + 1 < nblk && blks[id + 1].mat == B.mat) end = blks[id + 1].off;
    blks[id].n = (int)(end - B.off);
    if (B.roff == 0) mats[B.mat].blk0 = id;
}

__global__ void k_mat_blockcount(int nmat, MatDesc *mats, const int *nblk_dev, const BlkDesc *blks) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nmat) return;
    if (mats[b].n <= 0) { mats[b].nblk = 0; mats[b].blk0 = 0; return; }
    const int nblk = *nblk_dev;
    const int b0 = mats[b].blk0;
    int k = b0;
    while (k < nblk && blks[k].mat == b) ++k;
    mats[b].nblk = k - b0;
}

// Block list from the scanned split flags (nblk_host: the total read back by the host).
void build_blocks(long long nrows, const int *flags, const int *scanned, const int *nblk_dev,
                  int nblk_host, int nmat, MatDesc *mats, BlkDesc *blks, cudaStream_t s) {
    if (nrows <= 0) return;
    k_blocks_from_flags<<<(unsigned)((nrows + 255) / 256), 256, 0, s>>>(nrows, flags, scanned,
                                                                        nmat, mats, blks);
    if (nblk_host > 0)
        k_blocks_finish<<<(nblk_host + 255) / 256, 256, 0, s>>>(nblk_host, nblk_dev, blks, nmat,
                                                                 mats);
    k_mat_blockcount<<<(nmat + 255) / 256, 256, 0, s>>>(nmat, mats, nblk_dev, blks);
}

// ------------------------------------------------------------------ block setup

__global__ void k_blk_setup(int nblk, BlkDesc *blks, const MatDesc *__restrict__ mats,
                            const double *__restrict__ D, const double *__restrict__ E,
                            int range) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nblk) return;
    BlkDesc B = blks[b];
    const MatDesc M = mats[B.mat];
    const double *d = D + B.off;
    const double *e = E + B.off;
    const int n = B.n;
    // App. B, Alg. Gershgorin on the block (|beta_1| used for the first row).
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int i = lane; i < n; i += 32) {
        double r = 0.0;
        if (i > 0) r += fabs(e[i - 1]);
        if (i < n - 1) r += fabs(e[i]);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    const double bnorm = fmax(fabs(lo), fabs(hi));
    const double pad = (2.0 * n + 10.0) * bnorm * kEps;
    B.gl = lo - pad;
    B.gu = hi + pad;
    B.spdiam = B.gu - B.gl;
    int j0 = 1, j1 = n;
    if (range == MR3_RANGE_VALUE) {
        // (vl, vu]: local indices count_le(vl)+1 .. count_le(vu)
        int c = 0;
        if (lane < 2) c = count_le_T(n, d, e, lane == 0 ? M.vl : M.vu);
        const int c0 = __shfl_sync(FULL_MASK, c, 0), c1 = __shfl_sync(FULL_MASK, c, 1);
        j0 = c0 + 1;
        j1 = c1;
    } else if (range == MR3_RANGE_INDEX) {
        if (M.nblk == 1) { j0 = M.il; j1 = M.iu; } else { j0 = 1; j1 = 0; } // multi-block: later
    }
    B.j0 = j0;
    B.j1 = j1;
    if (lane == 0) blks[b] = B;
}

void launch_blk_setup(int nblk, BlkDesc *blks, int nmat, MatDesc *mats, const double *d,
                      const double *e, int range, cudaStream_t s) {
    (void)nmat;
    if (nblk <= 0) return;
    const int wpb = 4;
    k_blk_setup<<<(nblk + wpb - 1) / wpb, 32 * wpb, 0, s>>>(nblk, blks, mats, d, e, range);
}

// Range INDEX on a matrix that split into several blocks: eigenvalues il and iu of the
// whole (split) matrix are bracketed to full accuracy by 16-point multisection, then the
// requested set is distributed over the blocks by counts; eigenvalues that cannot be told
// apart at full accuracy are assigned in block order.
__global__ void k_index_multi(int nmat, MatDesc *mats, BlkDesc *blks, const double *__restrict__ D,
                              const double *__restrict__ E) {
    const int mi = blockIdx.x;
    const int lane = threadIdx.x;
    if (mi >= nmat) return;
    const MatDesc M = mats[mi];
    if (M.nblk <= 1 || M.n <= 0) return;
    double gl = DBL_MAX, gu = -DBL_MAX;
    for (int k = 0; k < M.nblk; ++k) { gl = fmin(gl, blks[M.blk0 + k].gl); gu = fmax(gu, blks[M.blk0 + k].gu); }
    const int half = lane >> 4, kk = lane & 15;
    const int target = half ? M.iu : M.il;
    double L = gl, H = gu;
    for (int sweep = 0; sweep < 80; ++sweep) {
        const double width = H - L;
        const double tol = fmax(4.0 * kEps * fmax(fabs(L), fabs(H)), 4.0 * kSafmin);
        const bool go0 = __shfl_sync(FULL_MASK, (int)(width > tol), 0);
        const bool go1 = __shfl_sync(FULL_MASK, (int)(width > tol), 16);
        if (!go0 && !go1) break;
        const double x = L + (kk + 1) * (width / 17.0);
        int cnt = 0;
        for (int k = 0; k < M.nblk; ++k) {
            const BlkDesc B = blks[M.blk0 + k];
            cnt += negcount_T_f64(B.n, D + B.off, E + B.off, x, 0);
        }
        const unsigned bal = __ballot_sync(FULL_MASK, cnt < target);
        const unsigned hm = (bal >> (16 * half)) & 0xffffu;
        const int t = __popc(hm);
        const double xl = __shfl_sync(FULL_MASK, x, 16 * half + (t > 0 ? t - 1 : 0));
        const double xh = __shfl_sync(FULL_MASK, x, 16 * half + (t < 16 ? t : 15));
        if (width > tol) {
            if (t > 0) L = xl;
            if (t < 16) H = xh;
        }
    }
    const double L1 = __shfl_sync(FULL_MASK, L, 0), H1 = __shfl_sync(FULL_MASK, H, 0);
    const double L2 = __shfl_sync(FULL_MASK, L, 16), H2 = __shfl_sync(FULL_MASK, H, 16);
    if (lane != 0) return;
    int cL1 = 0, cL2 = 0;
    for (int k = 0; k < M.nblk; ++k) {
        const BlkDesc B = blks[M.blk0 + k];
        cL1 += negcount_T_f64(B.n, D + B.off, E + B.off, L1, 0);
        cL2 += negcount_T_f64(B.n, D + B.off, E + B.off, L2, 0);
    }
    int excl = M.il - 1 - cL1; // eigenvalues in [L1, H1) to leave out (lowest first)
    int incl = M.iu - cL2;     // eigenvalues in [L2, H2) to take (lowest first)
    for (int k = 0; k < M.nblk; ++k) {
        BlkDesc &B = blks[M.blk0 + k];
        const double *d = D + B.off, *e = E + B.off;
        const int a1 = negcount_T_f64(B.n, d, e, L1, 0), b1 = negcount_T_f64(B.n, d, e, H1, 0);
        const int a2 = negcount_T_f64(B.n, d, e, L2, 0), b2 = negcount_T_f64(B.n, d, e, H2, 0);
        int x1 = b1 - a1;
        int takeout = excl < x1 ? excl : x1;
        if (takeout < 0) takeout = 0;
        excl -= takeout;
        int x2 = b2 - a2;
        int takein = incl < x2 ? incl : x2;
        if (takein < 0) takein = 0;
        incl -= takein;
        B.j0 = a1 + takeout + 1;
        B.j1 = a2 + takein;
    }
}

void launch_index_multi(int nmat, MatDesc *mats, BlkDesc *blks, const double *d, const double *e,
                        cudaStream_t s) {
    if (nmat > 0) k_index_multi<<<nmat, 32, 0, s>>>(nmat, mats, blks, d, e);
}

// Per matrix: output columns of each block (blocks in order) and m.
__global__ void k_assign_columns(int nmat, MatDesc *mats, BlkDesc *blks) {
    const int mi = blockIdx.x * blockDim.x + threadIdx.x;
    if (mi >= nmat) return;
    const MatDesc M = mats[mi];
    int run = 0;
    for (int k = 0; k < M.nblk; ++k) {
        BlkDesc &B = blks[M.blk0 + k];
        if (B.j0 < 1) B.j0 = 1;
        if (B.j1 > B.n) B.j1 = B.n;
        const int mb = B.j1 >= B.j0 ? B.j1 - B.j0 + 1 : 0;
        B.col0 = M.woff + run;
        run += mb;
    }
    mats[mi].m = run;
}

void launch_assign_columns(int nmat, MatDesc *mats, BlkDesc *blks, int range, cudaStream_t s) {
    (void)range;
    if (nmat > 0) k_assign_columns<<<(nmat + 127) / 128, 128, 0, s>>>(nmat, mats, blks);
}

// ------------------------------------------------------------------ root representation

// L D L^T = T - mu I by the homogeneous three-term recurrence
//   p_i = (alpha_i - mu) p_{i-1} - beta_{i-1}^2 p_{i-2},   d_i = p_i / p_{i-1},
// one dependent FMA per step: the unscaled p_i go to P[i] and the power-of-two rescale
// applied after step i to K[i * kstride], so that the pivots can be divided out later in
// parallel.  Reports whether every pivot has the sign of a definite factorization
// (want_pos: positive; sign(d_i) = sign(p_i) xor sign(p_{i-1})) and the largest |d_i|
// (element growth, a division only when the running maximum may grow).
__device__ void factor_root(int n, const double *__restrict__ d, const double *__restrict__ e,
                            double mu, double *P, int *K, int kstride, bool want_pos,
                            bool &definite, double &growth) {
    double pm2 = 0.0, pm1 = 1.0;
    bool ok = true;
    double g = 0.0;
    // operands of step i + 1 are loaded while step i runs (software prefetch)
    double dn = __ldg(d), bn = 0.0;
    for (int i = 0; i < n; ++i) {
        const double ai = dn - mu, b = bn;
        if (i + 1 < n) {
            dn = __ldg(d + i + 1);
            bn = __ldg(e + i);
        }
        double q = 0.0;
        if (i > 0) q = (b * b) * pm2;
        double p = fma(ai, pm1, -q);
        P[i] = p;
        const int neg = sign_bit(p) ^ sign_bit(pm1);
        if ((want_pos ? neg : !neg) || is_zero(p) || !is_finite(p)) ok = false;
        if (fabs(p) > g * fabs(pm1)) g = fmax(g, fabs(p / pm1));
        int k = 0;
        const int ex = biased_exp(p);
        if (!is_zero(p) && (unsigned)(ex - (1023 - 200)) > 400u) {
            k = 1023 - ex;
            const double s = pow2i(k);
            p *= s;
            pm1 *= s;
        }
        K[(size_t)i * kstride] = k;
        pm2 = pm1;
        pm1 = p;
    }
    definite = ok;
    growth = g;
}

// One warp per block.  (1) Rough extremal eigenvalues of T by 16-point multisection with
// FP32 Sturm counts (lanes 0-15: lambda_1, lanes 16-31: lambda_n).  (2) Candidate root
// shifts mu_L = lambda_1 - delta and mu_R = lambda_n + delta, delta = max(4 n eps ||T||,
// 2 width); both FP64 factorizations are computed (lanes 0, 1).  When both are definite
// the end holding clearly more eigenvalues wins (a 5:4 majority of the Sturm count at the
// middle of the spectrum): shifting next to the dense part keeps its relative gaps large,
// so fewer eigenvalues cluster; otherwise the smaller element growth, ties to the left
// (definite factorizations have no large element growth either way).  If neither is
// definite delta doubles
// (at most 10 tries, then mu = gl - spdiam/8 which is always definite).  (3) The chosen
// factorization's primary data d, l are perturbed by relative amounts xi u, xi = 8 eps,
// u uniform in (-1, 1) from SplitMix64 (Alg. MRRR, perturbation of the root), and dl, dll
// are derived.
__global__ void k_root(int nblk, BlkDesc *blks, const double *__restrict__ D,
                       const double *__restrict__ E, double *pool0, float *f32,
                       unsigned long long seed) {
    const int b = blockIdx.x;
    const int lane = threadIdx.x;
    if (b >= nblk) return;
    BlkDesc B = blks[b];
    const int n = B.n;
    if (n <= 0) return;
    const double *d = D + B.off;
    const double *e = E + B.off;
    float *af = f32 + 2 * B.off;
    float *b2f = af + n;
    for (int i = lane; i < n; i += 32) {
        af[i] = (float)d[i];
        if (i < n - 1) { const float eb = (float)e[i]; b2f[i] = eb * eb; }
    }
    __syncwarp();
    const int half = lane >> 4, k = lane & 15;
    const int target = half ? n : 1;
    double L = B.gl, H = B.gu;
    for (int sweep = 0; sweep < 6; ++sweep) {
        const double x = L + (k + 1) * ((H - L) / 17.0);
        const int cnt = negcount_T_f32(n, af, b2f, (float)x);
        const unsigned bal = __ballot_sync(FULL_MASK, cnt < target);
        const unsigned hm = (bal >> (16 * half)) & 0xffffu;
        const int t = __popc(hm);
        const double xl = __shfl_sync(FULL_MASK, x, 16 * half + (t > 0 ? t - 1 : 0));
        const double xh = __shfl_sync(FULL_MASK, x, 16 * half + (t < 16 ? t : 15));
        if (t > 0) L = xl;
        if (t < 16) H = xh;
    }
    const double L1 = __shfl_sync(FULL_MASK, L, 0), H1 = __shfl_sync(FULL_MASK, H, 0);
    const double Ln = __shfl_sync(FULL_MASK, L, 16), Hn = __shfl_sync(FULL_MASK, H, 16);
    // eigenvalues below the middle of the spectrum (binary32 count, one lane)
    int cmid = 0;
    if (lane == 0) cmid = negcount_T_f32(n, af, b2f, (float)(0.5 * (L1 + Hn)));
    cmid = __shfl_sync(FULL_MASK, cmid, 0);
    const int pref = (4 * cmid > 5 * (n - cmid)) ? 0 : ((4 * (n - cmid) > 5 * cmid) ? 1 : -1);
    const double tn = fmax(fabs(B.gl), fabs(B.gu));
    // the single-precision counts are exact for T perturbed by ~eps_32 |T| entrywise
    const double d32 = 4.0 * 0x1p-24 * tn;
    double dL = fmax(fmax(4.0 * n * kEps * tn, 2.0 * (H1 - L1)), d32);
    double dR = fmax(fmax(4.0 * n * kEps * tn, 2.0 * (Hn - Ln)), d32);
    if (!(dL > 0.0)) dL = kSafmin;
    if (!(dR > 0.0)) dR = kSafmin;
    double *reg0 = pool0 + B.rep, *reg1 = reg0 + n, *reg2 = reg0 + 2 * n;
    int *K = (int *)reg2; // int2 per index: rescale exponents of the two candidates
    double mu = 0.0;
    const double *src = reg0;
    int kofs = 0;
    bool found = false;
    for (int tr = 0; tr < 10 && !found; ++tr) {
        const double muL = L1 - dL, muR = Hn + dR;
        bool ok = false;
        double g = 0.0;
        if (lane < 2)
            factor_root(n, d, e, lane == 0 ? muL : muR, lane == 0 ? reg0 : reg1, K + lane, 2,
                        lane == 0, ok, g);
        const int ok0 = __shfl_sync(FULL_MASK, (int)ok, 0), ok1 = __shfl_sync(FULL_MASK, (int)ok, 1);
        const double g0 = __shfl_sync(FULL_MASK, g, 0), g1 = __shfl_sync(FULL_MASK, g, 1);
        if (ok0 || ok1) {
            found = true;
            const bool left = (ok0 && ok1) ? (pref == 0 || (pref < 0 && g0 <= g1)) : (ok0 != 0);
            if (left) { mu = muL; src = reg0; kofs = 0; }
            else { mu = muR; src = reg1; kofs = 1; }
        } else {
            dL *= 2.0;
            dR *= 2.0;
        }
    }
    if (!found) {
        mu = B.gl - 0.125 * B.spdiam - kSafmin;
        bool ok;
        double g;
        if (lane == 0) factor_root(n, d, e, mu, reg0, K, 2, true, ok, g);
        src = reg0;
        kofs = 0;
    }
    __syncwarp();
    const double xi = 8.0 * kEps;
    // pivots d_i = p_i / (p_{i-1} 2^k_{i-1}), by chunks of 32 (the previous chunk's last p
    // and exponent carried in registers: the chunk's writes reuse the slots it read)
    double carry_p = 1.0;
    int carry_k = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const double pi = (i < n) ? src[i] : 1.0;
        const int ki = (i < n) ? K[2 * i + kofs] : 0;
        double pp = __shfl_up_sync(FULL_MASK, pi, 1);
        int kp = __shfl_up_sync(FULL_MASK, ki, 1);
        if (lane == 0) { pp = carry_p; kp = carry_k; }
        carry_p = __shfl_sync(FULL_MASK, pi, 31);
        carry_k = __shfl_sync(FULL_MASK, ki, 31);
        __syncwarp();
        if (i >= n) continue;
        const double pv = (pi / pp) * pow2i(-kp);
        const unsigned long long ctr = 2ull * (unsigned long long)(B.roff + i);
        const double dp = pv * (1.0 + xi * splitmix_pm1(seed, ctr));
        double dl = 0.0, dll = 0.0;
        if (i < n - 1) {
            const double l = e[i] / pv;
            const double lp = l * (1.0 + xi * splitmix_pm1(seed, ctr + 1));
            dl = dp * lp;
            dll = dl * lp;
        }
        reg0[i] = dp;
        reg1[i] = dl;
        reg2[i] = dll;
    }
    int dfexp;
    const bool dfok = df_write_copy_warp(n, reg0, reg2, (float4 *)(reg0 + rep_df_offset(n)), dfexp);
    __syncwarp();
    build_prefix(n, reg0);
    if (lane == 0) { blks[b].mu = mu; blks[b].dfok = dfok ? 1 : 0; blks[b].dfexp = dfexp; }
}

void launch_root(int nblk, BlkDesc *blks, const double *d, const double *e, double *pool0,
                 float *f32scratch, unsigned long long seed, cudaStream_t s) {
    if (nblk > 0) k_root<<<nblk, 32, 0, s>>>(nblk, blks, d, e, pool0, f32scratch, seed);
}

// ------------------------------------------------------------------ level 0 state

// Node b = block b.  Columns of the block: local index j0 + (c - col0).  The starting
// interval is the Gershgorin interval of the block shifted by mu, widened for the
// perturbation of the root (relative 8 eps per datum).
__global__ void k_init_columns(int nblk, const BlkDesc *__restrict__ blks, Node *nodes, int *cnode,
                               int *jloc, double *lo, double *hi) {
    const int b = blockIdx.x;
    if (b >= nblk) return;
    const BlkDesc B = blks[b];
    const int m = B.j1 >= B.j0 ? B.j1 - B.j0 + 1 : 0;
    if (threadIdx.x == 0) {
        Node N;
        N.rep = B.rep;
        N.blk = b;
        N.c0 = B.col0;
        N.c1 = B.col0 + m - 1;
        N.depth = 0;
        N.dfok = B.dfok;
        N.dfexp = B.dfexp;
        N.sigma = B.mu;
        N.lnb = -INFINITY;
        N.rnb = INFINITY;
        nodes[b] = N;
    }
    const double a = B.gl - B.mu, z = B.gu - B.mu;
    const double pad = 64.0 * (B.n + 1) * kEps * fmax(fabs(a), fabs(z)) + 4.0 * kSafmin;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        const int c = B.col0 + t;
        cnode[c] = b;
        jloc[c] = B.j0 + t;
        lo[c] = a - pad;
        hi[c] = z + pad;
    }
}

void launch_init_columns(int nblk, const BlkDesc *blks, Node *nodes, int *cnode, int *jloc,
                         double *lo, double *hi, int mtotal, cudaStream_t s) {
    (void)mtotal;
    if (nblk > 0) k_init_columns<<<nblk, 256, 0, s>>>(nblk, blks, nodes, cnode, jloc, lo, hi);
}

// For a subset (range != ALL) the eigenvalues j0-1 and j1+1 of each block bound the gaps
// of the node's end eigenvalues (relgap of an index set ranges over all j outside it).
// They are bisected on the root representation to classification accuracy; the node
// keeps the upper bound of lambda_{j0-1} in lnb and the lower bound of lambda_{j1+1}
// in rnb.
__global__ void k_outer_gaps(int nblk, const BlkDesc *__restrict__ blks, Node *nodes,
                             const double *__restrict__ pool0, double rtol) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = t >> 1, side = t & 1;
    if (b >= nblk) return;
    const BlkDesc B = blks[b];
    if (B.j1 < B.j0) return;
    const int j = side ? B.j1 + 1 : B.j0 - 1;
    if (j < 1 || j > B.n) return;
    const int n = B.n;
    const double *dd = pool0 + B.rep, *dll = dd + 2 * n;
    const double a = B.gl - B.mu, z = B.gu - B.mu;
    const double pad = 64.0 * (n + 1) * kEps * fmax(fabs(a), fabs(z)) + 4.0 * kSafmin;
    double l = a - pad, h = z + pad;
    for (int it = 0; it < 200; ++it) {
        const double w = h - l;
        if (!(w > fmax(rtol * fmax(fabs(l), fabs(h)), 4.0 * kSafmin))) break;
        const double mid = l + 0.5 * w;
        if (!(mid > l && mid < h)) break;
        if (negcount_ldl(n, dd, dll, mid) < j) l = mid; else h = mid;
    }
    if (side) nodes[b].rnb = l; else nodes[b].lnb = h;
}

void launch_outer_gaps(int nblk, const BlkDesc *blks, Node *nodes, const double *pool0,
                       double rtol, DevInfo *info, cudaStream_t s) {
    (void)info;
    if (nblk > 0) k_outer_gaps<<<(2 * nblk + 127) / 128, 128, 0, s>>>(nblk, blks, nodes, pool0, rtol);
}

// Zero the Z columns of matrices that split into several blocks (rows outside a block
// are zero in its eigenvectors).
__global__ void k_zero_z(int nmat, const MatDesc *__restrict__ mats, double *Z) {
    const int mi = blockIdx.y;
    if (mi >= nmat) return;
    const MatDesc M = mats[mi];
    if (M.nblk <= 1) return;
    const long long total = (long long)M.m * M.ldz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long col = i / M.ldz, row = i % M.ldz;
        if (row < M.n) Z[M.zoff + col * M.ldz + row] = 0.0;
    }
}

void launch_zero_z(int nmat, const MatDesc *mats, double *Z, cudaStream_t s) {
    if (nmat > 0) {
        dim3 g(64, nmat);
        k_zero_z<<<g, 256, 0, s>>>(nmat, mats, Z);
    }
}

cudaError_t preload_prologue() {
    return load_kernels(k_mat_norm, k_split_flags, k_scan_tiles, k_scan_sums, k_scan_add,
                        k_blocks_from_flags, k_blocks_finish, k_mat_blockcount, k_blk_setup,
                        k_index_multi, k_assign_columns, k_root, k_init_columns, k_outer_gaps,
                        k_zero_z);
}

} // namespace mr3
