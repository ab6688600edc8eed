// mr3_rqi.cu -- eigenpairs of well-separated eigenvalues (singletons): Rayleigh quotient
// iteration on the twisted factorizations of Alg. Getvec, guarded by bisection
// (Alg. S-task and the remarks after Alg. Getvec, Sec. 3.2.3).
#include <float.h>
#include "mr3_kernels.h"

namespace mr3 {

#define FULL_MASK 0xffffffffu

// Per-thread scratch with the 32 lanes of a warp interleaved, so that the accesses of a
// warp at step i are contiguous: per index five 256-byte rows (a_i, c_{i-1}, h_i,
// d_i f_{i+1}, and the two scale exponents as an int2).
struct Scratch {
    double *base;
    __device__ __forceinline__ double &A(int i) const { return base[(size_t)i * 160]; }
    __device__ __forceinline__ double &C(int i) const { return base[(size_t)i * 160 + 32]; }
    __device__ __forceinline__ double &H(int i) const { return base[(size_t)i * 160 + 64]; }
    __device__ __forceinline__ double &Q(int i) const { return base[(size_t)i * 160 + 96]; }
    __device__ __forceinline__ int2 &E(int i) const { return *(int2 *)(base + (size_t)i * 160 + 128); }
};
constexpr int kScratchPerIndex = 160; // doubles per index per warp slot

// Rescale (x, y) by 2^k so that |x| is near 1 when x leaves [2^-200, 2^200]; returns k.
__device__ __forceinline__ int rescale2(double &x, double &y) {
    const int ex = biased_exp(x);
    if ((unsigned)(ex - (1023 - 200)) > 400u && !is_zero(x)) {
        const int k = 1023 - ex;
        const double sc = pow2i(k);
        x *= sc;
        y *= sc;
        return k;
    }
    return 0;
}

// x * 2^e for a double x and an int e of any size (saturating to 0 / inf).
__device__ __forceinline__ double scale2(double x, int e) {
    if (e > 1023) { x *= pow2i(1023); e -= 1023; if (e > 1023) e = 1023; }
    else if (e < -1022) { x *= pow2i(-1022); e += 1022; if (e < -1022) return 0.0 * x; }
    return x * pow2i(e);
}

// Approximate log2 |x| as a float (exponent field plus log2 of the mantissa): enough to
// rank the |gamma_k| of the twist-index search without an FP64 division or compare.
__device__ __forceinline__ float log2abs(double x) {
    const long long b = __double_as_longlong(x) & 0x7fffffffffffffffll;
    if (b == 0) return -4096.f;
    const int ex = (int)(b >> 52);
    const float mant = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff)); // [1, 2)
    return (float)(ex - 1023) + __log2f(mant);
}

// Getvec (Alg. Getvec) for L D L^T - lam I without divisions in the recurrences.
// With the homogeneous variables of the Sturm count (see negcount_ldl),
//   forward  (dstqds):  c_i = d_i c_{i-1} + a_i,      a_{i+1} = dll_i a_i - lam c_i,
//                       d+_i = c_i / c_{i-1},          s_i = a_i / c_{i-1};
//   backward (dqds, read as in the design notes: omega-_{i+1} = p_{i+1} + dll_i):
//                       h_i = dll_i h_{i+1} + f_{i+1}, f_i = d_i f_{i+1} - lam h_i,
//                       omega-_{i+1} = h_i / h_{i+1},  p_i = f_i / h_i,
// started from c_{-1} = 1, a_0 = -lam, h_{n-1} = 1, f_{n-1} = d_{n-1} - lam.  Then
//   gamma_i = s_i + d_i p_{i+1}/omega-_{i+1} = (a_i h_i + c_{i-1} d_i f_{i+1}) / (c_{i-1} h_i),
//   gamma_{n-1} = d+_{n-1},
// where numerator and denominator share one scale.  The twisted solve N_r^T z = e_r,
// z_i = -l+_i z_{i+1} (i < r), z_{i+1} = -u-_i z_i (i >= r), with l+_i = dl_i c_{i-1}/c_i and
// u-_i = dl_i h_{i+1}/h_i, telescopes to
//   z_i = c_{i-1}/c_{r-1} prod_{k=i}^{r-1} (-dl_k)   (i < r),
//   z_i = h_i/h_r prod_{k=r}^{i-1} (-dl_k)           (i > r),
// which also covers the zero-pivot rule of Alg. Getvec without a special case.  (a, c)
// and (f, h) carry power-of-two scales tracked as integer exponents.
// Pass 1 runs the forward and backward recurrences interleaved (two independent chains),
// pass 2 ranks |gamma_i| in the log domain (full factorization only), pass 3 solves
// outward from r in both directions at once.
//  r < 0 : full factorization, r = argmin |gamma_i|; the count is NegCount(LDL^T, lam).
//  r >= 0: only the twisted factorization at r; the count is the inertia of
//          diag(d+_0..d+_{r-1}, gamma_r, omega-_{r+1}..omega-_{n-1}).
__device__ void getvec_h(int n, const double *__restrict__ d, const double *__restrict__ dl,
                         const double *__restrict__ dll, double lam, int &r, const Scratch &S,
                         double *zc, double &gamma, double &nrm2, int &negc, int &imax,
                         unsigned long long &steps) {
    const bool full = r < 0;
    const bool need_last = full || r == n - 1;  // c_{n-1} (gamma_{n-1}) needed
    const int fend = full ? n - 1 : r;            // forward stores indices 0..fend
    const int blow = full ? 0 : r;                // backward computes h_i for blow..n-2
    // ---- pass 1: forward (index i = t) and backward (index n-2-t) interleaved
    double a = -lam, cp = 1.0;
    int F = 0, sp = 0, cntf = 0;
    double c_last = 1.0, cprev_last = 1.0;
    double f = __ldg(d + n - 1) - lam, h = 1.0;
    int G = 0, sh = 0, cntb = 0;
    const int nf = fend + 1, nb = n - 1 - blow;
    const int T = max(nf, nb);
    for (int t = 0; t < T; ++t) {
        if (t < nf) {
            const int i = t;
            S.A(i) = a;
            S.C(i) = cp;
            S.E(i).x = F;
            if (i < fend || need_last) {
                double c = fma(__ldg(d + i), cp, a);
                if (is_zero(c)) c = -cp * 0x1p-80;
                const int sc = sign_bit(c);
                if (full || i < r) cntf += sc ^ sp;
                if (i == n - 1) {
                    c_last = c;
                    cprev_last = cp;
                } else {
                    const double tt = __ldg(dll + i) * a;
                    a = fma(-lam, c, tt);
                    F -= rescale2(c, a);
                    cp = c;
                    sp = sc;
                }
            }
        }
        if (t < nb) {
            const int i = n - 2 - t;
            double hi = fma(__ldg(dll + i), h, f);
            if (is_zero(hi)) hi = -h * 0x1p-80;
            const int sgh = sign_bit(hi);
            cntb += sgh ^ sh; // omega-_{i+1} = h_i / h_{i+1}
            const double df = __ldg(d + i) * f;
            f = fma(-lam, hi, df);
            S.H(i) = hi;
            S.Q(i) = df;
            S.E(i).y = G;
            G -= rescale2(hi, f);
            h = hi;
            sh = sgh;
        }
    }
    steps += (unsigned long long)(nf + nb);
    // ---- pass 2: gamma and the twist index
    double gnum, gden;
    int cnt;
    if (full) {
        float best = log2abs(c_last) - log2abs(cprev_last);
        if (!(best == best)) best = 3.0e38f;
        int rr = n - 1;
#pragma unroll 4
        for (int i = 0; i < n - 1; ++i) {
            const double ci = S.C(i), hi = S.H(i);
            const double num = fma(S.A(i), hi, ci * S.Q(i));
            const float key = log2abs(num) - log2abs(ci * hi);
            if (key <= best) {
                if (key < best || i < rr) rr = i;
                best = key;
            }
        }
        r = rr;
        cnt = cntf;
    } else {
        cnt = cntf + cntb;
    }
    if (r == n - 1) {
        gnum = c_last;
        gden = cprev_last;
    } else {
        const double ci = S.C(r), hi = S.H(r);
        gnum = fma(S.A(r), hi, ci * S.Q(r));
        gden = ci * hi;
    }
    gamma = gnum / gden;
    if (!full) cnt += sign_bit(gamma);
    negc = cnt;
    // ---- pass 3: solve N_r^T z = e_r (z_r = 1), both directions at once
    const int rf = S.E(r).x;                               // scale of c_{r-1}
    const double icr = 1.0 / S.C(r);                        // 1 / c_{r-1} (stored)
    const double ihr = (r < n - 1) ? 1.0 / S.H(r) : 1.0;    // 1 / h_r (stored)
    const int rg = (r < n - 1) ? S.E(r).y : 0;
    zc[r] = 1.0;
    double ss0 = 1.0, ss1 = 0.0;
    long long zmaxb = 0x3ff0000000000000ll; // bits of 1.0
    int im = r;
    double Pd = 1.0, Pu = 1.0;
    int EPd = 0, EPu = 0;
    const int ndown = r, nup = n - 1 - r;
    const int T3 = max(ndown, nup);
    for (int t = 0; t < T3; ++t) {
        if (t < ndown) {
            const int i = r - 1 - t;
            Pd *= -__ldg(dl + i);
            if ((unsigned)(biased_exp(Pd) - (1023 - 200)) > 400u && !is_zero(Pd)) {
                const int k = 1023 - biased_exp(Pd);
                Pd *= pow2i(k);
                EPd -= k;
            }
            const double zi = scale2(Pd * S.C(i) * icr, EPd + S.E(i).x - rf);
            zc[i] = zi;
            ss0 = fma(zi, zi, ss0);
            const long long zb = __double_as_longlong(zi) & 0x7fffffffffffffffll;
            if (zb > zmaxb) { zmaxb = zb; im = i; }
        }
        if (t < nup) {
            const int i = r + 1 + t;
            Pu *= -__ldg(dl + i - 1);
            if ((unsigned)(biased_exp(Pu) - (1023 - 200)) > 400u && !is_zero(Pu)) {
                const int k = 1023 - biased_exp(Pu);
                Pu *= pow2i(k);
                EPu -= k;
            }
            const double hh = (i < n - 1) ? S.H(i) : 1.0;
            const int gi = (i < n - 1) ? S.E(i).y : 0;
            const double zi = scale2(Pu * hh * ihr, EPu + gi - rg);
            zc[i] = zi;
            ss1 = fma(zi, zi, ss1);
            const long long zb = __double_as_longlong(zi) & 0x7fffffffffffffffll;
            if (zb > zmaxb || (zb == zmaxb && i < im)) { zmaxb = zb; im = i; }
        }
    }
    nrm2 = ss0 + ss1;
    imax = im;
    steps += (unsigned long long)n;
}

// Persistent kernel: each warp takes 32 consecutive singletons at a time.  Per singleton
// (Alg. S-task): lam = midpoint of [lo, hi]; repeat Getvec; update [lo, hi] from the count;
// accept when |gamma_r|/||z|| < tol1 gap (tol1 = n eps, gap = distance to the nearest
// other eigenvalue) or |gamma_r|/||z||^2 < tol2 |lam| (tol2 = 2 eps); otherwise apply the
// Rayleigh quotient correction gamma_r/||z||^2 when its sign points toward the eigenvalue
// and the result stays in [lo, hi]; else (or after max_rqi Getvecs) bisect to full
// accuracy and accept after one more Getvec.  The eigenvalue returned is the Rayleigh
// quotient lam + gamma_r/||z||^2 (when inside [lo, hi]) plus the node's shift sigma; z is
// normalised with its largest entry positive.
__global__ void __launch_bounds__(32) k_rqi(int nsingle, const SingleItem *__restrict__ singles,
                                             const Node *__restrict__ nodes,
                                             const BlkDesc *__restrict__ blks,
                                             const MatDesc *__restrict__ mats,
                                             const double *__restrict__ pool,
                                             const int *__restrict__ jloc,
                                             const double *__restrict__ lo,
                                             const double *__restrict__ hi,
                                             const double *__restrict__ gapl,
                                             const double *__restrict__ gapr,
                                             const double *__restrict__ Din,
                                             const double *__restrict__ Ein, double *w, double *Z,
                                             double *scratch, int nmax, int max_rqi,
                                             unsigned fault_mask, int *work_counter, int lanes,
                                             DevInfo *info) {
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    Scratch S;
    S.base = scratch + (size_t)slot * kScratchPerIndex * (size_t)nmax + lane;
    unsigned long long steps = 0, iters = 0;
    int itmax = 0, nfb = 0, ncap = 0;
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(work_counter, lanes);
        chunk = __shfl_sync(FULL_MASK, chunk, 0);
        if (chunk >= nsingle) break;
        const int idx = chunk + lane;
        if (lane < lanes && idx < nsingle) {
            const SingleItem it = singles[idx];
            const int c = it.col;
            const Node N = nodes[it.node];
            const BlkDesc B = blks[N.blk];
            const MatDesc M = mats[B.mat];
            const int n = B.n;
            const double *d = pool + N.rep, *dl = d + n, *dll = d + 2 * n;
            const int j = jloc[c];
            double l = lo[c], h = hi[c];
            double gap = fmin(gapl[c], gapr[c]);
            if (!(gap > 0.0)) gap = kSafmin;
            double *zc = Z + M.zoff + (long long)(c - M.woff) * M.ldz + B.roff;
            const double tol1 = n * kEps, tol2 = 4.0 * kEps, tol_noise = n * kEps;
            double lam = l + 0.5 * (h - l);
            int r = -1, it_n = 0;
            bool fb = false, capped = false;
            double gamma = 0.0, nrm2 = 1.0, rqc = 0.0;
            int negc = 0, imax = 0;
            double prev_arqc = INFINITY;
            for (int guard = 0; guard < 64; ++guard) {
                getvec_h(n, d, dl, dll, lam, r, S, zc, gamma, nrm2, negc, imax, steps);
                ++it_n;
                if (negc >= j) h = fmin(h, lam); else l = fmax(l, lam);
                const double nz = sqrt(nrm2);
                const double resid = fabs(gamma) / nz;
                rqc = gamma / nrm2;
                const bool conv = (resid < tol1 * gap) || (fabs(rqc) < tol2 * fabs(lam));
                // RQI converges cubically; a correction that no longer shrinks (at least by
                // half) while tiny against the gap sits at the representation's noise level
                const bool stalled = it_n >= 2 && fabs(rqc) >= 0.5 * prev_arqc &&
                                     fabs(rqc) <= 1e-3 * gap;
                if (fb || ((conv || stalled) && !(fault_mask & MR3_FAULT_RQI_NOCONV))) break;
                prev_arqc = fabs(rqc);
                const bool sign_ok = (negc < j) ? (rqc > 0.0) : (rqc < 0.0);
                const double lnew = lam + rqc;
                if (it_n < max_rqi && sign_ok && lnew >= l && lnew <= h) {
                    lam = lnew;
                    continue;
                }
                // A correction at the level of the rounding noise of the twisted
                // factorization (|rqc| <= n eps |lam|) cannot improve lam: accept.
                if (!(fault_mask & MR3_FAULT_RQI_NOCONV) && fabs(rqc) <= tol_noise * fabs(lam)) break;
                if (it_n >= max_rqi) capped = true;
                // bisection to full accuracy, then one more Getvec
                for (int k = 0; k < 2100; ++k) {
                    const double wd = h - l;
                    if (!(wd > fmax(4.0 * kEps * fmax(fabs(l), fabs(h)), 4.0 * kSafmin))) break;
                    const double mid = l + 0.5 * wd;
                    if (!(mid > l && mid < h)) break;
                    steps += n;
                    if (negcount_ldl(n, d, dll, mid) < j) l = mid; else h = mid;
                }
                lam = l + 0.5 * (h - l);
                r = -1;
                fb = true;
            }
            // Normalise (largest entry positive) and return the Rayleigh quotient of z with
            // respect to the input T (accuracy remark 5 of Sec. 3.1.2): it removes the bias
            // of the root's random perturbation and minimises ||T z - w z||.
            const double zsign = (zc[imax] < 0.0) ? -1.0 : 1.0;
            const double scale = zsign / sqrt(nrm2);
            const double *td = Din + B.off, *te = Ein + B.off;
            double rq = 0.0, zprev = 0.0;
            for (int i = 0; i < n; ++i) {
                const double zi = zc[i] * scale;
                zc[i] = zi;
                rq = fma(__ldg(td + i) * zi, zi, rq);
                if (i > 0) rq = fma(2.0 * __ldg(te + i - 1) * zprev, zi, rq);
                zprev = zi;
            }
            w[c] = rq;
            iters += it_n;
            itmax = max(itmax, it_n);
            nfb += fb ? 1 : 0;
            ncap += capped ? 1 : 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        steps += __shfl_xor_sync(FULL_MASK, steps, o);
        iters += __shfl_xor_sync(FULL_MASK, iters, o);
        itmax = max(itmax, __shfl_xor_sync(FULL_MASK, itmax, o));
        nfb += __shfl_xor_sync(FULL_MASK, nfb, o);
        ncap += __shfl_xor_sync(FULL_MASK, ncap, o);
    }
    if (lane == 0) {
        if (steps) atomicAdd(&info->twisted_steps, steps);
        if (iters) atomicAdd(&info->rqi_iters, iters);
        atomicMax(&info->rqi_max, itmax);
        if (nfb) atomicAdd(&info->fallbacks, nfb);
        if (ncap) atomicAdd(&info->status[MR3_SCAP], ncap);
    }
}

// One warp per block so that the warps spread over all SMs (each SM has only two FP64
// FMA lanes per clock); with few singletons a warp takes 8 or 16 of them instead of 32.
void launch_rqi(int nsingle, const SingleItem *singles, const Node *nodes, const BlkDesc *blks,
                const MatDesc *mats, const double *pool, const int *jloc, const double *lo,
                const double *hi, const double *gapl, const double *gapr, const double *d,
                const double *e, double *w, double *Z, double *scratch, int nslots, int nmax,
                int max_rqi, unsigned fault_mask, int *work_counter, DevInfo *info,
                cudaStream_t s) {
    if (nsingle <= 0) return;
    int lanes = 32;
    while (lanes > 8 && (long long)nsingle < (long long)lanes * 2 * 152) lanes >>= 1;
    const int want = (nsingle + lanes - 1) / lanes;
    const int nblocks = want < nslots ? want : nslots;
    cudaMemsetAsync(work_counter, 0, sizeof(int), s);
    k_rqi<<<nblocks, 32, 0, s>>>(nsingle, singles, nodes, blks, mats, pool, jloc, lo, hi, gapl,
                                 gapr, d, e, w, Z, scratch, nmax, max_rqi, fault_mask,
                                 work_counter, lanes, info);
}

} // namespace mr3
