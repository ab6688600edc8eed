// mr3_ddpath.cu -- the mixed-precision variant of Ch. 5 (opts->prec = MR3_DD): binary64
// input and output, the representation tree in double-double (eps_y ~ 2^-104).
//
// What changes against the binary64 path (everything else is shared):
//  * every representation carries a second plane of low-order words: the pool of a level
//    holds the leading words in the binary64 layout and, right behind it, the low words
//    at the same offsets (d, dl, dll);
//  * the root L D L^T = T - mu I is refactored in double-double (same mu, same random
//    perturbation factors) -- k_root_dd;
//  * each child representation is recomputed in double-double from its parent with the
//    shift tau the binary64 shift kernel selected -- k_shift_dd.  dstqds keeps the
//    off-diagonal of L D L^T, so dl+ = dl and dll+ = dl^2 / d+;
//  * eigenvalues are approximated on the leading words (the rounded copy M_x of Ch. 5,
//    "Arithmetic used to approximate eigenvalues"), safe while (k_rr + k_bi) n eps_x <~
//    gaptol, the default gaptol being 1e-10: in double-float down to its accuracy, then
//    in binary64;
//  * singletons get their eigenvectors from a twisted factorization and Rayleigh-quotient
//    iteration in double-double, stopped when the local residual is below
//    gap eps_x sqrt(n) (the relaxed criterion of Ch. 5, k_rs = 1) or the correction is at
//    double-double rounding level; the vector is rounded to binary64 when written to Z.
#include <float.h>
#include <algorithm>
#include "mr3_kernels.h"
#include "mr3_dd.cuh"
#include "mr3_df.cuh"

namespace mr3 {

namespace {

constexpr double kEpsY = 0x1p-104; // unit roundoff of the double-double working format

__device__ __forceinline__ ddouble dd_load(const double *h, const double *l, long long i) {
    return {__ldg(h + i), __ldg(l + i)};
}

// power-of-two factor bringing |x| back near 1 when it leaves [2^-400, 2^400]; 1 otherwise
__device__ __forceinline__ double rescale_factor(double x) {
    const int ex = biased_exp(x);
    if (is_zero(x) || (unsigned)(ex - (1023 - 400)) <= 800u) return 1.0;
    return pow2i(1023 - ex);
}

// ---------------------------------------------------------------- root representation

// One thread per block: L D L^T = T - mu I in double-double by the homogeneous three-term
// recurrence p_i = (alpha_i - mu) p_{i-1} - beta_{i-1}^2 p_{i-2}, d_i = p_i / p_{i-1},
// l_i = beta_i / d_i; then the perturbation factors of the binary64 root (the same
// SplitMix64 stream: 1 + xi u, xi = 8 eps) are applied to d_i and l_i.
__global__ void k_root_dd(int nblk, BlkDesc *blks, const double *__restrict__ D,
                          const double *__restrict__ E, double *pool0, double *pool0_lo,
                          unsigned long long seed) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    const BlkDesc B = blks[b];
    const int n = B.n;
    if (n <= 0) return;
    const double *d = D + B.off, *e = E + B.off;
    double *h0 = pool0 + B.rep, *l0 = pool0_lo + B.rep;
    const double mu = B.mu, xi = 8.0 * kEps;
    ddouble pm2 = dd_make(0.0), pm1 = dd_make(1.0);
    for (int i = 0; i < n; ++i) {
        ddouble a;
        dd_two_sum(__ldg(d + i), -mu, a.h, a.l);
        ddouble p = dd_mul(a, pm1);
        if (i > 0) {
            const double bi = __ldg(e + i - 1);
            p = dd_sub(p, dd_mul(dd_prod(bi, bi), pm2));
        }
        const ddouble piv = dd_div(p, pm1);
        const unsigned long long ctr = 2ull * (unsigned long long)(B.roff + i);
        const ddouble dp = dd_mul_d(piv, 1.0 + xi * splitmix_pm1(seed, ctr));
        ddouble dl = dd_make(0.0), dll = dd_make(0.0);
        if (i < n - 1) {
            const ddouble li = dd_div(dd_make(__ldg(e + i)), piv);
            const ddouble lp = dd_mul_d(li, 1.0 + xi * splitmix_pm1(seed, ctr + 1));
            dl = dd_mul(dp, lp);
            dll = dd_mul(dl, lp);
        }
        h0[i] = dp.h;          l0[i] = dp.l;
        h0[n + i] = dl.h;      l0[n + i] = dl.l;
        h0[2 * n + i] = dll.h; l0[2 * n + i] = dll.l;
        const double s = rescale_factor(p.h);
        if (s != 1.0) { p = dd_scale(p, s); pm1 = dd_scale(pm1, s); }
        pm2 = pm1;
        pm1 = p;
    }
    // the bisection's double-float copy is rewritten from these leading words
    int dfexp;
    const bool dfok = df_write_copy_serial(n, h0, h0 + 2 * n, (float4 *)(h0 + rep_df_offset(n)), dfexp);
    blks[b].dfok = dfok ? 1 : 0;
    blks[b].dfexp = dfexp;
}

// ---------------------------------------------------------------- child representations

// Substitute for an exactly zero pivot d_i + s_i of the divided recurrences below: a
// number 2^-120 times |d_i| (below the double-double roundoff, so the count is that of
// the limit), at least 2^-1000 so that it stays normal.
__device__ __forceinline__ double dd_tiny_pivot(double di) {
    return fmax(fabs(di) * 0x1p-120, 0x1p-1000);
}

// One thread per cluster: L+ D+ L+^T = L D L^T - tau I in double-double by the homogeneous
// dstqds recurrence c_i = d_i c_{i-1} + a_i, a_{i+1} = dll_i a_i - tau c_i (c_i is the
// product of the first i+1 pivots d+; (c, a) rescaled together by powers of two), with
// d+_i = c_i / c_{i-1} and dll+_i = dl_i^2 / d+_i off the recurrence's critical path.
__global__ void k_shift_dd(int ncluster, const ClusterItem *__restrict__ clusters,
                           const long long *__restrict__ cluster_rep, const Node *__restrict__ nodes,
                           const BlkDesc *__restrict__ blks, const double *__restrict__ pool,
                           const double *__restrict__ pool_lo, double *childpool,
                           double *childpool_lo, Node *child_nodes,
                           const double *__restrict__ child_tau, DevInfo *info) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncluster) return;
    const ClusterItem C = clusters[ci];
    const Node P = nodes[C.node];
    const int n = blks[P.blk].n;
    const double *ph = pool + P.rep, *pl = pool_lo + P.rep;
    double *ch = childpool + cluster_rep[ci], *cl = childpool_lo + cluster_rep[ci];
    const double tau = child_tau[ci];
    ddouble a = dd_make(-tau), cp = dd_make(1.0);
    for (int i = 0; i < n; ++i) {
        ddouble c = dd_add(dd_mul(dd_load(ph, pl, i), cp), a);
        if (is_zero(c.h)) c = dd_make(-cp.h * dd_tiny_pivot(ph[i]));
        const ddouble dp = dd_div(c, cp);
        ch[i] = dp.h;
        cl[i] = dp.l;
        if (i < n - 1) {
            const ddouble dl = dd_load(ph, pl, n + i);
            const ddouble dllp = dd_div(dd_mul(dl, dl), dp);
            ch[n + i] = dl.h;
            cl[n + i] = dl.l;
            ch[2 * n + i] = dllp.h;
            cl[2 * n + i] = dllp.l;
            a = dd_sub(dd_mul(dd_load(ph, pl, 2 * n + i), a), dd_mul_d(c, tau));
            const double s = rescale_factor(c.h);
            if (s != 1.0) { c = dd_scale(c, s); a = dd_scale(a, s); }
        } else {
            ch[n + i] = 0.0;     cl[n + i] = 0.0;
            ch[2 * n + i] = 0.0; cl[2 * n + i] = 0.0;
        }
        cp = c;
    }
    // the bisection's double-float copy, rewritten from this child's leading words
    int dfexp;
    const bool dfok = df_write_copy_serial(n, ch, ch + 2 * n, (float4 *)(ch + rep_df_offset(n)), dfexp);
    child_nodes[ci].dfok = dfok ? 1 : 0;
    child_nodes[ci].dfexp = dfexp;
    atomicAdd(&info->shift_steps, (unsigned long long)n);
}

// ---------------------------------------------------------------- singletons

// NegCount(L D L^T - sigma I) in double-double (dstqds with divisions; fallback only).
__device__ int negcount_dd(int n, const double *__restrict__ h, const double *__restrict__ l,
                           ddouble sigma) {
    ddouble s = dd_neg(sigma);
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        ddouble dp = dd_add(dd_load(h, l, i), s);
        if (is_zero(dp.h)) dp = dd_make(-dd_tiny_pivot(h[i]));
        cnt += dd_neg_sign(dp) ? 1 : 0;
        if (i < n - 1) s = dd_sub(dd_mul(dd_load(h, l, 2 * n + i), dd_div(s, dp)), sigma);
    }
    return cnt;
}

// Per-thread scratch: four doubles per index (l+ and, first s then u-), interleaved over the
// launch's T threads so that a warp's accesses at one index are contiguous.
struct DDScratch {
    double *base;
    long long T;
    __device__ double &at(int i, int q) const { return base[((long long)i * 4 + q) * T]; }
};

// One thread per singleton (persistent over T threads).  Alg. Getvec in double-double:
//   forward  (dstqds):  d+_i = d_i + s_i, l+_i = dl_i / d+_i, s_{i+1} = dll_i s_i / d+_i - lam
//   backward (dqds):    r_{i+1} = dll_i + p_{i+1}, u-_i = dl_i / r_{i+1},
//                       p_i = p_{i+1} d_i / r_{i+1} - lam
//   gamma_i = s_i + p_i + lam, twist r = argmin |gamma_i|, z_r = 1,
//   z_i = -l+_i z_{i+1} (i < r), z_{i+1} = -u-_i z_i (i >= r), carried in double-double and
//   rounded to binary64 as written into Z.
// S-task acceptance (Ch. 5): |gamma_r| / ||z|| <= gap eps_x sqrt(n), or a Rayleigh
// correction gamma_r / ||z||^2 below 4 eps_y |lam|.  Otherwise lam += correction while it
// stays inside the Sturm bracket [l, h] (updated from the forward count), else bisection in
// double-double to full accuracy and one more Getvec.  The eigenvalue written to w is the
// Rayleigh quotient of the rounded unit vector with respect to the input T.
__global__ void __launch_bounds__(128) k_rqi_dd(
    int nsingle, const SingleItem *__restrict__ singles, const Node *__restrict__ nodes,
    const BlkDesc *__restrict__ blks, const MatDesc *__restrict__ mats,
    const double *__restrict__ pool, const double *__restrict__ pool_lo,
    const int *__restrict__ jloc, const double *__restrict__ lo, const double *__restrict__ hi,
    const double *__restrict__ gapl, const double *__restrict__ gapr,
    const double *__restrict__ Din, const double *__restrict__ Ein, double *w, double *Z,
    double *scratch, int max_rqi, unsigned fault_mask, DevInfo *info) {
    const long long T = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    DDScratch S{scratch + tid, T};
    unsigned long long steps = 0, iters = 0;
    int itmax = 0, nfb = 0, ncap = 0;
    for (long long idx = tid; idx < nsingle; idx += T) {
        const SingleItem it = singles[idx];
        const int c = it.col;
        const Node N = nodes[it.node];
        const BlkDesc B = blks[N.blk];
        const MatDesc M = mats[B.mat];
        const int n = B.n;
        const double *Rh = pool + N.rep, *Rl = pool_lo + N.rep;
        const int j = jloc[c];
        double l = lo[c], h = hi[c];
        double gap = fmin(gapl[c], gapr[c]);
        if (!(gap > 0.0)) gap = kSafmin;
        double *zc = Z + M.zoff + (long long)(c - M.woff) * M.ldz + B.roff;
        const double tol1 = sqrt((double)n) * kEps;
        ddouble lam = dd_make(l + 0.5 * (h - l));
        bool fb = false, capped = false;
        int it_n = 0, imax = 0;
        double nrm2 = 1.0;
        for (int guard = 0; guard < 64; ++guard) {
            // ---- forward (one reciprocal of d+_i serves l+_i and the next s)
            ddouble s = dd_neg(lam);
            int negc = 0;
            for (int i = 0; i < n - 1; ++i) {
                ddouble dp = dd_add(dd_load(Rh, Rl, i), s);
                if (is_zero(dp.h)) dp = dd_make(-dd_tiny_pivot(Rh[i]));
                negc += dd_neg_sign(dp) ? 1 : 0;
                const ddouble rdp = dd_rcp(dp);
                const ddouble lp = dd_mul(dd_load(Rh, Rl, n + i), rdp);
                S.at(i, 0) = lp.h;
                S.at(i, 1) = lp.l;
                S.at(i, 2) = s.h;
                S.at(i, 3) = s.l;
                s = dd_sub(dd_mul(dd_mul(dd_load(Rh, Rl, 2 * n + i), s), rdp), lam);
            }
            {
                ddouble dp = dd_add(dd_load(Rh, Rl, n - 1), s);
                if (is_zero(dp.h)) dp = dd_make(-dd_tiny_pivot(Rh[n - 1]));
                negc += dd_neg_sign(dp) ? 1 : 0;
            }
            // ---- backward, gamma and the twist index
            ddouble p = dd_sub(dd_load(Rh, Rl, n - 1), lam);
            ddouble gam = dd_add(dd_add(s, p), lam);
            int r = n - 1;
            double agmin = fabs(gam.h);
            for (int i = n - 2; i >= 0; --i) {
                ddouble rr = dd_add(dd_load(Rh, Rl, 2 * n + i), p);
                if (is_zero(rr.h)) rr = dd_make(dd_tiny_pivot(Rh[2 * n + i]));
                const ddouble rrr = dd_rcp(rr);
                const ddouble um = dd_mul(dd_load(Rh, Rl, n + i), rrr);
                const ddouble x = dd_mul(dd_mul(p, dd_load(Rh, Rl, i)), rrr); // p_i + lam
                p = dd_sub(x, lam);
                const ddouble si = {S.at(i, 2), S.at(i, 3)};
                const ddouble g = dd_add(si, x); // gamma_i = s_i + p_i + lam
                S.at(i, 2) = um.h;
                S.at(i, 3) = um.l;
                if (fabs(g.h) < agmin) { agmin = fabs(g.h); gam = g; r = i; }
            }
            steps += 3ull * n;
            // ---- solve, z written to Z in binary64
            double ss = 1.0, zmax = 1.0;
            imax = r;
            zc[r] = 1.0;
            {
                ddouble z = dd_make(1.0), z2 = dd_make(0.0); // z_{i+1}, z_{i+2}
                for (int i = r - 1; i >= 0; --i) {
                    ddouble zi;
                    if (z.h != 0.0) {
                        zi = dd_neg(dd_mul(ddouble{S.at(i, 0), S.at(i, 1)}, z));
                    } else {
                        // zero-pivot rule of Alg. Getvec: z_i = -(dl_{i+1} / dl_i) z_{i+2}
                        zi = dd_neg(dd_mul(dd_div(dd_load(Rh, Rl, n + i + 1), dd_load(Rh, Rl, n + i)), z2));
                    }
                    zc[i] = zi.h;
                    ss = fma(zi.h, zi.h, ss);
                    if (fabs(zi.h) > zmax) { zmax = fabs(zi.h); imax = i; }
                    z2 = z;
                    z = zi;
                }
            }
            {
                ddouble z = dd_make(1.0), z2 = dd_make(0.0); // z_{i-1}, z_{i-2}
                for (int i = r + 1; i < n; ++i) {
                    ddouble zi;
                    if (z.h != 0.0) {
                        zi = dd_neg(dd_mul(ddouble{S.at(i - 1, 2), S.at(i - 1, 3)}, z));
                    } else {
                        zi = dd_neg(dd_mul(dd_div(dd_load(Rh, Rl, n + i - 2), dd_load(Rh, Rl, n + i - 1)), z2));
                    }
                    zc[i] = zi.h;
                    ss = fma(zi.h, zi.h, ss);
                    if (fabs(zi.h) > zmax) { zmax = fabs(zi.h); imax = i; }
                    z2 = z;
                    z = zi;
                }
            }
            nrm2 = ss;
            if (fb) break;
            ++it_n;
            if (negc >= j) h = fmin(h, lam.h); else l = fmax(l, lam.h);
            const double resid = fabs(gam.h) / sqrt(nrm2);
            const ddouble rqc = dd_div(gam, dd_make(nrm2));
            const bool conv = resid <= tol1 * gap || fabs(rqc.h) <= 4.0 * kEpsY * fabs(lam.h);
            const bool nofault = !(fault_mask & MR3_FAULT_RQI_NOCONV);
            if (conv && nofault) break;
            const ddouble lnew = dd_add(lam, rqc);
            const bool sign_ok = (negc < j) ? (rqc.h > 0.0) : (rqc.h < 0.0);
            if (nofault && it_n < max_rqi && sign_ok && lnew.h >= l && lnew.h <= h) {
                lam = lnew;
                continue;
            }
            if (it_n >= max_rqi) capped = true;
            // ---- bisection in double-double on a verified bracket, then one more Getvec
            ddouble bl = dd_make(l), bh = dd_make(h);
            const double wid0 = fmax(h - l, 4.0 * kEps * fmax(fabs(l), fabs(h)) + 4.0 * kSafmin);
            for (int t = 0; t < 60 && negcount_dd(n, Rh, Rl, bl) >= j; ++t)
                bl = dd_add_d(bl, -ldexp(wid0, t));
            for (int t = 0; t < 60 && negcount_dd(n, Rh, Rl, bh) < j; ++t)
                bh = dd_add_d(bh, ldexp(wid0, t));
            for (int t = 0; t < 400; ++t) {
                const ddouble wd = dd_sub(bh, bl);
                if (!(wd.h > 4.0 * kEpsY * fmax(fabs(bl.h), fabs(bh.h)) + 4.0 * kSafmin)) break;
                const ddouble mid = dd_add(bl, dd_mul_d(wd, 0.5));
                steps += n;
                if (negcount_dd(n, Rh, Rl, mid) < j) bl = mid; else bh = mid;
            }
            lam = dd_add(bl, dd_mul_d(dd_sub(bh, bl), 0.5));
            fb = true;
        }
        // ---- normalise (an entry of largest magnitude positive) and the Rayleigh quotient
        const double scale = ((zc[imax] < 0.0) ? -1.0 : 1.0) / sqrt(nrm2);
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
    if (steps) atomicAdd(&info->twisted_steps, steps);
    if (iters) atomicAdd(&info->rqi_iters, iters);
    if (itmax) atomicMax(&info->rqi_max, itmax);
    if (nfb) atomicAdd(&info->fallbacks, nfb);
    if (ncap) atomicAdd(&info->status[MR3_SCAP], ncap);
}

} // namespace

void launch_root_dd(int nblk, BlkDesc *blks, const double *d, const double *e, double *pool0,
                    double *pool0_lo, unsigned long long seed, cudaStream_t s) {
    if (nblk <= 0) return;
    k_root_dd<<<(nblk + 31) / 32, 32, 0, s>>>(nblk, blks, d, e, pool0, pool0_lo, seed);
}

void launch_shift_dd(int ncluster, const ClusterItem *clusters, const long long *cluster_rep,
                     const Node *nodes, const BlkDesc *blks, const double *pool,
                     const double *pool_lo, double *childpool, double *childpool_lo,
                     Node *child_nodes, const double *child_tau, DevInfo *info, cudaStream_t s) {
    if (ncluster <= 0) return;
    k_shift_dd<<<(ncluster + 31) / 32, 32, 0, s>>>(ncluster, clusters, cluster_rep, nodes, blks,
                                                  pool, pool_lo, childpool, childpool_lo,
                                                  child_nodes, child_tau, info);
}

// Threads of a singleton launch: one per singleton, rounded up to whole blocks of 128,
// within the scratch budget (the launch then loops over the singletons).
long long rqi_dd_threads(long long nsingle, int nmax, long long cap_bytes) {
    const long long per = 4ll * nmax * (long long)sizeof(double);
    const long long cap = std::max<long long>(128, (cap_bytes / per) / 128 * 128);
    return std::min<long long>((nsingle + 127) / 128 * 128, cap);
}

void launch_rqi_dd(int nsingle, const SingleItem *singles, const Node *nodes, const BlkDesc *blks,
                   const MatDesc *mats, const double *pool, const double *pool_lo, const int *jloc,
                   const double *lo, const double *hi, const double *gapl, const double *gapr,
                   const double *d, const double *e, double *w, double *Z, double *scratch,
                   long long nthreads, int max_rqi, unsigned fault_mask, DevInfo *info,
                   cudaStream_t s) {
    if (nsingle <= 0 || nthreads <= 0) return;
    // The kernel is bound by the binary64 pipe of the SMs it runs on: spread the singletons
    // over all 152 SMs (blocks of ceil(nsingle / 152) threads, at most 128).  Scratch holds
    // 4 nmax doubles for each of nthreads threads; the grid uses at most that many and loops
    // over the singletons.
    const long long per_sm = (nsingle + 151) / 152;
    const int bs = (int)std::max<long long>(1, std::min<long long>({128, per_sm, nthreads}));
    const long long need = (nsingle + bs - 1) / bs;
    const unsigned nb = (unsigned)std::min<long long>(need, nthreads / bs);
    k_rqi_dd<<<nb, bs, 0, s>>>(nsingle, singles, nodes, blks, mats, pool, pool_lo, jloc, lo,
                                     hi, gapl, gapr, d, e, w, Z, scratch, max_rqi, fault_mask,
                                     info);
}

} // namespace mr3
