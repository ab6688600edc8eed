// mr3_rqi.cu -- eigenpairs of well-separated eigenvalues (singletons): Rayleigh quotient
// iteration on the twisted factorizations of Alg. Getvec, guarded by bisection
// (Alg. S-task and the remarks after Alg. Getvec, Sec. 3.2.3).
#include <float.h>
#include "mr3_kernels.h"

namespace mr3 {

#define FULL_MASK 0xffffffffu

// A team of TEAM lanes finishes one singleton; a warp holds 32 / TEAM teams.  Lanes 0 and 1
// of a team run the two serial recurrences of a twisted factorization, after which all
// lanes of the team share the element-wise work (twist index, solve, normalisation).
// Teams of 8 keep a singleton's element-wise passes short (levels with few singletons are
// latency bound); teams of 2 fill 4x more lanes of every binary64 instruction in the
// recurrences, which wins when singletons far outnumber the resident warps (the binary64
// pipe costs the same per warp instruction whatever the number of active lanes).
constexpr int kScratchPerSingleton = 5; // doubles per index per singleton

// Scratch of one team: per index five values (a_i, c_{i-1}, h_i, d_i f_{i+1}, and the two
// scale exponents as an int2), interleaved with the other teams of the warp.
template <int TEAMS> struct Scratch {
    static constexpr int kSPI = kScratchPerSingleton * TEAMS; // doubles per index per warp slot
    double *base; // warp slot base + team
    __device__ __forceinline__ double &A(int i) const { return base[(size_t)i * kSPI]; }
    __device__ __forceinline__ double &C(int i) const { return base[(size_t)i * kSPI + TEAMS]; }
    __device__ __forceinline__ double &H(int i) const { return base[(size_t)i * kSPI + 2 * TEAMS]; }
    __device__ __forceinline__ double &Q(int i) const { return base[(size_t)i * kSPI + 3 * TEAMS]; }
    __device__ __forceinline__ int2 &E(int i) const { return *(int2 *)(base + (size_t)i * kSPI + 4 * TEAMS); }
};

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

// Reductions over the TEAM lanes of a team (all 32 lanes call them together).
template <int TEAM> __device__ __forceinline__ double team_sum(double v) {
    for (int o = TEAM / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, TEAM);
    return v;
}
template <int TEAM> __device__ __forceinline__ void team_argmin(float &key, int &idx) {
    for (int o = TEAM / 2; o > 0; o >>= 1) {
        const float k2 = __shfl_xor_sync(0xffffffffu, key, o, TEAM);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o, TEAM);
        if (k2 < key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
    }
}
template <int TEAM> __device__ __forceinline__ void team_argmax_bits(long long &b, int &idx) {
    for (int o = TEAM / 2; o > 0; o >>= 1) {
        const long long b2 = __shfl_xor_sync(0xffffffffu, b, o, TEAM);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o, TEAM);
        if (b2 > b || (b2 == b && i2 < idx)) { b = b2; idx = i2; }
    }
}

// Persistent kernel (one warp per block; each team takes one singleton at a time).
// Per singleton (Alg. S-task): lam = midpoint of [lo, hi]; repeat Getvec; update [lo, hi]
// from the inertia count; accept when |gamma_r|/||z|| < tol1 gap (tol1 = n eps, gap = the
// distance to the nearest other eigenvalue) or |gamma_r|/||z||^2 < tol2 |lam| (tol2 = 4 eps),
// or when the correction stalls at a level tiny against the gap; otherwise apply the
// Rayleigh quotient correction gamma_r/||z||^2 when its sign points toward the eigenvalue
// and the result stays in [lo, hi]; else (or after max_rqi Getvecs) bisect to full accuracy
// and accept after one more Getvec.
//
// Getvec (Alg. Getvec) is evaluated without divisions in the recurrences.  With the
// homogeneous variables of the Sturm count (see negcount_ldl),
//   forward  (dstqds):  c_i = d_i c_{i-1} + a_i,      a_{i+1} = dll_i a_i - lam c_i,
//                       d+_i = c_i / c_{i-1},          s_i = a_i / c_{i-1};
//   backward (Alg. dqds, App. B, whose printed assignment to u- stands for omega-:
//             omega-_{i+1} = p_{i+1} + dll_i):
//                       h_i = dll_i h_{i+1} + f_{i+1}, f_i = d_i f_{i+1} - lam h_i,
//                       omega-_{i+1} = h_i / h_{i+1},  p_i = f_i / h_i,
// from c_{-1} = 1, a_0 = -lam, h_{n-1} = 1, f_{n-1} = d_{n-1} - lam, so that
//   gamma_i = s_i + d_i p_{i+1}/omega-_{i+1} = (a_i h_i + c_{i-1} d_i f_{i+1}) / (c_{i-1} h_i),
//   gamma_{n-1} = d+_{n-1}.
// The twisted solve N_r^T z = e_r (z_i = -l+_i z_{i+1} for i < r, z_{i+1} = -u-_i z_i for i >= r,
// l+_i = dl_i c_{i-1}/c_i, u-_i = dl_i h_{i+1}/h_i) telescopes to
//   z_i = (Q_r / Q_i) c_{i-1} / c_{r-1}  (i < r),   z_i = (Q_i / Q_r) h_i / h_r  (i > r),
// with the representation's prefix products Q_i = prod_{k<i} (-dl_k); this covers the
// zero-pivot rule of Alg. Getvec and makes every element independent.  (a, c) and (f, h)
// carry power-of-two scales tracked as integer exponents.  The count returned with a full
// factorization is NegCount(LDL^T, lam); with a given twist index r it is the inertia of
// diag(d+_0..d+_{r-1}, gamma_r, omega-_{r+1}..omega-_{n-1}).  The eigenvalue returned is the
// Rayleigh quotient of z with respect to the input T (accuracy remark 5, Sec. 3.1.2), which
// removes the bias of the root's random perturbation.
template <int TEAM>
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
                                            unsigned fault_mask, int *work_counter,
                                            DevInfo *info) {
    constexpr int kTeam = TEAM, kTeams = 32 / TEAM;
    const int lane = threadIdx.x & 31;
    const int team = lane / kTeam, k = lane % kTeam, tbase = team * kTeam;
    const int slot = blockIdx.x;
    Scratch<kTeams> S;
    S.base = scratch + (size_t)slot * Scratch<kTeams>::kSPI * (size_t)nmax + team;
    unsigned long long steps = 0, iters = 0;
    int itmax = 0, nfb = 0, ncap = 0;
    for (;;) {
        int chunk = 0;
        if (lane == 0) chunk = atomicAdd(work_counter, kTeams);
        chunk = __shfl_sync(FULL_MASK, chunk, 0);
        if (chunk >= nsingle) break;
        const int idx = chunk + team;
        const bool active = idx < nsingle;
        // ---- singleton data (every lane of the team holds a copy)
        int c = 0, n = 1, j = 1;
        const double *d = pool, *dll = pool, *Qm = pool, *iQm = pool;
        const int *Qe = (const int *)pool;
        double l = 0.0, h = 0.0, gap = 1.0;
        double *zc = Z;
        const double *td = Din, *te = Ein;
        if (active) {
            const SingleItem it = singles[idx];
            c = it.col;
            const Node N = nodes[it.node];
            const BlkDesc B = blks[N.blk];
            const MatDesc M = mats[B.mat];
            n = B.n;
            d = pool + N.rep;
            dll = d + 2 * n;
            Qm = d + rep_q_offset(n);
            iQm = Qm + n;
            Qe = (const int *)(iQm + n);
            j = jloc[c];
            l = lo[c];
            h = hi[c];
            gap = fmin(gapl[c], gapr[c]);
            if (!(gap > 0.0)) gap = kSafmin;
            zc = Z + M.zoff + (long long)(c - M.woff) * M.ldz + B.roff;
            td = Din + B.off;
            te = Ein + B.off;
        }
        const double tol1 = n * kEps, tol2 = 4.0 * kEps, tol_noise = n * kEps;
        double lam = l + 0.5 * (h - l);
        int r = -1, it_n = 0;
        bool done = !active, fb = false, capped = false;
        double nrm2 = 1.0, rqc = 0.0, prev_arqc = INFINITY;
        int imax = 0;
        for (int guard = 0; guard < 64; ++guard) {
            if (__all_sync(FULL_MASK, done)) break;
            const bool full = r < 0;
            const bool need_last = full || r == n - 1;
            const int fend = full ? n - 1 : r;
            const int blow = full ? 0 : r;
            // ---- pass 1: lanes 0 and 1 run the forward and the backward recurrence in one
            // instruction stream.  Both read X' = p X + Y, Y' = q Y - lam X' with
            //   forward  (lane 0): X = c, Y = a, (p, q) = (d_i, dll_i), i = t upward;
            //   backward (lane 1): X = h, Y = f, (p, q) = (dll_i, d_i), i = n-2-t downward.
            int cntf = 0, cntb = 0;
            double c_last = 1.0, cprev_last = 1.0;
            if (!done && k < 2) {
                const bool bw = (k == 1);
                // regular steps (compute, store, next Y): forward indices 0..nreg-1 (then the
                // step at fend: c_{n-1} for a full factorization or r = n-1, else a store
                // only), backward indices n-2 .. blow
                const int nreg = bw ? (n - 1 - blow) : (need_last ? n - 1 : fend);
                const double *P = bw ? dll : d;
                const double *Qv = bw ? d : dll;
                double X = 1.0, Y = bw ? (__ldg(d + n - 1) - lam) : -lam;
                int Sx = 0, sp = 0, cnt = 0;
                if (bw) S.E(n - 1).y = 0;
                const int di = bw ? -1 : 1, i0 = bw ? (n - 2) : 0;
                // the lane's slots: forward (A, C, E.x) = (a_i, c_{i-1}, exponent) stored
                // before the step, backward (H, Q, E.y) = (h_i, d_i f_{i+1}, exponent) after it
                const int off1 = (bw ? 2 : 0) * kTeams, off2 = (bw ? 3 : 1) * kTeams;
                const int eoff = bw ? 1 : 0;
                auto store = [&](int i, double v1, double v2, int e) {
                    double *row = S.base + (size_t)i * Scratch<kTeams>::kSPI;
                    row[off1] = v1;
                    row[off2] = v2;
                    ((int *)(row + 4 * kTeams))[eoff] = e;
                };
                // one regular step with the per-step rules (zero-pivot substitute, rescale)
                auto step_exact = [&](int i, double pi, double qi) {
                    const double Yb = Y, Xb = X;
                    const double qY = qi * Y;
                    double Xn = fma(pi, X, Y);
                    // an exactly zero pivot becomes a negative one 2^-80 times the
                    // cancelled term |pi X| = |Y|: tiny relative to the data at any scale
                    if (is_zero(Xn)) Xn = is_zero(Y) ? -X * 0x1p-80 : copysign(fabs(Y) * 0x1p-80, -X);
                    const int sc = sign_bit(Xn);
                    cnt += sc ^ sp;
                    Y = fma(-lam, Xn, qY);
                    store(i, bw ? Xn : Yb, bw ? qY : Xb, Sx);
                    Sx -= rescale2(Xn, Y);
                    X = Xn;
                    sp = sc;
                };
                // blocks of 8 steps without a data-dependent branch (see negcount_ldl): the
                // per-step rescale is replaced by a normalisation at the end of the block;
                // a block in which some h or c was zero or left [2^-400, 2^400] (a flag
                // collected off the recurrence, so that products of two stored values, as
                // in the twist search, stay finite) is redone with the per-step rules
                int t = 0;
                double pn = (nreg > 0) ? __ldg(P + i0) : 0.0;
                double qn = (nreg > 0) ? __ldg(Qv + i0) : 0.0;
                for (; t + 8 <= nreg; t += 8) {
                    const double X0 = X, Y0 = Y;
                    const int Sx0 = Sx, sp0 = sp, cnt0 = cnt;
                    bool flag = false;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int i = i0 + di * (t + u);
                        const double pi = pn, qi = qn;
                        const int inext = (t + u + 1 < nreg) ? i + di : i;
                        pn = __ldg(P + inext);
                        qn = __ldg(Qv + inext);
                        const double Yb = Y, Xb = X;
                        const double qY = qi * Y;
                        const double Xn = fma(pi, X, Y);
                        flag |= (unsigned)(biased_exp(Xn) - (1023 - 400)) > 800u;
                        const int sc = sign_bit(Xn);
                        cnt += sc ^ sp;
                        sp = sc;
                        Y = fma(-lam, Xn, qY);
                        store(i, bw ? Xn : Yb, bw ? qY : Xb, Sx);
                        X = Xn;
                    }
                    const int ex = biased_exp(X), ey = biased_exp(Y);
                    if (__builtin_expect(flag || ey == 0x7ff, 0)) {
                        X = X0;
                        Y = Y0;
                        Sx = Sx0;
                        sp = sp0;
                        cnt = cnt0;
                        for (int u = 0; u < 8; ++u) {
                            const int i = i0 + di * (t + u);
                            step_exact(i, __ldg(P + i), __ldg(Qv + i));
                        }
                    } else {
                        const int kx = 1023 - ex;
                        const double q = pow2i(kx);
                        X *= q;
                        Y *= q;
                        Sx -= kx;
                    }
                }
                for (; t < nreg; ++t) {
                    const int i = i0 + di * t;
                    step_exact(i, __ldg(P + i), __ldg(Qv + i));
                }
                if (!bw) {
                    // the step at fend (= n-1 or r)
                    S.A(fend) = Y;
                    S.C(fend) = X;
                    S.E(fend).x = Sx;
                    if (need_last) {
                        double Xn = fma(__ldg(d + n - 1), X, Y);
                        if (is_zero(Xn)) Xn = is_zero(Y) ? -X * 0x1p-80 : copysign(fabs(Y) * 0x1p-80, -X);
                        const int sc = sign_bit(Xn);
                        if (full || n - 1 < r) cnt += sc ^ sp;
                        c_last = Xn;
                        cprev_last = X;
                    }
                }
                if (bw) cntb = cnt; else cntf = cnt;
                steps += (unsigned long long)(bw ? nreg : fend + 1);
            }
            __syncwarp();
            cntf = __shfl_sync(FULL_MASK, cntf, tbase);
            cntb = __shfl_sync(FULL_MASK, cntb, tbase + 1);
            c_last = __shfl_sync(FULL_MASK, c_last, tbase);
            cprev_last = __shfl_sync(FULL_MASK, cprev_last, tbase);
            // ---- pass 2: twist index (full factorizations)
            float best = 3.0e38f;
            int rr = n - 1;
            if (!done && full) {
                if (k == 0) {
                    best = log2abs(c_last) - log2abs(cprev_last);
                    if (!(best == best)) best = 3.0e38f;
                }
#pragma unroll 4
                for (int i = k; i < n - 1; i += kTeam) {
                    const double ci = S.C(i), hv = S.H(i);
                    const double num = fma(S.A(i), hv, ci * S.Q(i));
                    const float key = log2abs(num) - log2abs(ci * hv);
                    if (key < best || (key == best && i < rr)) { best = key; rr = i; }
                }
            }
            team_argmin<kTeam>(best, rr);
            double gamma = 1.0;
            int negc = 0;
            if (!done) {
                if (full) r = rr;
                double gnum, gden;
                if (r == n - 1) {
                    gnum = c_last;
                    gden = cprev_last;
                } else {
                    const double ci = S.C(r), hv = S.H(r);
                    gnum = fma(S.A(r), hv, ci * S.Q(r));
                    gden = ci * hv;
                }
                gamma = gnum / gden;
                negc = full ? cntf : cntf + cntb + sign_bit(gamma);
            }
            // ---- pass 3: solve (z_r = 1), each lane on every kTeam-th element
            double ss = 0.0;
            long long zb = 0;
            int zi_max = 0x7fffffff;
            if (!done) {
                const int rf = S.E(r).x;
                const double icr = 1.0 / S.C(r);
                const double ihr = (r < n - 1) ? 1.0 / S.H(r) : 1.0;
                const int rg = (r < n - 1) ? S.E(r).y : 0;
                const double qmr = Qm[r], iqmr = iQm[r];
                const int qer = Qe[r];
#pragma unroll 4
                for (int i = k; i < n; i += kTeam) {
                    double z;
                    if (i < r) {
                        z = scale2(qmr * iQm[i] * S.C(i) * icr, qer - Qe[i] + S.E(i).x - rf);
                    } else if (i > r) {
                        const double hv = (i < n - 1) ? S.H(i) : 1.0;
                        const int gi = (i < n - 1) ? S.E(i).y : 0;
                        z = scale2(Qm[i] * iqmr * hv * ihr, Qe[i] - qer + gi - rg);
                    } else {
                        z = 1.0;
                    }
                    zc[i] = z;
                    ss = fma(z, z, ss);
                    const long long b = __double_as_longlong(z) & 0x7fffffffffffffffll;
                    if (b > zb) { zb = b; zi_max = i; }
                }
                steps += (unsigned long long)((n + kTeam - 1) / kTeam);
            }
            ss = team_sum<kTeam>(ss);
            team_argmax_bits<kTeam>(zb, zi_max);
            if (done) continue;
            // ---- acceptance (uniform within the team)
            nrm2 = ss;
            imax = zi_max;
            ++it_n;
            if (negc >= j) h = fmin(h, lam); else l = fmax(l, lam);
            const double resid = fabs(gamma) / sqrt(nrm2);
            rqc = gamma / nrm2;
            const bool conv = (resid < tol1 * gap) || (fabs(rqc) < tol2 * fabs(lam));
            // RQI converges cubically; a correction that no longer shrinks (at least by
            // half) while tiny against the gap sits at the representation's noise level
            const bool stalled = it_n >= 2 && fabs(rqc) >= 0.5 * prev_arqc && fabs(rqc) <= 1e-3 * gap;
            const bool nofault = !(fault_mask & MR3_FAULT_RQI_NOCONV);
            if (fb || ((conv || stalled) && nofault)) { done = true; continue; }
            prev_arqc = fabs(rqc);
            const bool sign_ok = (negc < j) ? (rqc > 0.0) : (rqc < 0.0);
            const double lnew = lam + rqc;
            if (it_n < max_rqi && sign_ok && lnew >= l && lnew <= h) {
                lam = lnew;
                continue;
            }
            // a correction at the rounding noise of the factorization cannot improve lam
            if (nofault && fabs(rqc) <= tol_noise * fabs(lam)) { done = true; continue; }
            if (it_n >= max_rqi) capped = true;
            // bisection to full accuracy, as a multisection over the team's lanes (lane k
            // counts at the (k+1)-th of kTeam interior points; the team ballot of
            // "count < j" picks the part holding lambda_j), then one more Getvec
            {
                const unsigned tmask = (kTeam == 32) ? FULL_MASK : (((1u << kTeam) - 1u) << tbase);
                for (int kk = 0; kk < 2100; ++kk) {
                    const double wd = h - l;
                    if (!(wd > fmax(4.0 * kEps * fmax(fabs(l), fabs(h)), 4.0 * kSafmin))) break;
                    const double x = l + (k + 1) * (wd / (kTeam + 1));
                    if (__ballot_sync(tmask, !(x > l && x < h)) & tmask) {
                        // no representable interior points left: plain bisection
                        const double mid = l + 0.5 * wd;
                        if (!(mid > l && mid < h)) break;
                        if (k == 0) steps += n;
                        if (negcount_ldl(n, d, dll, mid) < j) l = mid; else h = mid;
                        continue;
                    }
                    steps += n;
                    const unsigned bal = __ballot_sync(tmask, negcount_ldl(n, d, dll, x) < j) & tmask;
                    const int t = __popc(bal);
                    const double xl = __shfl_sync(tmask, x, tbase + (t > 0 ? t - 1 : 0));
                    const double xh = __shfl_sync(tmask, x, tbase + (t < kTeam ? t : kTeam - 1));
                    if (t > 0) l = xl;
                    if (t < kTeam) h = xh;
                }
            }
            lam = l + 0.5 * (h - l);
            r = -1;
            fb = true;
        }
        // ---- normalise (an entry of largest magnitude positive) and the Rayleigh quotient
        double rq = 0.0;
        if (active) {
            const double zsign = (zc[imax] < 0.0) ? -1.0 : 1.0;
            const double scale = zsign / sqrt(nrm2);
#pragma unroll 4
            for (int i = k; i < n; i += kTeam) zc[i] *= scale;
        }
        __syncwarp();
        if (active) {
#pragma unroll 4
            for (int i = k; i < n; i += kTeam) {
                const double zi = zc[i];
                rq = fma(__ldg(td + i) * zi, zi, rq);
                if (i + 1 < n) rq = fma(2.0 * __ldg(te + i) * zi, zc[i + 1], rq);
            }
        }
        rq = team_sum<kTeam>(rq);
        if (active && k == 0) {
            w[c] = rq;
            iters += it_n;
            itmax = max(itmax, it_n);
            nfb += fb ? 1 : 0;
            ncap += capped ? 1 : 0;
        }
        __syncwarp();
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

void launch_rqi(int nsingle, const SingleItem *singles, const Node *nodes, const BlkDesc *blks,
                const MatDesc *mats, const double *pool, const int *jloc, const double *lo,
                const double *hi, const double *gapl, const double *gapr, const double *d,
                const double *e, double *w, double *Z, double *scratch, int nslots, int nmax,
                int max_rqi, unsigned fault_mask, int *work_counter, DevInfo *info,
                int team, cudaStream_t s) {
    if (nsingle <= 0) return;
    const int per = 32 / team;
    const int want = (nsingle + per - 1) / per;
    const int nblocks = want < nslots ? want : nslots;
    cudaMemsetAsync(work_counter, 0, sizeof(int), s);
    if (team == 2)
        k_rqi<2><<<nblocks, 32, 0, s>>>(nsingle, singles, nodes, blks, mats, pool, jloc, lo, hi,
                                        gapl, gapr, d, e, w, Z, scratch, nmax, max_rqi,
                                        fault_mask, work_counter, info);
    else
        k_rqi<8><<<nblocks, 32, 0, s>>>(nsingle, singles, nodes, blks, mats, pool, jloc, lo, hi,
                                        gapl, gapr, d, e, w, Z, scratch, nmax, max_rqi,
                                        fault_mask, work_counter, info);
}

// Teams of 2 once the singletons clearly outnumber what the resident warps hold with teams
// of 8 (about 17 warps per SM at this kernel's register count, 4 singletons each).  When a
// solve covers several matrices the singleton launch runs beside the other matrices' shift
// and refinement kernels on the main stream, and its fewer binary64 instructions with teams
// of 2 pay off from much smaller counts (measured on the n = 8192 three-matrix step).
#ifndef MR3_RQI_TEAM2_MIN
#define MR3_RQI_TEAM2_MIN 32768
#endif
#ifndef MR3_RQI_TEAM2_MIN_MULTI
#define MR3_RQI_TEAM2_MIN_MULTI 2048
#endif
int rqi_team(long long nsingle, int nmat) {
    return nsingle > (nmat > 1 ? MR3_RQI_TEAM2_MIN_MULTI : MR3_RQI_TEAM2_MIN) ? 2 : 8;
}
int rqi_scratch_per_index(int team) { return kScratchPerSingleton * (32 / team); }
int rqi_singles_per_slot(int team) { return 32 / team; }

cudaError_t preload_rqi() { return load_kernels(k_rqi<2>, k_rqi<8>); }

} // namespace mr3
