// mr3_rqi.cu -- eigenpairs of well-separated eigenvalues (singletons): Rayleigh quotient
// iteration on the twisted factorizations of Alg. Getvec, guarded by bisection
// (Alg. S-task and the remarks after Alg. Getvec, Sec. 3.2.3).
#include <float.h>
#include "mr3_kernels.h"

namespace mr3 {

#define FULL_MASK 0xffffffffu

// A team of TEAM lanes finishes one singleton; a warp holds 32 / TEAM teams.  Lanes 0 and 1
// of a team run the two serial recurrences of a twisted factorization (forward dstqds and
// backward dqds), after which all lanes of the team share the element-wise work.  Teams of
// 8 keep a singleton's element-wise pass short (levels with few singletons are latency
// bound); teams of 2 fill 4x more lanes of every binary64 instruction in the recurrences,
// which wins when singletons far outnumber the resident warps (the binary64 pipe costs the
// same per warp instruction whatever the number of active lanes).
//
// Memory traffic.  The vector is written once per iteration with a known twist index,
// straight from the recurrences, and rescaled once at the end; an iteration that has to
// find the twist index writes no vector at all.  That search needs, at every index i, the
// forward quantities (a_i, c_{i-1}) next to the backward ones (h_i, d_i f_{i+1}); the lane
// that reaches i first leaves a record of its pair for the other lane, which evaluates
// gamma_i when it passes i.  Records hold the two binary64 values, the running sum of
// squares of the lane's side of the vector (binary32 mantissa, integer exponent) and
// log2 |G(i)| (integer part exact, binary32 fraction), which give ||z||^2 for any twist
// index to ~1e-6 relative (enough to steer the first Rayleigh correction; the norms that
// normalise the output are exact).  The exponents are kept as integers because they reach
// tens of thousands (the prefix products Q_i of a glued matrix shrink by the glue at every
// block): a binary32 logarithm of that size resolves only ~0.4% and drops smaller terms.
#ifndef MR3_RQI2_MIN_BLOCKS
#define MR3_RQI2_MIN_BLOCKS 16
#endif
constexpr int kRecordDoubles = 4;                    // (X, Y, {S, frac}, {E, int})
constexpr int kScratchPerSingleton = 2 * kRecordDoubles; // forward and backward record

// log2 |G| = i + f with the integer part exact and f in (-2, 2).
struct LogG {
    int i;
    float f;
};
// A sum of squares S 2^e (S in binary32).
struct LSum {
    float s;
    int e;
};
constexpr int kEmpty = -(1 << 29); // exponent of an empty sum

// log2 of the mantissa of a normal double (in [0, 1)).
__device__ __forceinline__ float log2mant(double x) {
    const long long b = __double_as_longlong(x);
    return __log2f(__int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff)));
}

// S 2^e += 2^(2 g).
__device__ __forceinline__ void lsum_add(LSum &q, const LogG &g) {
    const int ne = max(q.e, 2 * g.i);
    q.s = q.s * exp2f((float)(q.e - ne)) + exp2f((float)(2 * g.i - ne) + 2.f * g.f);
    q.e = ne;
}

// log2(S 2^e / 2^(2 g)): log2 of one side's sum of z_k^2 for the twist index with G = g.
__device__ __forceinline__ float lsum_rel(const LSum &q, const LogG &g) {
    return __log2f(q.s) + (float)(q.e - 2 * g.i) - 2.f * g.f;
}

template <int TEAMS> struct Records {
    static constexpr int kSPI = kScratchPerSingleton * TEAMS; // doubles per index per slot
    double *base; // warp slot base + team; row i holds every team's two records
    __device__ __forceinline__ double *rec(int i, bool bw) const {
        return base + (size_t)i * kSPI + (bw ? kRecordDoubles * TEAMS : 0);
    }
    __device__ __forceinline__ void put(int i, bool bw, double x, double y, const LSum &q,
                                        const LogG &g) const {
        double *p = rec(i, bw);
        __stcg(p, x);
        __stcg(p + TEAMS, y);
        __stcg((float2 *)(p + 2 * TEAMS), make_float2(q.s, g.f));
        __stcg((int2 *)(p + 3 * TEAMS), make_int2(q.e, g.i));
    }
    __device__ __forceinline__ void get(int i, bool bw, double &x, double &y, LSum &q,
                                        LogG &g) const {
        const double *p = rec(i, bw);
        x = __ldcg(p);
        y = __ldcg(p + TEAMS);
        const float2 a = __ldcg((const float2 *)(p + 2 * TEAMS));
        const int2 b = __ldcg((const int2 *)(p + 3 * TEAMS));
        q.s = a.x;
        g.f = a.y;
        q.e = b.x;
        g.i = b.y;
    }
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

// x * 2^e by adding e to the exponent field (integer operations only): a zero or subnormal
// x, or a result below the normal range, gives a signed zero; a result above it, infinity.
// Used for vector entries, where anything below 2^-1022 is negligible.
__device__ __forceinline__ double ldexp_bits(double x, int e) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    const int ne = ex + e;
    const long long sgn = b & (long long)0x8000000000000000ull;
    const long long r = (ex == 0 || ne <= 0) ? sgn
                      : (ne >= 0x7ff ? (sgn | 0x7ff0000000000000ll) : b + ((long long)e << 52));
    return __longlong_as_double(r);
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

// Candidate twist index of one lane: the key log2 |gamma_i| ranks candidates; gamma_i is
// kept as numerator and denominator (they share one power-of-two scale); lf, lb are log2
// of sum_{k<i} z_k^2 and sum_{k>i} z_k^2 for z_i = 1; gf, gb are log2 |G_f(i)| and
// log2 |G_b(i)| (the scale of each side of the vector, reused by the next iteration).
struct Cand {
    float key;
    int idx;
    double gnum, gden;
    float lf, lb, gf, gb;
};

__device__ __forceinline__ void cand_reset(Cand &c) {
    c.key = 3.0e38f;
    c.idx = 0x7fffffff;
    c.gnum = 1.0;
    c.gden = 1.0;
    c.lf = c.lb = -INFINITY;
    c.gf = c.gb = 0.f;
}

// gamma_i = (a_i h_i + c_{i-1} d_i f_{i+1}) / (c_{i-1} h_i) from the forward pair
// (xf, yf) = (c_{i-1}, a_i) and the backward pair (xb, yb) = (h_i, d_i f_{i+1}), with the
// side sums (qf, qb) and side scales (gf, gb) at i.
__device__ __forceinline__ void cand_eval(Cand &c, int i, double xf, double yf, const LSum &qf,
                                          const LogG &gf, double xb, double yb, const LSum &qb,
                                          const LogG &gb) {
    const double num = fma(yf, xb, xf * yb);
    const double den = xf * xb;
    float key = log2abs(num) - log2abs(den);
    if (!(key == key)) key = 3.0e38f;
    if (key < c.key || (key == c.key && i < c.idx)) {
        c.key = key;
        c.idx = i;
        c.gnum = num;
        c.gden = den;
        c.lf = lsum_rel(qf, gf);
        c.lb = lsum_rel(qb, gb);
        c.gf = (float)gf.i + gf.f;
        c.gb = (float)gb.i + gb.f;
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
//   z_i = G_f(i) / G_f(r) (i < r),  G_f(i) = c_{i-1} / Q_i;   z_i = G_b(i) / G_b(r) (i > r),
//   G_b(i) = Q_i h_i,
// with the representation's prefix products Q_i = prod_{k<i} (-dl_k); this covers the
// zero-pivot rule of Alg. Getvec and makes every element independent.  (a, c) and (f, h)
// carry power-of-two scales tracked as integer exponents.  The count returned with a full
// factorization is NegCount(LDL^T, lam); with a given twist index r it is the inertia of
// diag(d+_0..d+_{r-1}, gamma_r, omega-_{r+1}..omega-_{n-1}).
//
// Iterations.  A full factorization (the first one, and the one after a bisection fallback)
// finds r = argmin |gamma_i| with the records described above and writes no vector.  An
// iteration with r known writes t_i = G(i) 2^-ref for i != r straight from the recurrences
// (ref = log2 |G(r)| of the previous iteration keeps t_i near z_i) and sums t_i^2 exactly,
// so ||z||^2 = 1 + f_f^2 sum_{i<r} t_i^2 + f_b^2 sum_{i>r} t_i^2 with f = 2^ref / G(r).  A
// full factorization that passes the acceptance test is followed by one such iteration at
// the same lam.  At acceptance one pass over the vector multiplies each side by its factor,
// 1/||z|| and the sign that makes an entry of largest magnitude positive, and forms the
// Rayleigh quotient of the unit vector with respect to the input T (accuracy remark 5,
// Sec. 3.1.2), which removes the bias of the root's random perturbation.
// Resident warps per SM the launch bounds ask for: teams of 2 run where singletons far
// outnumber the resident warps, so their register budget (128) admits 16 warps per SM, at
// the price of a few spilled values (measured on the 4096-matrix batch: 12 warps per SM
// 468 ms, 14: 455, 16: 456, against 557 at the 8 that 213 registers allowed); teams of 8
// keep the full budget and no stack frame.
template <int TEAM> struct RqiOccupancy { static constexpr int kMinBlocks = 1; };
template <> struct RqiOccupancy<2> { static constexpr int kMinBlocks = MR3_RQI2_MIN_BLOCKS; };

template <int TEAM>
__global__ void __launch_bounds__(32, RqiOccupancy<TEAM>::kMinBlocks) k_rqi(int nsingle, const SingleItem *__restrict__ singles,
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
                                            DevInfo *info, const int *dnsingle, int nmat,
                                            int forced_team) {
    // with a device count, both team sizes are launched and the one the host's rule would
    // not pick returns at once
    if (dnsingle) {
        nsingle = *dnsingle;
        if (rqi_team_rule(nsingle, nmat, forced_team) != TEAM) return;
    }
    constexpr int kTeam = TEAM, kTeams = 32 / TEAM;
    const int lane = threadIdx.x & 31;
    const int team = lane / kTeam, k = lane % kTeam, tbase = team * kTeam;
    const unsigned tmask = (kTeam == 32) ? FULL_MASK : (((1u << kTeam) - 1u) << tbase);
    const int slot = blockIdx.x;
    Records<kTeams> R;
    R.base = scratch + (size_t)slot * Records<kTeams>::kSPI * (size_t)nmax + team;
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
        bool done = !active, fb = false, capped = false, final_pending = false;
        double nrm2 = 1.0, rqc = 0.0, prev_arqc = INFINITY;
        int ref_f = 0, ref_b = 0;
        double Ff = 0.0, Fb = 0.0, Fr = 1.0; // output factors of the last vector written
        for (int guard = 0; guard < 64; ++guard) {
            if (__all_sync(FULL_MASK, done)) break;
            const bool full = r < 0;
            // ---- serial pass: lanes 0 and 1 run the forward and the backward recurrence
            // in one instruction stream.  Both read X' = p X + Y, Y' = q Y - lam X' with
            //   forward  (lane 0): X = c, Y = a, (p, q) = (d_i, dll_i), i = t upward;
            //   backward (lane 1): X = h, Y = f, (p, q) = (dll_i, d_i), i = n-2-t downward.
            int cnt = 0;
            Cand cd;
            cand_reset(cd);
            double ssum = 0.0;             // sum of t_i^2 over the lane's side
            long long mbits = -1;          // largest |t_i| (bits), its index and sign
            int midx = 0x7fffffff, mneg = 0;
            double Xe = 1.0, Ye = 0.0;     // the pair at the twist index (r known)
            int Se = 0;
            double c_last = 1.0, cprev_last = 1.0;
            if (!done && k < 2) {
                const bool bw = (k == 1);
                const int fend = full ? n - 1 : r;
                const bool need_last = full || r == n - 1;
                const int blow = full ? 0 : r;
                const int nreg = bw ? (n - 1 - blow) : (need_last ? n - 1 : fend);
                const double *P = bw ? dll : d;
                const double *Qv = bw ? d : dll;
                // full: Qm for log2 |Q_i|; r known: the factor of G (1/Q_i forward, Q_i backward)
                const double *Qs = (full || bw) ? Qm : iQm;
                const int qsgn = bw ? 1 : -1, ref = bw ? ref_b : ref_f;
                // the lane that reaches index i second evaluates gamma_i there when the other
                // lane's record is at least 16 steps old; indices in between are evaluated
                // after the pass
                const int iF = (n + 16) >> 1, iB = (n - 18) >> 1;
                double X = 1.0, Y = bw ? (__ldg(d + n - 1) - lam) : -lam;
                int Sx = 0, sp = 0;
                LSum lp = {0.f, kEmpty}; // running sum of G^2 on this side
                if (bw) {                // index n-1: h_{n-1} = 1, G_b(n-1) = Q_{n-1}
                    const double qm = __ldg(Qm + n - 1);
                    const int qe = __ldg(Qe + n - 1);
                    if (full) {
                        const LogG g0 = {qe, __log2f(fabsf((float)qm))};
                        lsum_add(lp, g0);
                    } else if (r < n - 1) {
                        const double t = ldexp_bits(qm, qe - ref);
                        zc[n - 1] = t;
                        ssum = t * t;
                        mbits = __double_as_longlong(t) & 0x7fffffffffffffffll;
                        midx = n - 1;
                        mneg = t < 0.0;
                    }
                }
                // side work at index i: (xv, yv) = (c_{i-1}, a_i) before a forward step,
                // (h_i, d_i f_{i+1}) after a backward step; s = their exponent
                auto visit = [&](int i, double xv, double yv, int s, double qm, int qe) {
                    if (full) {
                        const float mq = __log2f(fabsf((float)qm));
                        LogG lg;
                        lg.i = biased_exp(xv) - 1023 + s + (bw ? qe : -qe);
                        lg.f = log2mant(xv) + (bw ? mq : -mq);
                        if (bw ? (i <= iB) : (i >= iF)) {
                            double px, py;
                            LSum pq;
                            LogG pg;
                            R.get(i, !bw, px, py, pq, pg);
                            // forward pair first: the backward lane passes the record's pair
                            // as the forward one (selects, so the two lanes stay converged)
                            const double fx = bw ? px : xv, fy = bw ? py : yv;
                            const double bx = bw ? xv : px, by = bw ? yv : py;
                            const LSum fq = bw ? pq : lp, bq = bw ? lp : pq;
                            const LogG fg = bw ? pg : lg, bg = bw ? lg : pg;
                            cand_eval(cd, i, fx, fy, fq, fg, bx, by, bq, bg);
                        } else {
                            R.put(i, bw, xv, yv, lp, lg);
                        }
                        lsum_add(lp, lg);
                    } else if (bw ? (i > r) : (i < r)) {
                        const double t = ldexp_bits(xv * qm, s + qsgn * qe - ref);
                        zc[i] = t;
                        ssum = fma(t, t, ssum);
                        const long long b = __double_as_longlong(t) & 0x7fffffffffffffffll;
                        if (bw ? (b >= mbits) : (b > mbits)) { mbits = b; midx = i; mneg = t < 0.0; }
                    } else if (bw && i == r) {
                        Xe = xv;
                        Ye = yv;
                        Se = s;
                    }
                };
                const int di = bw ? -1 : 1, i0 = bw ? (n - 2) : 0;
                // one regular step with the per-step rules (zero-pivot substitute, rescale)
                auto step_exact = [&](int i, double pi, double qi, double qm, int qe) {
                    const double Yb = Y, Xb = X;
                    const double qY = qi * Y;
                    double Xn = fma(pi, X, Y);
                    // an exactly zero pivot becomes a negative one 2^-80 times the
                    // cancelled term |pi X| = |Y|: tiny relative to the data at any scale
                    if (is_zero(Xn)) Xn = is_zero(Y) ? -X * 0x1p-80 : copysign(fabs(Y) * 0x1p-80, -X);
                    const int sc = sign_bit(Xn);
                    cnt += sc ^ sp;
                    Y = fma(-lam, Xn, qY);
                    visit(i, bw ? Xn : Xb, bw ? qY : Yb, Sx, qm, qe);
                    Sx -= rescale2(Xn, Y);
                    X = Xn;
                    sp = sc;
                };
                // blocks of 8 steps without a data-dependent branch (see negcount_ldl): the
                // per-step rescale is replaced by a normalisation at the end of the block;
                // a block in which some h or c was zero or left [2^-400, 2^400] (a flag
                // collected off the recurrence, so that products of two values, as in gamma,
                // stay finite) is redone with the per-step rules
                int t = 0;
                double pn = (nreg > 0) ? __ldg(P + i0) : 0.0;
                double qn = (nreg > 0) ? __ldg(Qv + i0) : 0.0;
                double qmn = (nreg > 0) ? __ldg(Qs + i0) : 0.0;
                int qen = (nreg > 0) ? __ldg(Qe + i0) : 0;
                for (; t + 8 <= nreg; t += 8) {
                    const double X0 = X, Y0 = Y;
                    const int Sx0 = Sx, sp0 = sp, cnt0 = cnt;
                    const LSum lp0 = lp;
                    const Cand cd0 = cd;
                    const double ss0 = ssum, Xe0 = Xe, Ye0 = Ye;
                    const long long mb0 = mbits;
                    const int mi0 = midx, mn0 = mneg, Se0 = Se;
                    bool flag = false;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int i = i0 + di * (t + u);
                        const double pi = pn, qi = qn, qm = qmn;
                        const int qe = qen;
                        const int inext = (t + u + 1 < nreg) ? i + di : i;
                        pn = __ldg(P + inext);
                        qn = __ldg(Qv + inext);
                        qmn = __ldg(Qs + inext);
                        qen = __ldg(Qe + inext);
                        const double Yb = Y, Xb = X;
                        const double qY = qi * Y;
                        const double Xn = fma(pi, X, Y);
                        flag |= (unsigned)(biased_exp(Xn) - (1023 - 400)) > 800u;
                        const int sc = sign_bit(Xn);
                        cnt += sc ^ sp;
                        sp = sc;
                        Y = fma(-lam, Xn, qY);
                        visit(i, bw ? Xn : Xb, bw ? qY : Yb, Sx, qm, qe);
                        X = Xn;
                    }
                    const int ex = biased_exp(X), ey = biased_exp(Y);
                    if (__builtin_expect(flag || ey == 0x7ff, 0)) {
                        X = X0;
                        Y = Y0;
                        Sx = Sx0;
                        sp = sp0;
                        cnt = cnt0;
                        lp = lp0;
                        cd = cd0;
                        ssum = ss0;
                        Xe = Xe0;
                        Ye = Ye0;
                        Se = Se0;
                        mbits = mb0;
                        midx = mi0;
                        mneg = mn0;
                        for (int u = 0; u < 8; ++u) {
                            const int i = i0 + di * (t + u);
                            step_exact(i, __ldg(P + i), __ldg(Qv + i), __ldg(Qs + i), __ldg(Qe + i));
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
                    step_exact(i, __ldg(P + i), __ldg(Qv + i), __ldg(Qs + i), __ldg(Qe + i));
                }
                if (!bw) {
                    // the pair (c_{fend-1}, a_fend) at fend (= n-1 or r), and for a full
                    // factorization or r = n-1 the last pivot d+_{n-1} = c_{n-1} / c_{n-2}
                    Xe = X;
                    Ye = Y;
                    Se = Sx;
                    if (need_last) {
                        double Xn = fma(__ldg(d + n - 1), X, Y);
                        if (is_zero(Xn)) Xn = is_zero(Y) ? -X * 0x1p-80 : copysign(fabs(Y) * 0x1p-80, -X);
                        const int sc = sign_bit(Xn);
                        if (full) cnt += sc ^ sp;
                        c_last = Xn;
                        cprev_last = X;
                        if (full) { // candidate r = n-1: z_i = G_f(i) / G_f(n-1) for i < n-1
                            LogG lg;
                            lg.i = biased_exp(X) - 1023 + Sx - __ldg(Qe + n - 1);
                            lg.f = log2mant(X) - __log2f(fabsf((float)__ldg(Qm + n - 1)));
                            float key = log2abs(Xn) - log2abs(X);
                            if (!(key == key)) key = 3.0e38f;
                            if (key < cd.key || (key == cd.key && n - 1 < cd.idx)) {
                                cd.key = key;
                                cd.idx = n - 1;
                                cd.gnum = Xn;
                                cd.gden = X;
                                cd.lf = lsum_rel(lp, lg);
                                cd.lb = -INFINITY;
                                cd.gf = (float)lg.i + lg.f;
                                cd.gb = 0.f;
                            }
                        }
                    }
                }
                steps += (unsigned long long)(bw ? nreg : fend + 1);
            }
            __syncwarp();
            double gamma = 1.0;
            int negc = 0;
            bool bad_scale = false;
            // ---- twist index of a full factorization: indices next to the crossing point
            // of the two lanes are evaluated now from both records (visible after the
            // __syncwarp above), spread over the team's lanes; then the team's minimum.
            // Every shuffle below runs on all lanes (teams differ in state).
            if (!done && full) {
                const int iF = (n + 16) >> 1, iB = (n - 18) >> 1;
                const int w0 = max(iB + 1, 0), w1 = min(iF - 1, n - 2);
                for (int i = w0 + k; i <= w1; i += kTeam) {
                    double xf, yf, xb, yb;
                    LSum qf, qb;
                    LogG gf, gb;
                    R.get(i, false, xf, yf, qf, gf);
                    R.get(i, true, xb, yb, qb, gb);
                    cand_eval(cd, i, xf, yf, qf, gf, xb, yb, qb, gb);
                }
            }
            float bkey = cd.key;
            int bidx = cd.idx;
            team_argmin<kTeam>(bkey, bidx);
            const unsigned win = __ballot_sync(FULL_MASK, cd.key == bkey && cd.idx == bidx) & tmask;
            const int src = win ? (__ffs(win) - 1) : tbase;
            const double cgnum = __shfl_sync(FULL_MASK, cd.gnum, src);
            const double cgden = __shfl_sync(FULL_MASK, cd.gden, src);
            const float clf = __shfl_sync(FULL_MASK, cd.lf, src);
            const float clb = __shfl_sync(FULL_MASK, cd.lb, src);
            const float cgf = __shfl_sync(FULL_MASK, cd.gf, src);
            const float cgb = __shfl_sync(FULL_MASK, cd.gb, src);
            const int cntf = __shfl_sync(FULL_MASK, cnt, tbase);
            const int cntb = __shfl_sync(FULL_MASK, cnt, tbase + 1);
            const double xf = __shfl_sync(FULL_MASK, Xe, tbase);
            const double yf = __shfl_sync(FULL_MASK, Ye, tbase);
            const int sf = __shfl_sync(FULL_MASK, Se, tbase);
            const double xb = __shfl_sync(FULL_MASK, Xe, tbase + 1);
            const double yb = __shfl_sync(FULL_MASK, Ye, tbase + 1);
            const int sb = __shfl_sync(FULL_MASK, Se, tbase + 1);
            const double clast = __shfl_sync(FULL_MASK, c_last, tbase);
            const double cprev = __shfl_sync(FULL_MASK, cprev_last, tbase);
            const double ssf = __shfl_sync(FULL_MASK, ssum, tbase);
            const double ssb = __shfl_sync(FULL_MASK, ssum, tbase + 1);
            const long long mbf = __shfl_sync(FULL_MASK, mbits, tbase);
            const long long mbb = __shfl_sync(FULL_MASK, mbits, tbase + 1);
            const int mnf = __shfl_sync(FULL_MASK, mneg, tbase);
            const int mnb = __shfl_sync(FULL_MASK, mneg, tbase + 1);
            if (!done && full) {
                r = min(max(bidx, 0), n - 1);
                gamma = cgnum / cgden;
                negc = cntf;
                // ||z||^2 from the binary32 side sums (steers this iteration only)
                nrm2 = 1.0 + exp2((double)clf) + exp2((double)clb);
                ref_f = (int)rintf(cgf);
                ref_b = (int)rintf(cgb);
            } else if (!done) {
                // ---- r known: gamma_r from the two lanes' pairs at r, the exact ||z||^2
                // from the two side sums, and the factors that turn t_i into the unit vector
                double gnum, gden;
                if (r == n - 1) {
                    gnum = clast;
                    gden = cprev;
                } else {
                    gnum = fma(yf, xb, xf * yb);
                    gden = xf * xb;
                }
                gamma = gnum / gden;
                negc = cntf + cntb + sign_bit(gamma);
                // z_i = t_i f_f (i < r), f_f = 2^ref_f / G_f(r) = mf 2^ef;
                // z_i = t_i f_b (i > r), f_b = 2^ref_b / G_b(r) = mb 2^eb
                const double qmr = __ldg(Qm + r), iqmr = __ldg(iQm + r);
                const int qer = __ldg(Qe + r);
                const double mf = 1.0 / (xf * iqmr);
                const int ef = ref_f - sf + qer;
                const double mb = (r < n - 1) ? 1.0 / (qmr * xb) : 0.0;
                const int eb = ref_b - sb - qer;
                const double sumf = scale2(scale2(ssf * mf, ef) * mf, ef);
                const double sumb = (r < n - 1) ? scale2(scale2(ssb * mb, eb) * mb, eb) : 0.0;
                nrm2 = 1.0 + sumf + sumb;
                // the next iteration's scales: log2 |G(r)| of this one
                const int nref_f = ref_f - (ef + biased_exp(mf) - 1023);
                const int nref_b = (r < n - 1) ? ref_b - (eb + biased_exp(mb) - 1023) : ref_b;
                // the entry of largest magnitude (ties to the lowest index) becomes positive
                double zmax = -1.0;
                bool neg = false;
                if (mbf >= 0) {
                    zmax = fabs(scale2(__longlong_as_double(mbf) * mf, ef));
                    neg = (mnf != 0) != (mf < 0.0);
                }
                if (1.0 > zmax) { zmax = 1.0; neg = false; }
                if (mbb >= 0 && r < n - 1) {
                    const double zb = fabs(scale2(__longlong_as_double(mbb) * mb, eb));
                    if (zb > zmax) { zmax = zb; neg = (mnb != 0) != (mb < 0.0); }
                }
                const double inv = (neg ? -1.0 : 1.0) / sqrt(nrm2);
                Ff = scale2(mf * inv, ef);
                Fb = (r < n - 1) ? scale2(mb * inv, eb) : 0.0;
                Fr = inv;
                // scales far off: t_i = z_i / f, and a factor f beyond 2^+-400 means that
                // the t_i of this iteration sat near the ends of the binary64 range (small
                // entries flushed to zero, or an overflow): redo at the same lam with the
                // scales of this iteration, which make f = 1.  G(r) can move by such powers of
                // two between iterations when leading minors are nearly singular at lam
                // (glued matrices).
                const int lgf2 = (r > 0) ? ef + biased_exp(mf) - 1023 : 0;
                const int lgb2 = (r < n - 1) ? eb + biased_exp(mb) - 1023 : 0;
                bad_scale = !(nrm2 < 1e300) || !is_finite(Ff) || !is_finite(Fb) ||
                            !(ssf < 1e300) || !(ssb < 1e300) || lgf2 > 400 || lgf2 < -400 ||
                            lgb2 > 400 || lgb2 < -400;
                ref_f = nref_f;
                ref_b = nref_b;
            }
            if (done) continue;
            if (bad_scale) continue; // same lam, same r, new scales
            // ---- acceptance (uniform within the team)
            ++it_n;
            if (negc >= j) h = fmin(h, lam); else l = fmax(l, lam);
            if (!full && final_pending) { done = true; continue; }
            const double resid = fabs(gamma) / sqrt(nrm2);
            rqc = gamma / nrm2;
            const bool conv = (resid < tol1 * gap) || (fabs(rqc) < tol2 * fabs(lam));
            // RQI converges cubically; a correction that no longer shrinks (at least by
            // half) while tiny against the gap sits at the representation's noise level
            const bool stalled = it_n >= 2 && fabs(rqc) >= 0.5 * prev_arqc && fabs(rqc) <= 1e-3 * gap;
            const bool nofault = !(fault_mask & MR3_FAULT_RQI_NOCONV);
            // an accepted full factorization is followed by one iteration with its twist
            // index at the same lam, which writes the vector
            if (fb || ((conv || stalled) && nofault)) {
                if (full) final_pending = true; else done = true;
                continue;
            }
            prev_arqc = fabs(rqc);
            const bool sign_ok = (negc < j) ? (rqc > 0.0) : (rqc < 0.0);
            const double lnew = lam + rqc;
            if (it_n < max_rqi && sign_ok && lnew >= l && lnew <= h) {
                lam = lnew;
                continue;
            }
            // a correction at the rounding noise of the factorization cannot improve lam
            if (nofault && fabs(rqc) <= tol_noise * fabs(lam)) {
                if (full) final_pending = true; else done = true;
                continue;
            }
            if (it_n >= max_rqi) capped = true;
            // bisection to full accuracy, as a multisection over the team's lanes (lane k
            // counts at the (k+1)-th of kTeam interior points; the team ballot of
            // "count < j" picks the part holding lambda_j), then one more Getvec
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
                const int tt = __popc(bal);
                const double xl = __shfl_sync(tmask, x, tbase + (tt > 0 ? tt - 1 : 0));
                const double xh = __shfl_sync(tmask, x, tbase + (tt < kTeam ? tt : kTeam - 1));
                if (tt > 0) l = xl;
                if (tt < kTeam) h = xh;
            }
            lam = l + 0.5 * (h - l);
            r = -1;
            fb = true;
        }
        // ---- one pass over the vector: each side times its factor (1/||z|| and the sign
        // included), and the Rayleigh quotient z^T T z of the unit vector (lane k of a team
        // holds entries k, k + TEAM, ...; the neighbour entry comes from the next lane, or
        // from the team's last lane of the previous round)
        if (active && !done && k == 0) ++ncap; // guard exhausted: the last iteration stands
        const int nw = (int)__reduce_max_sync(FULL_MASK, (unsigned)(active ? n : 0));
        double rq = 0.0, carry = 0.0;
        for (int base = 0; base < nw; base += kTeam) {
            const int i = base + k;
            const bool act = active && r >= 0 && i < n;
            double z = 0.0;
            if (act) {
                const double tv = (i == r) ? 1.0 : zc[i];
                z = tv * ((i < r) ? Ff : ((i > r) ? Fb : Fr));
                zc[i] = z;
            }
            const double zn = __shfl_down_sync(FULL_MASK, z, 1, kTeam);
            const double zp = __shfl_sync(FULL_MASK, carry, tbase + kTeam - 1);
            if (act) {
                rq = fma(__ldg(td + i) * z, z, rq);
                if (k < kTeam - 1 && i + 1 < n) rq = fma(2.0 * __ldg(te + i) * z, zn, rq);
                if (k == 0 && i > 0) rq = fma(2.0 * __ldg(te + i - 1) * zp, z, rq);
            }
            carry = z;
        }
        if (active && k == 0) steps += (unsigned long long)((n + kTeam - 1) / kTeam);
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
                                        fault_mask, work_counter, info, nullptr, 0, 0);
    else
        k_rqi<8><<<nblocks, 32, 0, s>>>(nsingle, singles, nodes, blks, mats, pool, jloc, lo, hi,
                                        gapl, gapr, d, e, w, Z, scratch, nmax, max_rqi,
                                        fault_mask, work_counter, info, nullptr, 0, 0);
}

void launch_rqi_dev(int max_single, const int *dnsingle, int nmat, int forced_team,
                    const SingleItem *singles, const Node *nodes, const BlkDesc *blks,
                    const MatDesc *mats, const double *pool, const int *jloc, const double *lo,
                    const double *hi, const double *gapl, const double *gapr, const double *d,
                    const double *e, double *w, double *Z, double *scratch, int nslots2,
                    int nslots8, int nmax, int max_rqi, unsigned fault_mask, int *work_counter,
                    DevInfo *info, cudaStream_t s) {
    if (max_single <= 0) return;
    cudaMemsetAsync(work_counter, 0, sizeof(int), s);
    const int b2 = std::min(nslots2, (max_single + 15) / 16);
    const int b8 = std::min(nslots8, (max_single + 3) / 4);
    k_rqi<2><<<b2, 32, 0, s>>>(max_single, singles, nodes, blks, mats, pool, jloc, lo, hi, gapl,
                               gapr, d, e, w, Z, scratch, nmax, max_rqi, fault_mask, work_counter,
                               info, dnsingle, nmat, forced_team);
    k_rqi<8><<<b8, 32, 0, s>>>(max_single, singles, nodes, blks, mats, pool, jloc, lo, hi, gapl,
                               gapr, d, e, w, Z, scratch, nmax, max_rqi, fault_mask, work_counter,
                               info, dnsingle, nmat, forced_team);
}

int rqi_team(long long nsingle, int nmat) { return rqi_team_rule(nsingle, nmat, 0); }
int rqi_scratch_per_index(int team) { return kScratchPerSingleton * (32 / team); }
int rqi_singles_per_slot(int team) { return 32 / team; }

cudaError_t preload_rqi() { return load_kernels(k_rqi<2>, k_rqi<8>); }

} // namespace mr3
