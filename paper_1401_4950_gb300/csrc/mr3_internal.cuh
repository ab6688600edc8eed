// mr3_internal.cuh -- data structures and device numerics shared by the MRRR kernels.
//
// Notation follows the thesis (Ch. 3): a representation is an N-representation of a
// lower bidiagonal factorization L D L^T with d (n pivots) and l (n-1 multipliers);
// the derived data dl_i = d_i l_i and dll_i = d_i l_i^2 are kept beside d (remark on
// Alg. NegCount on LDL^T, App. B).  A representation of order n occupies rep_size(n)
// doubles of a pool starting at an even double offset:
//   d at [0, n), dl at [n, 2n), dll at [2n, 3n);
//   from the even offset rep_df_offset(n), a double-float copy {d.h, d.l, dll.h, dll.l}
//   (one 16-byte aligned float4 per index) for the bisection;
//   from rep_q_offset(n), the prefix products Q_i = prod_{k<i} (-dl_k) as a mantissa
//   Qm_i in [1, 2) (signed), its reciprocal iQm_i and an int exponent Qe_i (the twisted
//   solve of the singletons multiplies them instead of running a product chain).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mr3 {

constexpr double kEps = 1.1102230246251565e-16;     // unit roundoff 2^-53
constexpr double kSafmin = 2.2250738585072014e-308; // underflow threshold omega
constexpr int kRepStride = 8; // doubles per index in a representation (plus kRepPad)
constexpr int kRepPad = 4;
__host__ __device__ __forceinline__ long long rep_size(int n) { return (long long)kRepStride * n + kRepPad; }
__host__ __device__ __forceinline__ long long rep_df_offset(int n) { return 3ll * n + (n & 1); }
__host__ __device__ __forceinline__ long long rep_q_offset(int n) { return rep_df_offset(n) + 2ll * n; }

// Classification threshold of the binary64 tree when the caller leaves gaptol at its
// default (Sec. 3.2.3).  The loss of orthogonality the tree attains grows like
// eps / gaptol (the thesis quotes O(n eps / gaptol) as the observed worst case of the
// bound on orthogonality, Sec. 3.1.2): two eigenvalues that are classified as singletons
// at a relative gap just above gaptol get vectors whose inner product is a few eps /
// gaptol.  Measured on Wilkinson-type pairs, that is about 3.6 eps / relgap, which only
// stays below 10 n eps while gaptol >= 0.36 / n.  So blocks of small order n_b use
// gaptol = 2 / n_b, capped at 0.05 (gaptol must stay well below 1 for clusters to break,
// Ch. 5), and larger blocks keep the customary 1e-3.
__host__ __device__ __forceinline__ double auto_gaptol(int nb) {
    const double g = 2.0 / (double)(nb > 1 ? nb : 1);
    return g < 1e-3 ? 1e-3 : (g > 0.05 ? 0.05 : g);
}
// Sentinel passed as gaptol: choose auto_gaptol(n_b) per block.
constexpr double kGaptolAuto = 0.0;

// One input matrix of a (possibly batched) solve.
struct MatDesc {
    long long off;  // first row in the packed d/e arrays
    long long zoff; // Z element offset of the first eigenvector of this matrix
    int n;          // order
    int ldz;        // leading dimension of this matrix's Z
    int woff;       // first global column (index into w and the per-column state)
    int m;          // eigenpairs selected (set on the device)
    int blk0, nblk; // blocks after splitting
    int il, iu;     // index range (range INDEX), 1-based
    double vl, vu;  // value range (range VALUE): (vl, vu]
    double tnorm;   // max(|gl|, |gu|) of the Gershgorin interval of the whole matrix
};

// One irreducible block (Sec. 3.2.1): the unit the root representation is built for.
struct BlkDesc {
    long long off;  // first row in the packed d/e arrays
    long long rep;  // offset of the root representation in the level-0 pool
    int n;          // order
    int mat;        // owning matrix
    int roff;       // first row inside the matrix
    int j0, j1;     // local eigenvalue indices selected (1-based, inclusive; j1 < j0: none)
    int col0;       // global column of local index j0
    int dfok;       // the root's double-float copy is usable (see df_entry_ok)
    int dfexp;      // the copy holds 2^dfexp (d, dll)
    double gl, gu;  // Gershgorin interval of the block
    double mu;      // root shift: M_root = T_block - mu I (before the random perturbation)
    double spdiam;  // gu - gl
};

// A node {M, I, sigma} of the representation tree (Alg. MRRR): a representation, a
// contiguous range of global columns, and the accumulated shift.
struct Node {
    long long rep;     // offset of the representation in this level's pool
    int blk;           // owning block
    int c0, c1;        // global columns (inclusive)
    int depth;
    int dfok;          // the double-float copy is usable (see df_entry_ok)
    int dfexp;         // the copy holds 2^dfexp (d, dll)
    double sigma;      // eigenvalue of T = eigenvalue of the representation + sigma
    double lnb, rnb;   // bounds (in this representation's coordinates) of the nearest
                       // eigenvalues outside [c0, c1]: upper bound of the left one, lower
                       // bound of the right one; -inf / +inf when there is none
};

struct ClusterItem {
    int node;          // parent node (current level)
    int c0, c1;        // cluster columns
    int act;           // first slot of its columns in the next level's active list
    double lnb, rnb;   // neighbour bounds outside the cluster (parent coordinates)
};

struct SingleItem {
    int col;
    int node;
};

struct LevelCounters {
    int nsingle;
    int ncluster;
    int maxcluster;
    int nactive;         // columns in clusters (refined on the next level)
    long long pool_need; // doubles needed for the child representations
    int overflow;        // the child representations did not fit a fixed pool
    int pad;
};

// ---- launch-shape rules shared by the host-driven level loop and the one captured in a
// graph (where the kernels read the counts from the device): the same count gives the
// same shape, and the shapes change the Sturm-count samples, hence the results.

// Lanes per eigenvalue of the multisection: enough lanes to keep about warps_per_sm warps
// per SM busy on 152 SMs, a power of two up to 32; tpe > 0 forces one.
__host__ __device__ __forceinline__ int bisect_lanes(long long nactive, int warps_per_sm, int tpe) {
    int L = 1;
    if (tpe > 0) {
        while (L * 2 <= tpe && L < 32) L *= 2;
        return L;
    }
    const long long target = 152ll * 32 * warps_per_sm;
    while (L < 32 && (long long)(2 * L) * nactive <= target) L *= 2;
    return L;
}

// Lanes per cluster end of the end refinement (phase 0 double-float, phase 1 binary64):
// many ends -> fewer lanes (throughput), few ends -> more (latency).
#ifndef MR3_REFINE_WARPS_PER_SM
#define MR3_REFINE_WARPS_PER_SM 8
#endif
#ifndef MR3_REFINE1_LANES_PER_SM
#define MR3_REFINE1_LANES_PER_SM 128
#endif
__host__ __device__ __forceinline__ long long refine_lane_cap(int phase) {
    return phase == 0 ? 152ll * 32 * MR3_REFINE_WARPS_PER_SM : 152ll * MR3_REFINE1_LANES_PER_SM;
}
__host__ __device__ __forceinline__ int refine_lanes(long long ends, int phase) {
    const long long cap = refine_lane_cap(phase);
    int E = phase == 0 ? 4 : 1;
    while (E < 32 && ends * (2 * E) <= cap) E *= 2;
    return E;
}

// RQI team size: teams of 2 once the singletons clearly outnumber what the resident warps
// hold with teams of 8; several matrices in one solve switch earlier (their singleton
// launch runs beside the other matrices' shift kernels).  forced = 2 or 8 overrides.
#ifndef MR3_RQI_TEAM2_MIN
#define MR3_RQI_TEAM2_MIN 32768
#endif
#ifndef MR3_RQI_TEAM2_MIN_MULTI
#define MR3_RQI_TEAM2_MIN_MULTI 2048
#endif
__host__ __device__ __forceinline__ int rqi_team_rule(long long nsingle, int nmat, int forced) {
    if (forced == 2 || forced == 8) return forced;
    return nsingle > (nmat > 1 ? MR3_RQI_TEAM2_MIN_MULTI : MR3_RQI_TEAM2_MIN) ? 2 : 8;
}

struct DevInfo {
    unsigned long long sturm_steps;
    unsigned long long shift_steps;
    unsigned long long twisted_steps;
    unsigned long long rqi_iters;
    int rqi_max;
    int fallbacks;
    int new_rrr;
    int untested;
    int nclusters;
    int largest;
    int dmax;
    int status[8];
    int ladder;       // clusters whose first two shift candidates failed the plain test
    int recomputed;   // ... of which a back-off candidate passed the growth test
    int env_accepted; // ... of which a first candidate passed the envelope test
    // multisection statistics, gathered only while trace is nonzero: [0] the bisection,
    // [1] and [2] the two phases of the cluster-end refinement.  Per launch: the items,
    // their sweeps (sum and maximum), and the lanes that counted over the lanes of the
    // warps' sweeps (the lane utilisation)
    int trace;
    int tr_max[3];
    unsigned long long tr_items[3], tr_sweeps[3], tr_lane_counts[3], tr_warp_lanes[3];
};

// Adds one warp's multisection statistics (all 32 lanes call it): sw counts of this lane,
// rounds the warp ran, group leaders (lead) add their item with its sweeps.
__device__ __forceinline__ void trace_sweeps(DevInfo *info, int kind, bool lead, int sw,
                                             int rounds) {
    unsigned long long c = (unsigned long long)sw;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lead && sw > 0) {
        atomicAdd(&info->tr_items[kind], 1ull);
        atomicAdd(&info->tr_sweeps[kind], (unsigned long long)sw);
        atomicMax(&info->tr_max[kind], sw);
    }
    if ((threadIdx.x & 31) == 0 && c) {
        atomicAdd(&info->tr_lane_counts[kind], c);
        atomicAdd(&info->tr_warp_lanes[kind], 32ull * (unsigned long long)rounds);
    }
}

// ------------------------------------------------------------------ bit helpers

__device__ __forceinline__ int sign_bit(double x) {
    return (int)((unsigned long long)__double_as_longlong(x) >> 63);
}
__device__ __forceinline__ int biased_exp(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}
// 2^k for -1022 <= k <= 1023 (exact power of two built from the exponent field).
// Approximate reciprocal of the hardware (rcp.approx.ftz.f64): for magnitudes in tests
// that need no correct rounding.
__device__ __forceinline__ double rcp_approx(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    return r;
}

__device__ __forceinline__ double pow2i(int k) {
    return __longlong_as_double((long long)(k + 1023) << 52);
}
__device__ __forceinline__ bool is_zero(double x) {
    return (((unsigned long long)__double_as_longlong(x)) << 1) == 0ull;
}
__device__ __forceinline__ bool is_finite(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// Counter-based SplitMix64 (Steele, Lea, Flood 2014): output for counter i of stream
// seed, mapped to a uniform double in (-1, 1).  Draws the random relative perturbation
// of the root representation (Alg. MRRR).
__device__ __forceinline__ double splitmix_pm1(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// ------------------------------------------------------------------ Sturm counts
//
// NegCount on L D L^T (App. B, Alg. NegCount on LDL^T) counts the negative pivots d+_i
// of L+ D+ L+^T = L D L^T - sigma I, computed by the dstqds recurrence
//     d+_i = d_i + s_i,   s_{i+1} = (s_i / d+_i) dll_i - sigma,   s_1 = -sigma.
// On GB300 an FP64 division costs ~10 FMA slots of throughput and ~650 cycles of
// latency, so the recurrence is evaluated in homogeneous (division-free) form: with
// c_i = d+_1 ... d+_i (times a positive power-of-two scale) and a_i = s_i c_{i-1},
//     c_i = d_i c_{i-1} + a_i,    a_{i+1} = dll_i a_i - sigma c_i,
// and sign(d+_i) = sign(c_i) xor sign(c_{i-1}).  Each rounding error can be pushed onto
// d_i or dll_i as an O(eps) relative perturbation (the pair (a, c) only shares a
// positive scale), so the count is exact for a relatively perturbed representation,
// the property bisection on an RRR relies on.
//
// Zero pivots (App. B remarks: SignBit(-0) = 1).  The homogeneous form needs no division,
// so an exactly zero c_i is simply kept: the next step gives c_{i+1} = dll_i a_i, the
// pivot d+_{i+1} = c_{i+1} / c_i is infinite, and the pair (d+_i, d+_{i+1}) contributes
// exactly one negative pivot whatever sign the zero carries (sign(c_{i+1}) =
// sign(c_{i-1}) xor 1 when dll_i and d_i share a sign), which is the count of the limit
// sigma -> sigma+ .  Only the last pivot has no successor: an exactly zero d+_{n-1}
// counts as negative.  A tiny substitute pivot would have to be tiny relative to the
// data, which carry no fixed scale.
//
// Scaling.  (a, c) must stay in the binary64 range.  A data-dependent branch inside the
// serial loop costs ~380 cycles per step on GB300 (measured: 593 against 215 cycles per
// step without it, whose two dependent FMAs are the critical path), so the loop runs in
// blocks of 8 unrolled steps without a branch and normalises (a, c) by a power of two
// at the end of each block.  A block whose end value left [2^-923, 2^877] (data of
// extreme magnitude, or a pivot near underflow) is redone from its saved state with a
// rescale after every step; the last steps run that way too.
__device__ __forceinline__ double norm_pow2(double c) {
    const int ex = biased_exp(c);
    return (ex > 0 && ex < 0x7ff) ? pow2i(1023 - ex) : 1.0;
}

// One step with the per-step rules (used for redone blocks and the last steps).
__device__ __forceinline__ void count_step_exact(double di, double li, double sigma, double &a,
                                                 double &cp, int &sp, int &cnt) {
    double c = fma(di, cp, a);
    const bool z = is_zero(c);
    const int sc = z ? (sp ^ 1) : sign_bit(c);
    cnt += sc ^ sp;
    a = fma(-sigma, c, li * a);
    const int ex = biased_exp(c);
    if ((unsigned)(ex - (1023 - 200)) > 400u && !z) {
        const double s = pow2i(1023 - ex);
        c *= s;
        a *= s;
    }
    cp = c;
    sp = sc;
}

__device__ __forceinline__ int negcount_ldl(int n, const double *__restrict__ d,
                                            const double *__restrict__ dll, double sigma) {
    double a = -sigma, cp = 1.0;
    int sp = 0, cnt = 0, i = 0;
    double dn = __ldg(d), ln = (n > 1) ? __ldg(dll) : 0.0; // prefetched data of step i
    for (; i + 8 < n; i += 8) {
        const double a0 = a, c0 = cp;
        const int sp0 = sp, cnt0 = cnt;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double di = dn, li = ln;
            dn = __ldg(d + i + u + 1);
            ln = (i + u + 1 < n - 1) ? __ldg(dll + i + u + 1) : 0.0;
            const double t = li * a;
            const double c = fma(di, cp, a);
            const int sc = sign_bit(c);
            cnt += sc ^ sp;
            sp = sc;
            a = fma(-sigma, c, t);
            cp = c;
        }
        const int ex = biased_exp(cp), ea = biased_exp(a);
        if (__builtin_expect(ea == 0x7ff || (unsigned)(ex - 100) > 1800u, 0)) {
            a = a0;
            cp = c0;
            sp = sp0;
            cnt = cnt0;
            for (int k = i; k < i + 8; ++k)
                count_step_exact(__ldg(d + k), (k < n - 1) ? __ldg(dll + k) : 0.0, sigma, a, cp, sp, cnt);
        }
        const double q = norm_pow2(cp);
        cp *= q;
        a *= q;
    }
    for (; i < n - 1; ++i) {
        const double di = dn, li = ln;
        dn = __ldg(d + i + 1);
        ln = (i + 1 < n - 1) ? __ldg(dll + i + 1) : 0.0;
        count_step_exact(di, li, sigma, a, cp, sp, cnt);
    }
    const double c = fma(dn, cp, a);
    const int sc = is_zero(c) ? (sp ^ 1) : sign_bit(c);
    cnt += sc ^ sp;
    return cnt;
}

// NegCount on T itself (App. B, Alg. NegCount on T) in single precision, used only to
// locate the extremal eigenvalues roughly before the root shift is chosen (the FP64
// factorization then verifies definiteness).  Homogeneous three-term form of the pivot
// recurrence d_i = (alpha_i - sigma) - beta_{i-1}^2 / d_{i-1}:
//     p_i = (alpha_i - sigma) p_{i-1} - beta_{i-1}^2 p_{i-2},   d_i = p_i / p_{i-1}.
__device__ __forceinline__ int negcount_T_f32(int n, const float *__restrict__ af,
                                              const float *__restrict__ b2f, float sigma) {
    float pm2 = 0.f, pm1 = 1.f;
    int sp = 0, cnt = 0;
    for (int i = 0; i < n; ++i) {
        const float q = (i > 0) ? b2f[i - 1] * pm2 : 0.f;
        float p = fmaf(af[i] - sigma, pm1, -q);
        const bool z = (p == 0.f); // zero pivot: negative, p_i = 0 kept (see negcount_ldl)
        const int sc = z ? (sp ^ 1) : (__float_as_int(p) < 0 ? 1 : 0);
        cnt += sc ^ sp;
        const int ex = (__float_as_int(p) >> 23) & 0xff;
        if ((unsigned)(ex - (127 - 40)) > 80u && !z) {
            const float s = __int_as_float((254 - ex) << 23); // 2^(127-ex)
            p *= s;
            pm1 *= s;
        }
        pm2 = pm1;
        pm1 = p;
        sp = sc;
    }
    return cnt;
}

// Q_i = prod_{k<i} (-dl_k), i = 0..n-1, for a representation at rep (warp-collective: a
// chunk of indices per lane, an exclusive product scan over the lanes, then each lane
// walks its chunk).  Stored as Qm (signed mantissa in [1, 2)), iQm = 1/Qm, Qe (exponent).
__device__ __forceinline__ void split_exp(double x, double &m, int &e) {
    if (is_zero(x) || !is_finite(x)) { m = x; e = 0; return; }
    const int ex = biased_exp(x);
    if (ex == 0) { x *= 0x1p+600; e = biased_exp(x) - 1023 - 600; m = x * pow2i(-(biased_exp(x) - 1023)); return; }
    e = ex - 1023;
    m = x * pow2i(-e);
}

__device__ __forceinline__ void build_prefix(int n, double *rep) {
    const int lane = threadIdx.x & 31;
    const double *dl = rep + n;
    double *Qm = rep + rep_q_offset(n);
    double *iQm = Qm + n;
    int *Qe = (int *)(iQm + n);
    const int ch = (n + 31) / 32;
    const int i0 = min(lane * ch, n), i1 = min(i0 + ch, n);
    // product of -dl_k over this lane's chunk (k < n-1)
    double m = 1.0;
    int e = 0;
    for (int k = i0; k < i1 && k < n - 1; ++k) {
        double t;
        int te;
        split_exp(-dl[k], t, te);
        m *= t;
        e += te;
        double mm;
        int me;
        split_exp(m, mm, me);
        m = mm;
        e += me;
    }
    // exclusive scan of (m, e) over lanes
    double pm = m;
    int pe = e;
    for (int o = 1; o < 32; o <<= 1) {
        const double ym = __shfl_up_sync(0xffffffffu, pm, o);
        const int ye = __shfl_up_sync(0xffffffffu, pe, o);
        if (lane >= o) {
            double mm;
            int me;
            split_exp(pm * ym, mm, me);
            pm = mm;
            pe = pe + ye + me;
        }
    }
    double xm = __shfl_up_sync(0xffffffffu, pm, 1);
    int xe = __shfl_up_sync(0xffffffffu, pe, 1);
    if (lane == 0) { xm = 1.0; xe = 0; }
    for (int i = i0; i < i1; ++i) {
        Qm[i] = xm;
        Qe[i] = xe;
        iQm[i] = 1.0 / xm;
        if (i < n - 1) {
            double t;
            int te;
            split_exp(-dl[i], t, te);
            double mm;
            int me;
            split_exp(xm * t, mm, me);
            xm = mm;
            xe = xe + te + me;
        }
    }
}

} // namespace mr3
