// mr3_df.cuh -- double-float ("double-word" binary32) arithmetic and the Sturm count in it.
//
// The thesis' mixed-precision MRRR (Ch. 5, "Arithmetic used to approximate eigenvalues")
// computes eigenvalue approximations in a cheaper x-bit arithmetic on a rounded copy M_x of
// the representation M_y, which is safe as long as (k_rr + k_bi) n eps_x <~ gaptol.  On
// GB300 binary32 runs ~56x faster than binary64, so the bisection here works on a
// double-float copy of each representation (unit roundoff ~2^-47, so (k_rr + k_bi) n eps_x
// ~ 1e-9 at n = 8192, far below gaptol = 1e-3).
//
// Building blocks, all with explicitly rounded intrinsics so that no contraction can
// change them:
//   TwoSum (Knuth, TAOCP vol. 2), Fast2Sum (Dekker 1971), TwoProd via FMA;
//   double-word + double-word "accurate" addition and double-word x double-word
//   multiplication of Joldes, Muller and Popescu (ACM TOMS 44(2), 2017).
#pragma once
#include <cuda_runtime.h>

namespace mr3 {

struct dfloat {
    float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    float sh, sl, th, tl;
    two_sum(x.h, y.h, sh, sl);
    two_sum(x.l, y.l, th, tl);
    sl = __fadd_rn(sl, th);
    fast_two_sum(sh, sl, sh, sl);
    sl = __fadd_rn(sl, tl);
    dfloat r;
    fast_two_sum(sh, sl, r.h, r.l);
    return r;
}

__device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
    const float ch = __fmul_rn(x.h, y.h);
    float cl = __fmaf_rn(x.h, y.h, -ch);
    const float tl = __fmul_rn(x.h, y.l);
    cl = __fadd_rn(cl, __fmaf_rn(x.l, y.h, tl));
    dfloat r;
    fast_two_sum(ch, cl, r.h, r.l);
    return r;
}

__device__ __forceinline__ dfloat df_neg(dfloat x) { return {-x.h, -x.l}; }

// x y + z in one pass: the leading product exactly (TwoProd by FMA), the cross terms and
// the low words in single rounding, one TwoSum of the leading parts and a final Fast2Sum.
// The error is a few units of 2^-48 times |x y| + |z| (not of the result): in the Sturm
// count that is a relative perturbation of d_i and of s_i, which the mixed stability of
// dstqds admits, so the count stays exact for a slightly perturbed representation.
__device__ __forceinline__ dfloat df_fma(dfloat x, dfloat y, dfloat z) {
    const float p = __fmul_rn(x.h, y.h);
    const float pe = __fmaf_rn(x.h, y.h, -p);
    const float t = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.h));
    float s, e;
    two_sum(p, z.h, s, e);
    const float lo = __fadd_rn(e, __fadd_rn(pe, __fadd_rn(t, z.l)));
    dfloat r;
    fast_two_sum(s, lo, r.h, r.l);
    return r;
}

// x1 y1 + x2 y2 in one pass (same construction and error form as df_fma).
__device__ __forceinline__ dfloat df_dot2(dfloat x1, dfloat y1, dfloat x2, dfloat y2) {
    const float p1 = __fmul_rn(x1.h, y1.h);
    const float e1 = __fmaf_rn(x1.h, y1.h, -p1);
    const float t1 = __fmaf_rn(x1.h, y1.l, __fmul_rn(x1.l, y1.h));
    const float p2 = __fmul_rn(x2.h, y2.h);
    const float e2 = __fmaf_rn(x2.h, y2.h, -p2);
    const float t2 = __fmaf_rn(x2.h, y2.l, __fmul_rn(x2.l, y2.h));
    float s, e;
    two_sum(p1, p2, s, e);
    const float lo = __fadd_rn(e, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(t1, t2)));
    dfloat r;
    fast_two_sum(s, lo, r.h, r.l);
    return r;
}

// Nearest double-float to a double (exact when the double has at most 48 significant
// bits); the tail is computed in binary64 once per datum.
__device__ __forceinline__ dfloat df_from(double x) {
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(x - (double)h);
    return {h, l};
}
__device__ __forceinline__ double df_to(dfloat x) { return (double)x.h + (double)x.l; }

// ---- scaled double-float copies of a representation
//
// The error bound of the count below (a few units of 2^-48 per operation, relative) holds
// only while every binary32 product and the rounding error TwoProd extracts from it are
// normal numbers.  A representation of small norm breaks that: with entries ~2^-40 and
// (a, c) rescaled down to 2^-40, the error words fall to the subnormal range and carry
// ~2^-42 relative precision, 64 times the bound the bisection widens by.  Sturm counts
// do not change when d, dll and sigma are scaled by one power of two, so the copy of each
// representation holds 2^k (d, dll) with its largest entry in [1, 2), and the count runs
// at 2^k sigma.  A copy is used only when every scaled pivot is at least 2^-46 (with
// |c| >= 2^-40 the products d_i c_{i-1} then stay above 2^-86, and a binary32 product
// and its TwoProd error word are exact down to ~2^-101) and every nonzero scaled dll_i
// at least 2^-100 (its double-float tail normal); otherwise the node counts in binary64.
// Entries of order one also keep the growth of c over a few unrolled steps far from the
// binary32 overflow.
constexpr int kDfTopExp = 0;

// k with amax 2^k in [1, 2) (amax > 0 and finite).
__device__ __forceinline__ int df_scale_exp(double amax) {
    int e;
    (void)frexp(amax, &e); // amax in [2^(e-1), 2^e)
    return kDfTopExp + 1 - e;
}

// One scaled entry pair (pivot, dll) usable in double-float.
__device__ __forceinline__ bool df_entry_ok(double ds, double dlls) {
    const double a = fabs(ds), b = fabs(dlls);
    return a >= 0x1p-46 && a <= 0x1p100 && (b == 0.0 || (b >= 0x1p-100 && b <= 0x1p100));
}

// A scaled shift usable in double-float: zero, or in [2^-80, 2^100] (see the magnitudes
// of the count below).
__device__ __forceinline__ bool df_shift_ok(double xs) {
    const double a = fabs(xs);
    return a == 0.0 || (a >= 0x1p-80 && a <= 0x1p100);
}

// Writes the scaled copy of the representation with pivots d[0..n) and dll[0..n-1) to
// out[0..n) (float4 {d.h, d.l, dll.h, dll.l}; dll_{n-1} = 0), warp-collective.  Returns
// whether the copy is usable; kexp receives k.
__device__ __forceinline__ bool df_write_copy_warp(int n, const double *d, const double *dll,
                                                   float4 *out, int &kexp) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    double amax = 0.0;
    bool fin = true;
    for (int i = lane; i < n; i += 32) {
        const double x = d[i], y = (i < n - 1) ? dll[i] : 0.0;
        fin &= isfinite(x) && isfinite(y);
        amax = fmax(amax, fmax(fabs(x), fabs(y)));
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    fin = __all_sync(0xffffffffu, fin);
    const int k = (fin && amax > 0.0) ? df_scale_exp(amax) : 0;
    bool ok = fin && amax > 0.0;
    for (int i = lane; i < n; i += 32) {
        const double xs = scalbn(d[i], k), ys = (i < n - 1) ? scalbn(dll[i], k) : 0.0;
        ok &= df_entry_ok(xs, ys);
        const dfloat a = df_from(xs), b = df_from(ys);
        out[i] = make_float4(a.h, a.l, b.h, b.l);
    }
    ok = __all_sync(0xffffffffu, ok);
    kexp = k;
    return ok;
}

// The same for one thread.
__device__ __forceinline__ bool df_write_copy_serial(int n, const double *d, const double *dll,
                                                     float4 *out, int &kexp) {
    double amax = 0.0;
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        const double x = d[i], y = (i < n - 1) ? dll[i] : 0.0;
        ok &= isfinite(x) && isfinite(y);
        amax = fmax(amax, fmax(fabs(x), fabs(y)));
    }
    ok &= amax > 0.0;
    const int k = ok ? df_scale_exp(amax) : 0;
    for (int i = 0; i < n; ++i) {
        const double xs = scalbn(d[i], k), ys = (i < n - 1) ? scalbn(dll[i], k) : 0.0;
        ok &= df_entry_ok(xs, ys);
        const dfloat a = df_from(xs), b = df_from(ys);
        out[i] = make_float4(a.h, a.l, b.h, b.l);
    }
    kexp = k;
    return ok;
}

// Magnitudes.  c and a = s c share one scale, and s can be far below the data (s_1 =
// -sigma, and s stays of the order of sigma along stretches of the chain when sigma is
// tiny against the data).  So c is kept high, near 2^30 (rescaled when it leaves
// [2^-10, 2^70]), and shifts below 2^-80 count in binary64 (df_shift_ok): then sigma c
// >= 2^-90 and d_i c >= 2^-56, and in every sum of the recurrence the larger term keeps
// exact TwoProd error words (normal down to ~2^-101).  With c near 1 instead, a and its
// products fell below the binary32 range on a glued Wilkinson matrix at sigma ~ 2^-67
// (relative), the error words flushed to zero and a count came out one too high.
constexpr int kDfCExp = 30; // c is normalised to [2^30, 2^31)

// One step of the double-float count with per-step rules: an exactly zero c_i counts as a
// negative pivot (the limit sigma -> sigma+), (a, c) are rescaled to |c| in
// [2^30, 2^31) when c leaves [2^-10, 2^70]; false when the recurrence left the binary32
// range.
__device__ __forceinline__ bool df_step_exact(const float4 q, bool last, dfloat ns, dfloat &a,
                                              dfloat &cp, int &sp, int &cnt) {
    dfloat c = df_fma({q.x, q.y}, cp, a);
    const bool z = (c.h == 0.f);
    const int sc = z ? (sp ^ 1) : (__float_as_int(c.h) < 0 ? 1 : 0);
    cnt += sc ^ sp;
    if (!last) {
        a = df_dot2({q.z, q.w}, a, ns, c);
        const int ex = (__float_as_int(c.h) >> 23) & 0xff;
        if ((unsigned)(ex - (127 - 10)) > 80u && !z) {
            if (ex == 0xff) return false;
            // to [2^30, 2^31) in two exact factors: 2^(127-ex) (2^126 for a subnormal c),
            // each representable, then 2^30
            const float s1 = ex > 0 ? __int_as_float((254 - ex) << 23) : 0x1p126f;
            const float s2 = __int_as_float((127 + kDfCExp) << 23);
            c.h = __fmul_rn(__fmul_rn(c.h, s1), s2);
            c.l = __fmul_rn(__fmul_rn(c.l, s1), s2);
            a.h = __fmul_rn(__fmul_rn(a.h, s1), s2);
            a.l = __fmul_rn(__fmul_rn(a.l, s1), s2);
        }
        if (!(fabsf(a.h) < 0x1p120f)) return false;
    }
    cp = c;
    sp = sc;
    return true;
}

// NegCount on L D L^T at sigma in double-float, homogeneous form (see negcount_ldl in
// mr3_internal.cuh): c_i = d_i c_{i-1} + a_i, a_{i+1} = dll_i a_i - sigma c_i.  dd holds
// {d.h, d.l, dll.h, dll.l} per index, scaled as above, and sigma carries the same scale.
// As in negcount_ldl, the serial loop has no data-dependent branch: blocks of 4 unrolled
// steps (an exact zero pivot needs no test, its pair with the next pivot contributes one
// negative either way), then (a, c) normalised by a power of two (measured on GB300: 108
// cycles per step against 255 with the per-step rescale test).  A flag collected off the
// recurrence marks a block in which c fell below 2^-10 (see the magnitudes above) or a
// value left the range; such a block is redone with the per-step rules.  Returns -1 if the recurrence left the binary32
// range (the caller then counts in binary64).
__device__ __forceinline__ float df_norm_pow2(float c) {
    const int ex = (__float_as_int(c) >> 23) & 0xff;
    // called with |c| >= 2^-10 (ex >= 117) or an exact zero; other values left unscaled
    return (ex >= 1 + kDfCExp && ex < 0xff) ? __int_as_float((254 + kDfCExp - ex) << 23) : 1.f;
}

__device__ __forceinline__ int negcount_df(int n, const float4 *__restrict__ dd, dfloat sigma) {
    const dfloat ns = df_neg(sigma);
    const float c0s = __int_as_float((127 + kDfCExp) << 23); // 2^30
    dfloat a = {__fmul_rn(ns.h, c0s), __fmul_rn(ns.l, c0s)}, cp = {c0s, 0.f};
    int sp = 0, cnt = 0, i = 0;
    float4 qn = __ldg(dd); // prefetched data of step i
    for (; i + 4 < n; i += 4) {
        const dfloat a0 = a, c0 = cp;
        const int sp0 = sp, cnt0 = cnt;
        unsigned bad = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 q = qn;
            qn = __ldg(dd + i + u + 1);
            const dfloat c = df_fma({q.x, q.y}, cp, a);
            const int sc = __float_as_int(c.h) < 0 ? 1 : 0;
            cnt += sc ^ sp;
            sp = sc;
            a = df_dot2({q.z, q.w}, a, ns, c);
            const int ex = (__float_as_int(c.h) >> 23) & 0xff;
            bad |= ((unsigned)(ex - (127 - 10)) > 137u || !(fabsf(a.h) < 0x1p120f)) ? 1u : 0u;
            cp = c;
        }
        if (__builtin_expect(bad != 0, 0)) {
            a = a0;
            cp = c0;
            sp = sp0;
            cnt = cnt0;
            for (int k = i; k < i + 4; ++k)
                if (!df_step_exact(__ldg(dd + k), false, ns, a, cp, sp, cnt)) return -1;
        }
        const float q = df_norm_pow2(cp.h);
        cp.h = __fmul_rn(cp.h, q);
        cp.l = __fmul_rn(cp.l, q);
        a.h = __fmul_rn(a.h, q);
        a.l = __fmul_rn(a.l, q);
        if (!(fabsf(a.h) < 0x1p120f)) return -1;
    }
    for (; i < n; ++i) {
        const float4 q = qn;
        if (i + 1 < n) qn = __ldg(dd + i + 1);
        if (!df_step_exact(q, i == n - 1, ns, a, cp, sp, cnt)) return -1;
    }
    return cnt;
}

} // namespace mr3
