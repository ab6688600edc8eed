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

// Values whose double-float copy keeps full precision: normal binary32 tails need
// |x| >= 2^-100 (tail ~ 2^-24 |x|), and |x| <= 2^100 keeps head products finite.
__device__ __forceinline__ bool df_safe(double x) {
    const double a = fabs(x);
    return a == 0.0 || (a >= 0x1p-100 && a <= 0x1p100);
}

// NegCount on L D L^T at sigma in double-float, homogeneous form (see negcount_ldl in
// mr3_internal.cuh): c_i = d_i c_{i-1} + a_i, a_{i+1} = dll_i a_i - sigma c_i, with
// (a, c) rescaled by a power of two when c leaves [2^-40, 2^40].  dd holds
// {d.h, d.l, dll.h, dll.l} per index.  Returns -1 if the recurrence left the binary32
// range (the caller then counts in binary64).
__device__ __forceinline__ int negcount_df(int n, const float4 *__restrict__ dd, dfloat sigma) {
    const dfloat ns = df_neg(sigma);
    dfloat a = ns, cp = {1.f, 0.f};
    int sp = 0, cnt = 0;
    float4 qn = __ldg(dd); // prefetched data of step i
    for (int i = 0; i < n; ++i) {
        const float4 q = qn;
        if (i + 1 < n) qn = __ldg(dd + i + 1);
        const dfloat di = {q.x, q.y};
        dfloat c = df_fma(di, cp, a);
        if (c.h == 0.f) { c.h = -cp.h * 0x1p-30f; c.l = 0.f; }
        const int sc = __float_as_int(c.h) < 0 ? 1 : 0;
        cnt += sc ^ sp;
        if (i < n - 1) {
            const dfloat dlli = {q.z, q.w};
            a = df_dot2(dlli, a, ns, c);
            const int ex = (__float_as_int(c.h) >> 23) & 0xff;
            if ((unsigned)(ex - (127 - 40)) > 80u) {
                if (ex == 0xff) return -1;
                const float s = __int_as_float((254 - ex) << 23); // 2^(127-ex)
                c.h = __fmul_rn(c.h, s);
                c.l = __fmul_rn(c.l, s);
                a.h = __fmul_rn(a.h, s);
                a.l = __fmul_rn(a.l, s);
            }
            if (!(fabsf(a.h) < 0x1p120f)) return -1;
        }
        cp = c;
        sp = sc;
    }
    return cnt;
}

} // namespace mr3
