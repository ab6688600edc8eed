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
// representation holds 2^k (d, dll) with its largest entry in [2^20, 2^21), and the count
// runs at 2^k sigma.  A copy is used only when every scaled pivot is at least 2^-46 (with
// |c| >= 2^-40 the products d_i c_{i-1} then stay above 2^-86, and a binary32 product
// and its TwoProd error word are exact down to ~2^-101) and every nonzero scaled dll_i
// at least 2^-100 (its double-float tail normal); otherwise the node counts in binary64.
// On the other side, the largest entry at 2^21 keeps sigma c below 2^120 after the jump
// of c at a pivot as small as that.
constexpr int kDfTopExp = 20;

// k with amax 2^k in [2^20, 2^21) (amax > 0 and finite).
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

// A scaled shift usable in double-float (a tiny one loses only bits far below the data's).
__device__ __forceinline__ bool df_shift_ok(double xs) { return fabs(xs) <= 0x1p100; }

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

// NegCount on L D L^T at sigma in double-float, homogeneous form (see negcount_ldl in
// mr3_internal.cuh): c_i = d_i c_{i-1} + a_i, a_{i+1} = dll_i a_i - sigma c_i, with
// (a, c) rescaled by a power of two when c leaves [2^-40, 2^40].  dd holds
// {d.h, d.l, dll.h, dll.l} per index, scaled as above, and sigma carries the same scale.  Returns -1 if the recurrence left the binary32
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
        const bool z = (c.h == 0.f); // zero pivot: negative, c_i = 0 kept (see negcount_ldl)
        const int sc = z ? (sp ^ 1) : (__float_as_int(c.h) < 0 ? 1 : 0);
        cnt += sc ^ sp;
        if (i < n - 1) {
            const dfloat dlli = {q.z, q.w};
            a = df_dot2(dlli, a, ns, c);
            const int ex = (__float_as_int(c.h) >> 23) & 0xff;
            if ((unsigned)(ex - (127 - 40)) > 80u && !z) {
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
