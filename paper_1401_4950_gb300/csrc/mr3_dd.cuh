// mr3_dd.cuh -- double-double ("double-word" binary64) arithmetic for the mixed-precision
// variant of the thesis (Ch. 5): binary64 input and output, the representation tree
// (shifts, twisted factorizations, Rayleigh-quotient iteration) in a working format with
// unit roundoff eps_y ~ 2^-104, which allows gaptol down to ~eps_y sqrt(n) / eps_x
// (Eq. gaptolinterval) and so removes almost all clusters.
//
// Building blocks, with explicitly rounded intrinsics so that no contraction changes them:
//   TwoSum (Knuth, TAOCP vol. 2), Fast2Sum (Dekker 1971), TwoProd via FMA;
//   double-word + double-word "accurate" addition, double-word x double-word and
//   double-word x binary64 multiplication (Joldes, Muller and Popescu, ACM TOMS 44(2),
//   2017); reciprocal by one Newton step on the binary64 reciprocal, division as a product
//   with it.
#pragma once
#include <cuda_runtime.h>

namespace mr3 {

struct ddouble {
    double h, l;
};

__device__ __forceinline__ void dd_two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

__device__ __forceinline__ void dd_fast_two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    e = __dsub_rn(b, __dsub_rn(s, a));
}

__device__ __forceinline__ ddouble dd_make(double h) { return {h, 0.0}; }
__device__ __forceinline__ ddouble dd_neg(ddouble x) { return {-x.h, -x.l}; }

__device__ __forceinline__ ddouble dd_add(ddouble x, ddouble y) {
    double sh, sl, th, tl;
    dd_two_sum(x.h, y.h, sh, sl);
    dd_two_sum(x.l, y.l, th, tl);
    sl = __dadd_rn(sl, th);
    dd_fast_two_sum(sh, sl, sh, sl);
    sl = __dadd_rn(sl, tl);
    ddouble r;
    dd_fast_two_sum(sh, sl, r.h, r.l);
    return r;
}
__device__ __forceinline__ ddouble dd_sub(ddouble x, ddouble y) { return dd_add(x, dd_neg(y)); }

// x + b, b binary64
__device__ __forceinline__ ddouble dd_add_d(ddouble x, double b) {
    double sh, sl;
    dd_two_sum(x.h, b, sh, sl);
    sl = __dadd_rn(sl, x.l);
    ddouble r;
    dd_fast_two_sum(sh, sl, r.h, r.l);
    return r;
}

__device__ __forceinline__ ddouble dd_mul(ddouble x, ddouble y) {
    const double ch = __dmul_rn(x.h, y.h);
    double cl = __fma_rn(x.h, y.h, -ch);
    const double tl = __dmul_rn(x.h, y.l);
    cl = __dadd_rn(cl, __fma_rn(x.l, y.h, tl));
    ddouble r;
    dd_fast_two_sum(ch, cl, r.h, r.l);
    return r;
}

// x * b, b binary64
__device__ __forceinline__ ddouble dd_mul_d(ddouble x, double b) {
    const double ch = __dmul_rn(x.h, b);
    double cl = __fma_rn(x.h, b, -ch);
    cl = __fma_rn(x.l, b, cl);
    ddouble r;
    dd_fast_two_sum(ch, cl, r.h, r.l);
    return r;
}

// exact product of two binary64 numbers
__device__ __forceinline__ ddouble dd_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    return {p, __fma_rn(a, b, -p)};
}

// 1 / y: the binary64 reciprocal r0 of y.h, corrected by one Newton step carried in
// double-word, r = r0 + r0 (1 - y r0), with the residual 1 - y r0 formed from the exact
// product (relative error of r about 2^-104).
__device__ __forceinline__ ddouble dd_rcp(ddouble y) {
    const double r0 = __drcp_rn(y.h);
    const ddouble p = dd_mul_d(y, r0);
    const double e = __dsub_rn(__dsub_rn(1.0, p.h), p.l);
    ddouble r;
    dd_fast_two_sum(r0, __dmul_rn(r0, e), r.h, r.l);
    return r;
}

// x / y as x (1 / y): one binary64 reciprocal instead of two binary64 divisions.
__device__ __forceinline__ ddouble dd_div(ddouble x, ddouble y) { return dd_mul(x, dd_rcp(y)); }

// x * 2^k exactly (k within the normal range of both words)
__device__ __forceinline__ ddouble dd_scale(ddouble x, double pow2) {
    return {__dmul_rn(x.h, pow2), __dmul_rn(x.l, pow2)};
}

__device__ __forceinline__ bool dd_neg_sign(ddouble x) {
    // the sign of a normalised double-word is the sign of its leading word (signed zero
    // counts as negative, as SignBit in the Sturm counts)
    return ((unsigned long long)__double_as_longlong(x.h) >> 63) != 0;
}

__device__ __forceinline__ double dd_abs_h(ddouble x) { return fabs(x.h); }

} // namespace mr3
