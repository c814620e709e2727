// Float-float ("double-single") arithmetic on the float32 pipes.
//
// A value is an unevaluated sum h + l of two floats with |l| <= ulp(h)/2, about 48 significant bits.
// The error-free transformations are the classical ones: Knuth's TwoSum (6 flops, any operand
// order), Dekker's Fast2Sum (3 flops, |a| >= |b|) and TwoProd through a fused multiply-add (2 flops).
// On this GPU float64 issues at ~1/64 of float32, so float-float arithmetic at ~10-20 float32
// operations per product is several times faster than native float64 while keeping ~1e-14 relative
// precision (the exponent range stays that of float32).
//
// Every function forces the rounding steps with __fadd_rn / __fmul_rn / __fmaf_rn so the compiler
// cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace pswf {

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_make(float h) { return ff{h, 0.f}; }

__device__ __forceinline__ ff ff_from_double(double v) {
    const float h = __double2float_rn(v);
    return ff{h, __double2float_rn(v - static_cast<double>(h))};
}

__device__ __forceinline__ double ff_to_double(ff a) { return static_cast<double>(a.h) + static_cast<double>(a.l); }

// Knuth: s + e = a + b exactly
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fadd_rn(s, -a);
    const float e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -v)), __fadd_rn(b, -v));
    return ff{s, e};
}

// Dekker: s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff{s, __fadd_rn(b, -__fadd_rn(s, -a))};
}

// p + e = a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return ff{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.h, b.h);
    s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, s.l);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.h, b.h);
    p.l = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l));
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.h, b);
    p.l = __fmaf_rn(a.l, b, p.l);
    return fast_two_sum(p.h, p.l);
}

// a * b + c
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) { return ff_add(ff_mul(a, b), c); }

// Compensated accumulation acc += a * b in the manner of Ogita, Rump and Oishi's Dot2 (SIAM J. Sci.
// Comput. 26, 2005): acc.h carries the float32 running sum, acc.l the exact rounding errors of every
// product and sum (plus the cross terms of the float-float operands).  acc stays unnormalised until
// ff_norm; 12 float32 operations per term instead of 18 for ff_add(ff_mul(a, b), acc).
__device__ __forceinline__ void ff_acc(ff& acc, ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const ff s = two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}

// acc += a * b for a float32 factor b
__device__ __forceinline__ void ff_acc_f(ff& acc, ff a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    const ff s = two_sum(acc.h, p);
    acc.h = s.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}

// Horner step p * u + c keeping p unnormalised: the product's rounding error (FMA) and the cross terms
// go to the low word, the sum with c.h is exact (TwoSum) and its error joins the low word too; no
// renormalisation between steps (|p.l| stays within a few ulp(p.h)).  12 operations instead of 18 for
// ff_add(ff_mul(p, u), c).  Renormalise the result with ff_norm.
__device__ __forceinline__ ff ff_horner_step(ff p, ff u, ff c) {
    const float ph = __fmul_rn(p.h, u.h);
    float pl = __fmaf_rn(p.h, u.h, -ph);
    pl = __fmaf_rn(p.h, u.l, pl);
    pl = __fmaf_rn(p.l, u.h, pl);
    const ff s = two_sum(ph, c.h);
    return ff{s.h, __fadd_rn(s.l, __fadd_rn(pl, c.l))};
}

// renormalise an accumulator (|l| <= ulp(h)/2 afterwards)
__device__ __forceinline__ ff ff_norm(ff a) { return two_sum(a.h, a.l); }

// a^2 for a normalised a
__device__ __forceinline__ ff ff_sqr(ff a) {
    ff p = two_prod(a.h, a.h);
    p.l = __fmaf_rn(__fmul_rn(2.f, a.h), a.l, p.l);
    return fast_two_sum(p.h, p.l);
}

__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
    return ff{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

// 1/sqrt(v) for v > 0: float32 estimate y0 (rsqrtf, a few ulp), then the series
// v^(-1/2) = y0 (1 - r)^(-1/2) = y0 (1 + r/2 + 3 r^2/8 + O(r^3)) with r = 1 - v y0^2 formed in
// float-float (|r| < ~1e-6, so the float32 correction term is accurate to ~2^-46 of y0).
__device__ __forceinline__ ff ff_rsqrt(ff v) {
    const float y0 = rsqrtf(v.h);
    const ff vy2 = ff_mul(v, two_prod(y0, y0));
    const float r = __fadd_rn(__fadd_rn(1.f, -vy2.h), -vy2.l);   // 1 - vy2.h is exact (Sterbenz)
    const float corr = __fmul_rn(y0, __fmul_rn(r, __fmaf_rn(0.375f, r, 0.5f)));
    return fast_two_sum(y0, corr);
}

}  // namespace pswf
