// Paired-FP32 ("double-float") arithmetic for FP64-pipe-bound inner loops.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| at most
// a few units in the last place of hi: some 48 significant bits.  Every
// operation is built from the error-free transformations of FP32 sums and
// products -- Knuth's TwoSum (TAOCP vol. 2, Sec. 4.2.2), Dekker's fast
// two-sum (1971) and the exact product error fmaf(a, b, -a b) -- so it runs on
// the FP32 pipe, which on this GPU issues 64 times the FP64 rate.  Sums use
// the short form (exact error of the high parts, plain sum of the low
// parts): a few units of 2^-48 relative when both operands have the same
// sign, and a few units of 2^-48 of |a| + |b| absolute in general.  Sums and
// products leave the pair unnormalized (no closing two-sum: |lo| stays within
// a few ulp of hi, which every operation here accepts, and the error of the
// short chains the deposit forms stays near 2^-45); the square root and the
// conversion from a double return normalized pairs.  The
// explicit __f*_rn intrinsics keep the compiler from contracting or
// reordering the transformations.
#pragma once

#include <cuda_runtime.h>

#include "fpic_device.cuh"

namespace fpic {

struct ff {
    float hi, lo;
};

// s + e of two floats with |a| >= |b| (or a == 0): exact.
__device__ __forceinline__ ff ff_fast2(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_of(float a)
{
    return {a, 0.f};
}

// The double x as hi + lo, by integer operations on its bits (the FP64
// pipe's conversions would cost as much as FP64 arithmetic): hi takes the
// sign, exponent and leading 23 fraction bits, lo the remaining 29 bits
// rounded to a float (one fused multiply-add of two exact parts): within
// 2^-47 relative for 2^-70 <= |x| < 2^127; 0 below 2^-126 (and lo 0 below
// 2^-70), which only drops magnitudes under 2^-70 of the lattice values.
__device__ __forceinline__ ff ff_from(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
    const unsigned sign = hw & 0x80000000u;
    if (e < -126) return {0.f, 0.f};
    const float h = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    if (e < -70) return {h, 0.f};
    // remaining fraction m = lw mod 2^29 = mh 2^6 + ml; each part is a float
    // exactly (2^23 + m - 2^23), the sum is rounded once
    const unsigned m = lw & 0x1fffffffu;
    const float mh = __fsub_rn(__uint_as_float(0x4b000000u | (m >> 6)), 8388608.f);
    const float ml = __fsub_rn(__uint_as_float(0x4b000000u | (m & 63u)), 8388608.f);
    const float s46 = __uint_as_float((unsigned)(e - 46 + 127) << 23);   // 2^(e - 46)
    const float s52 = __uint_as_float((unsigned)(e - 52 + 127) << 23);   // 2^(e - 52)
    const float l = __fmaf_rn(mh, s46, __fmul_rn(ml, s52));
    return {h, __uint_as_float(__float_as_uint(l) | sign)};
}

// A normal float (or 0) as a double, by integer operations on its bits.
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e8 = (u >> 23) & 0xffu;
    if (e8 == 0u) return 0.0;
    const unsigned hw = (u & 0x80000000u) | ((e8 + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    return __longlong_as_double((long long)(((unsigned long long)hw << 32) | ((unsigned long long)(u & 7u) << 29)));
}

__device__ __forceinline__ double ff_to(ff a)
{
    return f2d_bits(a.hi) + f2d_bits(a.lo);
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float v = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
    return {s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

// a + b when a_hi >= b_hi >= 0 (more generally: a_hi's exponent at least
// b_hi's): Dekker's fast two-sum of the high parts gives the same sum and
// the same exact error as the two-sum in ff_add, so the same pair, with
// three additions fewer.
__device__ __forceinline__ ff ff_add_ge(ff a, ff b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    return {s, __fadd_rn(__fsub_rn(b.hi, __fsub_rn(s, a.hi)), __fadd_rn(a.lo, b.lo))};
}

__device__ __forceinline__ ff ff_neg(ff a)
{
    return {-a.hi, -a.lo};
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    return {p, __fmaf_rn(a.lo, b.hi, e)};
}

__device__ __forceinline__ ff ff_sqr(ff a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    const float e = __fmaf_rn(a.hi, a.hi, -p);
    return {p, __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, e)};
}

// a times a float b
__device__ __forceinline__ ff ff_mulf(ff a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    return {p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p))};
}

// a times a power of two (exact)
__device__ __forceinline__ ff ff_scale(ff a, float two_k)
{
    return {__fmul_rn(a.hi, two_k), __fmul_rn(a.lo, two_k)};
}

// sqrt(a) for a > 0 in the normal float range.  With the FP32 estimate y
// of 1/sqrt(a_hi) (relative error e up to 2 ulp, about 2^-22), s = a_hi y
// is corrected by one Newton step for the square root, s + (a - s^2) y / 2,
// with a - s^2 formed exactly from the product error of s^2 (a_hi - s^2 is
// exact: the two are within a factor 2).  The step leaves 3 e^2 / 2 of the
// estimate's error (at most about 2^-43.4) beside the roundings of the
// correction (about 2^-46): ample for the deposit's lattices, whose
// shares are held to 1e-10 (fpic_probe_math measures it).
__device__ __forceinline__ ff ff_sqrt(ff a)
{
    const float y = rsqrtf(a.hi);
    const float s = __fmul_rn(a.hi, y);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
    return ff_fast2(s, __fmul_rn(d, __fmul_rn(0.5f, y)));
}

// 1/a for a > 0 in the normal float range: the FP32 estimate y of 1/a_hi
// (relative error about 2^-23), e = 1 - a y from the exact product error of
// a_hi y (1 - a_hi y is exact: the two are within a factor 2 of 1), and
// 1/a = y / (1 - e) = y (1 + e + e^2 + ...) to second order: relative error
// about 2^-46 (the rounding of y (e + e^2)); fpic_probe_math measures it.
__device__ __forceinline__ ff ff_rcp(ff a)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.hi));
    const float p = __fmul_rn(a.hi, y);
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p), __fmaf_rn(a.hi, y, -p)), __fmul_rn(a.lo, y));
    return ff_fast2(y, __fmul_rn(y, __fmaf_rn(e, e, e)));
}

// sin h and cos h - 1 of a step h in paired FP32 (the deposit's th
// lattice rotations).  Below 2^-7 by the Maclaurin series: h - h^3/6 and
// -h^2/2 in paired arithmetic, the next terms (h^5/120; h^4/24 - h^6/720),
// below 2^-28 relative, in FP32, the omitted ones below 2^-48 of the
// result: sin h to about 2^-46 relative, cos h - 1 to about 2^-40 of
// itself (2^-55 absolute, which is what the rotations need); larger steps
// (coarse grids) through the FP64 routine sincos_step.
__device__ __forceinline__ void sincos_step_ff(ff h, ff& sh, ff& cm)
{
    if (fabsf(h.hi) >= 0.0078125f) {
        double s, c;
        sincos_step(ff_to(h), s, c);
        sh = ff_from(s);
        cm = ff_from(c);
        return;
    }
    const ff t = ff_sqr(h);
    const ff h3 = ff_mul(h, t);
    const ff sixth = {__uint_as_float(0x3e2aaaabu), __uint_as_float(0xb1aaaaabu)};   // 1/6
    const float h5 = __fmul_rn(__fmul_rn(h3.hi, t.hi), 1.f / 120.f);
    sh = ff_add(h, ff_add(ff_neg(ff_mul(h3, sixth)), ff_of(h5)));
    const float c4 = __fmul_rn(__fmul_rn(t.hi, t.hi), __fsub_rn(1.f / 24.f, __fmul_rn(t.hi, 1.f / 720.f)));
    cm = ff_add(ff_scale(t, -0.5f), ff_of(c4));
}

__device__ __forceinline__ void sincos_step_ff(double hd, ff& sh, ff& cm)
{
    sincos_step_ff(ff_from(hd), sh, cm);
}

}  // namespace fpic
