// Double-float arithmetic on the FP32 pipe, and double <-> float-pair conversions
// done with integer instructions only.
//
// The FP32-bulk form keeps every state of its RK sweeps (stage values, stored
// trajectory, adjoint variables) as a pair of FP32 planes, hi and lo, with
// value hi + lo (about 48 significant bits).  The stage accumulation u + dt a k
// then runs in pair arithmetic on the 128-lane FP32 pipe instead of the 2-lane
// FP64 pipe of GB300; conversions from and to FP64 at the API boundary use bit
// manipulation because an F2F conversion issues on the FP64 pipe as well.
//
// Error-free transformations (Knuth's two-sum, Dekker/FMA two-product) with
// round-to-nearest intrinsics so that no multiply-add is contracted.
#pragma once
#include <cuda_runtime.h>

namespace semk {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| or a == 0
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// a + b with both parts (the accurate pair sum)
__device__ __forceinline__ df df_add(df a, df b) {
    df s = df_two_sum(a.hi, b.hi);
    const df t = df_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = df_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return df_fast_two_sum(s.hi, s.lo);
}

// a * b
__device__ __forceinline__ df df_mul(df a, df b) {
    df p = df_two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_fast_two_sum(p.hi, p.lo);
}

// a * b with b a single float
__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = df_two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}

// x = hi + lo: hi keeps the leading 24 significand bits of x (truncated), lo the
// next 24 of the remaining 29 (truncated), so |x - hi - lo| <= 2^-47 |x|.
// |x| < 2^-126 flushes to signed zero, |x| >= 2^128 gives +-inf, NaN stays NaN.
// Integer instructions only.
__device__ __forceinline__ void split_bits(double x, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
    const unsigned sign = h & 0x80000000u;
    const int e = (int)((h >> 20) & 0x7ffu);
    const int fe = e - 896;  // float biased exponent of hi
    if (e == 0x7ff) {
        hi = __uint_as_float(sign | 0x7f800000u | ((((h & 0xfffffu) | l) != 0u) ? 0x400000u : 0u));
        lo = 0.f;
        return;
    }
    if (fe >= 255) {
        hi = __uint_as_float(sign | 0x7f800000u);
        lo = 0.f;
        return;
    }
    if (fe <= 0) {
        hi = __uint_as_float(sign);
        lo = 0.f;
        return;
    }
    hi = __uint_as_float(sign | ((unsigned)fe << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
    const unsigned m = l & 0x1fffffffu;  // remaining 29 significand bits, weight 2^(e - 1075)
    if (m == 0u) {
        lo = 0.f;
        return;
    }
    const int p = 31 - __clz((int)m);    // position of the leading one of m
    const int le = p + e - 948;          // float biased exponent of lo
    if (le <= 0) {
        lo = 0.f;
        return;
    }
    const unsigned mant = (p >= 23 ? (m >> (p - 23)) : (m << (23 - p))) & 0x7fffffu;
    lo = __uint_as_float(sign | ((unsigned)le << 23) | mant);
}

// exact float -> double (denormal floats flush to zero); integer instructions only
__device__ __forceinline__ double widen_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    if (e == 0u) return __hiloint2double((int)sign, 0);
    if (e == 0xffu) return __hiloint2double((int)(sign | 0x7ff00000u | (m ? 0x80000u : 0u)), 0);
    return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

__device__ __forceinline__ bool nonfinite_f(float v) {
    return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}

// ---------------------------------------------------------------- double-float element arithmetic
// Value type of the element kernels of the FP64-DF form: x = h + l in two floats
// (about 48 significand bits), with the operators the element kernels use.  The
// FP64 pipe of GB300 issues 2 lanes per SM and clock, the FP32 pipe 128; a
// multiply-add below costs 13 FP32 operations, so it runs about 5 times faster
// than a native FP64 FMA while its rounding error stays near 2^-48 relative to
// the magnitudes summed (Ogita, Rump & Oishi, "Accurate sum and dot product",
// SIAM J. Sci. Comput. 26 (2005): the compensated dot product, here with
// double-float inputs).  Sums and products leave the pair unnormalised (|l| may
// exceed half an ulp of h); its value h + l is what counts.  The operators live
// in their own namespace so that argument-dependent lookup finds them and an
// unqualified fma() on doubles still resolves to the CUDA math function.
namespace dfa {

struct dfloat {
    float h, l;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float x) : h(x), l(0.f) {}
    __host__ __device__ constexpr dfloat(float a, float b) : h(a), l(b) {}
};

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.h, -a.l); }

// a + b: two-sum of the leading parts, trailing parts added in FP32
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const df s = df_two_sum(a.h, b.h);
    return dfloat(s.hi, __fadd_rn(__fadd_rn(a.l, b.l), s.lo));
}

__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }

// a * b: exact product of the leading parts (FMA), cross terms in FP32
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.h, -p);
    const float q = __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h));
    return dfloat(p, __fadd_rn(e, q));
}

// a * b + c: one step of the compensated dot product
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.h, -p);
    const float q = __fmaf_rn(a.h, b.l, __fmul_rn(a.l, b.h));
    const df s = df_two_sum(c.h, p);
    return dfloat(s.hi, __fadd_rn(c.l, __fadd_rn(__fadd_rn(e, q), s.lo)));
}

__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }

}  // namespace dfa

using dfa::dfloat;

// Host: the double-float nearest to a double (h rounded, l the rounded remainder).
inline dfloat dfloat_of(double x) {
    const float h = (float)x;
    return dfloat(h, (float)(x - (double)h));
}

}  // namespace semk
