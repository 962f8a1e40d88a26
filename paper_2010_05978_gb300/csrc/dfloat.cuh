// Double-float arithmetic (an unevaluated sum hi + lo of two FP32 numbers,
// ~48 significant bits) for the FP32 fast mode's phase and grid-coordinate
// steps.  GB300 runs FP64 at 1/58 of the FP32 rate, and those steps need
// more than FP32's 24 bits (phases reach 1e3-1e4 rad, grid coordinates need
// ~1e-8 grid units on grids of 1e3-1e4 points), but far less than FP64's 53.
//
// Building blocks are the classical error-free transformations: Knuth's
// two-sum and the FMA-based exact product (Dekker/Kahan).  Nothing here may
// be compiled with reassociation (no fast-math).
#pragma once
#include <cuda_runtime.h>

namespace fres {

struct dflt {
    float hi, lo;
};

__device__ __forceinline__ dflt df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dflt df_quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ dflt df_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
    dflt s = df_two_sum(a.hi, b.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return df_quick_two_sum(s.hi, t);
}

__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
    dflt p = df_two_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return df_quick_two_sum(p.hi, t);
}

__device__ __forceinline__ dflt df_mul_f(dflt a, float b) {
    dflt p = df_two_prod(a.hi, b);
    return df_quick_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// FP64 -> double-float with integer operations only: hi keeps the top 24
// significant bits of x (truncated), lo the next 24 bits of the exact
// remainder.  |x| must lie in the normal FP32 range or be 0 (values below
// 2^-100 in magnitude are treated as 0).
__device__ __forceinline__ dflt df_from_double(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;   // unbiased exponent
    if (e < -100) return {0.0f, 0.0f};
    if (e > 126) return {__int_as_float(0x7fc00000), 0.0f};   // out of range / inf / nan
    const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
    const unsigned mant = (unsigned)((b >> 29) & 0x7FFFFF);
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | mant);
    // remainder: low 29 mantissa bits, worth (bits) * 2^(e - 52)
    const float rem = (float)(unsigned)(b & 0x1FFFFFFF);   // rounded to 24 bits
    const int se = e - 52 + 127;
    const float scale = se > 0 ? __uint_as_float((unsigned)se << 23) : 0.0f;
    const float lo = sign ? -rem * scale : rem * scale;
    return {hi, lo};
}

// Host-side split of an FP64 constant (round-to-nearest hi, then the rest).
inline dflt df_host(double x) {
    const float hi = (float)x;
    const float lo = (float)(x - (double)hi);
    return {hi, lo};
}

// Reduce a double-float phase to a float in [-pi, pi]: phi - 2 pi n with
// n = rint(phi / 2 pi), 2 pi carried as a double-float.
__device__ __forceinline__ float df_reduce_2pi(dflt ph) {
    const float n = rintf(ph.hi * 0.15915494309189533577f);
    const dflt twopi = {6.28318548202514648438f, -1.7484555314695172e-07f};   // fl32(2pi), rest
    const dflt r = df_add(ph, df_mul_f(twopi, -n));
    return r.hi + r.lo;
}

// Split a double-float grid coordinate into the integer cell floor(v) and the
// fraction v - floor(v) in [0, 1) (FP32).
__device__ __forceinline__ void df_floor_split(dflt v, int* cell, float* frac) {
    float c = floorf(v.hi);
    float f = __fadd_rn(__fsub_rn(v.hi, c), v.lo);   // v.hi - c is exact
    if (f < 0.0f) {
        c -= 1.0f;
        f += 1.0f;
    } else if (f >= 1.0f) {
        c += 1.0f;
        f -= 1.0f;
    }
    if (f >= 1.0f) f = 0.99999994f;   // rounding of f + 1 just below 0
    *cell = (int)c;
    *frac = f;
}

}  // namespace fres
