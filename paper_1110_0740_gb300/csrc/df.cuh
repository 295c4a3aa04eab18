// df.cuh -- float64 <-> float32 moves without the FP64 pipe, and
// double-float arithmetic for the mixed path.
//
// On GB300 the FP64 pipe issues 2 thread-operations per SM per cycle
// against 128 for FP32 (conversions F2F.F32.F64 / F2F.F64.F32 run on the
// FP64 pipe too).  The mixed path therefore
//   * splits a float64 value x into an unevaluated sum hi + lo of two floats
//     with integer and float32 operations only (hi: the sign, exponent and
//     top 23 mantissa bits of x; lo: the remaining 29 mantissa bits rounded
//     to 24 significant bits), which represents x to about 2^-47 relative;
//   * computes the one quantity that needs more than float32, the pressure
//     p = (Gamma-1)(E - m^2/(2 rho) - B^2/2) of a float64 state, in
//     double-float arithmetic built from the error-free transformations
//     TwoSum (Knuth) and TwoProd via FMA (Dekker / Ogita-Rump-Oishi);
//   * widens a float to a float64 by integer operations (exact).
// Zero and values below the normal float range split to signed zeros (a
// float32 path could not carry them either); values beyond the float range
// become +-inf and nan stays nan, so the status checks still see them.
// (On GB300 even the float <-> double conversion instructions issue on the
// FP64 pipe, so none is used, not even on a rarely taken branch, which the
// compiler may evaluate unconditionally.)  The low part is dropped when its
// scale 2^(e-1075) falls below the normal float range (|x| < ~2^-74), where x
// is then carried to float32 accuracy only.
#pragma once

#include <cuda_runtime.h>

namespace ctu {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_split(double x)
{
    const int hw = __double2hiint(x);
    const unsigned lw = (unsigned)__double2loint(x);
    const int e = (hw >> 20) & 0x7FF;
    const unsigned sign = (unsigned)hw & 0x80000000u;
    if (e > 1023 + 127) {  // beyond the float range: +-inf, or nan for a nan
        const bool nan = e == 0x7FF && ((((unsigned)hw & 0xFFFFFu) | lw) != 0u);
        return df{__uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.0f};
    }
    if (e < 1023 - 126) {  // zero, or below the normal float range: signed zero
        const float z = __uint_as_float(sign);
        return df{z, z};
    }
    const unsigned mant23 = (((unsigned)hw & 0xFFFFFu) << 3) | (lw >> 29);
    df r;
    r.hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | mant23);
    // remaining 29 mantissa bits: value rem * 2^(e - 1075), same sign as x.
    // rem = a * 2^23 + b is converted exactly with the 2^23 magic-number
    // trick (a float with exponent 2^23 holds a 23-bit integer in its
    // mantissa), then rounded once to float by the FMA.
    const unsigned rem = lw & 0x1FFFFFFFu;
    const float fa = __uint_as_float(0x4B000000u | (rem >> 23)) - 8388608.0f;
    const float fb = __uint_as_float(0x4B000000u | (rem & 0x7FFFFFu)) - 8388608.0f;
    const float v = fmaf(fa, 8388608.0f, fb);
    const int se = e - 1075 + 127;  // exponent field of 2^(e - 1075)
    const float scale = se > 0 ? __uint_as_float((unsigned)se << 23) : 0.0f;
    r.lo = __uint_as_float(__float_as_uint(v * scale) | sign);
    return r;
}

// float -> float64 by integer operations (exact for normal floats and zero).
__device__ __forceinline__ double f2d_int(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned sign = u & 0x80000000u;
    if (e == 0u) return __hiloint2double((int)sign, 0);  // zero (denormals flush to zero)
    if (e == 0xFFu)                                      // inf, nan
        return __hiloint2double((int)(sign | 0x7FF00000u | ((u & 0x7FFFFFu) ? 0x80000u : 0u)), 0);
    const unsigned hw = sign | ((e - 127u + 1023u) << 20) | ((u & 0x7FFFFFu) >> 3);
    const unsigned lw = (u & 0x7u) << 29;
    return __hiloint2double((int)hw, (int)lw);
}

// Error-free transformations.
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    const float err = (a - (s - bb)) + (b - bb);
    return df{s, err};
}

__device__ __forceinline__ df fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = a + b;
    return df{s, b - (s - a)};
}

__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = a * b;
    return df{p, fmaf(a, b, -p)};
}

// Accurate double-float sum (both parts with TwoSum).
__device__ __forceinline__ df df_add(df x, df y)
{
    df s = two_sum(x.hi, y.hi);
    df t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }

__device__ __forceinline__ df df_mul(df x, df y)
{
    df p = two_prod(x.hi, y.hi);
    p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_sqr(df x)
{
    df p = two_prod(x.hi, x.hi);
    p.lo = fmaf(2.0f * x.hi, x.lo, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_div(df x, df y)
{
    const float q1 = x.hi / y.hi;
    // r = x - q1 * y
    df p = two_prod(q1, y.hi);
    p.lo = fmaf(q1, y.lo, p.lo);
    df r = df_add(x, df_neg(p));
    const float q2 = r.hi / y.hi;
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ df df_scale(df x, float s)  // s a power of two or exact small int
{
    return df{x.hi * s, x.lo * s};
}

// Pressure of a float64 MHD state, p = (Gamma-1)(E - m^2/(2 rho) - B^2/2),
// in double-float: ~2^-44 relative to E, i.e. float32-exact p even when E
// exceeds p by many orders of magnitude.  u: the state's first 8 components
// split (df_split).
__device__ __forceinline__ float df_pressure_split(const df (&u)[8], float gm1)
{
    const df rho = u[0];
    const df mx = u[1], my = u[2], mz = u[3];
    const df E = u[4];
    const df bx = u[5], by = u[6], bz = u[7];
    const df m2 = df_add(df_add(df_sqr(mx), df_sqr(my)), df_sqr(mz));
    const df b2 = df_add(df_add(df_sqr(bx), df_sqr(by)), df_sqr(bz));
    const df ke = df_scale(df_div(m2, rho), 0.5f);
    const df eint = df_add(df_add(E, df_neg(ke)), df_neg(df_scale(b2, 0.5f)));
    return gm1 * (eint.hi + eint.lo);
}


} // namespace ctu
