// Exact FP64 <-> FP32 conversions on the integer and FP32 pipes.
//
// On GB300 a hardware conversion between double and float issues on the FP64
// pipe, which runs at a small fraction of the FP32 rate; the FP32 arithmetic
// form converts the FP64 state of every staged cell (halo included), every
// residual and every wavespeed, so those conversions cost it a measurable
// share of its time. These functions give the same bits with integer
// operations, written from the IEEE 754 binary64 and binary32 layouts:
//
//   double -> float, round to nearest, ties to even: for a double whose
//   result is a normal float (biased exponent 897..1150) the float's bits are
//   the double's bits shifted right by 29 with the exponent rebiased by
//   1023 - 127 = 896, plus one if the 29 dropped bits exceed half an ulp, or
//   equal it with an odd result (a carry into the exponent is the correct
//   rounding up, to infinity included). Zero and double subnormals give a
//   signed zero; anything else (float subnormals, infinities, NaN) takes the
//   hardware conversion.
//
//   float -> double (exact): a normal float's exponent is rebiased by 896
//   and its 23 mantissa bits become the top of the 52; a signed zero stays
//   one; subnormals, infinities and NaN take the hardware conversion.
//
// Both are __host__ __device__ so that a host test checks this very source
// against the compiler's conversions bit for bit.
#pragma once

#include <cstdint>
#include <cstring>

namespace gbr {

__host__ __device__ __forceinline__ float f64_to_f32_rn(double x)
{
#ifdef __CUDA_ARCH__
    const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
    const unsigned sh = __funnelshift_r(lo, hi, 29);  // low 32 bits of (hi:lo) >> 29
#else
    uint64_t u;
    memcpy(&u, &x, 8);
    const unsigned lo = (unsigned)u, hi = (unsigned)(u >> 32);
    const unsigned sh = (unsigned)(u >> 29);
#endif
    const unsigned e = (hi >> 20) & 0x7ffu;
    unsigned f;
    if (e - 897u <= 253u) {
        f = sh - (896u << 23);  // exponent field: low 9 bits of e, rebiased
        f += ((lo & 0x1fffffffu) + (f & 1u)) > 0x10000000u;
        f |= hi & 0x80000000u;
    } else if (e == 0u) {
        f = hi & 0x80000000u;
    } else {
        return (float)x;
    }
#ifdef __CUDA_ARCH__
    return __uint_as_float(f);
#else
    float r;
    memcpy(&r, &f, 4);
    return r;
#endif
}

__host__ __device__ __forceinline__ double f32_to_f64(float x)
{
#ifdef __CUDA_ARCH__
    const unsigned b = __float_as_uint(x);
#else
    unsigned b;
    memcpy(&b, &x, 4);
#endif
    const unsigned e = (b >> 23) & 0xffu;
    unsigned hi, lo;
    if (e - 1u <= 253u) {
        hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
        lo = b << 29;
    } else if ((b & 0x7fffffffu) == 0u) {
        hi = b & 0x80000000u;
        lo = 0u;
    } else {
        return (double)x;
    }
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)hi, (int)lo);
#else
    const uint64_t u = ((uint64_t)hi << 32) | lo;
    double r;
    memcpy(&r, &u, 8);
    return r;
#endif
}

// The state (always FP64) in the arithmetic type T, and back.
template <typename T>
__device__ __forceinline__ T from_f64(double x) { return T(x); }
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return f64_to_f32_rn(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }

}  // namespace gbr
