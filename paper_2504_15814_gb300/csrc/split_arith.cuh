// Float64 data handled without float64 instructions.
//
// GB300 executes float64 arithmetic at about 1/73 of the float32 rate, so the
// split-precision path keeps the float64 pipe out of its inner loop:
//   * a float64 value x is split exactly into floats hi + lo (+ a tail below
//     2^-46 |x|) with integer bit operations;
//   * differences x_j - x_c are formed from the pairs in float32, which keeps
//     the cancellation exact up to float32 rounding of the difference itself;
//   * a float64 result base + increment is rebuilt from a float32 two-sum and
//     an integer assembly of the float64 bit pattern.
// Error-free float32 transformations follow Knuth's TwoSum.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace amr {

struct F2 {
  float hi, lo;
};

// x -> (hi, lo): hi keeps the sign, exponent and leading 24 significand bits
// of x (truncation), lo the next 23 bits.  |x - hi - lo| < 2^-46 |x|.
// |x| < 2^-126 gives (0, 0); |x| >= 2^128 gives hi = +-inf; a NaN gives a
// NaN hi, so that it propagates as NaN.
__device__ __forceinline__ F2 split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t h = (uint32_t)(b >> 32), l = (uint32_t)b;
  const uint32_t sign = h & 0x80000000u;
  const int E = (int)((h >> 20) & 0x7ffu);
  F2 r;
  if (E < 897) {  // below the float normal range (or zero)
    r.hi = 0.f;
    r.lo = 0.f;
    return r;
  }
  if (E > 1150) {
    const bool nan = E == 2047 && ((h & 0xfffffu) | l) != 0u;
    r.hi = __uint_as_float(sign | (nan ? 0x7fc00000u : 0x7f800000u));
    r.lo = 0.f;
    return r;
  }
  r.hi = __uint_as_float(sign | ((uint32_t)(E - 896) << 23) | ((h & 0xfffffu) << 3) | (l >> 29));
  // next 23 significand bits as an exact float integer, scaled by 2^(E-1069)
  const float m = __uint_as_float(0x4b000000u | ((l >> 6) & 0x7fffffu)) - 8388608.0f;
  const float scale = E >= 943 ? __uint_as_float((uint32_t)(E - 942) << 23) : 0.f;
  r.lo = __uint_as_float(__float_as_uint(m * scale) | sign);
  return r;
}

// a + b = s + e exactly (Knuth TwoSum, any magnitudes).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float aa = __fsub_rn(s, bb);
  e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
  return s;
}

// float64 value of s + e for a float pair with |e| <= ulp(s) (the output of
// a TwoSum), assembled from the bit patterns: double(s) exactly, plus e in
// units of the float64 ulp of s rounded to an integer.  Error <= 2^-53 |s|
// beyond the rounding of e.  |s| < 2^-75 returns double(s) without e; an
// infinite or NaN s gives the float64 infinity or a NaN.
__device__ __forceinline__ double pair_to_f64(float s, float e) {
  const uint32_t sb = __float_as_uint(s);
  const uint32_t E = (sb >> 23) & 0xffu;
  const uint32_t mag = sb & 0x7fffffffu;
  // double(s): exponent rebias 127 -> 1023, significand shifted into place
  uint32_t hi = (sb & 0x80000000u) | ((mag >> 3) + (896u << 20));
  uint32_t lo = sb << 29;
  if (E == 0) {  // zero (or a float denormal, not produced here): signed zero
    hi = sb & 0x80000000u;
    lo = 0u;
  }
  if (E == 255u) {  // infinity or NaN: the float64 infinity or a NaN
    hi = (sb & 0x80000000u) | 0x7ff00000u | ((mag & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)lo);
  }
  long long bits = ((long long)hi << 32) | lo;
  if (E >= 52u) {
    // e * 2^(179 - E): e in units of ulp_double(s) = 2^(E - 127 - 52)
    const float scale = __uint_as_float((306u - E) << 23);
    int n = __float2int_rn(e * scale);
    if (sb & 0x80000000u) n = -n;  // sign-magnitude: work on |value|
    if ((sb & 0x7fffffu) == 0u && n < 0) n *= 2;  // s a power of two, magnitude decreasing
    bits += n;
  }
  return __longlong_as_double(bits);
}

// s + e = a + b exactly when |a| >= |b| (Dekker FastTwoSum).
__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

// base + incr as float64, base given by its split pair (error < 2^-46 |base|
// from the split, plus float32 rounding of the small correction terms).  The
// second renormalisation uses FastTwoSum: its precondition |s1| >= |t| fails
// only when the result is 2^23 times smaller than the base, and then the
// error stays below 2^-47 |base|.
__device__ __forceinline__ double add_back(F2 base, float incr) {
  float e1, e2;
  const float s1 = two_sum(base.hi, incr, e1);
  const float t = __fadd_rn(e1, base.lo);
  const float s2 = fast_two_sum(s1, t, e2);
  return pair_to_f64(s2, e2);
}

// Exact float64 value of a float, assembled from its bits with integer
// operations (float-to-double conversion runs on the float64 unit on GB300).
// Float denormals become signed zero; infinities and NaNs stay so.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t mag = b & 0x7fffffffu;
  uint32_t hi = (b & 0x80000000u) | ((mag >> 3) + (896u << 20));
  uint32_t lo = b << 29;
  if (mag < 0x00800000u) {
    hi = b & 0x80000000u;
    lo = 0u;
  }
  if (mag >= 0x7f800000u) hi = (b & 0x80000000u) | 0x7ff00000u | ((mag & 0x7fffffu) >> 3);  // inf / NaN
  return __hiloint2double((int)hi, (int)lo);
}

}  // namespace amr
