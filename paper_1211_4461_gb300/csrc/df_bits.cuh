// Bit-level conversions between FP64 values and pairs of FP32 words.
//
// FP64 arithmetic and conversions run at 1/61 of the FP32 rate on this part, so
// the one-pass kernels that split FP64 fields into double-float pairs (and
// back) are bound by the FP64 pipe rather than by memory.  The helpers below
// do the same work with integer operations on the IEEE-754 fields:
//   - frexp's exponent of a finite nonzero value;
//   - the round-to-nearest split of x 2^-e into hi + lo, hi = RN_24(x 2^-e) and
//     lo = RN_24(x 2^-e - hi), equal to what the FP64 conversions give while
//     the scaled exponent s (x 2^-e = +-1.f 2^s) is at least -70.  Below, lo
//     (and, below -126, hi) may be rounded once more into FP32's subnormal
//     range; |x 2^-e| < 2^-69 there and the pair stays within 2^-149 of it.
//     Below -150 the pair is zero, as RN_24 gives;
//   - the exact widening of an FP32 value to FP64, times a power of two.
// Zero, subnormal and non-finite FP64 inputs, and scaled exponents above 100,
// take the FP64 conversions instead.
#pragma once

namespace csff {
namespace bits {

constexpr unsigned long long ABS_MASK = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long MANT_MASK = 0x000FFFFFFFFFFFFFull;

// biased exponent field of x (0: zero or subnormal, 0x7ff: inf or NaN)
__device__ __forceinline__ int exp_field(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
}

// e with |x| = f 2^e, f in [1/2, 1) (frexp's exponent); x finite and nonzero
__device__ __forceinline__ int frexp_exp(double x) {
  const int E = exp_field(x);
  if (E != 0) return E - 1022;
  int e;
  frexp(x, &e);                 // subnormal
  return e;
}

// (hi, lo) with hi = RN_24(x 2^-e), lo = RN_24(x 2^-e - hi)
__device__ __forceinline__ float2 split_scaled(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  const int s = E - 1023 - e;   // x 2^-e = +-1.f 2^s
  if (E == 0 || E == 0x7ff || s > 100) {
    const double xs = ldexp(x, -e);
    const float h = __double2float_rn(xs);
    return make_float2(h, __double2float_rn(xs - (double)h));
  }
  const float sg = (b >> 63) ? -1.f : 1.f;
  if (s < -150) return make_float2(0.f * sg, 0.f * sg);
  // 53-bit significand = hm 2^29 + rem, rounded to 24 bits (ties to even)
  const long long m53 = (long long)((b & MANT_MASK) | (1ull << 52));
  int hm = (int)(m53 >> 29);
  int rem = (int)(m53 & ((1ll << 29) - 1));
  if (rem > (1 << 28) || (rem == (1 << 28) && (hm & 1))) {
    hm += 1;
    rem -= 1 << 29;
  }
  // x 2^-e = hm 2^(s-23) + rem 2^(s-52)
  if (s >= -70) {
    // both powers of two are normal floats: hm (<= 2^24) converts exactly, rem
    // rounds once, in the conversion
    const float hi = __int2float_rn(hm) * __int_as_float((s - 23 + 127) << 23);
    const float lo = __int2float_rn(rem) * __int_as_float((s - 52 + 127) << 23);
    return make_float2(sg * hi, sg * lo);
  }
  // scale by 2^100 first so that every factor is a normal float; the final
  // multiply by 2^-100 rounds into the subnormal range where it must
  const float down = __int_as_float((-100 + 127) << 23);
  const float hi = (__int2float_rn(hm) * __int_as_float((s - 23 + 100 + 127) << 23)) * down;
  const float lo = s >= -126 ? (__int2float_rn(rem) * __int_as_float((s - 52 + 100 + 127) << 23)) * down : 0.f;
  return make_float2(sg * hi, sg * lo);
}

// f 2^e in FP64, exactly (a subnormal f is first scaled by 2^64 in FP32, which
// is exact; a non-finite f or a result outside the normal FP64 range goes
// through the FP64 conversion and an ldexp)
__device__ __forceinline__ double widen(float f, int e = 0) {
  const unsigned u0 = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u0 >> 31) << 63;
  if ((u0 & 0x7fffffffu) == 0) return __longlong_as_double((long long)sign);
  const bool sub = (u0 & 0x7f800000u) == 0;
  const unsigned u = sub ? __float_as_uint(f * 18446744073709551616.f) : u0;   // 2^64
  const int E = (int)((u >> 23) & 0xff);
  const int Ed = E + 896 + e - (sub ? 64 : 0);
  if (E == 0xff || Ed < 1 || Ed > 2046) return ldexp((double)f, e);
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)Ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

}  // namespace bits
}  // namespace csff
