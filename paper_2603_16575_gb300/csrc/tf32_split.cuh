// Fixed-point slicing of FP64 operands for the split-precision tensor-core
// contraction (tc_tf32x3.cuh).
//
// The 32 values of one operand row inside one k-chunk share the scale 2^e,
// e the smallest exponent with max|x| < 2^e.  Each value is rounded to a
// fixed-point number with 36 fractional bits relative to 2^e and cut into four
// 9-bit digits:
//   x ~= sign(x) 2^e (a_1 2^-9 + a_2 2^-18 + a_3 2^-27 + a_4 2^-36),
//   0 <= a_1 <= 2^9, 0 <= a_s < 2^9 (s > 1), |error| <= 2^(e-37),
// and the slice values v_s = sign(x) a_s 2^(e - 9 s) are exactly
// representable in TF32.  Everything is integer arithmetic on the bit pattern
// (FP64 throughput is 1/64 of FP32 on this part).
#pragma once
#include <stdint.h>

#include "tc_job.h"

namespace osv {
namespace tc {

// Biased FP64 exponent field of x (0 for zero and subnormals).
__device__ __forceinline__ unsigned exp_field(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// Slices of x for the chunk whose largest biased exponent field is emax
// (emax == 0: the chunk is zero).
__device__ __forceinline__ void fixed_slices(double x, unsigned emax, float v[NSL]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
#pragma unroll
  for (int s = 0; s < NSL; s++) v[s] = 0.f;
  if (emax == 0 || ex == 0) return;
  const int e = (int)emax - 1022;                                 // max|x| < 2^e
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // |x| = mant 2^(ex-1075)
  const int sh = 1075 - 36 + e - ex;                              // > 16 since |x| < 2^e
  if (sh >= 64) return;
  const unsigned long long F = (mant + (1ull << (sh - 1))) >> sh; // round(|x| 2^(36-e)) <= 2^36
  const float sg = (bits >> 63) ? -1.f : 1.f;
#pragma unroll
  for (int s = 0; s < NSL; s++) {
    const int sc = e - 9 * (s + 1);
    const unsigned d = (s == 0) ? (unsigned)(F >> 27) : (unsigned)((F >> (27 - 9 * s)) & 511u);
    if (sc >= -126) v[s] = sg * (float)d * __int_as_float((sc + 127) << 23);
  }
}

// One k-chunk of one row held by a full warp (lane = k offset, x = 0 past the
// end): the shared exponent from the warp's largest exponent field, then the
// slices.
__device__ __forceinline__ void warp_fixed_slices(double x, float v[NSL]) {
  const unsigned emax = __reduce_max_sync(0xffffffffu, exp_field(x));
  fixed_slices(x, emax, v);
}

}  // namespace tc
}  // namespace osv
