// Fixed-point slicing of FP64 operands for the split-precision tensor-core
// contraction (tc_tf32x3.cuh).
//
// The 32 values of one operand row inside one k-chunk share the scale 2^e,
// e = the exponent with max|x| < 2^e.  Each value is written as
//   x = 2^e * (a_1 2^-9 + a_2 2^-18 + a_3 2^-27 + a_4 2^-36) + r,
// a_s integers with |a_1| <= 2^9, |a_s| <= 2^8 (s > 1), |r| <= 2^(e-37); the
// slice values v_s = a_s 2^(e - 9 s) are exactly representable in TF32.
#pragma once
#include <stdint.h>

#include "tc_job.h"

namespace osv {
namespace tc {

// Exponent e with amax < 2^e (amax > 0), or INT_MIN-like sentinel for amax == 0.
__device__ __forceinline__ int chunk_exponent(double amax) {
  if (!(amax > 0.0)) return -100000;
  int e;
  frexp(amax, &e);     // amax = f 2^e, f in [0.5, 1)
  return e;
}

// Slices of x for the chunk exponent e (values below the FP32 normal range are dropped).
__device__ __forceinline__ void fixed_slices(double x, int e, float v[NSL]) {
  if (e < -900) {
#pragma unroll
    for (int s = 0; s < NSL; s++) v[s] = 0.f;
    return;
  }
  double q = ldexp(x, 9 - e);            // |q| < 2^9
#pragma unroll
  for (int s = 0; s < NSL; s++) {
    const double a = rint(q);
    const int ex = e - 9 * (s + 1);
    v[s] = (ex > -120) ? (float)ldexp(a, ex) : 0.f;
    q = (q - a) * 512.0;
  }
}

// One k-chunk of one row held by a full warp (lane = k offset, x = 0 past the
// end): the shared exponent from the warp's max |x|, then the slices.
__device__ __forceinline__ void warp_fixed_slices(double x, float v[NSL]) {
  double m = fabs(x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  fixed_slices(x, chunk_exponent(m), v);
}

}  // namespace tc
}  // namespace osv
