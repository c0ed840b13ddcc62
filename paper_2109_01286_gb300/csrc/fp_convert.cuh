// Integer-only rounding of FP64 values to FP32, shared by the 2D and 3D kernels: GB300
// converts between FP64 and FP32 at its FP64 rate, so kernels bound by the FP64 pipe round
// their FP32 sensor inputs this way.
#pragma once
#include <cuda_runtime.h>

namespace hfd {

// x rounded to the nearest float, ties to even, as the FP64-to-FP32 conversion rounds it, by
// integer operations only (the FP64 kernels convert their sensor inputs this way, off the FP64
// pipe).  Finite values and infinities give the conversion's result bit for bit, subnormal
// floats included; NaN gives a quiet NaN of the same sign.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ffull);
  const unsigned long long m = b & 0xfffffffffffffull;
  if (E == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u : 0u));
  if (E == 0) return __uint_as_float(sign);                // FP64 subnormals round to zero
  const int e = E - 1023;
  if (e > 127) return __uint_as_float(sign | 0x7f800000u);
  // the 53-bit significand loses 29 bits for a normal float, more for a subnormal one
  const int sh = e >= -126 ? 29 : 29 + (-126 - e);
  if (sh > 54) return __uint_as_float(sign);               // below half the smallest subnormal
  const unsigned long long M = m | (1ull << 52);
  const unsigned long long q = M >> sh, rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  const unsigned qr = (unsigned)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
  // a normal result: the significand's leading bit adds one to the exponent field (and a
  // rounding carry to 2^24 adds one more, up to infinity)
  const unsigned bits = e >= -126 ? ((unsigned)(e + 126) << 23) + qr : qr;
  return __uint_as_float(sign | bits);
}
}  // namespace hfd
