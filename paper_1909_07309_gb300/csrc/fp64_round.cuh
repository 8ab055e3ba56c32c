// Assembly of an FP64 result from an exact integer magnitude with integer
// instructions (shared by the seven-digit mode product and the integer-limb
// band products): the rare case of a result below the normal range.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

namespace stfd {

// (hi, lo): the magnitude as 128 bits with its leading bit at 127; be0 <= 0:
// the biased exponent the FP64 result would have. The subnormal significand
// keeps the 53 - (1 - be0) leading bits, hi >> (12 - be0), rounded once to
// nearest even (a carry to 2^52 gives the smallest normal number, whose bits
// are the same).
__device__ __forceinline__ double round_sub(unsigned long long hi, unsigned long long lo, int be0, bool neg) {
  const int k = 12 - be0;                                     // >= 12
  if (k > 64) return neg ? -0.0 : 0.0;                        // below half the smallest subnormal
  const unsigned long long q0 = k < 64 ? hi >> k : 0ull;
  const unsigned long long r = k < 64 ? hi & ((1ull << k) - 1) : hi, h = 1ull << (k - 1);
  const bool above = r > h || (r == h && lo != 0ull);
  const bool half = r == h && lo == 0ull;
  const unsigned long long q = q0 + ((above || (half && (q0 & 1ull))) ? 1ull : 0ull);
  return __longlong_as_double((long long)(((unsigned long long)neg << 63) | q));
}

}  // namespace stfd
