// Double-float ("df") arithmetic on the FP32 pipes: a value is the unevaluated
// sum h + l of two floats with |l| <= ulp(h)/2 after normalisation, about 48
// significant bits. Products use the exact FMA split (two-product), sums the
// error-free two-sum (Knuth). GB300 issues FP32 about 70 times faster than
// FP64, so FP64-accurate kernels run on these instead of the FP64 pipe.
#pragma once
#include <cuda_runtime.h>

namespace stfd {
namespace dfa {

struct df {
  float h, l;
};

__device__ __forceinline__ df norm(df a) {
  const float s = a.h + a.l;
  return df{s, a.l - (s - a.h)};
}

// 2^e as a float, exact for e in [-126, 127].
__device__ __forceinline__ float pow2(int e) { return __int_as_float((e + 127) << 23); }

// Conversions between FP64 and double-float. A conversion instruction that
// touches FP64 issues on the FP64 pipe, which on GB300 runs at ~1/64 of the
// FP32 rate, so the values are assembled from the IEEE 754 bit fields with
// integer and FP32 instructions. Only FP64 inputs of magnitude outside
// [2^-70, 2^127) (FP32 subnormals or overflow) take FP64 instructions, in a
// function that is not inlined so that the common path never executes them.

__device__ __noinline__ static df from_double_fp64(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}

// FP64 -> double-float: the 53-bit significand is cut into its top 24 bits
// (exact in a float) and the remaining 29 bits (rounded to 24), then
// renormalised; h + l carries at least 48 significant bits of x.
__device__ __forceinline__ df from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
  const int E = (int)((hi >> 20) & 0x7FFu);
  if (E == 0) return df{0.f, 0.f};   // zero, or below 2^-1022: beyond the FP32 range
  const int e = E - 1023;
  if (e < -70 || e > 126) return from_double_fp64(x);
  // the sign, the exponent and the top 23 fraction bits form the float h exactly
  const unsigned int sgn = hi & 0x80000000u;
  const float h = __uint_as_float(sgn | ((unsigned int)(e + 127) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
  const float l = __uint_as_float(__float_as_uint(__uint2float_rn(lo & 0x1FFFFFFFu) * pow2(e - 52)) | sgn);
  return norm(df{h, l});
}
__device__ __forceinline__ df from_float2(float2 v) { return df{v.x, v.y}; }

// FP64 -> FP32, rounded (the leading float of from_double).
__device__ __forceinline__ float d2f(double x) { return from_double(x).h; }

// FP32 -> FP64, exact (subnormals normalised, infinities and NaNs kept).
__device__ __forceinline__ double f2d(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
  unsigned int e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  unsigned long long field;
  if (e == 0xFFu) {
    field = 0x7FFull;
  } else if (e != 0u) {
    field = e + 896u;
  } else {
    if (m == 0u) return __longlong_as_double((long long)sgn);
    const int sh = __clz((int)m) - 8;   // moves the leading bit to position 23
    m = (m << sh) & 0x7FFFFFu;
    field = (unsigned long long)(897 - sh);
  }
  return __longlong_as_double((long long)(sgn | (field << 52) | ((unsigned long long)m << 29)));
}

// One float of a pair as a signed integer in units of 2^{eb - 181} (the
// larger float's binade, 2^-54 of it); bits below the unit are rounded off.
__device__ __forceinline__ long long df_term(unsigned int bits, int eb) {
  int e = (int)((bits >> 23) & 0xFFu);
  unsigned long long m = bits & 0x7FFFFFu;
  if (e != 0) m |= 0x800000u;
  else e = 1;   // subnormal
  const int sh = e - eb + 31;
  unsigned long long t = 0;
  if (sh >= 0) t = m << sh;
  else if (sh > -32) t = (m + (1ull << (-sh - 1))) >> -sh;
  return (bits >> 31) ? -(long long)t : (long long)t;
}

// double-float -> FP64 for any pair: h + l summed exactly as one integer
// (whenever h + l is itself a double, as for every normalised pair from
// from_double), then normalised to a 53-bit significand (round half up).
__device__ __noinline__ static double to_double_general(df a) {
  const unsigned int bh = __float_as_uint(a.h), bl = __float_as_uint(a.l);
  const int eh = (int)((bh >> 23) & 0xFFu), el = (int)((bl >> 23) & 0xFFu);
  if (eh == 0xFF || el == 0xFF) {   // infinity or NaN: that float's value
    const unsigned int w = eh == 0xFF ? bh : bl;
    return __longlong_as_double((long long)(((unsigned long long)(w >> 31) << 63) | (0x7FFull << 52) |
                                            ((unsigned long long)(w & 0x7FFFFFu) << 29)));
  }
  const int eb = max(max(eh, el), 1);
  const long long S = df_term(bh, eb) + df_term(bl, eb);
  if (S == 0) return 0.0;
  const unsigned long long sgn = S < 0 ? (1ull << 63) : 0ull;
  unsigned long long mag = (unsigned long long)(S < 0 ? -S : S);
  const int lz = __clzll((long long)mag);
  if (lz < 11) {
    const int r = 11 - lz;
    mag = (mag + (1ull << (r - 1))) >> r;
  } else {
    mag <<= (lz - 11);
  }
  // the significand's leading bit adds one to the exponent field (also after a rounding carry)
  const unsigned long long field = (unsigned long long)(eb + 905 - lz - 1);
  return __longlong_as_double((long long)(sgn | ((field << 52) + mag)));
}

// double-float -> FP64, rounded to nearest: h is exact as a double; l,
// measured in units of the double ulp of h's binade (a power-of-two scaling,
// exact), is rounded to an integer k and added to the bit pattern of h, which
// adds k ulps (a normalised pair, |l| <= ulp_float(h) / 2, never carries out of
// the binade; when h is a power of two and the sum falls below it, the units
// are those of the binade below). Pairs that are not normalised or have
// |h| < 2^-75 take to_double_general.
__device__ __forceinline__ double to_double(df a) {
  const unsigned int bh = __float_as_uint(a.h);
  if ((bh << 1) == 0u && (__float_as_uint(a.l) << 1) == 0u) return 0.0;
  const int eh = (int)((bh >> 23) & 0xFFu);
  float v = a.l * pow2(179 - max(eh, 52));
  if (bh >> 31) v = -v;
  if ((bh & 0x7FFFFFu) == 0u && v < 0.f) v *= 2.f;
  if (eh < 52 || eh == 0xFF || !(fabsf(v) < 1073741824.f)) return to_double_general(a);
  const unsigned long long B = ((unsigned long long)(bh >> 31) << 63) | ((unsigned long long)(eh + 896) << 52) |
                               ((unsigned long long)(bh & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)(B + (unsigned long long)(long long)__float2int_rn(v)));
}

// acc += b * x (the b.l * x.l term, ~2^-48 relative, is dropped)
__device__ __forceinline__ void fma_acc(df& acc, float2 b, df x) {
  const float p = b.x * x.h;
  const float e = fmaf(b.x, x.h, -p);
  const float lo = fmaf(b.x, x.l, fmaf(b.y, x.h, e));
  const float s = acc.h + p;
  const float bp = s - acc.h;
  const float err = (acc.h - (s - bp)) + (p - bp);
  acc.h = s;
  acc.l += err + lo;
}

__device__ __forceinline__ df mul(df a, df b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p);
  return norm(df{p, fmaf(a.h, b.l, fmaf(a.l, b.h, e))});
}

__device__ __forceinline__ df add(df a, df b) {
  const float s = a.h + b.h;
  const float bp = s - a.h;
  const float err = (a.h - (s - bp)) + (b.h - bp);
  return norm(df{s, err + a.l + b.l});
}

__device__ __forceinline__ df neg(df a) { return df{-a.h, -a.l}; }
__device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }

// 1 / a: FP32 reciprocal refined by one Newton step in df arithmetic
__device__ __forceinline__ df recip(df a) {
  const float r = 1.0f / a.h;
  // e = 1 - a r (in df), result r + r e
  const df ar = mul(a, df{r, 0.0f});
  const df e = add(df{1.0f, 0.0f}, neg(ar));
  return add(df{r, 0.0f}, mul(df{r, 0.0f}, e));
}

}  // namespace dfa
}  // namespace stfd
