// Exact integer sums rounded once to FP64 with integer instructions, shared by
// the seven-digit mode product (tc_oz7.cu) and the integer-limb band products
// (band_fx.cu). Host and device: the host build lets the CPU tests check every
// path against exact rational rounding.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <cstring>

#ifdef __CUDACC__
#define FR_NOINLINE __noinline__
#else
#define FR_NOINLINE __attribute__((noinline))
#endif

namespace stfd {

__host__ __device__ __forceinline__ int fr_clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}
__host__ __device__ __forceinline__ double fr_as_double(unsigned long long bits) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)bits);
#else
  double d;
  std::memcpy(&d, &bits, 8);
  return d;
#endif
}
__host__ __device__ __forceinline__ double fr_inf(bool neg) {
#ifdef __CUDA_ARCH__
  return neg ? -CUDART_INF : CUDART_INF;
#else
  return fr_as_double(neg ? 0xFFF0000000000000ull : 0x7FF0000000000000ull);
#endif
}

// (hi, lo): the magnitude as 128 bits with its leading bit at 127; be0 <= 0:
// the biased exponent the FP64 result would have. The subnormal significand
// keeps the 53 - (1 - be0) leading bits, hi >> (12 - be0), rounded once to
// nearest even (a carry to 2^52 gives the smallest normal number, whose bits
// are the same).
__host__ __device__ __forceinline__ double round_sub(unsigned long long hi, unsigned long long lo, int be0, bool neg) {
  const int k = 12 - be0;                                     // >= 12
  if (k > 64) return neg ? -0.0 : 0.0;                        // below half the smallest subnormal
  const unsigned long long q0 = k < 64 ? hi >> k : 0ull;
  const unsigned long long r = k < 64 ? hi & ((1ull << k) - 1) : hi, h = 1ull << (k - 1);
  const bool above = r > h || (r == h && lo != 0ull);
  const bool half = r == h && lo == 0ull;
  const unsigned long long q = q0 + ((above || (half && (q0 & 1ull))) ? 1ull : 0ull);
  return fr_as_double(((unsigned long long)neg << 63) | q);
}

// The top 64 bits `top` of a magnitude normalised to its leading bit (bit 63),
// the bits below as `rest`, its biased exponent be0 before rounding: the FP64
// value rounded once to nearest even (round bit at 10, the rest as sticky; a
// rounding carry moves into the exponent through the addition).
__host__ __device__ __forceinline__ double round_top(unsigned long long top, unsigned long long rest, int be0, bool neg) {
  if (be0 < 1) return round_sub(top, rest, be0, neg);          // below the normal range: rare
  if (be0 > 2046) return fr_inf(neg);
  const unsigned low = ((unsigned)top & 0x7FFu) | (rest != 0ull ? 1u : 0u);
  const unsigned up = (low + 0x3FFu + ((unsigned)(top >> 11) & 1u)) >> 11;     // ties to even
  const unsigned long long bits = ((unsigned long long)(be0 - 1) << 52) + ((top >> 11) + up);
  return fr_as_double(bits | ((unsigned long long)neg << 63));
}

// ---- integer-limb band products
// acc += C U for 27-bit limbs: hh = sum C_h U_h, ll = sum C_l U_l,
// mm = sum (C_h + C_l)(U_h + U_l); S = hh 2^54 + (mm - hh - ll) 2^27 + ll.
struct Acc {
  long long hh, mm, ll;
};

// S as a signed 128-bit integer (hi: high word, two's complement; |S| < 2^126).
struct S128 {
  long long hi;
  unsigned long long lo;
};
// The cross term mm - hh - ll is formed modulo 2^64: exact whenever it fits in
// 64 bits, even if mm itself was accumulated with wrap-around.
__host__ __device__ __forceinline__ S128 to_s128(const Acc& a) {
  const long long hl =
      (long long)((unsigned long long)a.mm - (unsigned long long)a.hh - (unsigned long long)a.ll);
  const long long t1 = hl + (a.ll >> 27);
  const unsigned long long r0 = (unsigned long long)a.ll & ((1ull << 27) - 1);
  const long long t2 = a.hh + (t1 >> 27);
  const unsigned long long R = ((unsigned long long)(t1 & ((1ll << 27) - 1)) << 27) | r0;   // S = t2 2^54 + R
  return S128{t2 >> 10, ((unsigned long long)t2 << 54) | R};
}

// x 2^g + y for 0 <= g <= 16 (no overflow when |x 2^g| + |y| < 2^127).
__host__ __device__ __forceinline__ S128 shl_add(S128 x, int g, S128 y) {
  const unsigned long long xh = g ? ((unsigned long long)x.hi << g) | (x.lo >> (64 - g)) : (unsigned long long)x.hi;
  const unsigned long long xl = x.lo << g;
  const unsigned long long lo = xl + y.lo;
  const unsigned long long hi = xh + (unsigned long long)y.hi + (lo < xl ? 1ull : 0ull);
  return S128{(long long)hi, lo};
}

// S 2^{SE - 2150} rounded once, to nearest even, to FP64: the top 64 bits of
// the normalised magnitude with the rest as a sticky bit, then round_top.
__host__ __device__ __forceinline__ double round_s128(S128 s, int SE) {
  const bool neg = s.hi < 0;
  const unsigned long long ml = neg ? 0ull - s.lo : s.lo;
  const unsigned long long mh = neg ? ~(unsigned long long)s.hi + (s.lo == 0ull ? 1ull : 0ull) : (unsigned long long)s.hi;
  if ((mh | ml) == 0ull) return 0.0;
  int lz;
  unsigned long long top, rest;
  if (mh) {
    lz = fr_clz64(mh);                      // >= 1: |S| < 2^127
    top = (mh << lz) | (ml >> (64 - lz));
    rest = ml << lz;
  } else {
    lz = 64 + fr_clz64(ml);
    top = ml << (lz - 64);
    rest = 0ull;
  }
  return round_top(top, rest, 127 - lz + SE - 2150 + 1023, neg);
}

// One product: S 2^{SE - 2150} rounded once.
__host__ __device__ __forceinline__ double round_acc(const Acc& a, int SE) { return round_s128(to_s128(a), SE); }

// Two products x 2^{SX - 2150} + y 2^{SY - 2150} summed exactly and rounded
// once; the caller keeps |SX - SY| small enough for shl_add (2^16 for sums
// below 2^110, 2^10 for sums below 2^116).
__host__ __device__ __forceinline__ double round_pair_exact(const Acc& x, int SX, const Acc& y, int SY) {
  const int g = SX - SY;
  const bool xs = g >= 0;   // shift the operand of the larger scale
  const S128 sx = to_s128(x), sy = to_s128(y);
  const S128 big{xs ? sx.hi : sy.hi, xs ? sx.lo : sy.lo}, small{xs ? sy.hi : sx.hi, xs ? sy.lo : sx.lo};
  return round_s128(shl_add(big, xs ? g : -g, small), xs ? SY : SX);
}

// ---- integer-limb stencil row sums (up to 729 taps)
// Balanced 27-bit limbs of a signed integer |U| < 2^53: U = h 2^27 + l with
// l in [-2^26, 2^26), |h| <= 2^26.
__host__ __device__ __forceinline__ int2 split_balanced(long long U) {
  const long long lo = ((U + (1ll << 26)) & ((1ll << 27) - 1)) - (1ll << 26);
  return make_int2((int)((U - lo) >> 27), (int)lo);
}

// The balanced limbs of U = round(m 2^{max(e,1) - E}) (halves away from zero)
// for an FP64 bit pattern u, m its 53-bit significand, under a frame
// E >= max(1, e): |U| < 2^53.
__host__ __device__ __forceinline__ int2 balanced_limbs(unsigned long long u, int E) {
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(e != 0) << 52);
  int s = E - (e > 1 ? e : 1);
  s = s < 63 ? s : 63;
  const unsigned long long mag = (m + ((1ull << s) >> 1)) >> s;
  return split_balanced((u >> 63) ? -(long long)mag : (long long)mag);
}

// sum_o C_o U_o of balanced limbs in three words: hh = sum C_h U_h and
// ll = sum C_l U_l (each term at most 2^52 in magnitude), mm = sum (C_h + C_l)
// (U_h + U_l) modulo 2^64. For up to 729 taps the cross term mm - hh - ll =
// sum (C_h U_l + C_l U_h) is below 729 2^53 < 2^63 in magnitude, so to_s128
// recovers S exactly from the wrapped mm.
struct AccW {
  long long hh, ll;
  unsigned long long mm;
};
__host__ __device__ __forceinline__ void tapw(AccW& a, int2 c, int cs, int2 u) {
  a.hh += (long long)c.x * u.x;
  a.ll += (long long)c.y * u.y;
  a.mm += (unsigned long long)((long long)cs * (u.x + u.y));
}
__host__ __device__ __forceinline__ Acc as_acc(const AccW& a) { return Acc{a.hh, (long long)a.mm, a.ll}; }

// ---- seven-digit mode products
// Rare case of combine7: |Z| below 2^24 (then zh 2^24 + zl is exact in FP64
// and scalbn rounds once).
__host__ __device__ FR_NOINLINE inline double combine7_slow(long long zh, long long zl, int SE) {
  const double hi = (double)zh * 16777216.0, lo = (double)zl;
  return scalbn(hi + lo, SE);
}

// Z = sum_c I_c 256^{6-c} (integers |I_c| < 2^24, exact) rounded to nearest
// even, times 2^SE, as FP64. Z is formed exactly as zh 2^24 + zl in two 64-bit
// words; its magnitude Mt 2^24 + mr (0 <= mr < 2^24) is normalised as a
// 128-bit value and rounded once by round_top (the FP64 pipe is not used).
__host__ __device__ __forceinline__ double combine7_int(const int* I, int SE) {
  const long long zh = (long long)I[0] * 16777216ll + (long long)I[1] * 65536ll + (long long)I[2] * 256ll + I[3];
  const long long zl = (long long)I[4] * 65536ll + (long long)I[5] * 256ll + I[6];
  const long long Zt = zh + (zl >> 24);                     // Z = Zt 2^24 + zr, 0 <= zr < 2^24
  const unsigned zr = (unsigned)zl & 0xFFFFFFu;
  const bool neg = Zt < 0;
  const unsigned long long Mt = neg ? (unsigned long long)(~Zt) + (zr == 0u) : (unsigned long long)Zt;
  const unsigned mr = neg ? ((0x1000000u - zr) & 0xFFFFFFu) : zr;
  if (Mt == 0ull) return combine7_slow(zh, zl, SE);
  const int lz = fr_clz64(Mt);                             // 13 .. 63
  const unsigned long long lo64 = (unsigned long long)mr << 40;
  const unsigned long long hi = (Mt << lz) | (lo64 >> (64 - lz));
  const unsigned long long lo = lo64 << lz;
  return round_top(hi, lo, 87 - lz + SE + 1023, neg);
}

}  // namespace stfd
