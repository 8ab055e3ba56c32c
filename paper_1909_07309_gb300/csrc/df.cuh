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

__device__ __forceinline__ df from_double(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ df from_float2(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ double to_double(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df norm(df a) {
  const float s = a.h + a.l;
  return df{s, a.l - (s - a.h)};
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
