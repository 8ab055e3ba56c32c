// Banded mode products of the system matvec (eq. syst_mat through eq.
// kron_vec_multi) in double-float arithmetic on the FP32 pipes.
//
// GB300 issues FP64 at about 1/70 of its FP32 rate, so the FP64-accurate
// matvec keeps every value as an unevaluated sum hi + lo of two floats
// (about 48 significant bits): products are split exactly with an FMA
// (two-product), sums are accumulated with Knuth's error-free two-sum, and
// the low-order parts are summed separately. Intermediate tensors are stored
// as float2 (8 bytes, the size of a double); the first pass reads FP64 and the
// last writes FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "df.cuh"
#include "device_state.h"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {
namespace {

constexpr int kTC = 32;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct df {
  float h, l;
};

__device__ __forceinline__ df to_df(double x) {
  const float h = __double2float_rn(x);
  return df{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ df to_df(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ double to_double(df a) { return (double)a.h + (double)a.l; }

// acc += b * x, b and x double-floats; the b.l * x.l term (~2^-48 relative) is dropped.
__device__ __forceinline__ void df_fma(df& acc, float2 b, df x) {
  const float p = b.x * x.h;
  const float e = fmaf(b.x, x.h, -p);                  // exact: b.h x.h = p + e
  const float lo = fmaf(b.x, x.l, fmaf(b.y, x.h, e));
  const float s = acc.h + p;                           // two-sum(acc.h, p)
  const float bp = s - acc.h;
  const float err = (acc.h - (s - bp)) + (p - bp);
  acc.h = s;
  acc.l += err + lo;
}

__device__ __forceinline__ df df_norm(df a) {
  const float s = a.h + a.l;
  return df{s, a.l - (s - a.h)};
}

// a * s with s a double-float scalar
__device__ __forceinline__ df df_scale(df a, float2 s) {
  const float p = a.h * s.x;
  const float e = fmaf(a.h, s.x, -p);
  const float lo = fmaf(a.h, s.y, fmaf(a.l, s.x, e));
  return df_norm(df{p, lo});
}

__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.h + b.h;
  const float bp = s - a.h;
  const float err = (a.h - (s - bp)) + (b.h - bp);
  return df_norm(df{s, err + a.l + b.l});
}

template <typename T>
__device__ __forceinline__ df load_df(const T* p, long long i);
template <>
__device__ __forceinline__ df load_df<double>(const double* p, long long i) { return to_df(p[i]); }
template <>
__device__ __forceinline__ df load_df<float2>(const float2* p, long long i) { return to_df(p[i]); }

__device__ __forceinline__ void store_df(double* p, long long i, df v) { p[i] = to_double(v); }
__device__ __forceinline__ void store_df(float2* p, long long i, df v) { p[i] = make_float2(v.h, v.l); }

// One direction of the sum-factorised matvec in a single pass over the data:
//   Uo = U x_m A1                         (if TWO_OUT)
//   Vo = s2 (U x_m A2) + s3 (V x_m A3)    (V term if HAS_V)
// with |a - i| <= bw. U is FP64 (first direction) or float2, V float2, Vo float2
// or FP64 (time direction). The three accumulations are independent chains.
template <typename TIn, typename TOut, bool HAS_V, bool TWO_OUT>
__global__ void __launch_bounds__(kThreads)
k_band_pair_df(const TIn* __restrict__ U, const float2* __restrict__ V, const float2* __restrict__ A1,
               const float2* __restrict__ A2, const float2* __restrict__ A3, float2 s2, float2 s3,
               float2* __restrict__ Uo, TOut* __restrict__ Vo, int n, long long inner, long long Q, int bw,
               int scale) {
  extern __shared__ float2 sm2[];
  float2* xu = sm2;
  float2* xv = sm2 + (size_t)n * kTC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long q = (long long)blockIdx.x * kTC + lane;
  const bool valid = q < Q;
  long long base = 0;
  if (valid) {
    const long long o = q / inner;
    base = o * (long long)n * inner + (q - o * inner);
  }
  for (int a = warp; a < n; a += kWarps) {
    const df v = valid ? load_df<TIn>(U, base + (long long)a * inner) : df{0.f, 0.f};
    xu[a * kTC + lane] = make_float2(v.h, v.l);
    if (HAS_V) xv[a * kTC + lane] = valid ? V[base + (long long)a * inner] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int i = warp; i < n; i += kWarps) {
    const int a0 = max(0, i - bw), a1 = min(n - 1, i + bw);
    const float2* r1 = A1 + (size_t)i * n;
    const float2* r2 = A2 + (size_t)i * n;
    const float2* r3 = A3 + (size_t)i * n;
    df c1{0.f, 0.f}, c2{0.f, 0.f}, c3{0.f, 0.f};
    for (int a = a0; a <= a1; ++a) {
      const df xa = to_df(xu[a * kTC + lane]);
      if (TWO_OUT) df_fma(c1, __ldg(r1 + a), xa);
      df_fma(c2, __ldg(r2 + a), xa);
      if (HAS_V) df_fma(c3, __ldg(r3 + a), to_df(xv[a * kTC + lane]));
    }
    df vo = df_norm(c2);
    if (scale) vo = df_scale(vo, s2);
    if (HAS_V) {
      df t = df_norm(c3);
      if (scale) t = df_scale(t, s3);
      vo = df_add(vo, t);
    }
    if (valid) {
      if (TWO_OUT) store_df(Uo, base + (long long)i * inner, df_norm(c1));
      store_df(Vo, base + (long long)i * inner, vo);
    }
  }
}

// ---- Band passes with compile-time half-bandwidth P: two accumulation chains of a
// pass that share their operand layout are issued together with the sm_100
// float2 instructions (fma.rn.f32x2 and friends; per component the scalar
// steps of df_fma in the same order, so the results equal those of scalar
// double-float code): KIND 0 (first direction) pairs M x and K x, the tile holding
// (x.h, x.h, x.l, x.l); KIND 1 (middle directions) pairs M u and M v, the tile
// holding (u.h, v.h, u.l, v.l), with K u as a scalar chain; KIND 2 (time) pairs
// W u and M_t v on the same tile layout. The coefficient tables hold the
// matching pairs (hi_1, hi_2, lo_1, lo_2) per tap.
struct df2 {
  float2 h, l;
};

// FP64 loads of the paired kernel convert with integer and FP32 instructions
// (df.cuh) rather than on the FP64 pipe.
__device__ __forceinline__ df ld_pk(const double* p, long long i) {
  const dfa::df v = dfa::from_double(p[i]);
  return df{v.h, v.l};
}
__device__ __forceinline__ df ld_pk(const float2* p, long long i) { return to_df(p[i]); }

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // a - b
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

// acc += b * x for two independent triples; the steps of df_fma
__device__ __forceinline__ void df_fma2(df2& acc, float2 bh, float2 bl, float2 xh, float2 xl) {
  const float2 p = __fmul2_rn(bh, xh);
  const float2 e = __ffma2_rn(bh, xh, make_float2(-p.x, -p.y));
  const float2 lo = __ffma2_rn(bh, xl, __ffma2_rn(bl, xh, e));
  const float2 s = __fadd2_rn(acc.h, p);
  const float2 bp = sub2(s, acc.h);
  const float2 err = __fadd2_rn(sub2(acc.h, sub2(s, bp)), sub2(p, bp));
  acc.h = s;
  acc.l = __fadd2_rn(acc.l, __fadd2_rn(err, lo));
}

template <typename TIn, typename TOut, int KIND, int P>
__global__ void __launch_bounds__(kThreads)
k_band_pk(const TIn* __restrict__ U, const float2* __restrict__ V, const float4* __restrict__ T4,
          const float2* __restrict__ T2, float2 s2, float2 s3, float2* __restrict__ Uo, TOut* __restrict__ Vo, int n,
          long long inner, long long Q, int scale, int rot) {
  constexpr int W = 2 * P + 1;
  constexpr int kLd = kTC + 1;   // tile row stride in float4 (the padding keeps the transposed stores conflict-free)
  extern __shared__ float4 sm4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long q = (long long)blockIdx.x * kTC + lane;
  const bool valid = q < Q;
  long long base = 0;
  if (valid) {
    const long long o = q / inner;
    base = o * (long long)n * inner + (q - o * inner);
  }
  tc::grid_dependency_wait();   // programmatic dependent launch: inputs from here on
  if (rot || inner == 1) {
    // the CTA's fibres are consecutive rows of length n: one contiguous block,
    // read with consecutive threads on consecutive words and transposed into the tile
    const long long q0 = (long long)blockIdx.x * kTC;
    const int nf = (int)min((long long)kTC, Q - q0);
    const TIn* src = U + q0 * n;
    const float2* srcv = KIND == 0 ? nullptr : V + q0 * n;
    // (f, a) of element e = f n + a, advanced by kThreads without a division per element
    const int df_step = kThreads / n, da_step = kThreads - df_step * n;
    int f = threadIdx.x / n, a = threadIdx.x - f * n;
    for (int e = threadIdx.x; e < kTC * n; e += kThreads) {
      const df u = f < nf ? ld_pk(src, e) : df{0.f, 0.f};
      if (KIND == 0) {
        sm4[a * kLd + f] = make_float4(u.h, u.h, u.l, u.l);
      } else {
        const float2 v = f < nf ? srcv[e] : make_float2(0.f, 0.f);
        sm4[a * kLd + f] = make_float4(u.h, v.x, u.l, v.y);
      }
      f += df_step;
      a += da_step;
      if (a >= n) {
        a -= n;
        ++f;
      }
    }
  } else {
    for (int a = warp; a < n; a += kWarps) {
      const df u = valid ? ld_pk(U, base + (long long)a * inner) : df{0.f, 0.f};
      if (KIND == 0) {
        sm4[a * kLd + lane] = make_float4(u.h, u.h, u.l, u.l);
      } else {
        const float2 v = valid ? V[base + (long long)a * inner] : make_float2(0.f, 0.f);
        sm4[a * kLd + lane] = make_float4(u.h, v.x, u.l, v.y);
      }
    }
  }
  __syncthreads();
  tc::grid_launch_dependents();
  for (int i = warp; i < n; i += kWarps) {
    const float4* r4 = T4 + (size_t)i * W;
    const float2* r2 = T2 + (size_t)i * W;
    df2 c{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    df ck{0.f, 0.f};
    if (i >= P && i < n - P) {
      const float4* xr = sm4 + (i - P) * kLd + lane;
#pragma unroll
      for (int t = 0; t < W; ++t) {
        const float4 e = xr[t * kLd];
        const float4 cf = __ldg(r4 + t);
        df_fma2(c, make_float2(cf.x, cf.y), make_float2(cf.z, cf.w), make_float2(e.x, e.y), make_float2(e.z, e.w));
        if (KIND == 1) df_fma(ck, __ldg(r2 + t), df{e.x, e.z});
      }
    } else {
      const int a0 = max(0, i - P), a1 = min(n - 1, i + P);
      for (int a = a0; a <= a1; ++a) {
        const int t = a - i + P;
        const float4 e = sm4[a * kLd + lane];
        const float4 cf = __ldg(r4 + t);
        df_fma2(c, make_float2(cf.x, cf.y), make_float2(cf.z, cf.w), make_float2(e.x, e.y), make_float2(e.z, e.w));
        if (KIND == 1) df_fma(ck, __ldg(r2 + t), df{e.x, e.z});
      }
    }
    if (!valid) continue;
    // rotated layout: entry i of fibre q goes to i Q + q, so that the direction
    // just applied becomes the slowest index and the next one the fastest
    const long long off = rot ? q + (long long)i * Q : base + (long long)i * inner;
    const df c1 = df_norm(df{c.h.x, c.l.x}), c2 = df_norm(df{c.h.y, c.l.y});
    if (KIND == 0) {          // (M x, K x)
      store_df(Uo, off, c1);
      store_df(Vo, off, c2);
    } else if (KIND == 1) {   // (M u, K u + M v)
      store_df(Uo, off, c1);
      store_df(Vo, off, df_add(df_norm(ck), c2));
    } else {                  // gamma W u + nu M_t v
      df a2 = c1, a3 = c2;
      if (scale) {
        a2 = df_scale(a2, s2);
        a3 = df_scale(a3, s3);
      }
      store_df(Vo, off, df_add(a2, a3));
    }
  }
}

template <typename TIn, typename TOut, int KIND, int P>
cudaError_t launch_pk(const TIn* U, const float2* V, const float4* T4, const float2* T2, double s2, double s3,
                      float2* Uo, TOut* Vo, int n, long long inner, long long outer, int rot, cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  {
    const cudaError_t e = ensure_smem_attr(k_band_pk<TIn, TOut, KIND, P>, 256 * (kTC + 1) * (int)sizeof(float4));
    if (e != cudaSuccess) return e;
  }
  const size_t smem = (size_t)n * (kTC + 1) * sizeof(float4);
  if (smem > (size_t)256 * (kTC + 1) * sizeof(float4)) return cudaErrorInvalidValue;
  double entries = 0.0;
  for (int i = 0; i < n; ++i) entries += (double)(std::min(n - 1, i + P) - std::max(0, i - P) + 1);
  const int nprod = KIND == 1 ? 3 : 2;
  const int nio = KIND == 0 ? 3 : KIND == 1 ? 4 : 3;
  ProfScope ps("band_pair_df", 2.0 * entries * (double)Q * nprod, 8.0 * (double)Q * n * nio, st);
  const float h2 = (float)s2, h3 = (float)s3;
  const float2 c2 = make_float2(h2, (float)(s2 - (double)h2)), c3 = make_float2(h3, (float)(s3 - (double)h3));
  const int scale = (s2 != 1.0 || s3 != 1.0) ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((Q + kTC - 1) / kTC));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_band_pk<TIn, TOut, KIND, P>, U, V, T4, T2, c2, c3, Uo, Vo, n,
                                           inner, Q, scale, rot);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename TIn, typename TOut, bool HAS_V, bool TWO_OUT>
cudaError_t launch_pair(const TIn* U, const float2* V, const float2* A1, const float2* A2, const float2* A3,
                        double s2, double s3, float2* Uo, TOut* Vo, int n, long long inner, long long outer, int bw,
                        cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  {
    const cudaError_t e = ensure_smem_attr(k_band_pair_df<TIn, TOut, HAS_V, TWO_OUT>, 2 * 256 * kTC * (int)sizeof(float2));
    if (e != cudaSuccess) return e;
  }
  const size_t smem = (size_t)(HAS_V ? 2 : 1) * n * kTC * sizeof(float2);
  double entries = 0.0;
  for (int i = 0; i < n; ++i) entries += (double)(std::min(n - 1, i + bw) - std::max(0, i - bw) + 1);
  const int nprod = (TWO_OUT ? 1 : 0) + 1 + (HAS_V ? 1 : 0);
  const int nio = (HAS_V ? 2 : 1) + (TWO_OUT ? 2 : 1);
  ProfScope ps("band_pair_df", 2.0 * entries * (double)Q * nprod, 8.0 * (double)Q * n * nio, st);
  const float h2 = (float)s2, h3 = (float)s3;
  const float2 c2 = make_float2(h2, (float)(s2 - (double)h2)), c3 = make_float2(h3, (float)(s3 - (double)h3));
  const int scale = (s2 != 1.0 || s3 != 1.0) ? 1 : 0;
  k_band_pair_df<TIn, TOut, HAS_V, TWO_OUT><<<(unsigned)((Q + kTC - 1) / kTC), kThreads, smem, st>>>(
      U, V, A1, A2, A3, c2, c3, Uo, Vo, n, inner, Q, bw, scale);
  return cudaGetLastError();
}

}  // namespace

#define STFD_BAND_DISPATCH(P_, CALL) \
  switch (P_) {                            \
    case 1: return CALL(1);                \
    case 2: return CALL(2);                \
    case 3: return CALL(3);                \
    case 4: return CALL(4);                \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_band_first_pk(const double* x, const float4* MK, float2* Uo, float2* Vo, int n, long long inner,
                                 long long outer, int p, int rot, cudaStream_t st) {
#define CALL(PP) launch_pk<double, float2, 0, PP>(x, nullptr, MK, nullptr, 1.0, 1.0, Uo, Vo, n, inner, outer, rot, st)
  STFD_BAND_DISPATCH(p, CALL)
#undef CALL
}

cudaError_t launch_band_mid_pk(const float2* u, const float2* v, const float4* MM, const float2* Kb, float2* Uo,
                               float2* Vo, int n, long long inner, long long outer, int p, int rot, cudaStream_t st) {
#define CALL(PP) launch_pk<float2, float2, 1, PP>(u, v, MM, Kb, 1.0, 1.0, Uo, Vo, n, inner, outer, rot, st)
  STFD_BAND_DISPATCH(p, CALL)
#undef CALL
}

cudaError_t launch_band_last_pk(const float2* u, const float2* v, const float4* WMt, double gamma, double nu,
                                double* y, int n, long long inner, long long outer, int p, int rot, cudaStream_t st) {
#define CALL(PP) launch_pk<float2, double, 2, PP>(u, v, WMt, nullptr, gamma, nu, nullptr, y, n, inner, outer, rot, st)
  STFD_BAND_DISPATCH(p, CALL)
#undef CALL
}

cudaError_t launch_band_first_df(const double* x, const float2* M, const float2* K, float2* Uo, float2* Vo, int n,
                                 long long inner, long long outer, int bw, cudaStream_t st) {
  return launch_pair<double, float2, false, true>(x, nullptr, M, K, nullptr, 1.0, 1.0, Uo, Vo, n, inner, outer, bw, st);
}

cudaError_t launch_band_mid_df(const float2* u, const float2* v, const float2* M, const float2* K, float2* Uo,
                               float2* Vo, int n, long long inner, long long outer, int bw, cudaStream_t st) {
  return launch_pair<float2, float2, true, true>(u, v, M, K, M, 1.0, 1.0, Uo, Vo, n, inner, outer, bw, st);
}

cudaError_t launch_band_last_df(const float2* u, const float2* v, const float2* W, double gamma, const float2* Mt,
                                double nu, double* y, int n, long long inner, long long outer, int bw,
                                cudaStream_t st) {
  return launch_pair<float2, double, true, false>(u, v, nullptr, W, Mt, gamma, nu, nullptr, y, n, inner, outer, bw, st);
}

}  // namespace stfd
