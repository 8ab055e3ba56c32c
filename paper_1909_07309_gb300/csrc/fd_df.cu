// Algorithm 1 (Steps 2-4) in double-float arithmetic on the FP32 pipes: the
// FP64-accurate preconditioner for a GPU whose FP64 pipe is ~1/70 of its FP32
// rate. Dense mode products (eq. kron_vec_multi with the eigenvector factors)
// and the real arrowhead block LU (eq. block_LU, 2 x 2 blocks of the Remark in
// Sec. 4.5) both carry every value as a (hi, lo) float pair.
#include <cuda_runtime.h>

#include <algorithm>

#include "arrow_df.cuh"
#include "df.cuh"
#include "device_state.h"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {
namespace {

using dfa::df;

constexpr int kTC = 32;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kIB = 4;   // output rows per thread and pass (register blocking)

template <typename T>
__device__ __forceinline__ df ld(const T* p, long long i);
template <>
__device__ __forceinline__ df ld<double>(const double* p, long long i) { return dfa::from_double(p[i]); }
template <>
__device__ __forceinline__ df ld<float2>(const float2* p, long long i) { return dfa::from_float2(p[i]); }
__device__ __forceinline__ void st(double* p, long long i, df v) { p[i] = dfa::to_double(v); }
__device__ __forceinline__ void st(float2* p, long long i, df v) { p[i] = make_float2(v.h, v.l); }

// Y[o, i, c] = sum_a J[i, a] X[o, a, c]; J row-major (hi, lo) pairs.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kThreads)
k_mode_df(const TIn* __restrict__ X, const float2* __restrict__ J, TOut* __restrict__ Y, int n, long long inner,
          long long Q) {
  extern __shared__ float2 xs[];   // [n][kTC]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long q = (long long)blockIdx.x * kTC + lane;
  const bool valid = q < Q;
  long long base = 0;
  if (valid) {
    const long long o = q / inner;
    base = o * (long long)n * inner + (q - o * inner);
  }
  for (int a = warp; a < n; a += kWarps) {
    const df v = valid ? ld<TIn>(X, base + (long long)a * inner) : df{0.f, 0.f};
    xs[a * kTC + lane] = make_float2(v.h, v.l);
  }
  __syncthreads();
  for (int i0 = warp; i0 < n; i0 += kWarps * kIB) {
    df acc[kIB];
    const float2* row[kIB];
#pragma unroll
    for (int b = 0; b < kIB; ++b) {
      acc[b] = df{0.f, 0.f};
      const int i = min(i0 + b * kWarps, n - 1);
      row[b] = J + (size_t)i * n;
    }
    for (int a = 0; a < n; ++a) {
      const df x = dfa::from_float2(xs[a * kTC + lane]);
#pragma unroll
      for (int b = 0; b < kIB; ++b) dfa::fma_acc(acc[b], __ldg(row[b] + a), x);
    }
    if (valid) {
#pragma unroll
      for (int b = 0; b < kIB; ++b) {
        const int i = i0 + b * kWarps;
        if (i < n) st(Y, base + (long long)i * inner, dfa::norm(acc[b]));
      }
    }
  }
}

// Step 3 per spatial index k (see k_arrowhead in kernels.cu for the algebra).
__global__ void k_arrowhead_df(float2* __restrict__ X, ArrowDF p) {
  tc::grid_dependency_wait();   // programmatic dependent launch
  tc::grid_launch_dependents();
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < p.Ns;
       k += (long long)gridDim.x * blockDim.x)
    arrowhead_df_point(X, p, k);
}

int sms() { return sm_count_current(); }

template <typename TIn, typename TOut>
cudaError_t launch_mode(const TIn* X, const float2* J, TOut* Y, int n, long long inner, long long outer,
                        cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  {
    const cudaError_t e = ensure_smem_attr(k_mode_df<TIn, TOut>, 256 * kTC * (int)sizeof(float2));
    if (e != cudaSuccess) return e;
  }
  ProfScope ps("fd_mode_df", 2.0 * (double)Q * n * n, 8.0 * (double)Q * n * 2, st);
  k_mode_df<TIn, TOut><<<(unsigned)((Q + kTC - 1) / kTC), kThreads, (size_t)n * kTC * sizeof(float2), st>>>(
      X, J, Y, n, inner, Q);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fd_mode_df(const void* X, int x_is_double, const float2* J, void* Y, int y_is_double, int n,
                              long long inner, long long outer, cudaStream_t st) {
  if (x_is_double)
    return launch_mode<double, float2>((const double*)X, J, (float2*)Y, n, inner, outer, st);
  if (y_is_double)
    return launch_mode<float2, double>((const float2*)X, J, (double*)Y, n, inner, outer, st);
  return launch_mode<float2, float2>((const float2*)X, J, (float2*)Y, n, inner, outer, st);
}

cudaError_t launch_arrowhead_df(float2* X, int d, int n1, int n2, int nt, int n_pairs, int has_zero, long long Ns,
                                const float2* const* lam, const float2* B, const float2* BB, const float2* G,
                                const float2* Sinv, double nu, int sgn, cudaStream_t st) {
  if (Ns <= 0) return cudaSuccess;
  ArrowDF p;
  p.sgn = sgn < 0 ? -1.0f : 1.0f;
  p.d = d;
  p.n1 = n1;
  p.n2 = n2;
  p.nt = nt;
  p.n_pairs = n_pairs;
  p.has_zero = has_zero;
  p.Ns = Ns;
  for (int l = 0; l < 3; ++l) p.lam[l] = l < d ? lam[l] : nullptr;
  p.B = B;
  p.BB = BB;
  p.G = G;
  p.Sinv = Sinv;
  const float nh = (float)nu;
  p.nu = make_float2(nh, (float)(nu - (double)nh));
  ProfScope ps("arrowhead_df", (double)Ns * (10.0 * n_pairs + 4.0), 16.0 * (double)Ns * nt, st);
  const long long want = (Ns + 255) / 256;
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sms() * 8));
  return tc::launch_pdl(k_arrowhead_df, dim3(grid), dim3(256), 0, st, X, p);
}

}  // namespace stfd
