// FP64 device kernels: mode products (Steps 2 and 4 of Algorithm 1, and the
// banded products of the system matvec), the arrowhead block-LU solve (Step
// 3, eq. block_LU with the 2 x 2 blocks of the Remark in Sec. 4.5), and the
// BLAS-1/2 pieces of GMRES.
//
// On GB300 the FP64 pipe delivers about 1 TFLOP/s (DFMA and DMMA alike), so
// these kernels are bound by FP64 issue, not by HBM: they stage the data
// tile in shared memory once and spend their time in DFMA.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_state.h"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {
namespace {

constexpr int kTC = 32;        // tensor columns per block (one per lane)
constexpr int kThreads = 256;  // 8 warps; warp w computes rows i = w, w+8, ...
constexpr int kWarps = kThreads / 32;

// Y[o, i, c] = s1 sum_a J1[i,a] X1[o,a,c] + s2 sum_a J2[i,a] X2[o,a,c], |a - i| <= bw.
// Column q = o * inner + c; block b handles q in [32 b, 32 b + 32).
// BAND selects the instantiation used by the system matvec (banded univariate
// factors) versus the dense eigenvector products of Algorithm 1.
template <bool BAND>
__global__ void __launch_bounds__(kThreads)
k_mode_fp64(const double* __restrict__ X1, const double* __restrict__ J1, double s1,
            const double* __restrict__ X2, const double* __restrict__ J2, double s2,
            double* __restrict__ Y, int n, long long inner, long long Q, int bw) {
  extern __shared__ double smem[];
  double* xs1 = smem;             // [n][kTC]
  double* xs2 = smem + (size_t)n * kTC;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long q = (long long)blockIdx.x * kTC + lane;
  const bool valid = q < Q;
  long long base = 0;
  if (valid) {
    const long long o = q / inner;
    base = o * (long long)n * inner + (q - o * inner);
  }
  for (int a = warp; a < n; a += kWarps) {
    xs1[a * kTC + lane] = valid ? X1[base + (long long)a * inner] : 0.0;
    if (X2) xs2[a * kTC + lane] = valid ? X2[base + (long long)a * inner] : 0.0;
  }
  __syncthreads();
  for (int i = warp; i < n; i += kWarps) {
    const int a0 = max(0, i - bw), a1 = min(n - 1, i + bw);
    const double* j1 = J1 + (size_t)i * n;
    double acc1 = 0.0, acc2 = 0.0;
    for (int a = a0; a <= a1; ++a) acc1 = fma(__ldg(j1 + a), xs1[a * kTC + lane], acc1);
    if (X2) {
      const double* j2 = J2 + (size_t)i * n;
      for (int a = a0; a <= a1; ++a) acc2 = fma(__ldg(j2 + a), xs2[a * kTC + lane], acc2);
    }
    if (valid) Y[base + (long long)i * inner] = X2 ? fma(s1, acc1, s2 * acc2) : s1 * acc1;
  }
}

// Step 3 per spatial index k, with a = nu mu_k (mu_k = sum_l lambda_l[i_l]):
//  pairs j:  H_j = [[a, b_j], [-b_j, a]], b_j = gamma lam_j, B_j = gamma [g_2j; g_2j+1]
//  zero block (if any): H = a, B = gamma g_z;   last: H_n = gamma sigma + a
//  y_n = x_n + sum_j B_j^T H_j^{-1} x_j,  q_n = y_n / S_k,  q_j = H_j^{-1} (x_j - B_j q_n).
template <typename T>
__global__ void k_arrowhead(T* __restrict__ X, ArrowParamsT<T> p) {
  const long long Ns = p.Ns;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < Ns;
       k += (long long)gridDim.x * blockDim.x) {
    long long rest = k;
    const int i1 = (int)(rest % p.n1);
    rest /= p.n1;
    T mu = p.lam[0][i1];
    if (p.d >= 2) {
      const int i2 = (int)(rest % p.n2);
      rest /= p.n2;
      mu += p.lam[1][i2];
    }
    if (p.d >= 3) mu += p.lam[2][rest];
    const T a = p.nu * mu;
    const T gam = p.gamma * p.sgn;   // transposed system: b_j -> -b_j, B_j -> -B_j
    T y = X[(long long)(p.nt - 1) * Ns + k];
    // unrolled: the loads of eight pairs are in flight together
#pragma unroll 8
    for (int j = 0; j < p.n_pairs; ++j) {
      const T x1 = X[(long long)(2 * j) * Ns + k], x2 = X[(long long)(2 * j + 1) * Ns + k];
      const T b = gam * p.lamt[j];
      const T inv = T(1) / fma(a, a, b * b);
      const T h1 = (a * x1 - b * x2) * inv, h2 = (b * x1 + a * x2) * inv;
      y = fma(gam, fma(p.g[2 * j], h1, p.g[2 * j + 1] * h2), y);
    }
    const int z = 2 * p.n_pairs;
    T x0 = 0.0;
    if (p.has_zero) {
      x0 = X[(long long)z * Ns + k];
      y = fma(gam * p.g[z], x0 / a, y);
    }
    const T qn = y * p.Sinv[k];
    X[(long long)(p.nt - 1) * Ns + k] = qn;
    // unrolled: the loads of eight pairs are in flight together
#pragma unroll 8
    for (int j = 0; j < p.n_pairs; ++j) {
      const long long o1 = (long long)(2 * j) * Ns + k, o2 = (long long)(2 * j + 1) * Ns + k;
      const T b = gam * p.lamt[j];
      const T inv = T(1) / fma(a, a, b * b);
      const T r1 = X[o1] - gam * p.g[2 * j] * qn, r2 = X[o2] - gam * p.g[2 * j + 1] * qn;
      X[o1] = (a * r1 - b * r2) * inv;
      X[o2] = (b * r1 + a * r2) * inv;
    }
    if (p.has_zero) X[(long long)z * Ns + k] = (x0 - gam * p.g[z] * qn) / a;
  }
}

// FP32 Step 3 of the mixed-precision preconditioner, staged: a CTA owns 128
// consecutive spatial indices; each thread copies its own index's n_t entries
// into shared memory (asynchronous copies, all in flight together, column t of
// an [n_t][128] tile), computes the block LU above on them and writes the
// results back (coalesced per time index). One thread per index, as
// k_arrowhead, without its chain of dependent global loads.
constexpr int kArrowTile = 128;
__global__ void __launch_bounds__(kArrowTile) k_arrowhead_staged(float* __restrict__ X, ArrowParamsT<float> p) {
  extern __shared__ __align__(16) float sx[];   // [nt][kArrowTile]
  const long long Ns = p.Ns;
  const int t = threadIdx.x;
  const long long k = (long long)blockIdx.x * kArrowTile + t;
  tc::grid_dependency_wait();
  if (k >= Ns) return;   // no barrier below: each thread reads only its own column
  for (int j = 0; j < p.nt; ++j) tc::cp_async4(&sx[j * kArrowTile + t], X + (long long)j * Ns + k);
  long long rest = k;
  const int i1 = (int)(rest % p.n1);
  rest /= p.n1;
  float mu = p.lam[0][i1];
  if (p.d >= 2) {
    const int i2 = (int)(rest % p.n2);
    rest /= p.n2;
    mu += p.lam[1][i2];
  }
  if (p.d >= 3) mu += p.lam[2][rest];
  const float a = p.nu * mu;
  const float gam = p.gamma * p.sgn;   // transposed system: b_j -> -b_j, B_j -> -B_j
  const float sinv = p.Sinv[k];
  tc::cp_async_wait_all();
  const float* col = sx + t;
  float y = col[(p.nt - 1) * kArrowTile];
  for (int j = 0; j < p.n_pairs; ++j) {
    const float x1 = col[(2 * j) * kArrowTile], x2 = col[(2 * j + 1) * kArrowTile];
    const float b = gam * p.lamt[j];
    const float inv = 1.0f / fmaf(a, a, b * b);
    const float h1 = (a * x1 - b * x2) * inv, h2 = (b * x1 + a * x2) * inv;
    y = fmaf(gam, fmaf(p.g[2 * j], h1, p.g[2 * j + 1] * h2), y);
  }
  const int z = 2 * p.n_pairs;
  float x0 = 0.0f;
  if (p.has_zero) {
    x0 = col[z * kArrowTile];
    y = fmaf(gam * p.g[z], x0 / a, y);
  }
  const float qn = y * sinv;
  X[(long long)(p.nt - 1) * Ns + k] = qn;
  for (int j = 0; j < p.n_pairs; ++j) {
    const float b = gam * p.lamt[j];
    const float inv = 1.0f / fmaf(a, a, b * b);
    const float r1 = col[(2 * j) * kArrowTile] - gam * p.g[2 * j] * qn;
    const float r2 = col[(2 * j + 1) * kArrowTile] - gam * p.g[2 * j + 1] * qn;
    X[(long long)(2 * j) * Ns + k] = (a * r1 - b * r2) * inv;
    X[(long long)(2 * j + 1) * Ns + k] = (b * r1 + a * r2) * inv;
  }
  if (p.has_zero) X[(long long)z * Ns + k] = (x0 - gam * p.g[z] * qn) / a;
}

// Table of Step 3 (FP64, once per handle): for every pair j and spatial index
// k, w_jk = (a_k + i b_j) / (a_k^2 + b_j^2) with a_k = nu mu_k and b_j = gamma
// lam_j, so that H_j^{-1} x_j is the complex product w_jk z_j, z_j = x_2j + i
// x_2j+1 (the 2 x 2 blocks of the Remark in Sec. 4.5). Stored [j][k].
__global__ void k_arrow_wtab(double2* __restrict__ W, ArrowParamsT<double> p) {
  const long long total = p.Ns * (long long)p.n_pairs;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / p.Ns);
    const long long k = idx - (long long)j * p.Ns;
    long long rest = k;
    const int i1 = (int)(rest % p.n1);
    rest /= p.n1;
    double mu = p.lam[0][i1];
    if (p.d >= 2) {
      const int i2 = (int)(rest % p.n2);
      rest /= p.n2;
      mu += p.lam[1][i2];
    }
    if (p.d >= 3) mu += p.lam[2][rest];
    const double a = p.nu * mu, b = p.gamma * p.lamt[j];
    const double inv = 1.0 / fma(a, a, b * b);
    W[idx] = make_double2(a * inv, b * inv);
  }
}

// FP64 Step 3 with the table above: per pair and index 12 FP64 operations
// (pass 1: h_j = w z_j and y += G_j . h_j; pass 2: q_j = w (z_j - G_j q_n)).
// The transposed system (sgn = -1) flips b_j and G_j: w's imaginary part and
// G change sign (sign-bit flips, no arithmetic).
__global__ void k_arrowhead_f64(double* __restrict__ X, ArrowParamsT<double> p, const double2* __restrict__ W,
                                const double* __restrict__ G) {
  const long long Ns = p.Ns;
  const unsigned long long flip = p.sgn < 0.0 ? 0x8000000000000000ull : 0ull;
  auto fl = [&](double v) { return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(v) ^ flip)); };
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < Ns;
       k += (long long)gridDim.x * blockDim.x) {
    double y = X[(long long)(p.nt - 1) * Ns + k];
    // unrolled: the loads of eight pairs are in flight together
#pragma unroll 8
    for (int j = 0; j < p.n_pairs; ++j) {
      const double x1 = X[(long long)(2 * j) * Ns + k], x2 = X[(long long)(2 * j + 1) * Ns + k];
      const double2 w = W[(long long)j * Ns + k];
      const double wi = fl(w.y);
      const double h1 = fma(w.x, x1, -wi * x2), h2 = fma(wi, x1, w.x * x2);
      y = fma(fl(G[2 * j]), h1, fma(fl(G[2 * j + 1]), h2, y));
    }
    const int z = 2 * p.n_pairs;
    double x0 = 0.0, a = 1.0;
    if (p.has_zero) {
      long long rest = k;
      const int i1 = (int)(rest % p.n1);
      rest /= p.n1;
      double mu = p.lam[0][i1];
      if (p.d >= 2) {
        const int i2 = (int)(rest % p.n2);
        rest /= p.n2;
        mu += p.lam[1][i2];
      }
      if (p.d >= 3) mu += p.lam[2][rest];
      a = p.nu * mu;
      x0 = X[(long long)z * Ns + k];
      y = fma(fl(G[z]), x0 / a, y);
    }
    const double qn = y * p.Sinv[k];
    X[(long long)(p.nt - 1) * Ns + k] = qn;
    // unrolled: the loads of eight pairs are in flight together
#pragma unroll 8
    for (int j = 0; j < p.n_pairs; ++j) {
      const long long o1 = (long long)(2 * j) * Ns + k, o2 = (long long)(2 * j + 1) * Ns + k;
      const double2 w = W[(long long)j * Ns + k];
      const double wi = fl(w.y);
      const double r1 = fma(-fl(G[2 * j]), qn, X[o1]), r2 = fma(-fl(G[2 * j + 1]), qn, X[o2]);
      X[o1] = fma(w.x, r1, -wi * r2);
      X[o2] = fma(wi, r1, w.x * r2);
    }
    if (p.has_zero) X[(long long)z * Ns + k] = fma(-fl(G[z]), qn, x0) / a;
  }
}

// ---- exact power-of-two range scaling for the double-float paths
// (their FP32 exponent range would otherwise clip very large or very small inputs)
__global__ void k_max_bexp(const double* __restrict__ x, long long N, int* __restrict__ out) {
  int m = 0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x)
    m = max(m, (int)(((unsigned long long)__double_as_longlong(x[k]) >> 52) & 0x7FF));
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// y = x 2^{dir (E - 1023)} with E = *bexp (the largest biased exponent of the
// vector the scale was taken from; E = 2047 (Inf/NaN) leaves x unscaled). Normal
// results are formed by adding to the exponent field (integer pipe); the rare
// others by one FP64 multiplication by the exact power of two (k >= -1023, so
// 2^k is a double: one correctly rounded result).
__global__ void k_scale_pow2(const double* __restrict__ x, double* __restrict__ y, long long N,
                             const int* __restrict__ bexp, int dir) {
  const int E = max(*bexp, 1);                                    // only subnormals: as exponent 1
  const int k = E >= 2047 ? 0 : dir * (E - 1023);                // dir -1: 1023 - E; dir +1: E - 1023
  const double f = k >= -1022 ? __longlong_as_double((long long)(k + 1023) << 52)
                              : __longlong_as_double(0x0008000000000000ll);   // 2^-1023
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const long long b = __double_as_longlong(x[i]);
    const int e = (int)(((unsigned long long)b >> 52) & 0x7FF);
    const int ne = e + k;
    y[i] = (e > 0 && e < 2047 && ne > 0 && ne < 2047) ? __longlong_as_double(b + ((long long)k << 52)) : x[i] * f;
  }
}

constexpr int kDotThreads = 256;
constexpr int kDotGroup = 4;

__device__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;   // valid in thread 0
}

// Sum over this block's share of C vectors dotted with w (C is a compile-time
// group size, so no vector is loaded twice), unrolled 4x along the vectors.
template <int C>
__device__ __forceinline__ void dot_group(const double* const* __restrict__ V, int i0, const double* __restrict__ w,
                                          long long N, long long k0, long long stride, double* acc) {
  const double* v[C];
#pragma unroll
  for (int b = 0; b < C; ++b) v[b] = V[i0 + b];
  long long k = k0;
  for (; k + 3 * stride < N; k += 4 * stride) {
    double wk[4], x[4][C];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      wk[u] = __ldg(w + k + u * stride);
#pragma unroll
      for (int b = 0; b < C; ++b) x[u][b] = __ldg(v[b] + k + u * stride);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int b = 0; b < C; ++b) acc[b] = fma(x[u][b], wk[u], acc[b]);
  }
  for (; k < N; k += stride) {
    const double wk = __ldg(w + k);
#pragma unroll
    for (int b = 0; b < C; ++b) acc[b] = fma(__ldg(v[b] + k), wk, acc[b]);
  }
}

// partial[b*m + i] = sum over block b's share of V_i . w
__global__ void __launch_bounds__(kDotThreads)
k_dot_multi(const double* const* __restrict__ V, int m, const double* __restrict__ w, long long N,
            double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int i0 = 0; i0 < m; i0 += kDotGroup) {
    const int cnt = min(kDotGroup, m - i0);
    double acc[kDotGroup] = {0.0, 0.0, 0.0, 0.0};
    switch (cnt) {
      case 1: dot_group<1>(V, i0, w, N, k0, stride, acc); break;
      case 2: dot_group<2>(V, i0, w, N, k0, stride, acc); break;
      case 3: dot_group<3>(V, i0, w, N, k0, stride, acc); break;
      default: dot_group<4>(V, i0, w, N, k0, stride, acc); break;
    }
    for (int b = 0; b < cnt; ++b) {
      const double s = block_sum(acc[b], red);
      if (threadIdx.x == 0) partial[(size_t)blockIdx.x * m + i0 + b] = s;
    }
  }
}

// out[i] = sum_b partial[b*m + i]: one warp per entry, lanes stride over blocks.
__global__ void k_reduce_partial(const double* __restrict__ partial, int m, int nblocks,
                                 double* __restrict__ out, int accumulate) {
  const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)b * m + i];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) out[i] = accumulate ? out[i] + s : s;
}

// w[k] += sign * sum_i h[i] V_i[k]: each thread owns 4 strided elements and
// walks the vectors with the pointer and signed coefficient hoisted per vector;
// the update starts from w[k], one FP64 FMA per vector and element (the FP64
// pipe, ~1/64 of the FP32 rate on GB300, is as close a bound as the memory).
__global__ void __launch_bounds__(256)
k_multi_axpy(double* __restrict__ w, const double* const* __restrict__ V, const double* __restrict__ h, int m,
             long long N, double sign) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; k0 < N; k0 += 4 * stride) {
    double acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long k = k0 + u * stride;
      acc[u] = k < N ? w[k] : 0.0;
    }
    for (int i = 0; i < m; ++i) {
      const double* vi = V[i];
      const double hi = sign * h[i];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long k = k0 + u * stride;
        if (k < N) acc[u] = fma(hi, __ldg(vi + k), acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long k = k0 + u * stride;
      if (k < N) w[k] = acc[u];
    }
  }
}

// w[k] -= sum_{i<C} h[i] V_i[k], and partial[block*C + i] = the block's share of
// V_i . w (of the updated w): the first update of classical Gram-Schmidt fused
// with the dot products of the second (one pass instead of two).
template <int C>
__global__ void __launch_bounds__(kDotThreads)
k_axpy_dot(double* __restrict__ w, const double* const* __restrict__ V, const double* __restrict__ h, long long N,
           double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  const double* v[C];
  double nh[C], d[C];
#pragma unroll
  for (int b = 0; b < C; ++b) {
    v[b] = V[b];
    nh[b] = -h[b];
    d[b] = 0.0;
  }
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + stride < N; k += 2 * stride) {
    double wk[2], x[2][C];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      wk[u] = w[k + u * stride];
#pragma unroll
      for (int b = 0; b < C; ++b) x[u][b] = __ldg(v[b] + k + u * stride);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
#pragma unroll
      for (int b = 0; b < C; ++b) wk[u] = fma(nh[b], x[u][b], wk[u]);
      w[k + u * stride] = wk[u];
#pragma unroll
      for (int b = 0; b < C; ++b) d[b] = fma(x[u][b], wk[u], d[b]);
    }
  }
  for (; k < N; k += stride) {
    double wk = w[k], x[C];
#pragma unroll
    for (int b = 0; b < C; ++b) {
      x[b] = __ldg(v[b] + k);
      wk = fma(nh[b], x[b], wk);
    }
    w[k] = wk;
#pragma unroll
    for (int b = 0; b < C; ++b) d[b] = fma(x[b], wk, d[b]);
  }
#pragma unroll
  for (int b = 0; b < C; ++b) {
    const double t = block_sum(d[b], red);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * C + b] = t;
  }
}

// w[k] = (set ? 0 : w[k]) + sign * sum_i h[i] V_i[k], and partial[block] = the
// block's share of sum_k w[k]^2 of the result (the norm fused into the update).
__global__ void __launch_bounds__(kDotThreads)
k_axpy_norm(double* __restrict__ w, const double* const* __restrict__ V, const double* __restrict__ h, int m,
            long long N, double sign, int set, double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  double sq = 0.0;
  for (long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; k0 < N; k0 += 4 * stride) {
    double acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long k = k0 + u * stride;
      acc[u] = (set || k >= N) ? 0.0 : w[k];
    }
    for (int i = 0; i < m; ++i) {
      const double* vi = V[i];
      const double hi = sign * h[i];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long k = k0 + u * stride;
        if (k < N) acc[u] = fma(hi, __ldg(vi + k), acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const long long k = k0 + u * stride;
      if (k < N) {
        w[k] = acc[u];
        if (partial) sq = fma(acc[u], acc[u], sq);
      }
    }
  }
  if (partial) {
    const double t = block_sum(sq, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// r = f - y (y may be NULL: r = f); out[k] = r if out is not NULL; partial[block]
// = the block's share of sum_k r^2.
__global__ void __launch_bounds__(kDotThreads)
k_sub_norm(double* __restrict__ out, const double* __restrict__ f, const double* __restrict__ y, long long N,
           double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32];
  double sq = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    const double r = y ? f[k] - y[k] : f[k];
    if (out) out[k] = r;
    sq = fma(r, r, sq);
  }
  const double t = block_sum(sq, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// y = x / den (or x / sqrt(den)); leaves x unscaled when the divisor is not positive.
__global__ void k_scale_by_inverse(double* y, const double* x,   // may be the same vector
                                   const double* __restrict__ den, long long N, int sqrt_den) {
  const double dv = sqrt_den ? sqrt(den[0]) : den[0];
  const double inv = dv > 0.0 ? 1.0 / dv : 1.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (long long)gridDim.x * blockDim.x)
    y[k] = x[k] * inv;
}

__global__ void k_sub(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                      long long N) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (long long)gridDim.x * blockDim.x)
    y[k] = a[k] - b[k];
}

int sm_count() { return sm_count_current(); }

int grid_for(long long n, int threads) {
  const long long want = (n + threads - 1) / threads;
  const long long cap = (long long)sm_count() * 8;
  return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

int dot_blocks() { return sm_count() * 4; }

template <bool BAND>
static cudaError_t launch_mode_impl(const char* name, const double* X1, const double* J1, double s1,
                                   const double* X2, const double* J2, double s2, double* Y, int n,
                                   long long inner, long long outer, int bw, cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  const size_t smem = (size_t)(X2 ? 2 : 1) * n * kTC * sizeof(double);
  {
    const cudaError_t e = ensure_smem_attr(k_mode_fp64<BAND>, 2 * 256 * kTC * (int)sizeof(double));
    if (e != cudaSuccess) return e;
  }
  // algorithmic work: 2 flops per stored band entry per column and input
  double entries = 0.0;
  for (int i = 0; i < n; ++i) entries += (double)(std::min(n - 1, i + bw) - std::max(0, i - bw) + 1);
  const int nin = X2 ? 2 : 1;
  const double flops = 2.0 * entries * (double)Q * nin;
  const double bytes = 8.0 * (double)Q * n * (nin + 1);
  ProfScope ps(name, flops, bytes, st);
  const long long blocks = (Q + kTC - 1) / kTC;
  k_mode_fp64<BAND><<<(unsigned)blocks, kThreads, smem, st>>>(X1, J1, s1, X2, J2, s2, Y, n, inner, Q, bw);
  return cudaGetLastError();
}

cudaError_t launch_fd_mode_fp64(const double* X, const double* J, double* Y, int n, long long inner,
                                long long outer, cudaStream_t st) {
  return launch_mode_impl<false>("fd_mode_fp64", X, J, 1.0, nullptr, nullptr, 0.0, Y, n, inner, outer, n, st);
}

cudaError_t launch_band_mode_fp64(const double* X1, const double* J1, double s1,
                                  const double* X2, const double* J2, double s2,
                                  double* Y, int n, long long inner, long long outer, int bw,
                                  cudaStream_t st) {
  return launch_mode_impl<true>("band_mode_fp64", X1, J1, s1, X2, J2, s2, Y, n, inner, outer, bw, st);
}

cudaError_t launch_arrowhead_fp64(double* X, const ArrowParams& p, cudaStream_t st) {
  if (p.Ns <= 0) return cudaSuccess;
  ProfScope ps("arrowhead_fp64", (double)p.Ns * (10.0 * p.n_pairs + 4.0), 16.0 * (double)p.Ns * p.nt, st);
  k_arrowhead<double><<<grid_for(p.Ns, 256), 256, 0, st>>>(X, p);
  return cudaGetLastError();
}

cudaError_t launch_arrow_wtab(double2* W, const ArrowParams& p, cudaStream_t st) {
  if (p.Ns <= 0 || p.n_pairs <= 0) return cudaSuccess;
  count_launch();
  k_arrow_wtab<<<grid_for(p.Ns * p.n_pairs, 256), 256, 0, st>>>(W, p);
  return cudaGetLastError();
}

cudaError_t launch_arrowhead_fp64_tab(double* X, const ArrowParams& p, const double2* W, const double* G,
                                      cudaStream_t st) {
  if (p.Ns <= 0) return cudaSuccess;
  ProfScope ps("arrowhead_fp64", (double)p.Ns * (12.0 * p.n_pairs + 4.0),
               16.0 * (double)p.Ns * p.nt + 16.0 * (double)p.Ns * p.n_pairs, st);
  k_arrowhead_f64<<<grid_for(p.Ns, 128), 128, 0, st>>>(X, p, W, G);
  return cudaGetLastError();
}

cudaError_t launch_arrowhead_fp32(float* X, const ArrowParamsT<float>& p, cudaStream_t st) {
  if (p.Ns <= 0) return cudaSuccess;
  ProfScope ps("arrowhead_fp32", (double)p.Ns * (10.0 * p.n_pairs + 4.0), 8.0 * (double)p.Ns * p.nt, st);
  const size_t smem = (size_t)p.nt * kArrowTile * sizeof(float);
  if (smem <= 96 * 1024) {
    const cudaError_t e = ensure_smem_attr(k_arrowhead_staged, 96 * 1024);
    if (e != cudaSuccess) return e;
    return tc::launch_pdl(k_arrowhead_staged, dim3((unsigned)((p.Ns + kArrowTile - 1) / kArrowTile)),
                          dim3(kArrowTile), smem, st, X, p);
  }
  k_arrowhead<float><<<grid_for(p.Ns, 256), 256, 0, st>>>(X, p);
  return cudaGetLastError();
}

cudaError_t launch_range_scale(const double* x, double* y, long long N, int* bexp, int dir, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (dir < 0) {   // a new scale from x
    cudaError_t e = cudaMemsetAsync(bexp, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    count_launch();
    k_max_bexp<<<grid_for(N, 256), 256, 0, st>>>(x, N, bexp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  count_launch();
  k_scale_pow2<<<grid_for(N, 256), 256, 0, st>>>(x, y, N, bexp, dir);
  return cudaGetLastError();
}

cudaError_t launch_dot_multi(const double* const* V, int m, const double* w, long long N,
                             double* partial, int nblocks, cudaStream_t st) {
  ProfScope ps("gmres_dot_multi", 2.0 * N * m, 8.0 * N * (m + 1), st);
  k_dot_multi<<<nblocks, kDotThreads, 0, st>>>(V, m, w, N, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partial(const double* partial, int m, int nblocks, double* out,
                                  int accumulate, cudaStream_t st) {
  ProfScope ps("gmres_reduce", (double)m * nblocks, 8.0 * m * nblocks, st);
  k_reduce_partial<<<(m + 3) / 4, 128, 0, st>>>(partial, m, nblocks, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(double* w, const double* const* V, const double* h, int m,
                              long long N, double sign, cudaStream_t st) {
  ProfScope ps("gmres_multi_axpy", 2.0 * N * m, 8.0 * N * (m + 2), st);
  k_multi_axpy<<<grid_for((N + 3) / 4, 256), 256, 0, st>>>(w, V, h, m, N, sign);
  return cudaGetLastError();
}

cudaError_t launch_axpy_dot(double* w, const double* const* V, const double* h, int m, long long N,
                            double* partial, int nblocks, cudaStream_t st) {
  if (m < 1 || m > 4) return cudaErrorInvalidValue;
  ProfScope ps("gmres_axpy_dot", 4.0 * N * m, 8.0 * N * (m + 2), st);
  switch (m) {
    case 1: k_axpy_dot<1><<<nblocks, kDotThreads, 0, st>>>(w, V, h, N, partial); break;
    case 2: k_axpy_dot<2><<<nblocks, kDotThreads, 0, st>>>(w, V, h, N, partial); break;
    case 3: k_axpy_dot<3><<<nblocks, kDotThreads, 0, st>>>(w, V, h, N, partial); break;
    default: k_axpy_dot<4><<<nblocks, kDotThreads, 0, st>>>(w, V, h, N, partial); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_scale_by_inverse(double* y, const double* x, const double* den, long long N,
                                    int sqrt_den, cudaStream_t st) {
  ProfScope ps("gmres_scale", (double)N, 16.0 * N, st);
  k_scale_by_inverse<<<grid_for(N, 256), 256, 0, st>>>(y, x, den, N, sqrt_den);
  return cudaGetLastError();
}

cudaError_t launch_axpy_norm(double* w, const double* const* V, const double* h, int m, long long N, double sign,
                             int set, double* partial, int nblocks, cudaStream_t st) {
  ProfScope ps("gmres_multi_axpy", 2.0 * N * m + 2.0 * N, 8.0 * N * (m + (set ? 1 : 2)), st);
  k_axpy_norm<<<nblocks, kDotThreads, 0, st>>>(w, V, h, m, N, sign, set, partial);
  return cudaGetLastError();
}

cudaError_t launch_sub_norm(double* out, const double* f, const double* y, long long N, double* partial,
                            int nblocks, cudaStream_t st) {
  ProfScope ps("gmres_sub_norm", 3.0 * N, 8.0 * N * ((y ? 2 : 1) + (out ? 1 : 0)), st);
  k_sub_norm<<<nblocks, kDotThreads, 0, st>>>(out, f, y, N, partial);
  return cudaGetLastError();
}

// A few doubles between device memory and host-mapped pinned memory, copied by
// a kernel: the solver's scalars do not queue on a copy engine behind bulk
// transfers that other streams may have in flight.
__global__ void k_copy_doubles(double* __restrict__ dst, const double* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_copy_doubles(double* dst, const double* src, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launch();
  k_copy_doubles<<<1, 128, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_sub(double* y, const double* a, const double* b, long long N, cudaStream_t st) {
  ProfScope ps("gmres_sub", (double)N, 24.0 * N, st);
  k_sub<<<grid_for(N, 256), 256, 0, st>>>(y, a, b, N);
  return cudaGetLastError();
}

}  // namespace stfd
