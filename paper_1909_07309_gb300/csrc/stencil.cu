// System matvec with general (sparse) spatial matrices, as on a mapped domain
// with variable coefficients (Sec. 4.6.1):
//     y = gamma (W_t (x) M_s) x + nu (M_t (x) K_s) x.
// Pass 1 (time): Z1 = gamma (W_t (x) I) x, Z2 = nu (M_t (x) I) x with the
// banded time factors. Pass 2 (space): y_t = M_s Z1_t + K_s Z2_t for every
// time slice t, with M_s and K_s in the tensor-product stencil layout (for each
// of the (2p+1)^d offsets a coefficient array over the N_s rows). A CTA owns
// R consecutive rows and TC time slices: for every pair of outer offsets it
// stages the R + 2p needed entries of Z1 and Z2 per time slice in shared
// memory, then every thread applies the 2p+1 innermost offsets of its row to
// all TC slices. The time chunks of one row block are consecutive block
// indices, so they run together and share that block's coefficients in L2.
//
// Also: the per-element conductivity gradient -nu lam^T (M_t (x) K_e) u and
// the diagonal scaling of the geometry-aware preconditioner (eq. prec_geo).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "df.cuh"
#include "device_state.h"
#include "kernels.h"
#include "profile.h"

namespace stfd {
namespace {

using dfa::df;

constexpr int kRows = 256;   // rows per CTA (threads)

template <typename T>
struct Num;
template <>
struct Num<double> {
  using acc = double;
  __device__ static acc zero() { return 0.0; }
  __device__ static void fma2(acc& a, double m, double z1, double k, double z2) { a = fma(m, z1, fma(k, z2, a)); }
  __device__ static double out(acc a) { return a; }
};
template <>
struct Num<float2> {
  using acc = df;
  __device__ static acc zero() { return df{0.f, 0.f}; }
  __device__ static void fma2(acc& a, float2 m, float2 z1, float2 k, float2 z2) {
    dfa::fma_acc(a, m, dfa::from_float2(z1));
    dfa::fma_acc(a, k, dfa::from_float2(z2));
  }
  __device__ static double out(acc a) { return dfa::to_double(dfa::norm(a)); }
};

// Pass 2. Block b handles time chunk b % n_chunks of row block b / n_chunks.
// PP > 0 fixes the half-bandwidth p at compile time (unrolled offsets,
// immediate shared-memory offsets); PP = 0 reads it from g.
template <typename T, int kTC, int PP>
__global__ void __launch_bounds__(kRows)
k_stencil(const T* __restrict__ Ms, const T* __restrict__ Ks, const T* __restrict__ Z1, const T* __restrict__ Z2,
          double* __restrict__ y, StencilDims g) {
  extern __shared__ unsigned char smem_raw[];
  const int p = PP > 0 ? PP : g.p;
  const int W = 2 * p + 1, span = kRows + 2 * p;
  T* z1s = reinterpret_cast<T*>(smem_raw);            // [kTC][span]
  T* z2s = z1s + kTC * span;
  const int n_chunks = (g.nt + kTC - 1) / kTC;
  const long long i0 = (long long)(blockIdx.x / n_chunks) * kRows;
  const int t0 = (int)(blockIdx.x % n_chunks) * kTC;
  const long long i = i0 + threadIdx.x;
  const bool valid = i < g.Ns;
  const int ntc = min(kTC, g.nt - t0);
  const int S23 = g.d >= 3 ? W * W : (g.d == 2 ? W : 1);
  const T* mrow = Ms + (valid ? i : 0);
  const T* krow = Ks + (valid ? i : 0);
  typename Num<T>::acc acc[kTC];
#pragma unroll
  for (int tt = 0; tt < kTC; ++tt) acc[tt] = Num<T>::zero();
  for (int o23 = 0; o23 < S23; ++o23) {
    const int o2 = g.d >= 2 ? o23 % W : p, o3 = g.d >= 3 ? o23 / W : p;
    const long long base = i0 - p + (long long)(o2 - p) * g.n1 + (long long)(o3 - p) * g.n1 * g.n2;
    __syncthreads();
    // stage Z1, Z2 at columns base .. base + span - 1 for the kTC slices
    for (int c = threadIdx.x; c < span; c += kRows) {
      long long j = base + c;
      j = j < 0 ? 0 : (j >= g.Ns ? g.Ns - 1 : j);   // the coefficient is 0 for columns outside the box
#pragma unroll
      for (int tt = 0; tt < kTC; ++tt) {
        T v1{}, v2{};
        if (tt < ntc) {
          v1 = Z1[(long long)(t0 + tt) * g.Ns + j];
          v2 = Z2[(long long)(t0 + tt) * g.Ns + j];
        }
        z1s[tt * span + c] = v1;
        z2s[tt * span + c] = v2;
      }
    }
    __syncthreads();
    const long long ob = (long long)W * o23 * g.Ns;
#pragma unroll
    for (int o1 = 0; o1 < (PP > 0 ? 2 * PP + 1 : W); ++o1) {
      if (PP == 0 && o1 >= W) break;
      const T m = mrow[ob + (long long)o1 * g.Ns], kk = krow[ob + (long long)o1 * g.Ns];
#pragma unroll
      for (int tt = 0; tt < kTC; ++tt)
        Num<T>::fma2(acc[tt], m, z1s[tt * span + threadIdx.x + o1], kk, z2s[tt * span + threadIdx.x + o1]);
    }
  }
  if (valid) {
#pragma unroll
    for (int tt = 0; tt < kTC; ++tt)   // static indices keep acc[] in registers
      if (tt < ntc) y[(long long)(t0 + tt) * g.Ns + i] = Num<T>::out(acc[tt]);
  }
}

// Pass 2 in double-float with two time slices per paired FP32 instruction
// (fma.rn.f32x2 and friends; per slice the scalar steps of dfa::fma_acc in the
// same order, so the results equal those of k_stencil<float2>). The staged
// slices are stored as high and low planes of slice pairs, [kTC/2][span] of
// float2 (slice 2u, slice 2u + 1), so that one 8-byte load gives an operand.
struct df2 {
  float2 h, l;
};

__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }

// acc += b * x on two slices (b the same coefficient for both); the steps of fma_acc
__device__ __forceinline__ void fma_acc2(df2& acc, float2 bh, float2 bl, float2 xh, float2 xl) {
  const float2 p = __fmul2_rn(bh, xh);
  const float2 e = __ffma2_rn(bh, xh, make_float2(-p.x, -p.y));
  const float2 lo = __ffma2_rn(bh, xl, __ffma2_rn(bl, xh, e));
  const float2 s = __fadd2_rn(acc.h, p);
  const float2 bp = sub2(s, acc.h);
  const float2 err = __fadd2_rn(sub2(acc.h, sub2(s, bp)), sub2(p, bp));
  acc.h = s;
  acc.l = __fadd2_rn(acc.l, __fadd2_rn(err, lo));
}

template <int kTC, int PP>
__global__ void __launch_bounds__(kRows)
k_stencil_pk(const float2* __restrict__ Ms, const float2* __restrict__ Ks, const float2* __restrict__ Z1,
             const float2* __restrict__ Z2, double* __restrict__ y, StencilDims g) {
  constexpr int kTP = kTC / 2;
  extern __shared__ unsigned char smem_raw[];
  const int p = PP > 0 ? PP : g.p;
  const int W = 2 * p + 1, span = kRows + 2 * p;
  float2* z1h = reinterpret_cast<float2*>(smem_raw);   // [kTP][span] each
  float2* z1l = z1h + kTP * span;
  float2* z2h = z1l + kTP * span;
  float2* z2l = z2h + kTP * span;
  const int n_chunks = (g.nt + kTC - 1) / kTC;
  const long long i0 = (long long)(blockIdx.x / n_chunks) * kRows;
  const int t0 = (int)(blockIdx.x % n_chunks) * kTC;
  const long long i = i0 + threadIdx.x;
  const bool valid = i < g.Ns;
  const int ntc = min(kTC, g.nt - t0);
  const int S23 = g.d >= 3 ? W * W : (g.d == 2 ? W : 1);
  const float2* mrow = Ms + (valid ? i : 0);
  const float2* krow = Ks + (valid ? i : 0);
  df2 acc[kTP];
#pragma unroll
  for (int u = 0; u < kTP; ++u) acc[u] = df2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  for (int o23 = 0; o23 < S23; ++o23) {
    const int o2 = g.d >= 2 ? o23 % W : p, o3 = g.d >= 3 ? o23 / W : p;
    const long long base = i0 - p + (long long)(o2 - p) * g.n1 + (long long)(o3 - p) * g.n1 * g.n2;
    __syncthreads();
    for (int c = threadIdx.x; c < span; c += kRows) {
      long long j = base + c;
      j = j < 0 ? 0 : (j >= g.Ns ? g.Ns - 1 : j);   // the coefficient is 0 for columns outside the box
#pragma unroll
      for (int u = 0; u < kTP; ++u) {
        float2 a1{0.f, 0.f}, b1{0.f, 0.f}, a2{0.f, 0.f}, b2{0.f, 0.f};   // slices 2u, 2u + 1
        if (2 * u < ntc) {
          a1 = Z1[(long long)(t0 + 2 * u) * g.Ns + j];
          a2 = Z2[(long long)(t0 + 2 * u) * g.Ns + j];
        }
        if (2 * u + 1 < ntc) {
          b1 = Z1[(long long)(t0 + 2 * u + 1) * g.Ns + j];
          b2 = Z2[(long long)(t0 + 2 * u + 1) * g.Ns + j];
        }
        z1h[u * span + c] = make_float2(a1.x, b1.x);
        z1l[u * span + c] = make_float2(a1.y, b1.y);
        z2h[u * span + c] = make_float2(a2.x, b2.x);
        z2l[u * span + c] = make_float2(a2.y, b2.y);
      }
    }
    __syncthreads();
    const long long ob = (long long)W * o23 * g.Ns;
#pragma unroll
    for (int o1 = 0; o1 < (PP > 0 ? 2 * PP + 1 : W); ++o1) {
      if (PP == 0 && o1 >= W) break;
      const float2 m = mrow[ob + (long long)o1 * g.Ns], kk = krow[ob + (long long)o1 * g.Ns];
      const float2 mh = make_float2(m.x, m.x), ml = make_float2(m.y, m.y);
      const float2 kh = make_float2(kk.x, kk.x), kl = make_float2(kk.y, kk.y);
      const int c = threadIdx.x + o1;
#pragma unroll
      for (int u = 0; u < kTP; ++u) {
        fma_acc2(acc[u], mh, ml, z1h[u * span + c], z1l[u * span + c]);
        fma_acc2(acc[u], kh, kl, z2h[u * span + c], z2l[u * span + c]);
      }
    }
  }
  if (valid) {
#pragma unroll
    for (int u = 0; u < kTP; ++u) {   // static indices keep acc[] in registers
      if (2 * u < ntc)
        y[(long long)(t0 + 2 * u) * g.Ns + i] = dfa::to_double(dfa::norm(df{acc[u].h.x, acc[u].l.x}));
      if (2 * u + 1 < ntc)
        y[(long long)(t0 + 2 * u + 1) * g.Ns + i] = dfa::to_double(dfa::norm(df{acc[u].h.y, acc[u].l.y}));
    }
  }
}

// Pass 1: Z1[t] = gamma sum_tau W[t, tau] x[tau], Z2[t] = nu sum_tau Mt[t, tau] x[tau]
// with band-compressed rows Wb[t][k] = W[t][t - pt + k] (already scaled).
template <typename T>
__global__ void k_time_pair(const double* __restrict__ x, const T* __restrict__ Wb, const T* __restrict__ Mb,
                            T* __restrict__ Z1, T* __restrict__ Z2, long long Ns, int nt, int pt) {
  const int B = 2 * pt + 1;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += (long long)gridDim.x * blockDim.x) {
    for (int t = 0; t < nt; ++t) {
      typename Num<T>::acc a1 = Num<T>::zero(), a2 = Num<T>::zero();
      for (int k = 0; k < B; ++k) {
        const int tau = t - pt + k;
        if (tau < 0 || tau >= nt) continue;
        const double xv = x[(long long)tau * Ns + i];
        if constexpr (std::is_same<T, double>::value) {
          a1 = fma((double)Wb[t * B + k], xv, a1);
          a2 = fma((double)Mb[t * B + k], xv, a2);
        } else {
          const df xd = dfa::from_double(xv);
          dfa::fma_acc(a1, Wb[t * B + k], xd);
          dfa::fma_acc(a2, Mb[t * B + k], xd);
        }
      }
      if constexpr (std::is_same<T, double>::value) {
        Z1[(long long)t * Ns + i] = a1;
        Z2[(long long)t * Ns + i] = a2;
      } else {
        const df n1 = dfa::norm(a1), n2 = dfa::norm(a2);
        Z1[(long long)t * Ns + i] = make_float2(n1.h, n1.l);
        Z2[(long long)t * Ns + i] = make_float2(n2.h, n2.l);
      }
    }
  }
}

int sm_count() { return sm_count_current(); }

template <typename T, int kTC, int PP>
cudaError_t run_stencil(const StencilOpDev& op, T* Z1, T* Z2, double* y, const StencilDims& g, cudaStream_t st) {
  const size_t smem = (size_t)2 * kTC * (kRows + 2 * op.p) * sizeof(T);
  {
    const cudaError_t e = ensure_smem_attr(k_stencil<T, kTC, PP>, 96 * 1024);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = ((g.Ns + kRows - 1) / kRows) * ((g.nt + kTC - 1) / kTC);
  if constexpr (std::is_same<T, float2>::value) {   // double-float: slices paired on the FP32 pipes
    {
      const cudaError_t e = ensure_smem_attr(k_stencil_pk<kTC, PP>, 96 * 1024);
      if (e != cudaSuccess) return e;
    }
    k_stencil_pk<kTC, PP><<<(unsigned)blocks, kRows, smem, st>>>(static_cast<const float2*>(op.Ms),
                                                                  static_cast<const float2*>(op.Ks), Z1, Z2, y, g);
    return cudaGetLastError();
  }
  k_stencil<T, kTC, PP><<<(unsigned)blocks, kRows, smem, st>>>(static_cast<const T*>(op.Ms),
                                                                static_cast<const T*>(op.Ks), Z1, Z2, y, g);
  return cudaGetLastError();
}

template <typename T>
cudaError_t stencil_matvec(const StencilOpDev& op, const double* x, double* y, int trans, cudaStream_t st) {
  const T* Wb = static_cast<const T*>(trans ? op.WbT : op.Wb);
  const T* Mb = static_cast<const T*>(op.Mtb);
  T* Z1 = static_cast<T*>(op.Z1);
  T* Z2 = static_cast<T*>(op.Z2);
  const long long Ns = op.Ns;
  const int nt = op.nt;
  {
    ProfScope ps("stencil_time", 4.0 * (2 * op.pt + 1) * (double)Ns * nt, 24.0 * (double)Ns * nt, st);
    const long long want = (Ns + 255) / 256;
    const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sm_count() * 16));
    k_time_pair<T><<<grid, 256, 0, st>>>(x, Wb, Mb, Z1, Z2, Ns, nt, op.pt);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  StencilDims g;
  g.d = op.d;
  g.p = op.p;
  g.n1 = op.n[0];
  g.n2 = op.d >= 2 ? op.n[1] : 1;
  g.Ns = Ns;
  g.nt = nt;
  if constexpr (std::is_same<T, double>::value) {
    if (op.fx) return launch_stencil_space_fx(op, Z1, Z2, y, g, st);
  }
  int S = 1;
  for (int l = 0; l < op.d; ++l) S *= 2 * op.p + 1;
  ProfScope ps("stencil_space", 4.0 * S * (double)Ns * nt,
               (2.0 * S * sizeof(T)) * (double)Ns + 2.0 * sizeof(T) * (double)Ns * nt + 8.0 * (double)Ns * nt, st);
  switch (op.p) {
    case 1: return run_stencil<T, 8, 1>(op, Z1, Z2, y, g, st);
    case 2: return run_stencil<T, 8, 2>(op, Z1, Z2, y, g, st);
    case 3: return run_stencil<T, 8, 3>(op, Z1, Z2, y, g, st);
    case 4: return run_stencil<T, 8, 4>(op, Z1, Z2, y, g, st);
    default: return run_stencil<T, 8, 0>(op, Z1, Z2, y, g, st);
  }
}

// g[e] = -nu sum_t lam_t^T K_e ubar_t over the element's reduced rows, with
// ubar = (M_t (x) I) u. One CTA per element, threads over time slices.
__global__ void k_grad_elements(const double* __restrict__ Ke, const double* __restrict__ lam,
                                const double* __restrict__ ubar, double* __restrict__ g, int d, int p, int n_el,
                                int n_s, long long Ns, int nt, double nu) {
  extern __shared__ double sh[];
  const int L = p + 1;
  int Ld = 1;
  for (int l = 0; l < d; ++l) Ld *= L;
  double* K = sh;                                   // Ld * Ld
  long long* rows = reinterpret_cast<long long*>(sh + (size_t)Ld * Ld);   // Ld (-1 = removed)
  double* red = reinterpret_cast<double*>(rows + Ld);                     // blockDim.x / 32
  const long long e = blockIdx.x;
  const double* Kg = Ke + (size_t)e * Ld * Ld;
  for (int k = threadIdx.x; k < Ld * Ld; k += blockDim.x) K[k] = Kg[k];
  for (int a = threadIdx.x; a < Ld; a += blockDim.x) {
    long long r = e, row = 0, stride = 1;
    int ra = a;
    bool ok = true;
    for (int l = 0; l < d; ++l) {
      const int il = (int)(r % n_el) + ra % L - 1;
      r /= n_el;
      ra /= L;
      if (il < 0 || il >= n_s) ok = false;
      row += (long long)il * stride;
      stride *= n_s;
    }
    rows[a] = ok ? row : -1;
  }
  __syncthreads();
  double part = 0.0;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const double* lt = lam + (long long)t * Ns;
    const double* ut = ubar + (long long)t * Ns;
    for (int a = 0; a < Ld; ++a) {
      if (rows[a] < 0) continue;
      double s = 0.0;
      for (int b = 0; b < Ld; ++b)
        if (rows[b] >= 0) s = fma(K[a * Ld + b], ut[rows[b]], s);
      part = fma(lt[rows[a]], s, part);
    }
  }
  for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    g[e] = -nu * s;
  }
}

__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ s, double* __restrict__ y,
                        long long N) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x)
    y[k] = x[k] * s[k];
}

}  // namespace

cudaError_t launch_stencil_matvec(const StencilOpDev& op, const double* x, double* y, int trans, cudaStream_t st) {
  if (op.Ns <= 0 || op.nt <= 0) return cudaSuccess;
  if (op.df) return stencil_matvec<float2>(op, x, y, trans, st);
  return stencil_matvec<double>(op, x, y, trans, st);
}

size_t grad_elements_smem(int d, int p) {
  int Ld = 1;
  for (int l = 0; l < d; ++l) Ld *= p + 1;
  return (size_t)Ld * Ld * sizeof(double) + (size_t)Ld * sizeof(long long) + 8 * sizeof(double);
}

cudaError_t launch_grad_elements(const double* Ke, const double* lam, const double* ubar, double* g, int d, int p,
                                 int n_el, int n_s, long long Ns, int nt, double nu, cudaStream_t st) {
  long long n_elem = 1;
  for (int l = 0; l < d; ++l) n_elem *= n_el;
  if (n_elem <= 0) return cudaSuccess;
  const size_t smem = grad_elements_smem(d, p);
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_grad_elements, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  ProfScope ps("grad_elements", 2.0 * n_elem * (double)nt * (double)smem / 8.0, 16.0 * (double)Ns * nt, st);
  k_grad_elements<<<(unsigned)n_elem, 256, smem, st>>>(Ke, lam, ubar, g, d, p, n_el, n_s, Ns, nt, nu);
  return cudaGetLastError();
}

cudaError_t launch_scale(const double* x, const double* s, double* y, long long N, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  ProfScope ps("diag_scale", (double)N, 24.0 * (double)N, st);
  const long long want = (N + 255) / 256;
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sm_count() * 16));
  k_scale<<<grid, 256, 0, st>>>(x, s, y, N);
  return cudaGetLastError();
}

cudaError_t launch_time_mass_fp64(const double* x, const double* Mb, double* y, double* scratch, long long Ns, int nt,
                                  int pt, cudaStream_t st) {
  if (Ns <= 0) return cudaSuccess;
  ProfScope ps("time_mass", 2.0 * (2 * pt + 1) * (double)Ns * nt, 16.0 * (double)Ns * nt, st);
  const long long want = (Ns + 255) / 256;
  const int grid = (int)std::max<long long>(1, std::min<long long>(want, (long long)sm_count() * 16));
  k_time_pair<double><<<grid, 256, 0, st>>>(x, Mb, Mb, y, scratch, Ns, nt, pt);
  return cudaGetLastError();
}

}  // namespace stfd
