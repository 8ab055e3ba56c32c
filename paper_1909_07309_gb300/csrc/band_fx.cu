// Banded mode products of the system matvec (eq. syst_mat through eq.
// kron_vec_multi) with FP64 results, in exact 64-bit integer arithmetic on the
// integer pipes (GB300 issues FP64 at about 1/64 of its integer rate).
//
// Every fibre of an input tensor (the n entries one band product reads) is
// written under one power of two as 53-bit integers: with E the largest biased
// exponent of the fibre, an entry of biased exponent e and significand m
// becomes U = round(m 2^{e - E}) -- exact for the entries of the largest binade
// and rounded at 2^-53 of the fibre's largest entry for the others. Every row of
// a band matrix is written the same way (C, exponent E_c). Each product sum
// S = sum_t C_t U_t (2p + 1 taps) is formed exactly from 27-bit limbs,
// U = U_h 2^27 + U_l and C = C_h 2^27 + C_l with 0 <= U_l, C_l < 2^27, in three
// 64-bit sums (3 IMAD.WIDE per tap, Karatsuba) and rounded once, to nearest
// even, to FP64: S 2^{E + E_c - 2150}. An output that sums two products of
// different inputs (K u + M v; gamma W u + nu M_t v) adds the two exact sums
// in 128-bit integers and rounds once when their scales are within 2^16 of
// each other in every lane of the warp (the usual case); otherwise it adds the
// two rounded products with one FP64 addition, within one unit in the last
// place of the exact sum.
//
// The pass structure is that of the double-float passes (band_df.cu): a CTA
// owns 32 fibres; with rot = 1 the fibres are contiguous (the direction is the
// fastest index) and entry i of fibre q is written to i Q + q, so that each
// pass leaves the next direction fastest; intermediates are FP64.
//   KIND 0 (first direction):  (Uo, Vo) = (x x M, x x K)
//   KIND 1 (middle directions): (Uo, Vo) = (u x M, u x K + v x M)
//   KIND 2 (time):              Vo = u x (gamma W) + v x (nu M_t)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_state.h"
#include "fp64_round.cuh"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {
namespace {

constexpr int kTC = 32;          // fibres per CTA (one per lane)
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLd = kTC + 1;     // tile row stride in int2 (conflict-free transposed stores)

__device__ __forceinline__ int bexp_d(unsigned long long u) { return max(1, (int)((u >> 52) & 0x7FF)); }

// A fibre whose largest biased exponent is 2047 holds an infinity or NaN: the
// outputs it feeds are NaN (the flag is read from shared memory at the store,
// so that no register stays live across the row loop).
__device__ __forceinline__ bool nonfinite(int E) { return E >= 2047; }
#define kQNaN __longlong_as_double(0x7FF8000000000000ll)

// Entry (bit pattern u) of a fibre with largest biased exponent E as the limbs
// (U_h, U_l) of U = round(m 2^{e - E}), U = U_h 2^27 + U_l, 0 <= U_l < 2^27.
__device__ __forceinline__ int2 to_limbs(unsigned long long u, int E) {
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(e != 0) << 52);
  const int s = min(E - max(e, 1), 63);
  const unsigned long long mag = (m + ((1ull << s) >> 1)) >> s;
  const long long U = (u >> 63) ? -(long long)mag : (long long)mag;
  return make_int2((int)(U >> 27), (int)(U & ((1ll << 27) - 1)));
}

// acc += C U for 27-bit limbs (one tap), three 64-bit products (Karatsuba):
// hh += C_h U_h, ll += C_l U_l, mm += (C_h + C_l)(U_h + U_l); the cross term
// C_h U_l + C_l U_h = mm - hh - ll is recovered once per output. All sums are
// exact: |C_h + C_l|, |U_h + U_l| < 2^28, at most 2p + 1 <= 9 taps. The
// accumulator and its rounding to FP64 (to_s128, round_s128) are in
// fp64_round.cuh.
__device__ __forceinline__ void tap(Acc& a, int2 c, int2 u) {
  a.hh += (long long)c.x * u.x;
  a.ll += (long long)c.y * u.y;
  a.mm += (long long)(c.x + c.y) * (u.x + u.y);
}

// Two products of different inputs, x 2^{SX - 2150} + y 2^{SY - 2150}: summed
// exactly and rounded once when their scales are within 2^16 of each other
// in every lane of the warp (the usual case: the inputs' and the rows'
// exponents offset each other); otherwise each is rounded and the two are
// added in FP64. The choice is made per warp so that no warp runs both paths.
__device__ __forceinline__ double round_sum(const Acc& x, int SX, const Acc& y, int SY) {
  const int g = SX - SY;
  if (__all_sync(0xFFFFFFFFu, g >= -16 && g <= 16)) return round_pair_exact(x, SX, y, SY);
  return round_acc(x, SX) + round_acc(y, SY);
}

// Coefficient tables (host-built, see fx_tables): per row i, two sets of W =
// 2p + 1 taps as int2 limbs (0 outside the matrix) -- KIND 0, 1: (M, K);
// KIND 2: (gamma W or gamma W^T, nu M_t) -- and the two row exponents.
template <int KIND, int P>
__global__ void __launch_bounds__(kThreads)
k_band_fx(const double* __restrict__ U, const double* __restrict__ V, const int2* __restrict__ C,
          const int* __restrict__ Ce, double* __restrict__ Uo, double* __restrict__ Vo, int n, long long inner,
          long long Q, int rot) {
  constexpr int W = 2 * P + 1;
  constexpr bool HAS_V = KIND != 0;
  extern __shared__ int2 smx[];
  int2* tu = smx;                                            // [(n + 2P) rows][kLd]
  int2* tv = smx + (size_t)(n + 2 * P) * kLd;
  __shared__ int sEu[kTC], sEv[kTC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long q = (long long)blockIdx.x * kTC + lane;
  const bool valid = q < Q;
  long long base = 0;
  if (valid) {
    const long long o = q / inner;
    base = o * (long long)n * inner + (q - o * inner);
  }
  unsigned long long* ru = reinterpret_cast<unsigned long long*>(tu);
  unsigned long long* rv = reinterpret_cast<unsigned long long*>(tv);
  if (threadIdx.x < kTC) {
    sEu[threadIdx.x] = 1;
    sEv[threadIdx.x] = 1;
  }
  // zero the P halo rows above and below (their coefficients are 0; entries must be finite)
  for (int e = threadIdx.x; e < 2 * P * kLd; e += kThreads) {
    const int r = e / kLd, c = e - r * kLd;
    const int row = r < P ? r : n + r;
    ru[(size_t)row * kLd + c] = 0ull;
    if (HAS_V) rv[(size_t)row * kLd + c] = 0ull;
  }
  tc::grid_dependency_wait();   // programmatic dependent launch: inputs from here on
  // ---- raw FP64 words into the tile (row a + P, column = fibre)
  if (rot || inner == 1) {
    const long long q0 = (long long)blockIdx.x * kTC;
    const int nf = (int)min((long long)kTC, Q - q0);
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(U) + q0 * n;
    const unsigned long long* srcv = HAS_V ? reinterpret_cast<const unsigned long long*>(V) + q0 * n : nullptr;
    const int df_step = kThreads / n, da_step = kThreads - df_step * n;
    int f = threadIdx.x / n, a = threadIdx.x - f * n;
    for (int e = threadIdx.x; e < kTC * n; e += kThreads) {
      ru[(size_t)(a + P) * kLd + f] = f < nf ? __ldg(src + e) : 0ull;
      if (HAS_V) rv[(size_t)(a + P) * kLd + f] = f < nf ? __ldg(srcv + e) : 0ull;
      f += df_step;
      a += da_step;
      if (a >= n) {
        a -= n;
        ++f;
      }
    }
  } else {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(U);
    const unsigned long long* srcv = reinterpret_cast<const unsigned long long*>(V);
    for (int a = warp; a < n; a += kWarps) {
      ru[(size_t)(a + P) * kLd + lane] = valid ? __ldg(src + base + (long long)a * inner) : 0ull;
      if (HAS_V) rv[(size_t)(a + P) * kLd + lane] = valid ? __ldg(srcv + base + (long long)a * inner) : 0ull;
    }
  }
  __syncthreads();
  // ---- largest biased exponent per fibre and input
  {
    int Eu = 1, Ev = 1;
    for (int a = warp; a < n; a += kWarps) {
      Eu = max(Eu, bexp_d(ru[(size_t)(a + P) * kLd + lane]));
      if (HAS_V) Ev = max(Ev, bexp_d(rv[(size_t)(a + P) * kLd + lane]));
    }
    atomicMax(&sEu[lane], Eu);
    if (HAS_V) atomicMax(&sEv[lane], Ev);
  }
  __syncthreads();
  const int Eu = sEu[lane], Ev = sEv[lane];
  // ---- entries to limbs, in place
  for (int a = warp; a < n; a += kWarps) {
    const size_t o = (size_t)(a + P) * kLd + lane;
    tu[o] = to_limbs(ru[o], Eu);
    if (HAS_V) tv[o] = to_limbs(rv[o], Ev);
  }
  __syncthreads();
  tc::grid_launch_dependents();
  for (int i = warp; i < n; i += kWarps) {
    const int2* cr = C + (size_t)i * 2 * W;
    Acc a1{0, 0, 0}, a2{0, 0, 0}, a3{0, 0, 0};
#pragma unroll
    for (int t = 0; t < W; ++t) {
      const int2 u = tu[(size_t)(i + t) * kLd + lane];
      const int2 c0 = __ldg(cr + t), c1 = __ldg(cr + W + t);
      if (KIND == 0) {
        tap(a1, c0, u);   // M x
        tap(a2, c1, u);   // K x
      } else if (KIND == 1) {
        const int2 v = tv[(size_t)(i + t) * kLd + lane];
        tap(a1, c0, u);   // M u
        tap(a2, c1, u);   // K u
        tap(a3, c0, v);   // M v
      } else {
        const int2 v = tv[(size_t)(i + t) * kLd + lane];
        tap(a2, c0, u);   // gamma W u
        tap(a3, c1, v);   // nu M_t v
      }
    }
    // every lane rounds (fibres past the end hold zeros; the warp votes in round_sum)
    const long long off = rot ? q + (long long)i * Q : base + (long long)i * inner;
    const int e0 = __ldg(Ce + 2 * i), e1 = __ldg(Ce + 2 * i + 1);
    if (KIND == 0) {
      const double uo = round_acc(a1, Eu + e0), vo = round_acc(a2, Eu + e1);
      if (valid) {
        Uo[off] = nonfinite(sEu[lane]) ? kQNaN : uo;
        Vo[off] = nonfinite(sEu[lane]) ? kQNaN : vo;
      }
    } else if (KIND == 1) {
      const double uo = round_acc(a1, Eu + e0), vo = round_sum(a2, Eu + e1, a3, Ev + e0);
      if (valid) {
        Uo[off] = nonfinite(sEu[lane]) ? kQNaN : uo;
        Vo[off] = nonfinite(max(sEu[lane], sEv[lane])) ? kQNaN : vo;
      }
    } else {
      const double vo = round_sum(a2, Eu + e0, a3, Ev + e1);
      if (valid) Vo[off] = nonfinite(max(sEu[lane], sEv[lane])) ? kQNaN : vo;
    }
  }
}

template <int KIND, int P>
cudaError_t launch_fx_p(const double* U, const double* V, const int2* C, const int* Ce, double* Uo, double* Vo, int n,
                        long long inner, long long outer, int rot, cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  const size_t smem = (size_t)(KIND == 0 ? 1 : 2) * (n + 2 * P) * kLd * sizeof(int2);
  {
    const cudaError_t e = ensure_smem_attr(k_band_fx<KIND, P>, 2 * (256 + 8) * kLd * (int)sizeof(int2));
    if (e != cudaSuccess) return e;
  }
  const int nprod = KIND == 1 ? 3 : 2;
  const int nio = KIND == 0 ? 3 : KIND == 1 ? 4 : 3;
  double entries = 0.0;
  for (int i = 0; i < n; ++i) entries += (double)(std::min(n - 1, i + P) - std::max(0, i - P) + 1);
  ProfScope ps("band_fx64", 2.0 * entries * (double)Q * nprod, 8.0 * (double)Q * n * nio, st);
  return tc::launch_pdl(k_band_fx<KIND, P>, dim3((unsigned)((Q + kTC - 1) / kTC)), dim3(kThreads), smem, st, U, V, C,
                        Ce, Uo, Vo, n, inner, Q, rot);
}

template <int KIND>
cudaError_t launch_fx_k(const double* U, const double* V, const int2* C, const int* Ce, double* Uo, double* Vo, int n,
                        long long inner, long long outer, int p, int rot, cudaStream_t st) {
  switch (p) {
    case 1: return launch_fx_p<KIND, 1>(U, V, C, Ce, Uo, Vo, n, inner, outer, rot, st);
    case 2: return launch_fx_p<KIND, 2>(U, V, C, Ce, Uo, Vo, n, inner, outer, rot, st);
    case 3: return launch_fx_p<KIND, 3>(U, V, C, Ce, Uo, Vo, n, inner, outer, rot, st);
    case 4: return launch_fx_p<KIND, 4>(U, V, C, Ce, Uo, Vo, n, inner, outer, rot, st);
    default: return cudaErrorInvalidValue;
  }
}

// 53-bit integer of x under the exponent E >= max(1, biased exponent of x), as limbs.
int2 host_limbs(double x, int E) {
  unsigned long long u;
  std::memcpy(&u, &x, 8);
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(e != 0) << 52);
  const int s = std::min(E - std::max(e, 1), 63);
  const unsigned long long mag = (m + ((1ull << s) >> 1)) >> s;
  const long long U = (u >> 63) ? -(long long)mag : (long long)mag;
  return make_int2((int)(U >> 27), (int)(U & ((1ll << 27) - 1)));
}

int host_bexp(double x) {
  unsigned long long u;
  std::memcpy(&u, &x, 8);
  return std::max(1, (int)((u >> 52) & 0x7FF));
}

}  // namespace

cudaError_t launch_band_first_fx(const double* x, const int2* C, const int* Ce, double* Uo, double* Vo, int n,
                                 long long inner, long long outer, int p, int rot, cudaStream_t st) {
  return launch_fx_k<0>(x, nullptr, C, Ce, Uo, Vo, n, inner, outer, p, rot, st);
}
cudaError_t launch_band_mid_fx(const double* u, const double* v, const int2* C, const int* Ce, double* Uo, double* Vo,
                               int n, long long inner, long long outer, int p, int rot, cudaStream_t st) {
  return launch_fx_k<1>(u, v, C, Ce, Uo, Vo, n, inner, outer, p, rot, st);
}
cudaError_t launch_band_last_fx(const double* u, const double* v, const int2* C, const int* Ce, double* y, int n,
                                long long inner, long long outer, int p, int rot, cudaStream_t st) {
  return launch_fx_k<2>(u, v, C, Ce, nullptr, y, n, inner, outer, p, rot, st);
}

// Host: coefficient table of one pass from two row-major n x n band matrices
// A, B (first and middle passes: M, K; time pass: gamma W or gamma W^T, nu M_t):
// C[i][s][t] = limbs of row i of matrix s at column i - p + t (0 outside),
// Ce[i][s] = largest biased exponent of that row's band.
void fx_tables(const double* A, const double* B, int n, int p, std::vector<int2>& C, std::vector<int>& Ce) {
  const int W = 2 * p + 1;
  const double* mats[2] = {A, B};
  C.assign((size_t)n * 2 * W, make_int2(0, 0));
  Ce.assign((size_t)n * 2, 1);
  for (int i = 0; i < n; ++i)
    for (int s = 0; s < 2; ++s) {
      int E = 1;
      for (int t = 0; t < W; ++t) {
        const int a = i - p + t;
        if (a >= 0 && a < n) E = std::max(E, host_bexp(mats[s][(size_t)i * n + a]));
      }
      Ce[(size_t)i * 2 + s] = E;
      for (int t = 0; t < W; ++t) {
        const int a = i - p + t;
        if (a >= 0 && a < n) C[((size_t)i * 2 + s) * W + t] = host_limbs(mats[s][(size_t)i * n + a], E);
      }
    }
}

}  // namespace stfd
