// Spatial pass of the mapped-domain system matvec (Sec. 4.6.1),
//     y_t = M_s Z1_t + K_s Z2_t   for every time slice t,
// with FP64 results no narrower than IEEE FP64, in exact 64-bit integer
// arithmetic on the integer pipes (GB300 issues FP64 at about 1/64 of its
// integer multiply-add rate).
//
// Every stencil row i of M_s (and of K_s) is written under its own power of
// two as 53-bit integers C (exponent frame E_m(i), E_k(i): the largest biased
// exponent of the row's (2p+1)^d coefficients), once, when the operator is
// created. A CTA owns R rows and TC time slices; for each slice it writes the
// entries of Z1_t and Z2_t that its rows read (its stencil neighbourhood, one
// segment of R + 2p columns per pair of outer offsets, copied asynchronously
// while the previous segment is multiplied)
// under one power of two per slice (the neighbourhood's largest biased
// exponent), exact in the top binade and rounded at 2^-53 of the
// neighbourhood's largest entry below it. Both are split into balanced 27-bit
// limbs, C = C_h 2^27 + C_l with C_l in [-2^26, 2^26) and |C_h| <= 2^26, and
// every row sum S = sum_o C_o U_o over the (2p+1)^d <= 729 offsets is formed
// exactly in three 64-bit sums (3 multiply-adds per tap, Karatsuba):
//     hh = sum C_h U_h,  ll = sum C_l U_l  (each below 729 2^52 < 2^62),
//     mm = sum (C_h + C_l)(U_h + U_l) modulo 2^64,
// whose cross term mm - hh - ll = sum (C_h U_l + C_l U_h) is below 729 2^53 <
// 2^63 in magnitude, so the wrapped sum recovers it exactly. The two products
// of an output (mass and stiffness parts, different frames) are summed
// exactly in 128-bit integers and rounded once to FP64 when their frames are
// within 2^10 of each other in every lane of the warp (|S| < 2^116, so the
// shifted sum stays below 2^127), otherwise each is rounded and the two are
// added in FP64. A non-finite entry in a row's coefficients or in a slice's
// neighbourhood gives NaN for the outputs it reaches. The limb split, the
// three-word sums and the rounding are in fp64_round.cuh.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_state.h"
#include "fp64_round.cuh"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {
namespace {

constexpr int kRows = 256;          // rows per CTA (threads)
constexpr int kMaxTaps = 729;       // the exactness bound of the three sums
constexpr int kPairGap = 10;        // largest frame gap summed exactly

__device__ __forceinline__ int bexp_u(unsigned long long u) { return max(1, (int)((u >> 52) & 0x7FF)); }

// One row of the coefficient table: the frame and, in place of the FP64
// values, their balanced limbs (same 8 bytes). Thread per row.
__global__ void k_stencil_fx_table(double* __restrict__ C, int* __restrict__ E, int S, long long Ns) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ns) return;
  unsigned long long* w = reinterpret_cast<unsigned long long*>(C);
  int Ei = 1;
  for (int o = 0; o < S; ++o) Ei = max(Ei, bexp_u(w[(long long)o * Ns + i]));
  E[i] = Ei;
  int2* c = reinterpret_cast<int2*>(C);
  for (int o = 0; o < S; ++o) {
    const long long k = (long long)o * Ns + i;
    c[k] = balanced_limbs(w[k], Ei);
  }
}

// Time slices per CTA and CTAs per SM: two slices at four CTAs (64 registers)
// ran fastest on GB300 among 1, 2 or 4 slices at 2 to 8 CTAs (113.8 ms against
// 115.8 for one slice at eight CTAs and 142.9 for four slices at three, at
// 93M dofs, p = 4, d = 3).
constexpr int kSlices = 2;
constexpr int kCtasPerSm = 4;

template <int kTC, int PP>
__global__ void __launch_bounds__(kRows, kCtasPerSm)
k_stencil_fx(const int2* __restrict__ Ms, const int2* __restrict__ Ks, const int* __restrict__ Em,
             const int* __restrict__ Ek, const double* __restrict__ Z1, const double* __restrict__ Z2,
             double* __restrict__ y, StencilDims g) {
  extern __shared__ unsigned char smem_raw[];
  const int p = PP > 0 ? PP : g.p;
  const int W = 2 * p + 1, span = kRows + 2 * p;
  // raw FP64 words of the next segment (asynchronous copies), then the limbs of
  // two segments (double-buffered: one is converted while the other is read)
  unsigned long long* r1s = reinterpret_cast<unsigned long long*>(smem_raw);   // [kTC][span]
  unsigned long long* r2s = r1s + kTC * span;
  int2* lbuf = reinterpret_cast<int2*>(r2s + kTC * span);                      // [2][2][kTC][span]
  __shared__ int sE[2 * kTC];                         // neighbourhood frames of Z1_t, Z2_t
  const int n_chunks = (g.nt + kTC - 1) / kTC;
  const long long i0 = (long long)(blockIdx.x / n_chunks) * kRows;
  const int t0 = (int)(blockIdx.x % n_chunks) * kTC;
  const long long i = i0 + threadIdx.x;
  const bool valid = i < g.Ns;
  const int ntc = min(kTC, g.nt - t0);
  const int S23 = g.d >= 3 ? W * W : (g.d == 2 ? W : 1);
  const unsigned long long* w1 = reinterpret_cast<const unsigned long long*>(Z1);
  const unsigned long long* w2 = reinterpret_cast<const unsigned long long*>(Z2);
  if (threadIdx.x < 2 * kTC) sE[threadIdx.x] = 1;
  __syncthreads();
  // ---- frames: the largest biased exponent of each slice over the neighbourhood
  {
    int e1[kTC], e2[kTC];
#pragma unroll
    for (int tt = 0; tt < kTC; ++tt) e1[tt] = e2[tt] = 1;
    for (int o23 = 0; o23 < S23; ++o23) {
      const int o2 = g.d >= 2 ? o23 % W : p, o3 = g.d >= 3 ? o23 / W : p;
      const long long base = i0 - p + (long long)(o2 - p) * g.n1 + (long long)(o3 - p) * g.n1 * g.n2;
      for (int c = threadIdx.x; c < span; c += kRows) {
        long long j = base + c;
        j = j < 0 ? 0 : (j >= g.Ns ? g.Ns - 1 : j);
#pragma unroll
        for (int tt = 0; tt < kTC; ++tt)
          if (tt < ntc) {
            e1[tt] = max(e1[tt], bexp_u(__ldg(w1 + (long long)(t0 + tt) * g.Ns + j)));
            e2[tt] = max(e2[tt], bexp_u(__ldg(w2 + (long long)(t0 + tt) * g.Ns + j)));
          }
      }
    }
#pragma unroll
    for (int tt = 0; tt < kTC; ++tt) {
      int a = e1[tt], b = e2[tt];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        a = max(a, __shfl_xor_sync(0xFFFFFFFFu, a, s));
        b = max(b, __shfl_xor_sync(0xFFFFFFFFu, b, s));
      }
      if ((threadIdx.x & 31) == 0) {
        atomicMax(&sE[tt], a);
        atomicMax(&sE[kTC + tt], b);
      }
    }
  }
  __syncthreads();
  int E1[kTC], E2[kTC];
#pragma unroll
  for (int tt = 0; tt < kTC; ++tt) {
    E1[tt] = sE[tt];
    E2[tt] = sE[kTC + tt];
  }
  const int2* mrow = Ms + (valid ? i : 0);
  const int2* krow = Ks + (valid ? i : 0);
  AccW am[kTC], ak[kTC];
#pragma unroll
  for (int tt = 0; tt < kTC; ++tt) am[tt] = ak[tt] = AccW{0, 0, 0ull};
  // segment o23: columns base .. base + span - 1 of the slices (clamped: the
  // coefficient is 0 for columns outside the box)
  auto seg_base = [&](int o23) -> long long {
    const int o2 = g.d >= 2 ? o23 % W : p, o3 = g.d >= 3 ? o23 / W : p;
    return i0 - p + (long long)(o2 - p) * g.n1 + (long long)(o3 - p) * g.n1 * g.n2;
  };
  auto issue = [&](int o23) {
    const long long base = seg_base(o23);
    for (int c = threadIdx.x; c < span; c += kRows) {
      long long j = base + c;
      j = j < 0 ? 0 : (j >= g.Ns ? g.Ns - 1 : j);
#pragma unroll
      for (int tt = 0; tt < kTC; ++tt)
        if (tt < ntc) {
          tc::cp_async8(r1s + tt * span + c, w1 + (long long)(t0 + tt) * g.Ns + j);
          tc::cp_async8(r2s + tt * span + c, w2 + (long long)(t0 + tt) * g.Ns + j);
        }
    }
    tc::cp_async_commit();
  };
  auto convert = [&](int buf) {
    int2* l1 = lbuf + (size_t)buf * 2 * kTC * span;
    int2* l2 = l1 + kTC * span;
    for (int c = threadIdx.x; c < span; c += kRows) {
#pragma unroll
      for (int tt = 0; tt < kTC; ++tt) {
        const bool on = tt < ntc;
        l1[tt * span + c] = on ? balanced_limbs(r1s[tt * span + c], E1[tt]) : make_int2(0, 0);
        l2[tt * span + c] = on ? balanced_limbs(r2s[tt * span + c], E2[tt]) : make_int2(0, 0);
      }
    }
  };
  issue(0);
  tc::cp_async_wait_all();
  __syncthreads();
  convert(0);
  for (int o23 = 0; o23 < S23; ++o23) {
    __syncthreads();   // limbs of segment o23 complete; the raw buffer is free
    if (o23 + 1 < S23) issue(o23 + 1);
    const int2* z1s = lbuf + (size_t)(o23 & 1) * 2 * kTC * span;
    const int2* z2s = z1s + kTC * span;
    const long long ob = (long long)W * o23 * g.Ns;
#pragma unroll
    for (int o1 = 0; o1 < (PP > 0 ? 2 * PP + 1 : W); ++o1) {
      if (PP == 0 && o1 >= W) break;
      const int2 m = __ldg(mrow + ob + (long long)o1 * g.Ns), kk = __ldg(krow + ob + (long long)o1 * g.Ns);
      const int ms = m.x + m.y, ks = kk.x + kk.y;
#pragma unroll
      for (int tt = 0; tt < kTC; ++tt) {
        tapw(am[tt], m, ms, z1s[tt * span + threadIdx.x + o1]);
        tapw(ak[tt], kk, ks, z2s[tt * span + threadIdx.x + o1]);
      }
    }
    if (o23 + 1 < S23) {   // the next segment's words have arrived: its limbs
      tc::cp_async_wait_all();
      __syncthreads();
      convert((o23 + 1) & 1);
    }
  }
  // ---- one rounding per output (every lane rounds: the warp votes on the exact pair sum)
  const int em = valid ? __ldg(Em + i) : 1, ek = valid ? __ldg(Ek + i) : 1;
#pragma unroll
  for (int tt = 0; tt < kTC; ++tt) {
    const int SX = em + E1[tt], SY = ek + E2[tt], gap = SX - SY;
    double out;
    if (__all_sync(0xFFFFFFFFu, !valid || (gap >= -kPairGap && gap <= kPairGap)))
      out = round_pair_exact(as_acc(am[tt]), SX, as_acc(ak[tt]), SY);
    else
      out = round_acc(as_acc(am[tt]), SX) + round_acc(as_acc(ak[tt]), SY);
    if (em >= 2047 || ek >= 2047 || E1[tt] >= 2047 || E2[tt] >= 2047) out = __longlong_as_double(0x7FF8000000000000ll);
    if (valid && tt < ntc) y[(long long)(t0 + tt) * g.Ns + i] = out;
  }
}

template <int kTC, int PP>
cudaError_t run_fx(const int2* Ms, const int2* Ks, const int* Em, const int* Ek, const double* Z1, const double* Z2,
                   double* y, const StencilDims& g, cudaStream_t st) {
  const size_t smem = (size_t)6 * kTC * (kRows + 2 * g.p) * sizeof(int2);   // raw words + two limb tiles
  {
    const cudaError_t e = ensure_smem_attr(k_stencil_fx<kTC, PP>, 96 * 1024);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = ((g.Ns + kRows - 1) / kRows) * ((g.nt + kTC - 1) / kTC);
  k_stencil_fx<kTC, PP><<<(unsigned)blocks, kRows, smem, st>>>(Ms, Ks, Em, Ek, Z1, Z2, y, g);
  return cudaGetLastError();
}

}  // namespace

int stencil_fx_max_taps() { return kMaxTaps; }

cudaError_t launch_stencil_fx_table(double* C, int* E, int S, long long Ns, cudaStream_t st) {
  if (S < 1 || S > kMaxTaps || Ns < 1) return cudaErrorInvalidValue;
  k_stencil_fx_table<<<(unsigned)((Ns + 255) / 256), 256, 0, st>>>(C, E, S, Ns);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_stencil_space_fx(const StencilOpDev& op, const double* Z1, const double* Z2, double* y,
                                    const StencilDims& g, cudaStream_t st) {
  int S = 1;
  for (int l = 0; l < g.d; ++l) S *= 2 * g.p + 1;
  if (S > kMaxTaps) return cudaErrorInvalidValue;
  const int2* Ms = static_cast<const int2*>(op.Ms);
  const int2* Ks = static_cast<const int2*>(op.Ks);
  ProfScope ps("stencil_space_fx64", 4.0 * S * (double)g.Ns * g.nt,
               (2.0 * S * 8.0) * (double)g.Ns + 16.0 * (double)g.Ns * g.nt + 8.0 * (double)g.Ns * g.nt, st);
  switch (g.p) {
    case 1: return run_fx<kSlices, 1>(Ms, Ks, op.Em, op.Ek, Z1, Z2, y, g, st);
    case 2: return run_fx<kSlices, 2>(Ms, Ks, op.Em, op.Ek, Z1, Z2, y, g, st);
    case 3: return run_fx<kSlices, 3>(Ms, Ks, op.Em, op.Ek, Z1, Z2, y, g, st);
    case 4: return run_fx<kSlices, 4>(Ms, Ks, op.Em, op.Ek, Z1, Z2, y, g, st);
    default: return run_fx<kSlices, 0>(Ms, Ks, op.Em, op.Ek, Z1, Z2, y, g, st);
  }
}

}  // namespace stfd
