// FP64-accurate mode products of Algorithm 1 on the tcgen05 tensor cores by
// exact digit slicing (the error-free splitting of Ozaki, Ogita, Oishi and
// Rump): Y[q][i] = sum_a X[q][a] J[i][a] with
//
//   X[q][a] = 2^{u_q} sum_{k<6} dx_k[q][a],   J[i][a] = 2^{v_i} sum_{l<6} dj_l[i][a],
//
// one power of two per row (from the row's largest exponent) so that the row
// lies below 2^7, and signed round-to-nearest digits dx_k, dj_l that are
// integers times 2^{-8k} (2^{-8l}) with |integer| <= 128 (192 for dx_3, which
// also absorbs the low float of a double-float entry): BF16 holds every digit
// exactly and every digit product is exact. Then
// Y[q][i] = 2^{u_q + v_i} sum_{c<6} T_c[q][i], T_c = sum_{k+l=c} sum_a dx_k dj_l,
// each T_c accumulated in its own FP32 TMEM accumulator by BF16 tcgen05 MMAs.
// For n <= 80 every partial sum of T_c is an integer multiple of 2^{-8c}
// below 2^{24 - 8c}, so all six accumulators are exact; the pairs with
// k + l >= 6 and the digits beyond dx_5 are dropped (below 2^-47 of the row
// scale). The six T_c are combined in double-float arithmetic.
//
// The digits of an entry come from FP32 additions: adding 1.5 * 2^{23-8k}
// rounds a value below 2^{22-8k} to a multiple of 2^{-8k}, subtracting it again
// gives the digit exactly, and subtracting the digit leaves the exact remainder.
//
// One persistent CTA per SM (the six accumulators take 480 of the 512 TMEM
// columns). Per 128-column tile: every thread holds KC entries of one row in
// registers (strided modes: loaded while the previous tile's MMAs ran), the
// row exponent is reduced across the row's four threads, the digits of each
// entry go to the six digit planes at once; then one thread issues the digit
// pair MMAs against the resident planes of J and commits them to one mbarrier.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "device_state.h"
#include "df.cuh"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {

namespace {

constexpr int kTile = 128;
constexpr int kDig = 6;

__host__ __device__ inline size_t canon_off16(int r, int k, int kcores) {
  return (size_t)(r >> 3) * (kcores * 128) + (size_t)(k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

struct OzArgs {
  const void* X;
  void* Y;
  const unsigned char* B;   // kDig digit planes of J (npad x npad BF16 each)
  const int* v;             // per output row i: 2^{v_i} scale of J
  int n, npad;
  long long inner, Q, ntiles;
  int* status;              // host-mapped status word (kStatusTimeout), may be null
  long long wait;           // bounded-wait iteration limit
};

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {   // a - b
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}

__device__ __forceinline__ float pow2f(int e) {   // 2^e for e in [-126, 127]
  return __int_as_float((e + 127) << 23);
}

template <typename T>
struct IsDouble {
  static constexpr bool value = false;
};
template <>
struct IsDouble<double> {
  static constexpr bool value = true;
};

template <typename T>
struct StoreOut;
template <>
struct StoreOut<double> {
  __device__ static void put(double* p, long long i, dfa::df v) { p[i] = dfa::to_double(v); }
};
template <>
struct StoreOut<float2> {
  __device__ static void put(float2* p, long long i, dfa::df v) { p[i] = make_float2(v.h, v.l); }
};

// 512 threads: thread t owns tile row r = t % 128 (its TMEM lane) together with
// three other threads (parts p = t / 128); part p owns the contiguous block of
// KC (even) columns p KC .. p KC + KC - 1 of the row, held in registers.
constexpr int kParts = 4;
constexpr int kThreads = kTile * kParts;

// Columns per part for a factor of order n (4 KC >= n; KC = 18 leaves the
// padding columns 72 .. 79 to a separate zero fill).
inline int oz_cols(int n) { return n <= 32 ? 8 : n <= 48 ? 12 : n <= 64 ? 16 : n <= 72 ? 18 : 20; }

// Rounding constants: x + kRound[k] - kRound[k] is x rounded to a multiple of
// 2^{-8k} (for |x| < 2^{22-8k}).
__device__ __forceinline__ float round_const(int k) { return 12582912.0f * pow2f(-8 * k); }

// Byte distance between 8-row groups of an A digit plane: the dense value plus
// 16 bytes (the tensor cores read the planes faster with the padding).
__host__ __device__ inline uint32_t a_sbo(int kcores) { return (uint32_t)kcores * 128u + 16u; }

// Column of the c-th entry held by digit-phase part p: part p owns the column
// pairs j = 4m + p (columns 8m + 2p and 8m + 2p + 1), so that when the 8 rows x 4
// parts of a warp store the same m, each thread's 32-bit word lands in its own
// bank (bank 4 (row mod 8) + p of the 16-byte row chunk, plus the row group's offset).
__device__ __forceinline__ int part_col(int p, int c) { return 8 * (c >> 1) + 2 * p + (c & 1); }

// Raw 8-byte words of tile `tile`, row r, the KC columns of part p (0 outside).
template <int KC>
__device__ __forceinline__ void load_raw(const long long* __restrict__ Xw, long long tile, int r, int p, int n,
                                         long long inner, long long Q, long long* raw) {
  const long long q = tile * kTile + r;
  const bool valid = q < Q;
  long long base = 0;
  if (valid) {
    const long long o = q / inner;
    base = o * (long long)n * inner + (q - o * inner);
  }
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    const int a = part_col(p, c);
    raw[c] = (valid && a < n) ? __ldg(Xw + base + (long long)a * inner) : 0ll;
  }
}

// An entry as a double-float (h, l): FP64 words are split with integer and
// FP32 instructions, double-float words are the two floats.
template <bool DBL>
__device__ __forceinline__ dfa::df entry(long long w) {
  if (DBL) return dfa::from_double(__longlong_as_double(w));
  return dfa::df{__int_as_float((int)(unsigned int)((unsigned long long)w & 0xFFFFFFFFull)),
                 __int_as_float((int)(unsigned int)((unsigned long long)w >> 32))};
}

// The six digits of one entry, already scaled below 2^7: d_0 .. d_2 from the
// high float, then the low float joins the remainder (one rounding, below the
// resolution 2^-40 of d_5) and d_3 .. d_5 follow.
__device__ __forceinline__ void digits6(float yh, float yl, float* d) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float C = round_const(k);
    d[k] = (yh + C) - C;
    yh -= d[k];
  }
  float y = yh + yl;
#pragma unroll
  for (int k = 3; k < kDig; ++k) {
    const float C = round_const(k);
    d[k] = (y + C) - C;
    y -= d[k];
  }
}

template <typename TIn, typename TOut, int KC>
__global__ void __launch_bounds__(kThreads, 1) k_tc_ozaki(OzArgs args) {
  constexpr bool DBL = IsDouble<TIn>::value;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int n = args.n, npad = args.npad;
  const int kcores = npad / 8;                  // 16-byte core matrices along K (8 BF16 each)
  const uint32_t sbo_b = (uint32_t)kcores * 128u, sbo_a = a_sbo(kcores);
  const size_t plane_b = (size_t)npad * npad * 2;
  const size_t plane_a = (size_t)(kTile / 8) * sbo_a;
  const long long inner = args.inner, Q = args.Q;
  unsigned char* sB = smem;                                            // kDig planes of J
  unsigned char* sA = sB + kDig * plane_b;                             // kDig planes of the tile
  int* sv = reinterpret_cast<int*>(sA + kDig * plane_a);              // npad
  int* sE = sv + ((npad + 3) & ~3);                                    // kTile row exponents
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sE + kParts * kTile);   // MMA, bulk copy
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  int* sflag = reinterpret_cast<int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, r = t & (kTile - 1), part = t >> 7;
  const int nchunk4 = (n + 3) / 4;
  // digit phase: warp w holds rows 32 (w mod 4) + 8 (w / 4) .. + 7 (inside its TMEM
  // lane quarter) and, per row, the four parts dp = lane / 8 of the columns
  const int dk = t & 7, dp = (t >> 3) & 3;
  const int drow = 32 * (warp & 3) + 8 * (warp >> 2) + dk;

  {
    const uint4* src = reinterpret_cast<const uint4*>(args.B);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    const int nv = (int)(kDig * plane_b / 16);
    for (int e = t; e < nv; e += kThreads) dst[e] = src[e];
    for (int i = t; i < npad; i += kThreads) sv[i] = i < n ? args.v[i] : 0;
  }
  if (t == 0) {
    tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
    tc::mbar_init(tc::smem_u32(&mbar[1]), 1);
    *sflag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const int mgroup = 256 / npad;                // B planes per MMA (N = mgroup npad <= 256)
  const uint32_t a_addr = tc::smem_u32(sA), b_addr = tc::smem_u32(sB);
  const int ksteps = npad / 16;
  const uint64_t da0 = tc::smem_desc(a_addr, 128u, sbo_a), db0 = tc::smem_desc(b_addr, 128u, sbo_b);
  uint32_t ph = 0u, ph_in = 0u;
  int pend_mma = -1, pend_in = -1;   // thread 0: phases of an MMA commit / bulk load not yet seen complete
  const long long* Xw = static_cast<const long long*>(args.X);
  // mode 1: the tile is one contiguous block of rows x n words in and out, moved
  // by bulk copies when the tensors are 16-byte aligned (the block offsets
  // q0 n 8 bytes are multiples of 1024)
  const bool bulk_in = (reinterpret_cast<uintptr_t>(args.X) & 15u) == 0u;
  const bool bulk_out = (reinterpret_cast<uintptr_t>(args.Y) & 15u) == 0u;
  long long raw[KC];
  // strided modes: each warp's loads are coalesced (consecutive rows are
  // consecutive addresses), so entries go straight to registers and the next
  // tile's are fetched while the MMAs run. Mode 1 (inner == 1): a row is
  // contiguous, so the tile is a contiguous block, copied through shared memory.
  // everything above (factor planes, TMEM, barriers) overlaps the end of the
  // preceding kernel; its output is read, and this kernel's written, only from here
  tc::grid_dependency_wait();
  if (inner != 1 && (long long)blockIdx.x < args.ntiles) load_raw<KC>(Xw, blockIdx.x, drow, dp, n, inner, Q, raw);
  // padding column pairs 2 KC .. npad / 2 - 1 (KC = 18): zero digits, written once
  // here and again per tile where the staging area overwrites them (mode 1)
  const size_t drbase = (size_t)(drow >> 3) * sbo_a + (size_t)(drow & 7) * 16;
  const auto zero_tail = [&]() {
    for (int j = 2 * KC + dp; j < npad / 2; j += kParts)
#pragma unroll
      for (int k = 0; k < kDig; ++k)
        *reinterpret_cast<uint32_t*>(sA + k * plane_a + drbase + (size_t)(j >> 2) * 128 + (size_t)(j & 3) * 4) = 0u;
  };
  zero_tail();

  for (long long tile = blockIdx.x; tile < args.ntiles; tile += gridDim.x) {
    if (tile + gridDim.x >= args.ntiles) tc::grid_launch_dependents();   // this CTA's last tile
    const long long q0 = tile * kTile;
    const int rows = (int)min((long long)kTile, Q - q0);
    const long long q = q0 + r;
    long long base = 0;
    if (q < Q) {
      const long long o = q / inner;
      base = o * (long long)n * inner + (q - o * inner);
    }
    if (inner == 1) {   // the tile's rows into the (free) plane area, row stride n
      long long* blk = reinterpret_cast<long long*>(sA);
      const long long* src = Xw + q0 * n;
      const int cnt = rows * n;
      if (bulk_in) {
        const int cnt2 = cnt & ~1;   // whole 16-byte units; an odd last word by thread 1
        if (t == 0) {
          if (bulk_out) tc::bulk_wait_read_all();   // the previous tile's output block has been read out
          tc::fence_async_smem();
          if (cnt2 > 0) {
            tc::mbar_arrive_expect_tx(tc::smem_u32(&mbar[1]), (uint32_t)cnt2 * 8u);
            tc::bulk_g2s(tc::smem_u32(blk), src, (uint32_t)cnt2 * 8u, tc::smem_u32(&mbar[1]));
          } else {
            tc::mbar_arrive(tc::smem_u32(&mbar[1]));
          }
        }
        if (t == 1 && (cnt & 1)) blk[cnt - 1] = __ldg(src + cnt - 1);
        if (tc::mbar_wait(tc::smem_u32(&mbar[1]), ph_in, args.wait)) {
          if (t == 0) pend_in = -1;
        } else {
          *sflag = 1;
          if (t == 0) pend_in = (int)ph_in;   // the copy may still be landing: drained below
        }
        ph_in ^= 1u;
      } else {
        if (bulk_out) {
          if (t == 0) tc::bulk_wait_read_all();
          __syncthreads();
        }
        for (int e = t; e < cnt; e += kThreads) blk[e] = __ldg(src + e);
      }
      __syncthreads();
      if (*sflag) break;
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const int a = part_col(dp, c);
        raw[c] = (drow < rows && a < n) ? blk[drow * n + a] : 0ll;
      }
      __syncthreads();   // the planes overwrite the block below
      zero_tail();
    }
    // ---- entries as double-floats; row exponent: max over this thread's
    // columns, then over the four parts
    float xh[KC], xl[KC];
    int Erow;
    {
      int E0 = 0, E1 = 0;
#pragma unroll
      for (int c = 0; c < KC; c += 2) {
        const dfa::df v0 = entry<DBL>(raw[c]), v1 = entry<DBL>(raw[c + 1]);
        xh[c] = v0.h;
        xl[c] = v0.l;
        xh[c + 1] = v1.h;
        xl[c + 1] = v1.l;
        E0 = max(E0, (int)((__float_as_uint(v0.h) >> 23) & 0xFFu));
        E1 = max(E1, (int)((__float_as_uint(v1.h) >> 23) & 0xFFu));
      }
      E0 = max(E0, E1);
      E0 = max(E0, __shfl_xor_sync(0xFFFFFFFFu, E0, 8));    // over the row's four parts
      E0 = max(E0, __shfl_xor_sync(0xFFFFFFFFu, E0, 16));
      Erow = max(E0, 7);   // rows below 2^-120 keep fewer than 48 bits
      if (dp == 0) sE[drow] = Erow;   // for the epilogue, whose threads own other rows
    }
    // X[q][a] = 2^{Erow - 133} y_a with |y_a| < 2^7
    const float S = pow2f(133 - Erow);
    // ---- six digit planes, two columns per 32-bit store
    {
#pragma unroll
      for (int c = 0; c < KC; c += 2) {
        const int a = part_col(dp, c);   // columns n .. 4 KC - 1 hold zero entries
        if (a >= npad) continue;
        float d0[kDig], d1[kDig];
        digits6(xh[c] * S, xl[c] * S, d0);
        digits6(xh[c + 1] * S, xl[c + 1] * S, d1);
        const size_t off = drbase + (size_t)(a >> 3) * 128 + (size_t)(a & 7) * 2;
#pragma unroll
        for (int k = 0; k < kDig; ++k) {
          const __nv_bfloat162 b = __floats2bfloat162_rn(d0[k], d1[k]);   // exact: digits are BF16 numbers
          *reinterpret_cast<__nv_bfloat162*>(sA + k * plane_a + off) = b;
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- all 21 digit pairs of the tile, one commit. The B planes are stacked
    // (plane l + 1 follows plane l as the next npad rows) and the accumulators
    // are adjacent (diagonal c at columns c npad), so one MMA of N = m npad
    // multiplies A plane k by B planes l .. l + m - 1 into diagonals
    // k + l .. k + l + m - 1: with N <= 256, 9 MMAs per K step instead of 21.
    if (t == 0) {
      for (int k = 0; k < kDig; ++k)
        for (int l = 0; l + k < kDig; l += mgroup) {
          const int m = min(mgroup, kDig - k - l);
          const uint32_t dcol = tmem + (uint32_t)((k + l) * npad);
          const uint32_t idesc_m = tc::instr_desc(1u, kTile, m * npad);
          for (int s = 0; s < ksteps; ++s) {
            const uint64_t da = da0 + (uint64_t)((k * plane_a + s * 256) >> 4);
            const uint64_t db = db0 + (uint64_t)((l * plane_b + s * 256) >> 4);
            tc::mma<0>(dcol, da, db, idesc_m, (k > 0 || s > 0) ? 1u : 0u);
          }
        }
      tc::mma_commit(tc::smem_u32(&mbar[0]));
      pend_mma = (int)ph;
    }
    // ---- the next tile's words travel while the tensor cores work
    if (inner != 1) {
      const long long nt = tile + gridDim.x;
      if (nt < args.ntiles) load_raw<KC>(Xw, nt, drow, dp, n, inner, Q, raw);
    }
    if (tc::mbar_wait(tc::smem_u32(&mbar[0]), ph, args.wait)) {
      if (t == 0) pend_mma = -1;
    } else {
      *sflag = 1;
    }
    ph ^= 1u;
    __syncthreads();
    if (*sflag) break;
    tc::fence_after_sync();
    // ---- epilogue: part p combines the six diagonals of row r on the 4-column
    // chunks p, p+4, ... that hold output columns (i < n)
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const int urow_e = sE[r] - 133;   // the exponent of epilogue row r, from the digit phase
    float2* stage = reinterpret_cast<float2*>(sA);   // free once the MMAs are done
    for (int c4 = part; c4 < nchunk4; c4 += kParts) {
      uint32_t Tr[kDig][4];
#pragma unroll
      for (int c = 0; c < kDig; ++c) tc::tmem_ld4_async(lane_base + (uint32_t)(c * npad + 4 * c4), Tr[c]);
      tc::tmem_wait_ld4x6(Tr);
      // two output columns at a time on the paired FP32 instructions (per
      // column the scalar steps: the results do not depend on the pairing)
#pragma unroll
      for (int j = 0; j < 4; j += 2) {
        const int i = 4 * c4 + j;   // i + 1 < npad: sv is padded
        if (i >= n || r >= rows) continue;
        float2 T[kDig];
#pragma unroll
        for (int c = 0; c < kDig; ++c) T[c] = make_float2(__uint_as_float(Tr[c][j]), __uint_as_float(Tr[c][j + 1]));
        // every T_c is exact; two-sums fold in the two leading diagonals below
        // T_0, the trailing three (below 2^-23 of the total) are summed in FP32
        float2 hi = T[0], lo = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 1; c < 3; ++c) {
          const float2 sm = __fadd2_rn(hi, T[c]), bp = sub2(sm, hi);
          lo = __fadd2_rn(lo, __fadd2_rn(sub2(hi, sub2(sm, bp)), sub2(T[c], bp)));
          hi = sm;
        }
        lo = __fadd2_rn(lo, __fadd2_rn(__fadd2_rn(T[3], T[4]), T[5]));
        const float2 nh = __fadd2_rn(hi, lo), nl = sub2(lo, sub2(nh, hi));   // normalised pair
        int sc0 = urow_e + sv[i], sc1 = urow_e + sv[i + 1];
        sc0 = max(-250, min(250, sc0));
        sc1 = max(-250, min(250, sc1));
        const float2 f1 = make_float2(pow2f(sc0 >> 1), pow2f(sc1 >> 1));
        const float2 f2 = make_float2(pow2f(sc0 - (sc0 >> 1)), pow2f(sc1 - (sc1 >> 1)));
        const float2 yh = __fmul2_rn(__fmul2_rn(nh, f1), f2), yl = __fmul2_rn(__fmul2_rn(nl, f1), f2);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          if (i + e >= n) break;
          const dfa::df y{e == 0 ? yh.x : yh.y, e == 0 ? yl.x : yl.y};
          if (inner == 1) {
            StoreOut<TOut>::put(reinterpret_cast<TOut*>(stage), (long long)r * n + i + e, y);
          } else {
            StoreOut<TOut>::put(static_cast<TOut*>(args.Y), base + (long long)(i + e) * inner, y);
          }
        }
      }
    }
    if (inner == 1) {   // the stage (row stride n) is the output block
      TOut* dst = static_cast<TOut*>(args.Y) + q0 * n;
      const TOut* sst = reinterpret_cast<const TOut*>(stage);
      const int cnt = rows * n;
      if (bulk_out) {
        tc::fence_async_smem();   // the stage writes, visible to the bulk copy
        __syncthreads();
        const int cnt2 = cnt & ~1;
        if (t == 0 && cnt2 > 0) tc::bulk_s2g(dst, tc::smem_u32(stage), (uint32_t)cnt2 * 8u);
        if (t == 1 && (cnt & 1)) dst[cnt - 1] = sst[cnt - 1];
      } else {
        __syncthreads();
        for (int e = t; e < cnt; e += kThreads) dst[e] = sst[e];
      }
    }
    tc::fence_before_sync();
    __syncthreads();   // the staging area and sE are rewritten by the next tile
  }
  tc::fence_after_sync();
  if (t == 0) {
    tc::bulk_wait_all();   // the last output block has left shared memory
    if (*sflag) {
      // a wait ran out: report it, and let this CTA's own MMAs and bulk loads
      // still in flight finish (bounded) before tensor memory is released
      if (args.status) atomicOr(args.status, kStatusTimeout);
      if (pend_mma >= 0) tc::mbar_wait(tc::smem_u32(&mbar[0]), (uint32_t)pend_mma, kDrainIters);
      if (pend_in >= 0) tc::mbar_wait(tc::smem_u32(&mbar[1]), (uint32_t)pend_in, kDrainIters);
      tc::fence_after_sync();
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

size_t oz_smem_bytes(int n) {
  const int npad = (n + 15) / 16 * 16;
  const int kcores = npad / 8;
  return (size_t)kDig * npad * npad * 2 + (size_t)kDig * (kTile / 8) * a_sbo(kcores) +
         (size_t)((npad + 3) & ~3) * 4 + (size_t)kParts * kTile * 4 + 32;
}

template <typename TIn, typename TOut, int KC>
cudaError_t launch_oz(const TIn* X, TOut* Y, const unsigned char* B, const int* v, int n, long long inner,
                      long long outer, cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  const size_t smem = oz_smem_bytes(n);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = ensure_smem_attr(k_tc_ozaki<TIn, TOut, KC>, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  const long long ntiles = (Q + kTile - 1) / kTile;
  const long long grid = std::min<long long>(ntiles, sm_count_current());
  OzArgs a{X, Y, B, v, n, (n + 15) / 16 * 16, inner, Q, ntiles, status_word(), wait_limit()};
  ProfScope ps("fd_mode_ozaki", 2.0 * (double)Q * n * n, 8.0 * (double)Q * n * 2, st);
  // 227 KB requested so that exactly one CTA (which owns all 512 TMEM columns) fits per SM
  // programmatic dependent launch: the next kernel's prologue may overlap this one's tail
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 227 * 1024;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_tc_ozaki<TIn, TOut, KC>, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename TIn, typename TOut>
cudaError_t launch_oz_cols(const TIn* X, TOut* Y, const unsigned char* B, const int* v, int n, long long inner,
                           long long outer, cudaStream_t st) {
  switch (oz_cols(n)) {
    case 8: return launch_oz<TIn, TOut, 8>(X, Y, B, v, n, inner, outer, st);
    case 12: return launch_oz<TIn, TOut, 12>(X, Y, B, v, n, inner, outer, st);
    case 16: return launch_oz<TIn, TOut, 16>(X, Y, B, v, n, inner, outer, st);
    case 18: return launch_oz<TIn, TOut, 18>(X, Y, B, v, n, inner, outer, st);
    default: return launch_oz<TIn, TOut, 20>(X, Y, B, v, n, inner, outer, st);
  }
}

}  // namespace

int ozaki_max_n() { return 80; }

// Host: digit planes of a row-major n x n factor J (J[i*n + a]) and the
// per-row scale exponents v_i: J[i][a] = 2^{v_i} (sum_l dj_l + remainder), with
// w = 2^{-v_i} J[i][a] below 2^7 and dj_l = round(w_l 2^{8l}) 2^{-8l} taken from
// the running remainder w_l (exact in FP64: scalings by powers of two, integer
// rounding, and the subtraction of a value within half a digit unit).
std::vector<unsigned char> ozaki_planes(const double* J, int n, std::vector<int>& v) {
  const int npad = (n + 15) / 16 * 16;
  const int kcores = npad / 8;
  const size_t plane = (size_t)npad * npad * 2;
  std::vector<unsigned char> img(kDig * plane, 0);
  v.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    int E = 0;
    for (int a = 0; a < n; ++a) {
      unsigned long long bits;
      std::memcpy(&bits, &J[(size_t)i * n + a], 8);
      E = std::max(E, (int)((bits >> 52) & 0x7FF));
    }
    E = std::max(E, 1);
    v[i] = E - 1029;   // |J[i][a]| < 2^{E - 1022} = 2^{v_i + 7}
    for (int a = 0; a < n; ++a) {
      double w = std::ldexp(J[(size_t)i * n + a], -v[i]);
      for (int l = 0; l < kDig; ++l) {
        const double dl = std::nearbyint(std::ldexp(w, 8 * l));
        const double d = std::ldexp(dl, -8 * l);
        w -= d;
        const __nv_bfloat16 h = __float2bfloat16_rn((float)d);
        std::memcpy(&img[l * plane + canon_off16(i, a, kcores)], &h, 2);
      }
    }
  }
  return img;
}

cudaError_t launch_fd_mode_ozaki(const void* X, int x_is_double, const unsigned char* B, const int* v, void* Y,
                                 int y_is_double, int n, long long inner, long long outer, cudaStream_t st) {
  if (x_is_double) return launch_oz_cols<double, float2>((const double*)X, (float2*)Y, B, v, n, inner, outer, st);
  if (y_is_double) return launch_oz_cols<float2, double>((const float2*)X, (double*)Y, B, v, n, inner, outer, st);
  return launch_oz_cols<float2, float2>((const float2*)X, (float2*)Y, B, v, n, inner, outer, st);
}

}  // namespace stfd
