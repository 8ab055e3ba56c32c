// FP64 mode products of Algorithm 1 (Steps 2 and 4) on the tcgen05 tensor
// cores, no narrower than IEEE FP64: Y[q][i] = sum_a X[q][a] J[i][a] with FP64
// input and output, by exact digit slicing (the error-free splitting of Ozaki,
// Ogita, Oishi and Rump) with seven 8-bit digits per entry.
//
// Every row of X (and of J) is written under its own power of two as a 55-bit
// integer: with E the largest biased exponent of the row, an entry of biased
// exponent e and 53-bit significand m becomes V = round(m 2^{2 - (E - e)}),
// exact for the entries within a factor 4 of the row maximum and rounded at
// 2^-55 of the row scale for the others. V is cut into seven signed digits,
//     V = sum_{k<7} d_k 256^{6-k},   d_k in [-128, 127] (d_0 in [-128, 129]),
// read off the bytes of V + 0x80808080808080 (each byte minus 128): integers of
// at most 8 significant bits, exact in BF16, whose products are exact in FP32.
// With T_c = sum_{k+l=c} sum_a dx_k[q][a] dj_l[i][a] (c <= 6, 28 digit pairs),
//     Y[q][i] ~ 2^{Ex_q + Ej_i - 2106} Z,   Z = sum_{c<=6} T_c 256^{6-c},
// and the pairs dropped (c >= 7) sum to at most 6 n 129^2 256^5 in units where
// the kept sum is up to n 2^110: below 2^-44 of n max|X| max|J| -- under the
// error bound n u sum|X||J| of an IEEE FP64 dot product, and about the size
// of one FP64 rounding of a typical entry. Each T_c is accumulated exactly in
// its own FP32 tensor-memory accumulator (|T_c| <= 7 n 129^2 < 2^24 for
// n <= 144); the seven are converted to integers, Z is formed exactly in two
// 64-bit limbs and rounded once, to nearest even, to the FP64 result.
//
// Tile: M = 128 tensor rows q (R = 112 of them valid when n > 64, so that the
// seven digit planes of the tile and of J fit in shared memory; the MMA's
// rows 112..127 read the next plane and are ignored), K = N = n rounded up to
// 16. Tensor memory holds the seven accumulators of 32 output columns at a time
// (224 columns), double-buffered: the MMAs of output chunk j + 1 run while the
// epilogue of chunk j reads its accumulators and writes FP64 results, and the
// MMAs of chunk j + 2 are issued as soon as chunk j's accumulators are read.
// One persistent 512-thread CTA per SM; the next tile's entries are loaded into
// registers while the MMAs run.
#include <cuda_bf16.h>
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

constexpr int kDig = 7;
constexpr int kChunk = 32;                 // output columns per tensor-memory buffer
constexpr int kBufCols = kDig * kChunk;    // 224 columns per buffer
constexpr unsigned long long kByteBias = 0x80808080808080ull;

struct Oz7Args {
  const double* X;
  double* Y;
  const unsigned char* B;   // digit planes of J, chunk-stacked (see oz7_planes)
  const int* ej;            // per output column i: largest biased exponent of row i of J
  int n, npad, R, nchunk;
  long long inner, Q, ntiles;
  int* status;
  long long wait;
};

// Column of the c-th entry held by digit-phase part p (pairs 4m + p: conflict-free
// 32-bit digit stores, as in the six-digit kernel).
__device__ __forceinline__ int part_col(int p, int c) { return 8 * (c >> 1) + 2 * p + (c & 1); }

__host__ __device__ inline uint32_t a_sbo(int kcores) { return (uint32_t)kcores * 128u + 16u; }

__host__ __device__ inline size_t canon_off16(int r, int k, int kcores, uint32_t sbo) {
  return (size_t)(r >> 3) * sbo + (size_t)(k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Largest of 1 and the biased exponent of an FP64 bit pattern.
__device__ __forceinline__ int bexp(long long w) {
  return max(1, (int)(((unsigned long long)w >> 52) & 0x7FF));
}

// Z = sum_c T_c 256^{6-c} (exact) rounded to nearest even, times 2^SE, as FP64:
// the seven FP32 sums are integers below 2^24, converted exactly, then
// combined and rounded once by combine7_int (fp64_round.cuh).
__device__ __forceinline__ double combine7(const float* T, int SE) {
  int I[kDig];
#pragma unroll
  for (int c = 0; c < kDig; ++c) I[c] = __float2int_rn(T[c]);   // exact: integers below 2^24
  return combine7_int(I, SE);
}

// Raw 8-byte words of tile `tile`, row r, the KC columns of part p (0 outside).
template <int KC>
__device__ __forceinline__ void load_raw(const long long* __restrict__ Xw, long long tile, int R, int r, int p, int n,
                                         long long inner, long long Q, long long* raw) {
  const long long q = tile * R + r;
  const bool valid = r < R && q < Q;
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

// The biased integer W = V + 0x80808080808080 of one entry, V = +-round(4 m
// 2^-s) the signed 55-bit integer of the entry in a row of largest biased
// exponent E (s = E - max(e, 1); branch-free). |V| < 2^55 < the bias, so W > 0,
// and the bytes of W minus 128 are the signed digits of V (d_0 from the top
// bits: W >> 48 minus 128, in [-128, 129]; the others in [-128, 127]).
__device__ __forceinline__ unsigned long long wbias(long long w, int E) {
  const unsigned long long u = (unsigned long long)w;
  const int e = (int)((u >> 52) & 0x7FF);
  const unsigned long long m = (u & 0xFFFFFFFFFFFFFull) | ((unsigned long long)(e != 0) << 52);
  const int s = min(E - max(e, 1), 63);
  const long long mag = (long long)(((m << 2) + ((1ull << s) >> 1)) >> s);
  return (unsigned long long)((u >> 63) ? -mag : mag) + kByteBias;
}

// Digit k of an entry with biased integer (hi, lo) as a float: byte k from the
// top (the top one up to 9 bits) minus 128.
// For k >= 1 one byte permute moves the byte next to the exponent bits of 2^23.
template <int k>
__device__ __forceinline__ float digit_of(uint32_t hi, uint32_t lo) {
  uint32_t f;
  if (k == 0) {
    f = 0x4B000000u | (hi >> 16);
  } else {
    // selector: result bytes (b0, b1, b2, b3) = (byte of the word, 0, 0, 0x4B) from {word, 0x4B000000}
    constexpr uint32_t byte_sel = k == 1 ? 1u : k == 2 ? 0u : k == 3 ? 3u : k == 4 ? 2u : k == 5 ? 1u : 0u;
    f = __byte_perm(k <= 2 ? hi : lo, 0x4B000000u, byte_sel | 0x4440u | 0x7000u);
  }
  return __uint_as_float(f) - 8388736.0f;   // (2^23 + b) - (2^23 + 128)
}

// 17 warps: warps 0..15 convert the tile's entries into digit planes, one plane
// at a time (each plane announced on its own mbarrier), then read the
// accumulators chunk by chunk and write the FP64 results; warp 16 issues the
// MMAs of each plane as soon as it is written (so the digit conversion and the
// tensor cores overlap), and the MMAs of a chunk once its tensor-memory buffer
// has been read out (empty/full mbarrier pairs per buffer).
constexpr int kWorkers = 512;
constexpr int kThreadsTotal = kWorkers + 32;

template <int KC>
__global__ void __launch_bounds__(kThreadsTotal, 1) k_tc_oz7(Oz7Args args) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int n = args.n, npad = args.npad, R = args.R, nchunk = args.nchunk;
  const int kcores = npad / 8;
  const uint32_t sbo_a = a_sbo(kcores), sbo_b = (uint32_t)kcores * 128u;
  const size_t plane_a = (size_t)(R / 8) * sbo_a;
  const long long inner = args.inner, Q = args.Q;
  unsigned char* sB = smem;                                        // 7 npad x npad BF16
  unsigned char* sA = sB + (size_t)kDig * npad * npad * 2;         // 7 planes of R rows (+ overrun)
  const size_t a_bytes = (size_t)(kDig * (R / 8) + (128 - R) / 8) * sbo_a;
  int* sEj = reinterpret_cast<int*>(sA + a_bytes);                 // npad
  int* sEx = sEj + npad;                                           // 2 x 128 row exponents (by tile parity)
  uint64_t* bar = reinterpret_cast<uint64_t*>(sEx + 256);          // pl[7], full[2], empty[2], exq[4]
  uint64_t* pl = bar;
  uint64_t* full = bar + kDig;
  uint64_t* empty = bar + kDig + 2;
  uint64_t* exq = bar + kDig + 4;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + kDig + 8);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool mma_warp = warp == kWorkers / 32;

  {
    const uint4* src = reinterpret_cast<const uint4*>(args.B);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    const int nv = kDig * npad * npad * 2 / 16;
    for (int e = t; e < nv; e += kThreadsTotal) dst[e] = src[e];
    uint4* za = reinterpret_cast<uint4*>(sA);   // zero the digit planes once (padding, overrun)
    for (size_t e = t; e < a_bytes / 16; e += kThreadsTotal) za[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = t; i < npad; i += kThreadsTotal) sEj[i] = i < n ? args.ej[i] : 1;
  }
  if (t == 0) {
    for (int k = 0; k < kDig; ++k) tc::mbar_init(tc::smem_u32(&pl[k]), kWorkers);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(tc::smem_u32(&full[b]), 1);
      tc::mbar_init(tc::smem_u32(&empty[b]), kWorkers);
    }
    for (int qd = 0; qd < 4; ++qd) tc::mbar_init(tc::smem_u32(&exq[qd]), 128);
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  bool timed_out = false;
  int pend0 = -1, pend1 = -1;   // MMA thread: phases of commits not yet seen complete

  if (mma_warp) {
    // ================= MMA issue: the whole warp waits, lane 0 issues =================
    const uint32_t a_addr = tc::smem_u32(sA), b_addr = tc::smem_u32(sB);
    const int ksteps = npad / 16;
    uint32_t ph_pl = 0u, ph_e0 = 0u, ph_e1 = 0u;
    int uses0 = 0, uses1 = 0;     // buffer uses so far (the first needs no drain wait)
    // descriptors: the start-address field (low word) advances by 16 (256 bytes) per K step
    const uint64_t da_base = tc::smem_desc(a_addr, 128u, sbo_a);
    const uint64_t db_base = tc::smem_desc(b_addr, 128u, sbo_b);
    const uint32_t a_hi = (uint32_t)(da_base >> 32), b_hi = (uint32_t)(db_base >> 32);
    const uint32_t a_lo0 = (uint32_t)da_base, b_lo0 = (uint32_t)db_base;
    // MMAs of plane k for chunks j0 .. j0 + cnt - 1, their K steps interleaved so
    // that consecutive MMAs accumulate into different tensor-memory buffers
    auto issue_plane = [&](int j0, int cnt, int k) {
      if (lane != 0) return;
      uint32_t dcol[2], db[2], idesc[2];
      for (int u = 0; u < cnt; ++u) {
        const int j = j0 + u;
        const int nc = min(kChunk, npad - kChunk * j);
        dcol[u] = tmem + (uint32_t)((j & 1) * kBufCols + k * nc);
        db[u] = b_lo0 + (uint32_t)(kDig * kChunk * j / 8) * (sbo_b >> 4);
        idesc[u] = tc::instr_desc(1u, 128, (kDig - k) * nc);
      }
      uint32_t da = a_lo0 + (uint32_t)(k * (plane_a >> 4));
      for (int s = 0; s < ksteps; ++s) {
        for (int u = 0; u < cnt; ++u) {
          tc::mma_bf16_lohi(dcol[u], da, a_hi, db[u], b_hi, idesc[u], (k > 0 || s > 0) ? 1u : 0u);
          db[u] += 16u;
        }
        da += 16u;
      }
    };
    auto wait_empty = [&](int b) -> bool {   // buffer b drained by the workers
      if ((b ? uses1 : uses0) == 0) return true;
      const bool ok = __all_sync(0xFFFFFFFFu, tc::mbar_wait(tc::smem_u32(&empty[b]), b ? ph_e1 : ph_e0, args.wait));
      if (b) ph_e1 ^= 1u;
      else ph_e0 ^= 1u;
      return ok;
    };
    auto commit = [&](int b) {
      if (lane == 0) tc::mma_commit(tc::smem_u32(&full[b]));
      if (b) pend1 = uses1++ & 1;
      else pend0 = uses0++ & 1;
    };
    const int first = min(nchunk, 2);
    for (long long tile = blockIdx.x; tile < args.ntiles && !timed_out; tile += gridDim.x) {
      if (tile + gridDim.x >= args.ntiles) tc::grid_launch_dependents();
      for (int j = 0; j < first && !timed_out; ++j) timed_out = !wait_empty(j);
      for (int k = 0; k < kDig && !timed_out; ++k) {
        if (!__all_sync(0xFFFFFFFFu, tc::mbar_wait(tc::smem_u32(&pl[k]), ph_pl, args.wait))) {
          timed_out = true;
          break;
        }
        tc::fence_after_sync();
        issue_plane(0, first, k);
        if (k == kDig - 1)
          for (int j = 0; j < first; ++j) commit(j);
      }
      ph_pl ^= 1u;
      for (int j = 2; j < nchunk && !timed_out; ++j) {
        if (!wait_empty(j & 1)) {
          timed_out = true;
          break;
        }
        tc::fence_after_sync();
        for (int k = 0; k < kDig; ++k) issue_plane(j, 1, k);
        commit(j & 1);
      }
    }
  } else {
    // ================= workers: digits, then the epilogue =================
    const int dk = lane & 7, dp = (lane >> 3) & 3;
    const int drow = 32 * (warp & 3) + 8 * (warp >> 2) + dk;
    const int erow = 32 * (warp & 3) + lane, epart = warp >> 2;
    const size_t drbase = (size_t)(drow >> 3) * sbo_a + (size_t)(drow & 7) * 16;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const long long* Xw = reinterpret_cast<const long long*>(args.X);
    long long raw[KC];
    uint32_t ph_f0 = 0u, ph_f1 = 0u;
    tc::grid_dependency_wait();   // the preceding kernel's output is read from here on
    if ((long long)blockIdx.x < args.ntiles) load_raw<KC>(Xw, blockIdx.x, R, drow, dp, n, inner, Q, raw);
    int par = 0;
    for (long long tile = blockIdx.x; tile < args.ntiles && !timed_out; tile += gridDim.x, par ^= 1) {
      if (tile + gridDim.x >= args.ntiles) tc::grid_launch_dependents();
      const long long q0 = tile * R;
      // ---- row exponent, the biased integers, then the seven planes one by one
      int E = 1;
#pragma unroll
      for (int c = 0; c < KC; ++c) E = max(E, bexp(raw[c]));
      E = max(E, __shfl_xor_sync(0xFFFFFFFFu, E, 8));
      E = max(E, __shfl_xor_sync(0xFFFFFFFFu, E, 16));
      if (dp == 0) sEx[par * 128 + drow] = E;
      uint32_t whi[KC], wlo[KC];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const unsigned long long W = wbias(raw[c], E);
        whi[c] = (uint32_t)(W >> 32);
        wlo[c] = (uint32_t)W;
      }
      const bool rows_ok = drow < R;   // rows >= R of the MMA read the next plane
#define STFD_OZ7_PLANE(k)                                                                                  \
  {                                                                                                      \
    if (rows_ok) {                                                                                       \
      _Pragma("unroll") for (int c = 0; c < KC; c += 2) {                                                \
        const int a = part_col(dp, c);                                                                   \
        if (a >= npad) continue;                                                                         \
        const __nv_bfloat162 v = __floats2bfloat162_rn(digit_of<k>(whi[c], wlo[c]),                      \
                                                       digit_of<k>(whi[c + 1], wlo[c + 1]));             \
        *reinterpret_cast<__nv_bfloat162*>(sA + (k) * plane_a + drbase + (size_t)(a >> 3) * 128 +        \
                                           (size_t)(a & 7) * 2) = v;                                     \
      }                                                                                                  \
    }                                                                                                    \
    tc::fence_async_smem();                                                                              \
    tc::mbar_arrive(tc::smem_u32(&pl[k]));                                                               \
  }
      STFD_OZ7_PLANE(0)
      STFD_OZ7_PLANE(1)
      STFD_OZ7_PLANE(2)
      STFD_OZ7_PLANE(3)
      STFD_OZ7_PLANE(4)
      STFD_OZ7_PLANE(5)
      STFD_OZ7_PLANE(6)
#undef STFD_OZ7_PLANE
      // the row exponents of this quadrant's rows (written above by the four
      // warps that also read them in the epilogue) are complete: a bounded wait,
      // so that a warp that left on a timeout cannot stall the others
      tc::mbar_arrive(tc::smem_u32(&exq[warp & 3]));
      if (!__all_sync(0xFFFFFFFFu, tc::mbar_wait(tc::smem_u32(&exq[warp & 3]), (uint32_t)par, args.wait))) {
        timed_out = true;
        break;
      }
      // ---- the next tile's entries travel while the tensor cores work
      {
        const long long nt = tile + gridDim.x;
        if (nt < args.ntiles) load_raw<KC>(Xw, nt, R, drow, dp, n, inner, Q, raw);
      }
      // ---- epilogue, chunk by chunk
      const long long q = q0 + erow;
      const bool row_ok = erow < R && q < Q;
      long long base = 0;
      if (row_ok) {
        const long long o = q / inner;
        base = o * (long long)n * inner + (q - o * inner);
      }
      for (int j = 0; j < nchunk; ++j) {
        const int b = j & 1;
        const int nc = min(kChunk, npad - kChunk * j);
        const int per = nc / 4;   // 8 or 4 columns of this part
        const bool ok = __all_sync(0xFFFFFFFFu, tc::mbar_wait(tc::smem_u32(&full[b]), b ? ph_f1 : ph_f0, args.wait));
        if (b) ph_f1 ^= 1u;
        else ph_f0 ^= 1u;
        if (!ok) {
          timed_out = true;
          break;
        }
        tc::fence_after_sync();
        const int ex = sEx[par * 128 + erow];
        for (int g = 0; g < per; g += 4) {
          const int col0 = kChunk * j + epart * per + g;
          uint32_t Tr[kDig][4];
#pragma unroll
          for (int c = 0; c < kDig; ++c)
            tc::tmem_ld4_async(lane_base + (uint32_t)(b * kBufCols + c * nc + epart * per + g), Tr[c]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < kDig; ++c)
            asm volatile("" : "+r"(Tr[c][0]), "+r"(Tr[c][1]), "+r"(Tr[c][2]), "+r"(Tr[c][3]) : : "memory");
          if (g + 4 >= per) {   // this thread has read its share of the buffer
            tc::fence_before_sync();
            tc::mbar_arrive(tc::smem_u32(&empty[b]));
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = col0 + e;
            if (!row_ok || i >= n) continue;
            float T[kDig];
#pragma unroll
            for (int c = 0; c < kDig; ++c) T[c] = __uint_as_float(Tr[c][e]);
            const int ej = sEj[i];
            const double y = (ex >= 2047 || ej >= 2047) ? __longlong_as_double(0x7FF8000000000000ll)
                                                        : combine7(T, ex + ej - 2106);
            args.Y[base + (long long)i * inner] = y;
          }
        }
      }
    }
  }
  // ---- exit: a wait that ran out is reported; the MMA thread lets its own
  // MMAs in flight finish (bounded) before tensor memory is released
  const bool any_timeout = __syncthreads_or(timed_out ? 1 : 0) != 0;
  if (mma_warp && lane == 0 && any_timeout) {   // pend*: the last commit on each buffer
    if (args.status) atomicOr(args.status, kStatusTimeout);
    if (pend0 >= 0) tc::mbar_wait(tc::smem_u32(&full[0]), (uint32_t)pend0, kDrainIters);
    if (pend1 >= 0) tc::mbar_wait(tc::smem_u32(&full[1]), (uint32_t)pend1, kDrainIters);
  }
  tc::fence_after_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

inline int oz7_cols(int n) { return n <= 32 ? 8 : n <= 48 ? 12 : n <= 64 ? 16 : n <= 72 ? 18 : 20; }
inline int oz7_rows(int n) { return n <= 64 ? 128 : 112; }

size_t oz7_smem_bytes(int n) {
  const int npad = (n + 15) / 16 * 16;
  const int R = oz7_rows(n);
  const size_t a_bytes = (size_t)(kDig * (R / 8) + (128 - R) / 8) * a_sbo(npad / 8);
  return (size_t)kDig * npad * npad * 2 + a_bytes + (size_t)npad * 4 + 256 * 4 + (kDig + 8) * 8 + 16;
}

template <int KC>
cudaError_t launch_oz7(const double* X, double* Y, const unsigned char* B, const int* ej, int n, long long inner,
                       long long outer, cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  const size_t smem = oz7_smem_bytes(n);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  {
    const cudaError_t e = ensure_smem_attr(k_tc_oz7<KC>, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  const int npad = (n + 15) / 16 * 16;
  const int R = oz7_rows(n);
  const long long ntiles = (Q + R - 1) / R;
  const long long grid = std::min<long long>(ntiles, sm_count_current());
  Oz7Args a{X, Y, B, ej, n, npad, R, (npad + kChunk - 1) / kChunk, inner, Q, ntiles, status_word(), wait_limit()};
  ProfScope ps("fd_mode_tc7", 2.0 * (double)Q * n * n, 8.0 * (double)Q * n * 2, st);
  // 227 KB requested so that exactly one CTA (which owns all 512 TMEM columns) fits per SM
  return tc::launch_pdl(k_tc_oz7<KC>, dim3((unsigned)grid), dim3(kThreadsTotal), (size_t)227 * 1024, st, a);
}

}  // namespace

int oz7_max_n() { return 80; }

// Host: the seven digit planes of a row-major n x n factor J (J[i*n + a]) in the
// chunk-stacked B layout of the kernel, and per row i the largest biased
// exponent ej[i] (rows scaled exactly as the kernel scales rows of X). Row
// r of the stacked image, for output column i in chunk j (i = 32 j + u) and
// digit l, is 7 * 32 * j + l * nc_j + u with nc_j the chunk's width.
std::vector<unsigned char> oz7_planes(const double* J, int n, std::vector<int>& ej) {
  const int npad = (n + 15) / 16 * 16;
  const int kcores = npad / 8;
  const uint32_t sbo = (uint32_t)kcores * 128u;
  std::vector<unsigned char> img((size_t)kDig * npad * npad * 2, 0);
  ej.assign(n, 1);
  for (int i = 0; i < n; ++i) {
    int E = 1;
    for (int a = 0; a < n; ++a) {
      unsigned long long bits;
      std::memcpy(&bits, &J[(size_t)i * n + a], 8);
      E = std::max(E, std::max(1, (int)((bits >> 52) & 0x7FF)));
    }
    ej[i] = E;
    const int j = i / kChunk, u = i % kChunk;
    const int nc = std::min(kChunk, npad - kChunk * j);
    for (int a = 0; a < n; ++a) {
      unsigned long long bits;
      std::memcpy(&bits, &J[(size_t)i * n + a], 8);
      const int e = (int)((bits >> 52) & 0x7FF);
      unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
      if (e) m |= 1ull << 52;
      const int s = E - std::max(e, 1);
      unsigned long long V;
      if (s <= 2) {
        V = m << (2 - s);
      } else {
        const int sh = s - 2;
        V = sh >= 60 ? 0ull : (m + (1ull << (sh - 1))) >> sh;
      }
      const unsigned long long W = V + kByteBias;
      const int sg = (bits >> 63) ? -1 : 1;
      for (int l = 0; l < kDig; ++l) {
        const int byte = l == 0 ? (int)(W >> 48) : (int)((W >> (8 * (6 - l))) & 0xFF);
        const float dl = (float)(sg * (byte - 128));
        const __nv_bfloat16 h = __float2bfloat16_rn(dl);   // exact: at most 8 significant bits
        const int row = kDig * kChunk * j + l * nc + u;
        std::memcpy(&img[canon_off16(row, a, kcores, sbo)], &h, 2);
      }
    }
  }
  return img;
}

cudaError_t launch_fd_mode_tc7(const double* X, const unsigned char* B, const int* ej, double* Y, int n,
                               long long inner, long long outer, cudaStream_t st) {
  switch (oz7_cols(n)) {
    case 8: return launch_oz7<8>(X, Y, B, ej, n, inner, outer, st);
    case 12: return launch_oz7<12>(X, Y, B, ej, n, inner, outer, st);
    case 16: return launch_oz7<16>(X, Y, B, ej, n, inner, outer, st);
    case 18: return launch_oz7<18>(X, Y, B, ej, n, inner, outer, st);
    default: return launch_oz7<20>(X, Y, B, ej, n, inner, outer, st);
  }
}

}  // namespace stfd
