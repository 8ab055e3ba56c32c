// FP64-accurate mode products of Algorithm 1 on the tcgen05 tensor cores by
// exact digit slicing (the error-free splitting of Ozaki, Ogita, Oishi and
// Rump): Y[q][i] = sum_a X[q][a] J[i][a] with
//
//   X[q][a] = 2^{u_q} F[q][a],  F = sum_{k<6} dx_k 2^{40-8k},  |dx_k| <= 255,
//   J[i][a] = 2^{v_i} G[i][a],  G = sum_{l<6} dj_l 2^{40-8l},  |dj_l| <= 255,
//
// one power of two per row (the row's largest exponent), so that every digit
// is an integer that BF16 holds exactly and every digit product is exact.
// Then Y[q][i] = 2^{u_q + v_i + 80} sum_{c<6} 2^{-8c} T_c[q][i] with
// T_c = sum_{k+l=c} sum_a dx_k[q][a] dj_l[i][a]. Each T_c is accumulated in its
// own FP32 TMEM accumulator by BF16 tcgen05 MMAs: for c <= 2 every partial sum
// is an integer below 2^24 (n <= 80), hence exact; for c >= 3 the FP32 rounding
// sits below 2^-44 of the result scale. Pairs with k + l >= 6 are dropped
// (< 2^-47 relative). The six T_c are combined in double-float arithmetic.
//
// One persistent CTA per SM (the six accumulators take 480 of the 512 TMEM
// columns). Per 128-column tile: every thread holds its 20 entries of one row
// in registers (loaded while the previous tile's MMAs ran), the row exponent is
// reduced across the row's four threads, each entry is converted to 48-bit
// fixed point and its six digits are written to the six digit planes at once;
// then one thread issues all 21 digit-pair MMAs against the resident planes of
// J and commits them to one mbarrier.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "df.cuh"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {

extern __device__ int g_tc_status;

namespace {

constexpr int kTile = 128;
constexpr int kDig = 6;
constexpr long kWaitIters = 1L << 22;

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
};

// Largest biased exponent over the entries a = a0, a0 + step, ... < n of a
// staged row (FP64 words or double-float words).
template <bool DBL>
__device__ __forceinline__ int row_max_exp(const long long* F, int n, int a0, int step) {
  int E0 = 0, E1 = 0;   // two independent maxima for instruction-level parallelism
  int a = a0;
  for (; a + step < n; a += 2 * step) {
    const unsigned long long w0 = (unsigned long long)F[a], w1 = (unsigned long long)F[a + step];
    E0 = max(E0, DBL ? (int)((w0 >> 52) & 0x7FF) : (int)((w0 >> 23) & 0xFF));
    E1 = max(E1, DBL ? (int)((w1 >> 52) & 0x7FF) : (int)((w1 >> 23) & 0xFF));
  }
  if (a < n) {
    const unsigned long long w = (unsigned long long)F[a];
    E0 = max(E0, DBL ? (int)((w >> 52) & 0x7FF) : (int)((w >> 23) & 0xFF));
  }
  return max(E0, E1);
}

// Staged entry -> signed 48-bit fixed point under the row exponent E:
// FP64:         x = F 2^{E-1070};   double-float: x = F 2^{E-174}.
template <bool DBL>
__device__ __forceinline__ long long to_fixed(long long word, int E) {
  if (DBL) {
    const int ex = (int)(((unsigned long long)word >> 52) & 0x7FF);
    if (ex == 0) return 0;
    const unsigned long long m = ((unsigned long long)word & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - ex + 5;
    const long long f = sh < 64 ? (long long)(m >> sh) : 0;
    return word < 0 ? -f : f;
  }
  const unsigned long long w = (unsigned long long)word;
  const unsigned int hb = (unsigned int)(w & 0xFFFFFFFFull), lb = (unsigned int)(w >> 32);
  long long fh = 0, fl = 0;
  const int eh = (hb >> 23) & 0xFF, el = (lb >> 23) & 0xFF;
  if (eh != 0) {
    const long long mh = (long long)((hb & 0x7FFFFF) | 0x800000);
    const int sh = 24 + eh - E;          // |h| = mh 2^{eh-150}
    fh = sh >= 0 ? (mh << sh) : (sh > -64 ? (mh >> -sh) : 0);
    if (hb >> 31) fh = -fh;
  }
  if (el != 0) {
    const long long ml = (long long)((lb & 0x7FFFFF) | 0x800000);
    const int sh = 24 + el - E;
    fl = sh >= 0 ? (ml << sh) : (sh > -64 ? (ml >> -sh) : 0);
    if (lb >> 31) fl = -fl;
  }
  return fh + fl;
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
// three other threads (parts p = t / 128); part p owns a contiguous block of
// kCols (even) columns of the row, held in registers from global memory.
constexpr int kParts = 4;
constexpr int kThreads = kTile * kParts;
constexpr int kCols = 20;                      // columns per part: 4 x 20 covers n <= 80

// Byte distance between 8-row groups of an A digit plane: the dense value plus
// 16 bytes, so that the 4 row groups a warp writes fall in different banks.
__host__ __device__ inline uint32_t a_sbo(int kcores) { return (uint32_t)kcores * 128u + 16u; }

// Raw 8-byte words of tile `tile`, row r, columns a0 .. a0 + kCols - 1 (0 outside).
__device__ __forceinline__ void load_raw(const long long* __restrict__ Xw, long long tile, int r, int a0, int a1,
                                         int n, long long inner, long long Q, long long* raw) {
  const long long q = tile * kTile + r;
  const bool valid = q < Q;
  long long base = 0;
  if (valid) {
    const long long o = q / inner;
    base = o * (long long)n * inner + (q - o * inner);
  }
#pragma unroll
  for (int c = 0; c < kCols; ++c) {
    const int a = a0 + c;
    raw[c] = (valid && a < a1) ? __ldg(Xw + base + (long long)a * inner) : 0ll;
  }
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kThreads, 1) k_tc_ozaki(OzArgs args) {
  constexpr bool DBL = IsDouble<TIn>::value;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int n = args.n, npad = args.npad;
  const int kcores = npad / 8;                  // 16-byte core matrices along K (8 BF16 each)
  const uint32_t sbo_b = (uint32_t)kcores * 128u, sbo_a = a_sbo(kcores);
  const size_t plane_b = (size_t)npad * npad * 2;
  const size_t plane_a = (size_t)(kTile / 8) * sbo_a;
  const int ld = n + 1;                         // output staging row stride (8-byte words)
  const long long inner = args.inner, Q = args.Q;
  unsigned char* sB = smem;                                            // kDig planes of J
  unsigned char* sA = sB + kDig * plane_b;                             // kDig planes of the tile
  int* sv = reinterpret_cast<int*>(sA + kDig * plane_a);              // npad
  int* sE = sv + ((npad + 3) & ~3);                                    // kParts x kTile
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sE + kParts * kTile);   // 1 barrier
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* sflag = reinterpret_cast<int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, r = t & (kTile - 1), part = t >> 7;
  const int nchunk_pad = npad / 8;
  const int a0 = part * kCols, a1 = min(n, a0 + kCols);   // this thread's columns

  {
    const uint4* src = reinterpret_cast<const uint4*>(args.B);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    const int nv = (int)(kDig * plane_b / 16);
    for (int e = t; e < nv; e += kThreads) dst[e] = src[e];
    for (int i = t; i < npad; i += kThreads) sv[i] = i < n ? args.v[i] : 0;
  }
  if (t == 0) {
    tc::mbar_init(tc::smem_u32(&mbar[0]), 1);
    *sflag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc::instr_desc(1u, kTile, npad);
  const uint32_t a_addr = tc::smem_u32(sA), b_addr = tc::smem_u32(sB);
  const int ksteps = npad / 16;
  const uint64_t da0 = tc::smem_desc(a_addr, 128u, sbo_a), db0 = tc::smem_desc(b_addr, 128u, sbo_b);
  uint32_t ph = 0u;
  const long long* Xw = static_cast<const long long*>(args.X);
  long long raw[kCols];
  // strided modes: each warp's loads are coalesced (consecutive rows are
  // consecutive addresses), so entries go straight to registers and the next
  // tile's are fetched while the MMAs run. Mode 1 (inner == 1): a row is
  // contiguous, so the tile is a contiguous block, copied through shared memory.
  if (inner != 1 && (long long)blockIdx.x < args.ntiles) load_raw(Xw, blockIdx.x, r, a0, a1, n, inner, Q, raw);

  for (long long tile = blockIdx.x; tile < args.ntiles; tile += gridDim.x) {
    const long long q0 = tile * kTile;
    const int rows = (int)min((long long)kTile, Q - q0);
    const long long q = q0 + r;
    long long base = 0;
    if (q < Q) {
      const long long o = q / inner;
      base = o * (long long)n * inner + (q - o * inner);
    }
    if (inner == 1) {   // coalesced copy of the tile's rows into the (free) plane area
      long long* blk = reinterpret_cast<long long*>(sA);
      const long long* src = Xw + q0 * n;
      const int cnt = rows * n;
      for (int e = t; e < cnt; e += kThreads) {
        const int rr = e / n;
        blk[rr * ld + (e - rr * n)] = __ldg(src + e);
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        const int a = a0 + c;
        raw[c] = (r < rows && a < a1) ? blk[r * ld + a] : 0ll;
      }
      __syncthreads();   // the planes overwrite the block below
    }
    // ---- row exponent: max over this thread's columns, then over the four parts
    {
      int E0 = 0, E1 = 0;
#pragma unroll
      for (int c = 0; c < kCols; c += 2) {
        const unsigned long long w0 = (unsigned long long)raw[c], w1 = (unsigned long long)raw[c + 1];
        E0 = max(E0, DBL ? (int)((w0 >> 52) & 0x7FF) : (int)((w0 >> 23) & 0xFF));
        E1 = max(E1, DBL ? (int)((w1 >> 52) & 0x7FF) : (int)((w1 >> 23) & 0xFF));
      }
      sE[part * kTile + r] = max(E0, E1);
    }
    __syncthreads();
    int E = 0;
#pragma unroll
    for (int pp = 0; pp < kParts; ++pp) E = max(E, sE[pp * kTile + r]);
    const int urow = DBL ? E - 1070 : E - 174;
    // ---- 48-bit fixed point and its six digit planes, two columns per 32-bit store
    {
      const size_t rbase = (size_t)(r >> 3) * sbo_a + (size_t)(r & 7) * 16;
#pragma unroll
      for (int c = 0; c < kCols; c += 2) {
        const int a = a0 + c;   // columns n .. npad-1 are written as zero digits
        if (a >= npad) break;
        uint32_t h[2][kDig];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const long long f = to_fixed<DBL>(raw[c + e], E);
          const unsigned long long m = (unsigned long long)(f < 0 ? -f : f);
          const uint32_t sgn = f < 0 ? 0x8000u : 0u;
#pragma unroll
          for (int k = 0; k < kDig; ++k) {
            const uint32_t dg = (uint32_t)(m >> (40 - 8 * k)) & 0xFFu;
            // exact float of the digit (0x4B000000 | d is 2^23 + d); its top 16 bits are its BF16
            const float fv = __int_as_float(0x4B000000u | dg) - 8388608.0f;
            h[e][k] = ((uint32_t)__float_as_int(fv) >> 16) | sgn;
          }
        }
        const size_t off = rbase + (size_t)(a >> 3) * 128 + (size_t)(a & 7) * 2;
#pragma unroll
        for (int k = 0; k < kDig; ++k)
          *reinterpret_cast<uint32_t*>(sA + k * plane_a + off) = h[0][k] | (h[1][k] << 16);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- all 21 digit-pair MMAs of the tile, one commit
    if (t == 0) {
      for (int k = 0; k < kDig; ++k)
        for (int l = 0; l + k < kDig; ++l) {
          const uint32_t dcol = tmem + (uint32_t)((k + l) * npad);
          for (int s = 0; s < ksteps; ++s) {
            const uint64_t da = da0 + (uint64_t)((k * plane_a + s * 256) >> 4);
            const uint64_t db = db0 + (uint64_t)((l * plane_b + s * 256) >> 4);
            tc::mma<0>(dcol, da, db, idesc, (k > 0 || s > 0) ? 1u : 0u);
          }
        }
      tc::mma_commit(tc::smem_u32(&mbar[0]));
    }
    // ---- the next tile's words travel while the tensor cores work
    if (inner != 1) {
      const long long nt = tile + gridDim.x;
      if (nt < args.ntiles) load_raw(Xw, nt, r, a0, a1, n, inner, Q, raw);
    }
    if (!tc::mbar_wait(tc::smem_u32(&mbar[0]), ph, kWaitIters)) *sflag = 1;
    ph ^= 1u;
    __syncthreads();
    if (*sflag) {
      if (t == 0) atomicExch(&g_tc_status, 1);
      break;
    }
    tc::fence_after_sync();
    // ---- epilogue: part p combines the six diagonals of row r on chunks p, p+4, ...
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    float2* stage = reinterpret_cast<float2*>(sA);   // free once the MMAs are done
    for (int c8 = part; c8 < nchunk_pad; c8 += kParts) {
      uint32_t Tr[kDig][8];
#pragma unroll
      for (int c = 0; c < kDig; ++c) tc::tmem_ld8_async(lane_base + (uint32_t)(c * npad + 8 * c8), Tr[c]);
      tc::tmem_wait_ld8x6(Tr);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = 8 * c8 + j;
        if (i >= n || r >= rows) continue;
        float T[kDig];
#pragma unroll
        for (int c = 0; c < kDig; ++c) T[c] = __uint_as_float(Tr[c][j]);
        // exact two-sums for the three leading diagonals; the trailing three sit
        // below 2^-22 of the total and are summed in plain FP32 (error < 2^-46 of it)
        float hi = T[0], lo = 0.f;
#pragma unroll
        for (int c = 1; c < 3; ++c) {
          const float v = T[c] * pow2f(-8 * c);
          const float sm = hi + v, bp = sm - hi;
          lo += (hi - (sm - bp)) + (v - bp);
          hi = sm;
        }
        lo += fmaf(T[5], pow2f(-40), fmaf(T[4], pow2f(-32), T[3] * pow2f(-24)));
        const dfa::df sres = dfa::norm(dfa::df{hi, lo});
        int sc = urow + sv[i] + 80;
        sc = max(-250, min(250, sc));
        const float f1 = pow2f(sc / 2), f2 = pow2f(sc - sc / 2);
        const dfa::df y{sres.h * f1 * f2, sres.l * f1 * f2};
        if (inner == 1) {
          stage[r * ld + i] = make_float2(y.h, y.l);
        } else {
          StoreOut<TOut>::put(static_cast<TOut*>(args.Y), base + (long long)i * inner, y);
        }
      }
    }
    if (inner == 1) {
      __syncthreads();
      TOut* dst = static_cast<TOut*>(args.Y) + q0 * n;
      const int cnt = rows * n;
      for (int e = t; e < cnt; e += kThreads) {
        const int rr = e / n;
        const float2 v = stage[rr * ld + (e - rr * n)];
        StoreOut<TOut>::put(dst, e, dfa::df{v.x, v.y});
      }
    }
    tc::fence_before_sync();
    __syncthreads();   // the staging area and sE are rewritten by the next tile
  }
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

int sm_count_oz() {
  static int s = 0;
  if (s == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) s = 148;
  }
  return s;
}

size_t oz_smem_bytes(int n) {
  const int npad = (n + 15) / 16 * 16;
  const int kcores = npad / 8;
  return (size_t)kDig * npad * npad * 2 + (size_t)kDig * (kTile / 8) * a_sbo(kcores) +
         (size_t)((npad + 3) & ~3) * 4 + (size_t)kParts * kTile * 4 + 32;
}

template <typename TIn, typename TOut>
cudaError_t launch_oz(const TIn* X, TOut* Y, const unsigned char* B, const int* v, int n, long long inner,
                      long long outer, cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  const size_t smem = oz_smem_bytes(n);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  static bool attr_done = false;
  if (!attr_done) {
    const cudaError_t e = cudaFuncSetAttribute(k_tc_ozaki<TIn, TOut>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               227 * 1024);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const long long ntiles = (Q + kTile - 1) / kTile;
  const long long grid = std::min<long long>(ntiles, sm_count_oz());
  OzArgs a{X, Y, B, v, n, (n + 15) / 16 * 16, inner, Q, ntiles};
  ProfScope ps("fd_mode_ozaki", 2.0 * (double)Q * n * n, 8.0 * (double)Q * n * 2, st);
  // 227 KB requested so that exactly one CTA (which owns all 512 TMEM columns) fits per SM
  k_tc_ozaki<TIn, TOut><<<(unsigned)grid, kThreads, 227 * 1024, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int ozaki_max_n() { return 80; }

// Host: digit planes of a row-major n x n factor J (J[i*n + a]) and the
// per-row scale exponents v_i (J[i][a] ~= 2^{v_i} sum_l dj_l 2^{40-8l}).
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
    v[i] = E - 1070;
    for (int a = 0; a < n; ++a) {
      unsigned long long bits;
      std::memcpy(&bits, &J[(size_t)i * n + a], 8);
      const int ex = (int)((bits >> 52) & 0x7FF);
      unsigned long long f = 0;
      if (ex != 0) {
        const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = E - ex + 5;
        f = sh < 64 ? (m >> sh) : 0;
      }
      const bool neg = (bits >> 63) != 0;
      for (int l = 0; l < kDig; ++l) {
        const int dg = (int)((f >> (40 - 8 * l)) & 0xFF);
        const __nv_bfloat16 h = __float2bfloat16_rn((float)(neg ? -dg : dg));
        std::memcpy(&img[l * plane + canon_off16(i, a, kcores)], &h, 2);
      }
    }
  }
  return img;
}

cudaError_t launch_fd_mode_ozaki(const void* X, int x_is_double, const unsigned char* B, const int* v, void* Y,
                                 int y_is_double, int n, long long inner, long long outer, cudaStream_t st) {
  if (x_is_double) return launch_oz<double, float2>((const double*)X, (float2*)Y, B, v, n, inner, outer, st);
  if (y_is_double) return launch_oz<float2, double>((const float2*)X, (double*)Y, B, v, n, inner, outer, st);
  return launch_oz<float2, float2>((const float2*)X, (float2*)Y, B, v, n, inner, outer, st);
}

}  // namespace stfd
