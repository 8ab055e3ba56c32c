// Mode products of Algorithm 1 (Steps 2 and 4) on the tcgen05 tensor cores with
// BF16 or TF32 operands and FP32 accumulation in tensor memory -- the
// mixed-precision preconditioner used inside FP64 flexible GMRES.
//
// GEMM per tile: D[q][i] = sum_a X[q][a] J[i][a], where q runs over 128
// consecutive tensor columns (all indices but the mode's, UMMA M = 128) and
// i, a over the mode (UMMA N = K = n rounded up to 16). Operands sit in shared
// memory in the no-swizzle K-major canonical layout (8-row x 16-byte core
// matrices); the factor J stays resident for the CTA's lifetime, each X tile
// is converted on the fly. Persistent CTAs, one accumulator of N fp32 columns
// in TMEM per CTA.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "device_state.h"
#include "kernels.h"
#include "profile.h"
#include "tc_common.cuh"

namespace stfd {
namespace {

constexpr int kTile = 128;                 // UMMA M

__host__ __device__ inline int esz_of(int kind) { return kind == 0 ? 2 : 4; }

// Byte offset of element (row r, k) in a K-major no-swizzle operand with `kcores`
// core matrices (16 bytes each) along K.
__host__ __device__ inline size_t canon_off(int r, int k, int kcores, int esz) {
  const int epc = 16 / esz;
  return (size_t)(r >> 3) * (kcores * 128) + (size_t)(k / epc) * 128 + (r & 7) * 16 + (k % epc) * esz;
}

template <int KIND>
__device__ __forceinline__ void put_operand(unsigned char* base, size_t off, float v) {
  if (KIND == 0) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
  } else {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    *reinterpret_cast<uint32_t*>(base + off) = t;
  }
}

struct TcArgs {
  const void* X;
  void* Y;
  const unsigned char* B;   // factor image, npad x npad in the operand format
  int n, npad, ncols;
  long long inner, Q, ntiles;
  int* status;              // host-mapped status word (kStatusTimeout), may be null
  long long wait;           // bounded-wait iteration limit
};

template <int KIND, typename TIn, typename TOut>
__global__ void __launch_bounds__(kTile) k_tc_mode(TcArgs args) {
  constexpr int esz = KIND == 0 ? 2 : 4;
  constexpr int kstep_bytes = 32;          // one MMA consumes 32 bytes of K per row
  extern __shared__ __align__(1024) unsigned char smem[];
  const int n = args.n, npad = args.npad;
  const int kcores = npad * esz / 16;
  const uint32_t sbo = (uint32_t)kcores * 128u;
  const long long inner = args.inner, Q = args.Q;
  const TIn* X = static_cast<const TIn*>(args.X);
  TOut* Y = static_cast<TOut*>(args.Y);
  unsigned char* sB = smem;
  unsigned char* sA = sB + (size_t)npad * npad * esz;
  float* stage = reinterpret_cast<float*>(sA + (size_t)kTile * npad * esz);
  const size_t stage_bytes = (inner == 1) ? (((size_t)kTile * (n + 1) * sizeof(float) + 15) & ~(size_t)15) : 0;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(stage) + stage_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* sflag = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;

  // factor image -> smem (16-byte vectors), zero the A tile once (K padding stays 0)
  {
    const uint4* src = reinterpret_cast<const uint4*>(args.B);
    uint4* dstB = reinterpret_cast<uint4*>(sB);
    const int nv = npad * npad * esz / 16;
    for (int e = tid; e < nv; e += kTile) dstB[e] = src[e];
    uint4* dstA = reinterpret_cast<uint4*>(sA);
    const int na = kTile * npad * esz / 16;
    for (int e = tid; e < na; e += kTile) dstA[e] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(mbar), 1);
    *sflag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tslot), (uint32_t)args.ncols);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc::instr_desc(KIND == 0 ? 1u : 2u, kTile, npad);
  const uint32_t a_addr = tc::smem_u32(sA), b_addr = tc::smem_u32(sB);
  uint32_t phase = 0;
  int pend = -1;   // thread 0: phase of an MMA commit not yet seen complete

  for (long long tile = blockIdx.x; tile < args.ntiles; tile += gridDim.x) {
    const long long q0 = tile * kTile;
    const int rows = (int)min((long long)kTile, Q - q0);
    // ---- X tile -> operand A
    long long base = 0;
    const long long q = q0 + tid;
    if (q < Q) {
      const long long o = q / inner;
      base = o * (long long)n * inner + (q - o * inner);
    }
    if (inner == 1) {
      const TIn* src = X + q0 * n;
      const int cnt = rows * n;
      for (int e = tid; e < cnt; e += kTile) {
        const int r = e / n, k = e - r * n;
        put_operand<KIND>(sA, canon_off(r, k, kcores, esz), (float)src[e]);
      }
    } else if (q < Q) {
      for (int k = 0; k < n; ++k) put_operand<KIND>(sA, canon_off(tid, k, kcores, esz), (float)X[base + (long long)k * inner]);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- MMA (one thread), completion tracked by the mbarrier
    if (tid == 0) {
      const int ksteps = npad * esz / kstep_bytes;
      for (int s = 0; s < ksteps; ++s) {
        const uint64_t da = tc::smem_desc(a_addr + s * 256, 128u, sbo);
        const uint64_t db = tc::smem_desc(b_addr + s * 256, 128u, sbo);
        tc::mma<KIND>(tmem, da, db, idesc, s > 0 ? 1u : 0u);
      }
      tc::mma_commit(tc::smem_u32(mbar));
    }
    const bool ok = tc::mbar_wait(tc::smem_u32(mbar), phase, args.wait);
    if (!ok) *sflag = 1;
    if (tid == 0) pend = ok ? -1 : (int)phase;
    phase ^= 1u;
    __syncthreads();
    if (*sflag) break;
    tc::fence_after_sync();
    // ---- epilogue: TMEM row tid -> Y
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < npad; c0 += 16) {
      float v[16];
      tc::tmem_ld16(trow + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int i = c0 + j;
        if (i < n) {
          if (inner == 1) stage[tid * (n + 1) + i] = v[j];
          else if (q < Q) Y[base + (long long)i * inner] = (TOut)v[j];
        }
      }
    }
    if (inner == 1) {
      __syncthreads();
      TOut* dst = Y + q0 * n;
      const int cnt = rows * n;
      for (int e = tid; e < cnt; e += kTile) {
        const int r = e / n;
        dst[e] = (TOut)stage[r * (n + 1) + (e - r * n)];
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  tc::fence_after_sync();
  if (tid == 0 && *sflag) {
    // a wait ran out: report it and let the MMAs in flight finish (bounded)
    // before tensor memory is released
    if (args.status) atomicOr(args.status, kStatusTimeout);
    if (pend >= 0) tc::mbar_wait(tc::smem_u32(mbar), (uint32_t)pend, kDrainIters);
    tc::fence_after_sync();
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)args.ncols);
}

template <int KIND, typename TIn, typename TOut>
cudaError_t launch_impl(const TIn* X, TOut* Y, const unsigned char* B, int n, long long inner, long long outer,
                        cudaStream_t st) {
  const long long Q = inner * outer;
  if (Q <= 0) return cudaSuccess;
  const int esz = esz_of(KIND);
  const int npad = (n + 15) / 16 * 16;
  int ncols = 32;
  while (ncols < npad) ncols <<= 1;
  const size_t stage = (inner == 1) ? (((size_t)kTile * (n + 1) * sizeof(float) + 15) & ~(size_t)15) : 0;
  const size_t smem = (size_t)npad * npad * esz + (size_t)kTile * npad * esz + stage + 32;
  {
    const cudaError_t e = ensure_smem_attr(k_tc_mode<KIND, TIn, TOut>, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const int by_smem = (int)std::max<size_t>(1, (228 * 1024) / (smem + 1024));
  const int by_tmem = 512 / ncols;
  const int per_sm = std::max(1, std::min(by_smem, by_tmem));
  // Request enough shared memory that no SM can hold more CTAs than tensor
  // memory has columns for (a surplus CTA would block in tcgen05.alloc).
  const size_t smem_req = std::max(smem, (size_t)(228 * 1024) / per_sm - 1024 + 1);
  const long long ntiles = (Q + kTile - 1) / kTile;
  const long long grid = std::min<long long>(ntiles, (long long)sm_count_current() * per_sm);
  TcArgs a{X, Y, B, n, npad, ncols, inner, Q, ntiles, status_word(), wait_limit()};
  const double flops = 2.0 * (double)Q * n * n;
  const double bytes = (double)Q * n * (sizeof(TIn) + sizeof(TOut));
  ProfScope ps(KIND == 0 ? "tc_mode_bf16" : "tc_mode_tf32", flops, bytes, st);
  k_tc_mode<KIND, TIn, TOut><<<(unsigned)grid, kTile, std::min(smem_req, (size_t)227 * 1024), st>>>(a);
  return cudaGetLastError();
}

}  // namespace

std::vector<unsigned char> tc_operand_image(const double* J, int n, int kind) {
  const int esz = esz_of(kind);
  const int npad = (n + 15) / 16 * 16;
  const int kcores = npad * esz / 16;
  std::vector<unsigned char> img((size_t)npad * npad * esz, 0);
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) {
      const size_t off = canon_off(i, a, kcores, esz);
      const float v = (float)J[(size_t)i * n + a];
      if (kind == 0) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        std::memcpy(&img[off], &h, 2);
      } else {
        // round to the 10-bit TF32 mantissa (nearest, ties away) on the host
        uint32_t u;
        std::memcpy(&u, &v, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        std::memcpy(&img[off], &u, 4);
      }
    }
  return img;
}

cudaError_t launch_tc_mode(int kind, const void* X, int x_is_double, void* Y, int y_is_double,
                           const unsigned char* B, int n, long long inner, long long outer, cudaStream_t st) {
  if (kind == 0) {
    if (x_is_double) return launch_impl<0, double, float>((const double*)X, (float*)Y, B, n, inner, outer, st);
    if (y_is_double) return launch_impl<0, float, double>((const float*)X, (double*)Y, B, n, inner, outer, st);
    return launch_impl<0, float, float>((const float*)X, (float*)Y, B, n, inner, outer, st);
  }
  if (x_is_double) return launch_impl<1, double, float>((const double*)X, (float*)Y, B, n, inner, outer, st);
  if (y_is_double) return launch_impl<1, float, double>((const float*)X, (double*)Y, B, n, inner, outer, st);
  return launch_impl<1, float, float>((const float*)X, (float*)Y, B, n, inner, outer, st);
}

namespace {
// An mbarrier that expects one arrival which never comes: the bounded wait must
// give up and raise the status flag.
__global__ void k_probe_bounded_wait(int max_iters, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(tc::smem_u32(&bar), 1);
  if (!tc::mbar_wait(tc::smem_u32(&bar), 0, max_iters) && status) atomicOr(status, kStatusTimeout);
}
}  // namespace

cudaError_t launch_probe_bounded_wait(int max_iters, cudaStream_t st) {
  k_probe_bounded_wait<<<1, 32, 0, st>>>(max_iters, status_word());
  return cudaGetLastError();
}

}  // namespace stfd
