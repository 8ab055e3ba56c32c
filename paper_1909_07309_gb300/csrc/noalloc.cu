// stfd_st_matvec_noalloc: the Kronecker system matvec for callers that cannot
// allocate device memory. Its scratch (the partial sums of the sum-factorised
// product) lives in one file-scope static device array instead of memory from
// cudaMalloc; the caller passes the univariate matrices, x and y.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "device_state.h"
#include "profile.h"
#include "stfd.h"
#include "stfd_internal.h"

namespace stfd {
namespace {

constexpr long long kNoAllocMaxN = STFD_NOALLOC_MAX_N;
constexpr int kMaxDevices = 64;

// Four partial-sum tensors of up to kNoAllocMaxN doubles (16 MiB). Every
// GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_scratch[4 * kNoAllocMaxN];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device. It is looked up (with
// that device current) on every call made outside stream capture, so that a
// device reset, which reloads the module, is picked up; a call made while `st`
// is being captured uses the address cached by an earlier call on the device.
int scratch_address(cudaStream_t st, double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return STFD_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return STFD_ERR_ARG;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return STFD_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return STFD_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  } else if (!g_scratch_addr[dev]) {
    return STFD_ERR_ARG;   // first call on this device inside a capture
  }
  *out = g_scratch_addr[dev];
  return STFD_OK;
}

constexpr int kTC = 32;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Banded mode product with column-major factors J[i + n a]:
// Y[o, i, c] = s1 sum_a J1[i,a] X1[o,a,c] + s2 sum_a J2[i,a] X2[o,a,c], |a - i| <= bw.
__global__ void __launch_bounds__(kThreads)
k_band_mode_colmajor(const double* __restrict__ X1, const double* __restrict__ J1, double s1,
                     const double* __restrict__ X2, const double* __restrict__ J2, double s2,
                     double* __restrict__ Y, int n, long long inner, long long Q, int bw) {
  extern __shared__ double smem[];
  double* xs1 = smem;
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
    double acc1 = 0.0, acc2 = 0.0;
    for (int a = a0; a <= a1; ++a) acc1 = fma(__ldg(J1 + i + (size_t)n * a), xs1[a * kTC + lane], acc1);
    if (X2)
      for (int a = a0; a <= a1; ++a) acc2 = fma(__ldg(J2 + i + (size_t)n * a), xs2[a * kTC + lane], acc2);
    if (valid) Y[base + (long long)i * inner] = X2 ? fma(s1, acc1, s2 * acc2) : s1 * acc1;
  }
}

cudaError_t launch(const double* X1, const double* J1, double s1, const double* X2, const double* J2,
                   double s2, double* Y, int n, long long inner, long long outer, int bw, cudaStream_t st) {
  {
    const cudaError_t e = ensure_smem_attr(k_band_mode_colmajor, 2 * kMaxN * kTC * (int)sizeof(double));
    if (e != cudaSuccess) return e;
  }
  const long long Q = inner * outer;
  const size_t smem = (size_t)(X2 ? 2 : 1) * n * kTC * sizeof(double);
  count_launch();
  k_band_mode_colmajor<<<(unsigned)((Q + kTC - 1) / kTC), kThreads, smem, st>>>(X1, J1, s1, X2, J2, s2, Y, n,
                                                                                inner, Q, bw);
  return cudaGetLastError();
}

}  // namespace
}  // namespace stfd

using namespace stfd;

extern "C" int stfd_st_matvec_noalloc(int d, const int* n, const double* const* K_dev,
                                      const double* const* M_dev, const double* Wt_dev, const double* Mt_dev,
                                      const int* bw, double gamma, double nu, const double* x_dev,
                                      double* y_dev, void* stream) {
  if (d < 1 || d > kMaxDim || !n || !K_dev || !M_dev || !Wt_dev || !Mt_dev || !x_dev || !y_dev) return STFD_ERR_ARG;
  long long N = 1;
  for (int l = 0; l <= d; ++l) {
    if (n[l] < 1 || n[l] > kMaxN) return STFD_ERR_ARG;
    if (l < d && (!K_dev[l] || !M_dev[l])) return STFD_ERR_ARG;
    N *= n[l];
  }
  if (n[d] < 2 || N > kNoAllocMaxN) return STFD_ERR_ARG;
  // x and y may not overlap at all (a partial overlap would be read after written)
  const uintptr_t xb = reinterpret_cast<uintptr_t>(x_dev), yb = reinterpret_cast<uintptr_t>(y_dev);
  const uintptr_t bytes = static_cast<uintptr_t>(N) * sizeof(double);
  if (xb < yb + bytes && yb < xb + bytes) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  double* scratch = nullptr;
  const int rc = scratch_address(st, &scratch);
  if (rc != STFD_OK) return rc;
  double* T[4] = {scratch, scratch + kNoAllocMaxN, scratch + 2 * kNoAllocMaxN, scratch + 3 * kNoAllocMaxN};
  auto band = [&](int l) { return (bw && bw[l] >= 0) ? std::min(bw[l], n[l] - 1) : n[l] - 1; };
  // Same sum-factorisation as stfd_st_matvec: (u, v) = (x x_1 M_1, x x_1 K_1), then
  // (u, v) <- (u x_l M_l, u x_l K_l + v x_l M_l), and y = gamma u x W_t + nu v x M_t.
  // Every scratch element read was written earlier in the same call: nothing needs zeroing.
  long long inner = 1;
  const double* u = x_dev;
  const double* v = nullptr;
  for (int l = 0; l < d; ++l) {
    const long long outer = N / (inner * n[l]);
    double* uo = (l % 2 == 0) ? T[0] : T[2];
    double* vo = (l % 2 == 0) ? T[1] : T[3];
    if (launch(u, M_dev[l], 1.0, nullptr, nullptr, 0.0, uo, n[l], inner, outer, band(l), st) != cudaSuccess)
      return STFD_ERR_CUDA;
    if (l == 0) {
      if (launch(u, K_dev[l], 1.0, nullptr, nullptr, 0.0, vo, n[l], inner, outer, band(l), st) != cudaSuccess)
        return STFD_ERR_CUDA;
    } else if (launch(u, K_dev[l], 1.0, v, M_dev[l], 1.0, vo, n[l], inner, outer, band(l), st) != cudaSuccess) {
      return STFD_ERR_CUDA;
    }
    u = uo;
    v = vo;
    inner *= n[l];
  }
  if (launch(u, Wt_dev, gamma, v, Mt_dev, nu, y_dev, n[d], inner, 1, band(d), st) != cudaSuccess)
    return STFD_ERR_CUDA;
  return STFD_OK;
}
