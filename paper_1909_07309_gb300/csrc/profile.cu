// Per-kernel CUDA-event timing, launch counting and the DFMA throughput probe
// declared in stfd_profile.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "df.cuh"
#include "kernels.h"
#include "profile.h"
#include "stfd.h"
#include "stfd_profile.h"

namespace stfd {
namespace {

struct Pending {
  const char* name;
  cudaEvent_t e0, e1;
  double flops, bytes;
};

struct Total {
  std::string name;
  long long launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Pending> g_pending;
std::vector<Total> g_totals;
std::vector<cudaEvent_t> g_free;
std::atomic<long long> g_launches{0};

cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Fold pending records into totals (caller holds the lock).
void drain() {
  for (const Pending& p : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      Total* t = nullptr;
      for (Total& x : g_totals)
        if (x.name == p.name) t = &x;
      if (!t) {
        g_totals.push_back(Total());
        t = &g_totals.back();
        t->name = p.name;
      }
      t->launches += 1;
      t->ms += ms;
      t->flops += p.flops;
      t->bytes += p.bytes;
    }
    g_free.push_back(p.e0);
    g_free.push_back(p.e1);
  }
  g_pending.clear();
}

}  // namespace

ProfScope::ProfScope(const char* name, double flops, double bytes, cudaStream_t st)
    : name_(name), flops_(flops), bytes_(bytes), st_(st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  e0_ = take_event();
  e1_ = take_event();
  if (e0_ && e1_) {
    cudaEventRecord(e0_, st_);
    active_ = true;
  }
}

ProfScope::~ProfScope() {
  if (!active_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(e1_, st_);
  g_pending.push_back(Pending{name_, e0_, e1_, flops_, bytes_});
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

// Eight independent FMA chains per thread keep the FP64 pipe saturated.
__global__ void k_probe_dfma(double* out, int iters, double c) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  double a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  const double b = 0.999999;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// Eight independent chains of 32 x 32 -> 64-bit integer multiply-adds per
// thread (mad.wide.s32, the operation of the integer-limb band products).
__global__ void k_probe_imad_wide(long long* out, int iters, int b) {
  long long a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
            a7 = a0 + 7;
  // each chain multiplies by its own low word: no common subexpression to hoist
  for (int i = 0; i < iters; ++i) {
    a0 += (long long)(int)a0 * b; a1 += (long long)(int)a1 * b; a2 += (long long)(int)a2 * b;
    a3 += (long long)(int)a3 * b; a4 += (long long)(int)a4 * b; a5 += (long long)(int)a5 * b;
    a6 += (long long)(int)a6 * b; a7 += (long long)(int)a7 * b;
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

}  // namespace
}  // namespace stfd

using namespace stfd;

extern "C" int stfd_probe_imad_wide_peak(double* ops_per_s, void* stream) {
  if (!ops_per_s) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return STFD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return STFD_ERR_CUDA;
  const int threads = 256, blocks = sms * 8, iters = 4000;
  long long* out = nullptr;
  if (cudaMalloc((void**)&out, (size_t)threads * blocks * sizeof(long long)) != cudaSuccess) return STFD_ERR_ALLOC;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = STFD_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = STFD_ERR_CUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && rc == STFD_OK; ++rep) {
    cudaEventRecord(e0, st);
    k_probe_imad_wide<<<blocks, threads, 0, st>>>(out, iters, 3);
    count_launch();
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = STFD_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  if (rc == STFD_OK) *ops_per_s = 8.0 * iters * (double)threads * blocks / (best * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

extern "C" int stfd_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  return STFD_OK;
}

extern "C" int stfd_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  g_totals.clear();
  return STFD_OK;
}

extern "C" int stfd_profile_count(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  return (int)g_totals.size();
}

extern "C" int stfd_profile_get(int idx, char* name, int name_cap, long long* launches, double* ms,
                                double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  drain();
  if (idx < 0 || idx >= (int)g_totals.size()) return STFD_ERR_ARG;
  const Total& t = g_totals[idx];
  if (name && name_cap > 0) {
    std::strncpy(name, t.name.c_str(), (size_t)name_cap - 1);
    name[name_cap - 1] = '\0';
  }
  if (launches) *launches = t.launches;
  if (ms) *ms = t.ms;
  if (flops) *flops = t.flops;
  if (bytes) *bytes = t.bytes;
  return STFD_OK;
}

extern "C" long long stfd_launch_count(void) { return g_launches.load(); }

extern "C" int stfd_probe_bounded_wait(int max_iters, void* stream) {
  if (max_iters < 1 || max_iters > 1000000) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  count_launch();
  if (stfd::launch_probe_bounded_wait(max_iters, st) != cudaSuccess) return STFD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return STFD_ERR_CUDA;
  return STFD_OK;
}

extern "C" int stfd_probe_fp64_peak(double* flops_per_s, void* stream) {
  if (!flops_per_s) return STFD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return STFD_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return STFD_ERR_CUDA;
  const int threads = 256, blocks = sms * 8, iters = 4000;
  double* out = nullptr;
  if (cudaMalloc((void**)&out, (size_t)threads * blocks * sizeof(double)) != cudaSuccess) return STFD_ERR_ALLOC;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = STFD_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = STFD_ERR_CUDA;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && rc == STFD_OK; ++rep) {
    cudaEventRecord(e0, st);
    k_probe_dfma<<<blocks, threads, 0, st>>>(out, iters, 1e-7);
    count_launch();
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = STFD_ERR_CUDA;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;   // first launch is a warm-up
  }
  if (rc == STFD_OK) *flops_per_s = 16.0 * iters * (double)threads * blocks / (best * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

namespace stfd {
__global__ void k_probe_convert(const double* __restrict__ x, long long n, float* __restrict__ pairs,
                                double* __restrict__ back, float* __restrict__ f, double* __restrict__ fback) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const stfd::dfa::df v = stfd::dfa::from_double(x[i]);
    pairs[2 * i] = v.h;
    pairs[2 * i + 1] = v.l;
    back[i] = stfd::dfa::to_double(v);
    const float r = stfd::dfa::d2f(x[i]);
    f[i] = r;
    fback[i] = stfd::dfa::f2d(r);
  }
}
}  // namespace stfd

extern "C" int stfd_probe_convert(const double* x, long long n, float* pairs, double* back, float* f, double* fback,
                                  void* stream) {
  if (n < 0 || (n > 0 && (!x || !pairs || !back || !f || !fback))) return STFD_ERR_ARG;
  if (n == 0) return STFD_OK;
  const long long blocks = std::min<long long>((n + 255) / 256, 4096);
  stfd::k_probe_convert<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, n, pairs, back, f, fback);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? STFD_OK : STFD_ERR_CUDA;
}
