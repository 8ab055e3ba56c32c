// Process-wide device state: see device_state.h.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <set>
#include <tuple>

#include "device_state.h"
#include "stfd.h"

namespace stfd {
namespace {

std::mutex g_mu;
std::set<std::tuple<const void*, int, int>> g_attr_done;   // (function, device, bytes)
constexpr int kMaxDevices = 64;
int g_sms[kMaxDevices] = {0};
int* g_status = nullptr;          // pinned, mapped, portable (host address == device address under UVA)
bool g_status_tried = false;
std::atomic<long long> g_wait_limit{1LL << 22};

}  // namespace

cudaError_t ensure_smem_attr(const void* func, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  const auto key = std::make_tuple(func, dev, bytes);
  if (g_attr_done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) g_attr_done.insert(key);
  return e;
}

int sm_count_current() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 148;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_sms[dev] <= 0) {
    int s = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || s <= 0) return 148;
    g_sms[dev] = s;
  }
  return g_sms[dev];
}

int* status_word() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_status && !g_status_tried) {
    g_status_tried = true;
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess) {
      *static_cast<volatile int*>(p) = 0;
      void* dp = nullptr;
      if (cudaHostGetDevicePointer(&dp, p, 0) == cudaSuccess && dp == p) {
        g_status = static_cast<int*>(p);
      } else {
        cudaFreeHost(p);
      }
    }
  }
  return g_status;
}

int status_read_and_clear() {
  int* w = status_word();
  if (!w) return 0;
  volatile int* v = w;
  const int s = *v;
  if (s) *v = 0;
  return s;
}

long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }
void set_wait_limit(long long iters) { g_wait_limit.store(iters, std::memory_order_relaxed); }

}  // namespace stfd

extern "C" int stfd_set_wait_limit(long long iters) {
  if (iters < 0 || iters > (1LL << 40)) return STFD_ERR_ARG;
  stfd::set_wait_limit(iters);
  return STFD_OK;
}

extern "C" long long stfd_get_wait_limit(void) { return stfd::wait_limit(); }
