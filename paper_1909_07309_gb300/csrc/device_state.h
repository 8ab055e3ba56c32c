// Process-wide device state shared by the launchers: per-device kernel
// attributes, the host-mapped status word that device-side bounded waits
// raise, and the iteration limit of those waits.
#pragma once
#include <cuda_runtime.h>

namespace stfd {

// Sets cudaFuncAttributeMaxDynamicSharedMemorySize of `func` to `bytes` on the
// current device, once per (function, device, size); thread-safe. The
// attribute is per device, so a process that drives several GPUs sets it on
// each of them before the first launch there.
cudaError_t ensure_smem_attr(const void* func, int bytes);
template <typename... A>
cudaError_t ensure_smem_attr(void (*func)(A...), int bytes) {
  return ensure_smem_attr(reinterpret_cast<const void*>(func), bytes);
}

// Number of SMs of the current device (cached per device).
int sm_count_current();

// Status bits raised by device code in the host-mapped status word.
enum : int { kStatusTimeout = 1 };

// Device-visible address of the status word (pinned host memory mapped into
// every device's address space; allocated on first use). nullptr if the
// allocation failed, in which case kernels skip the report.
int* status_word();
// Host: the status bits raised so far, cleared on return. Only launches that
// have completed (the caller synchronised their stream) are guaranteed seen.
int status_read_and_clear();

// Iteration limit of every bounded mbarrier wait in the tensor-core kernels
// (default 1 << 22, about a second). A wait that runs out raises
// kStatusTimeout and the kernel abandons its remaining tiles.
long long wait_limit();
void set_wait_limit(long long iters);
// Limit of the drain wait with which a kernel whose wait ran out lets its own
// tensor-core operations and bulk copies in flight finish before it releases
// tensor memory and exits (independent of wait_limit()).
constexpr long long kDrainIters = 1LL << 24;

}  // namespace stfd
