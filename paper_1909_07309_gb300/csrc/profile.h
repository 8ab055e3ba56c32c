// Internal: scope object that counts a kernel launch and, while profiling is
// enabled, brackets it with CUDA events on its stream (see stfd_profile.h).
#pragma once
#include <cuda_runtime.h>

namespace stfd {

class ProfScope {
 public:
  // flops / bytes: algorithmic work of the launch (for achieved-rate reports)
  ProfScope(const char* name, double flops, double bytes, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* name_;
  double flops_, bytes_;
  cudaStream_t st_;
  cudaEvent_t e0_ = nullptr, e1_ = nullptr;
  bool active_ = false;
};

void count_launch();

}  // namespace stfd
