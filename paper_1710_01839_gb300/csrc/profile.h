#pragma once

#include <cuda_runtime.h>

namespace mpg {

// RAII bracket of one kernel launch when profiling is on (mpgemm_profile).
class ProfScope {
  public:
    explicit ProfScope(cudaStream_t s);
    ~ProfScope();

  private:
    cudaStream_t s_;
    cudaEvent_t end_;
};

}  // namespace mpg
