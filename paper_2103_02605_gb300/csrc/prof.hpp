// prof.hpp -- RAII bracket that records CUDA events around one launch while
// tracing is on (include/fcirc_prof.h).
#pragma once
#include <cuda_runtime.h>

namespace fcirc {

bool prof_on();

class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope &) = delete;
    ProfScope &operator=(const ProfScope &) = delete;

  private:
    const char *name_;
    cudaStream_t s_;
    int dev_ = 0;
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;
};

}  // namespace fcirc
