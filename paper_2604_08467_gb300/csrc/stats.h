// Kernel launch statistics (see ptn_stats_* in include/ptn.h).
#pragma once

#include <cuda_runtime.h>

#include "ptn_internal.h"

namespace ptn {

enum KernelId {
    K_CONTRACT_DIRECT = 0, K_CONTRACT_GEMM, K_FINALIZE, K_PRESAMPLE, K_LOGQ, K_DEDUP, K_VAR_IDS, K_SCAN,
    K_ALLOC, K_SAMPLE_PARENTS, K_EMIT, K_PACK, K_EXPVAL, K_MISC, K_HARVEST, K_CONTRACT_SMALL, K_CACHE, K_COUNT
};

// Counts n launches of kernel `kid` that no StatScope brackets (the launch
// total then equals the number of kernels launched).
void count_launches(int kid, int n = 1);

// Path step the calling thread is launching (recorded with each timed launch).
void set_step_tag(int block, int step);
struct StepTag {
    StepTag(int block, int step) { set_step_tag(block, step); }
    ~StepTag() { set_step_tag(-1, -1); }
};

// Counts one launch of kernel `kid`; with timing on, brackets it with events.
class StatScope {
  public:
    StatScope(int kid, cudaStream_t s, double bytes = 0, double flops = 0);
    ~StatScope();

  private:
    int kid_;
    cudaStream_t s_;
    bool timing_ = false;
    void* a_ = nullptr;
    void* b_ = nullptr;
    double bytes_ = 0, flops_ = 0;
    int block_ = -1, step_ = -1;
};

}  // namespace ptn
