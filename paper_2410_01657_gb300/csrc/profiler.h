// Optional per-kernel CUDA-event timing (gnn_profile_* in gnnmp.h).
#pragma once

#include <cuda_runtime.h>

namespace gnn {

// Brackets one kernel launch with CUDA events on stream `s` while profiling is
// on; costs one relaxed atomic load when it is off.
struct ProfScope {
    int slot;
    cudaStream_t s;
    ProfScope(cudaStream_t stream, const char* name);
    ~ProfScope();
};

}  // namespace gnn
