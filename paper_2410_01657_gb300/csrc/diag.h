// Diagnostics of libgnnmp (declarations used by the C-ABI layer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gnn {
namespace diag {

cudaError_t take_device_error(unsigned int* out);
int measure_fp32_fma(double* tflops, int32_t* sm_count, cudaStream_t s);
int selftest_bounded_wait(uint64_t limit_ns, int32_t* status, cudaStream_t s);

}  // namespace diag
}  // namespace gnn
