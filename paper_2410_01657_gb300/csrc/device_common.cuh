// Device-side helpers shared by the libgnnmp CUDA translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.h"

namespace gnn {

// Latched device error word (0 = ok), one per translation unit (the units are
// compiled separately, so each has its own copy). Kernels set it with atomicOr
// when a bounded wait gives up; gnn_check reads and clears the word of every
// unit that launches waiting kernels, through its take_device_error().
#define GNN_DEVERR_TIMEOUT 1u
static __device__ unsigned int g_device_error = 0;

// Host side: read and clear this translation unit's error word.
static inline cudaError_t take_device_error_word(unsigned int* out) {
    unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(out, g_device_error, sizeof(unsigned int));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_device_error, &zero, sizeof(unsigned int));
}

__device__ __forceinline__ void raise_device_error(unsigned int bits) { atomicOr(&g_device_error, bits); }

__device__ __forceinline__ float elu1(float z) { return z > 0.f ? z : expm1f(z); }
// ELU derivative from its output h = ELU(z): 1 above zero, e^z = h + 1 below.
__device__ __forceinline__ float elu1_deriv_from_out(float h) { return h > 0.f ? 1.f : h + 1.f; }

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

inline int cuda_fail(cudaError_t e, const char* what) {
    return set_error(GNN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace gnn

#define GNN_CUDA_CHECK(call, what)                                   \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return ::gnn::cuda_fail(_e, (what));  \
    } while (0)

#define GNN_LAUNCH_CHECK(what) GNN_CUDA_CHECK(cudaGetLastError(), (what))
