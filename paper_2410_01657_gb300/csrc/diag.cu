// Diagnostics of libgnnmp with no counterpart in the paper:
//   * the FP32 FMA throughput of the device, the peak the plain FP32 SIMT path
//     is measured against (a long chain of independent fused multiply-adds per
//     thread, CUDA-event timed);
//   * a self-test of the bounded device-side waits: a kernel waits on an
//     mbarrier that no thread ever arrives at, with a caller-given limit, and
//     must give up, latch the timeout in the error word and return, leaving the
//     context usable.

#include "diag.h"

#include "device_common.cuh"
#include "tc_common.cuh"

namespace gnn {
namespace diag {

cudaError_t take_device_error(unsigned int* out) { return take_device_error_word(out); }

namespace {

constexpr int kFmaThreads = 1024;
constexpr int kFmaChains = 8;    // independent FMA chains per thread (latency hiding)
constexpr int kFmaUnroll = 16;
__device__ float g_fma_sink[1024];

// b and c are kernel arguments so the chains cannot be folded at compile time;
// the final store is taken only for an impossible sum, which keeps the chains live.
__global__ void __launch_bounds__(kFmaThreads) k_fma_peak(int iters, float b, float c) {
    float v[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) v[j] = threadIdx.x * 1e-6f + (float)j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kFmaUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kFmaChains; ++j) v[j] = fmaf(v[j], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) s += v[j];
    if (s == -1.2345e-30f) g_fma_sink[blockIdx.x & 1023] = s;
}

__global__ void k_wait_selftest(uint64_t limit_ns, int32_t* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    // phase 0 of `bar` never completes: nobody arrives
    const bool done = tc::mbar_wait(&bar, 0, limit_ns);
    if (threadIdx.x == 0) *status = done ? 2 : 1;
}

}  // namespace

int measure_fp32_fma(double* tflops, int32_t* sm_count, cudaStream_t s) {
    int dev = 0, sms = 0;
    GNN_CUDA_CHECK(cudaGetDevice(&dev), "gnn_measure_fp32_fma: cudaGetDevice");
    GNN_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev),
                   "gnn_measure_fp32_fma: SM count");
    const int blocks = 2 * sms, iters = 4096;
    cudaEvent_t e0, e1;
    GNN_CUDA_CHECK(cudaEventCreate(&e0), "gnn_measure_fp32_fma: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(GNN_ECUDA, "gnn_measure_fp32_fma: event");
    }
    float best = 0.f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, s);
        k_fma_peak<<<blocks, kFmaThreads, 0, s>>>(iters, 0.9999f, 1e-4f);
        cudaEventRecord(e1, s);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GNN_CUDA_CHECK(err, "gnn_measure_fp32_fma: FMA kernel");
    const double flops = 2.0 * blocks * kFmaThreads * (double)iters * kFmaUnroll * kFmaChains;
    *tflops = flops / (best * 1e-3) / 1e12;
    *sm_count = sms;
    return GNN_OK;
}

int selftest_bounded_wait(uint64_t limit_ns, int32_t* status, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, status);
    GNN_LAUNCH_CHECK("k_wait_selftest");
    return GNN_OK;
}

}  // namespace diag
}  // namespace gnn
