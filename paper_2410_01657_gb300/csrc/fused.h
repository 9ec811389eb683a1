// Fused BF16 tcgen05 path of libgnnmp (declarations used by the C-ABI layer).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gnnmp.h"

namespace gnn {
namespace fused {

cudaError_t take_device_error(unsigned int* out);
size_t mp_forward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W);
size_t mp_backward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W);
int mp_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
               const __nv_bfloat16* e_in, float* x_out, __nv_bfloat16* e_out, float* a_star_out, void* ws,
               size_t ws_bytes, cudaStream_t s);
int mp_backward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                const __nv_bfloat16* e_in, const float* a_star, const float* dx_out, const __nv_bfloat16* de_out,
                float* dx_in, __nv_bfloat16* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes,
                cudaStream_t s);

// gnn_mp_forward without a caller workspace (built-in scratch area).
size_t static_scratch_bytes();
int mp_forward_static(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                      const __nv_bfloat16* e_in, float* x_out, __nv_bfloat16* e_out, float* a_star_out,
                      cudaStream_t s);

// Steps of the forward shared with the backward's recomputation.
int proj_forward(const gnn_graph_dev& G, int H, const gnn_mp_params& W, const float* x_in, __nv_bfloat16* pq,
                 cudaStream_t s);
int aggregate_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                      const __nv_bfloat16* e_in, const __nv_bfloat16* pq, __nv_bfloat16* e_out, float* a,
                      cudaStream_t s);
int node_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* a,
                 const float* x_in, float* x_out, cudaStream_t s);

// Fused BF16 row MLP (encoders / decoder of the network).
bool rowmlp_supported(const gnn_mlp& P);
size_t rowmlp_backward_ws(const gnn_mlp& P);
int rowmlp_forward(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, float eps,
                   cudaStream_t s);
int rowmlp_backward(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                    const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s);

}  // namespace fused
}  // namespace gnn
