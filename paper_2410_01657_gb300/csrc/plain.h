// Plain FP32 SIMT path of libgnnmp (declarations used by the C-ABI layer).
#pragma once

#include <cuda_runtime.h>

#include "gnnmp.h"

namespace gnn {
namespace plain {

cudaError_t take_device_error(unsigned int* out);
size_t mp_forward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W);
size_t mp_backward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W);
int mp_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
               const float* e_in, float* x_out, float* e_out, float* a_star_out, void* ws, size_t ws_bytes,
               cudaStream_t s);
int mp_backward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                const float* e_in, const float* a_star, const float* dx_out, const float* de_out, float* dx_in,
                float* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes, cudaStream_t s);
int halo(const gnn_graph_dev& G, float* rows, int width, cudaStream_t s);
size_t mlp_ws(const gnn_mlp& P, int64_t rows, bool bwd);
int mlp_forward(const gnn_mlp& P, int64_t rows, const float* X, void* Y, int y_bf16, float eps, void* ws,
                size_t ws_bytes, cudaStream_t s);
int mlp_backward(const gnn_mlp& P, int64_t rows, const float* X, const void* dY, int dy_bf16, float* dX,
                 const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s);
int consistent_loss(const gnn_graph_dev& G, const float* y, const float* t, int F, float* loss, float* dy,
                    void* ws, size_t ws_bytes, cudaStream_t s);

}  // namespace plain
}  // namespace gnn
