// Fused BF16 tcgen05 path of libgnnmp (declarations used by the C-ABI layer).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gnnmp.h"

namespace gnn {
namespace fused {

// Read and clear the device error word of fused.cu, fused_bwd.cu, bwd128.cu, rowmlp.cu, edge128.cu,
// rowenc128.cu, rowdec128.cu, node128.cu.
cudaError_t take_device_error(unsigned int* out);
cudaError_t take_device_error_bwd(unsigned int* out);
cudaError_t take_device_error_bwd128(unsigned int* out);
cudaError_t take_device_error_rowmlp(unsigned int* out);
cudaError_t take_device_error_edge128(unsigned int* out);
cudaError_t take_device_error_rowenc128(unsigned int* out);
cudaError_t take_device_error_rowdec128(unsigned int* out);
cudaError_t take_device_error_node128(unsigned int* out);
// The H = 128 edge forward with two tile groups per SM and the hidden
// activations in tensor memory (edge128.cu); supported for 2..4 Linears.
bool edge_fwd_tm_supported(const gnn_mp_params& W);
int edge_fwd_tm(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const __nv_bfloat16* e_in,
                const __nv_bfloat16* pq, __nv_bfloat16* e_out, float* a, cudaStream_t s);
// The H = 128 node forward in the same two-group tensor-memory form (node128.cu;
// 2..4 Linears); 16-byte aligned a*, x and x' rows.
bool node_fwd_tm_supported(const gnn_mp_params& W);
int node_fwd_tm(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* a,
                const float* x_in, float* x_out, cudaStream_t s);
size_t mp_forward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W);
size_t mp_backward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W);
// Bytes of the saved MLP activations (BF16 h_0 .. h_{L-2} of every edge, then
// of every node row) that mp_forward writes and mp_backward reads when given
// `act`; 0 where the backward recomputes them instead (H = 128 has its own
// layered adjoint).
size_t mp_act_bytes(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W);
// Elements of the edge part of those activations; the node MLP's h_0 .. h_{L-2}
// follow, block k of R = ceil(n_rows / 128) * 128 rows each, then the node
// MLP's BF16 input rows [a*, x] (R rows, 2H wide).
size_t mp_act_elems_edge(const gnn_graph_dev& G, const gnn_mp_params& W, int H);
int mp_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
               const __nv_bfloat16* e_in, float* x_out, __nv_bfloat16* e_out, float* a_star_out, void* ws,
               size_t ws_bytes, cudaStream_t s, __nv_bfloat16* act = nullptr);
int mp_backward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                const __nv_bfloat16* e_in, const float* a_star, const float* dx_out, const __nv_bfloat16* de_out,
                float* dx_in, __nv_bfloat16* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes,
                cudaStream_t s, const __nv_bfloat16* act = nullptr);

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
                      cudaStream_t s, __nv_bfloat16* act = nullptr);
int node_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* a,
                 const float* x_in, float* x_out, cudaStream_t s, __nv_bfloat16* act = nullptr);

// Backward recomputation of the edge or node MLP at H = 128 over the tiles
// [t0, t1): saves the hidden activations (and, for nodes, the BF16 [a*, x]
// input rows) to tile-padded scratch rows (t - t0) * 128 + i, and applies the
// LayerNorm adjoint to the gradient of the layer output. Writes per-CTA
// partials [dgamma | dbeta | db_last] (3H floats, pstride apart) for `grid` CTAs.
struct RecomputeSave {
    int64_t t0, t1;
    __nv_bfloat16* hs;            // h_0 .. h_{L-2}, hs_stride elements apart
    int64_t hs_stride;
    __nv_bfloat16* xa;            // nodes: [rows x 2H]
    __nv_bfloat16* dz;            // gradient of the last pre-activation [rows x H]
    const float* da;              // edges: aggregate gradient after the halo adjoint
    const __nv_bfloat16* de_out;  // edges: upstream gradient of e' (NULL: zero)
    const float* dx_out;          // nodes: upstream gradient of x'
    float* part;
    int64_t pstride;
    int grid;                     // out
};
int edge_recompute_save(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                        const __nv_bfloat16* e_in, const __nv_bfloat16* pq, RecomputeSave& o, cudaStream_t s);
// The same recomputation in the two-group tensor-memory form (edge128.cu; 2..4 Linears).
int edge_save_tm(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const __nv_bfloat16* e_in,
                 const __nv_bfloat16* pq, RecomputeSave& o, cudaStream_t s);
int node_recompute_save(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                        const float* a_star, const float* x_in, RecomputeSave& o, cudaStream_t s);

// Projection adjoint of the BF16 backward: dQ from dz1 over each row's sent
// edges, dx_in += dP W1a + dQ W1b, dW1a and dW1b added into dW.edge.W[0].
int proj_backward(const gnn_graph_dev& G, int H, const gnn_mp_params& W, const float* x_in, const float* dP,
                  const __nv_bfloat16* dz1, float* dx_in, const gnn_mp_params& dW, float* part, cudaStream_t s);

// Layered BF16 backward at H = 128 (recomputation, per-Linear adjoint kernels).
size_t backward_h128_ws(const gnn_graph_dev& G, const gnn_mp_params& W);
int backward_h128(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                  const __nv_bfloat16* e_in, const float* a_star, const float* dx_out, const __nv_bfloat16* de_out,
                  float* dx_in, __nv_bfloat16* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes,
                  cudaStream_t s);

// The per-Linear adjoint k = L-1 .. 1 of an H = 128 MLP (bwd128.cu) over n_tiles
// tiles of tile-padded BF16 scratch rows: reads dz_{L-1} from dzs[*cur] and
// h_{k-1} from hs + (k - 1) hs_stride, adds dW_k, db_{k-1} into dW and leaves
// dz_0 in dzs[*cur] (each pass writes the other buffer and flips *cur). With
// `pairs`, Linears k and k-1 share a pass (k_bwd_chain2, dz_{k-1} kept on chip)
// while two remain, else one pass per Linear (k_bwd_chain); the results are the
// same bit for bit. part holds pstride >= 2 H (H + 1) floats for each CTA of a
// persistent grid (one CTA per SM). k_last > 1 stops after Linear k_last (dz_{k_last - 1}
// left in dzs[*cur]).
int chain_backward_h128(const gnn_mlp& W, const gnn_mlp& dW, __nv_bfloat16* hs, int64_t hs_stride,
                        __nv_bfloat16* const dzs[2], float* part, int64_t pstride, int64_t n_tiles, int* cur,
                        cudaStream_t s, bool pairs = true, int k_last = 1);
// The same kernel on the first Linear of a row MLP whose input X is data: with
// dz_0 and the BF16 copy of X in tile-padded scratch rows (row i of the scratch
// is row row0 + i of X), writes dX = dz_0 W_0 (FP32 [n_rows x H], rows below
// n_rows only) and adds dW_0 = dz_0^T X into dW0 ([H x H]).
int chain_input_h128(const float* W0, float* dW0, const __nv_bfloat16* dz, const __nv_bfloat16* xb, float* dx,
                     int64_t row0, int64_t n_rows, float* part, int64_t pstride, int64_t n_tiles, cudaStream_t s);

// Fused BF16 encoder row MLP at H = 128 (rowenc128.cu): in <= 16, 2..4 Linears
// of width 128, LayerNorm; the adjoint recomputes the activations layer by layer
// in a workspace of rowenc128_backward_ws bytes (smaller ones run in more chunks).
bool rowenc128_shape(const gnn_mlp& P);
size_t rowenc128_backward_ws(const gnn_mlp& P, int64_t n_rows);
int rowenc128_forward(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, float eps,
                      cudaStream_t s);
int rowenc128_backward(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                       const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s);

// Fused BF16 decoder row MLP at H = 128 (rowdec128.cu): in = hidden = 128, out <= 16,
// 2..4 Linears, no LayerNorm; workspace and chunking as the encoder's.
bool rowdec128_shape(const gnn_mlp& P);
size_t rowdec128_backward_ws(const gnn_mlp& P, int64_t n_rows);
int rowdec128_forward(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, cudaStream_t s);
int rowdec128_backward(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                       const gnn_mlp& dP, void* ws, size_t ws_bytes, cudaStream_t s);

// Fused BF16 row MLP (encoders / decoder of the network).
bool rowmlp_supported(const gnn_mlp& P);
size_t rowmlp_backward_ws(const gnn_mlp& P, int64_t n_rows);
// Bytes of a row MLP's saved activations (n_lin - 1 blocks of ceil(n_rows / 128)
// * 128 BF16 rows of H), 0 where none are kept.
size_t rowmlp_act_bytes(const gnn_mlp& P, int64_t n_rows);
int rowmlp_forward(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, float eps,
                   cudaStream_t s, __nv_bfloat16* act = nullptr);
int rowmlp_backward(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                    const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s,
                    const __nv_bfloat16* act = nullptr);

}  // namespace fused
}  // namespace gnn
