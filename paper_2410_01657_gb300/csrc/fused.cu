// Fused BF16 path of libgnnmp (tcgen05 / TMEM kernels).
#include "device_common.cuh"
#include "fused.h"

namespace gnn {
namespace fused {

cudaError_t take_device_error(unsigned int* out) { return take_device_error_word(out); }

size_t mp_forward_ws(const gnn_graph_dev&, const gnn_mp_config&, const gnn_mp_params&) { return 0; }
size_t mp_backward_ws(const gnn_graph_dev&, const gnn_mp_config&, const gnn_mp_params&) { return 0; }

int mp_forward(const gnn_graph_dev&, const gnn_mp_config&, const gnn_mp_params&, const float*,
               const __nv_bfloat16*, float*, __nv_bfloat16*, float*, void*, size_t, cudaStream_t) {
    return set_error(GNN_EUNSUPPORTED, "gnn_mp_forward: BF16 fused path not built yet");
}

int mp_backward(const gnn_graph_dev&, const gnn_mp_config&, const gnn_mp_params&, const float*,
                const __nv_bfloat16*, const float*, const float*, const __nv_bfloat16*, float*, __nv_bfloat16*,
                const gnn_mp_params&, void*, size_t, cudaStream_t) {
    return set_error(GNN_EUNSUPPORTED, "gnn_mp_backward: BF16 fused path not built yet");
}

}  // namespace fused
}  // namespace gnn
