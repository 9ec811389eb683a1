// Autotuner of the fused BF16 layer forward (gnn_mp_autotune): times every
// launch choice of the edge forward on the caller's graph with CUDA events and
// keeps the fastest. The choices compute the same arithmetic, so the tuner
// picks a launch shape, never a different result.

#include <cuda_runtime.h>

#include <vector>

#include "device_common.cuh"

namespace {

struct Choice {
    int32_t kernel, ctas_per_sm;
};

std::vector<Choice> choices_for(int H) {
    std::vector<Choice> c;
    if (H <= 64) {
        c.push_back({GNN_EDGE_FWD_RT, 0});
        c.push_back({GNN_EDGE_FWD_WS, 0});
    }
    if (H == 128) c.push_back({GNN_EDGE_FWD_TM, 0});
    c.push_back({GNN_EDGE_FWD_ONE, 0});
    c.push_back({GNN_EDGE_FWD_ONE, 1});
    return c;
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" int gnn_mp_autotune(const gnn_graph_dev* G, gnn_mp_config* cfg, const gnn_mp_params* W,
                               const float* x_in, const void* e_in, float* x_out, void* e_out, float* a_star_out,
                               void* ws, size_t ws_bytes, int32_t reps, gnn_tune_entry* out, int32_t max_out,
                               int32_t* n_out, void* stream) {
    GNN_REQUIRE(cfg, GNN_EINVAL, "gnn_mp_autotune: NULL config");
    GNN_REQUIRE(cfg->precision == GNN_PREC_BF16, GNN_EDTYPE, "gnn_mp_autotune: only the BF16 path has launch choices");
    GNN_REQUIRE(reps >= 1 && reps <= 1000, GNN_EINVAL, "gnn_mp_autotune: reps %d outside 1..1000", reps);
    GNN_REQUIRE(max_out >= 0 && (out || max_out == 0), GNN_EINVAL, "gnn_mp_autotune: bad output array");
    if (n_out) *n_out = 0;
    cudaStream_t s = (cudaStream_t)stream;
    Events ev;
    GNN_CUDA_CHECK(cudaEventCreate(&ev.a), "cudaEventCreate");
    GNN_CUDA_CHECK(cudaEventCreate(&ev.b), "cudaEventCreate");
    gnn_mp_config best = *cfg;
    float best_ms = -1.f;
    int32_t written = 0;
    for (const Choice& c : choices_for(cfg->hidden)) {
        gnn_mp_config k = *cfg;
        k.edge_fwd_kernel = c.kernel;
        k.ctas_per_sm = c.ctas_per_sm;
        int rc = gnn_mp_forward(G, &k, W, x_in, e_in, x_out, e_out, a_star_out, ws, ws_bytes, stream);
        if (rc == GNN_EUNSUPPORTED) continue;   // does not fit this configuration
        if (rc) return rc;
        GNN_CUDA_CHECK(cudaEventRecord(ev.a, s), "cudaEventRecord");
        for (int r = 0; r < reps; ++r) {
            rc = gnn_mp_forward(G, &k, W, x_in, e_in, x_out, e_out, a_star_out, ws, ws_bytes, stream);
            if (rc) return rc;
        }
        GNN_CUDA_CHECK(cudaEventRecord(ev.b, s), "cudaEventRecord");
        GNN_CUDA_CHECK(cudaEventSynchronize(ev.b), "cudaEventSynchronize");
        rc = gnn_check(stream);
        if (rc) return rc;
        float ms = 0.f;
        GNN_CUDA_CHECK(cudaEventElapsedTime(&ms, ev.a, ev.b), "cudaEventElapsedTime");
        ms /= (float)reps;
        if (written < max_out) out[written++] = gnn_tune_entry{c.kernel, c.ctas_per_sm, ms};
        if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    GNN_REQUIRE(best_ms >= 0.f, GNN_EUNSUPPORTED, "gnn_mp_autotune: no launch choice fits");
    cfg->edge_fwd_kernel = best.edge_fwd_kernel;
    cfg->ctas_per_sm = best.ctas_per_sm;
    if (n_out) *n_out = written;
    return GNN_OK;
}
