// C-ABI compute entry points of libgnnmp: argument validation and dispatch to
// the plain FP32 path (plain.cu) or the fused BF16 tcgen05 path (fused.cu).

#include <cstdio>
#include <cstring>

#include "device_common.cuh"
#include "fused.h"
#include "plain.h"
#include "diag.h"

namespace {

using gnn::set_error;

int check_graph(const gnn_graph_dev* G, const char* fn) {
    GNN_REQUIRE(G, GNN_EINVAL, "%s: NULL graph", fn);
    GNN_REQUIRE(G->n_rows >= 0 && G->n_edges >= 0 && G->n_shared >= 0 && G->n_edge_tiles >= 0, GNN_ESHAPE,
                "%s: negative size", fn);
    GNN_REQUIRE(G->n_rows < (int64_t)1 << 31 && G->n_edges < (int64_t)1 << 31, GNN_ESHAPE,
                "%s: more than 2^31-1 rows or edges", fn);
    if (G->n_rows) GNN_REQUIRE(G->row_ptr && G->t_ptr && G->node_w, GNN_EINVAL, "%s: NULL row arrays", fn);
    if (G->n_edges) GNN_REQUIRE(G->col && G->edge_w && G->t_eid, GNN_EINVAL, "%s: NULL edge arrays", fn);
    if (G->n_shared) GNN_REQUIRE(G->halo_ptr && G->halo_rows, GNN_EINVAL, "%s: NULL halo arrays", fn);
    return GNN_OK;
}

int check_mlp(const gnn_mlp& P, int in, int hidden, int out, bool ln, const char* fn, const char* which) {
    GNN_REQUIRE(P.n_lin >= 2 && P.n_lin <= GNN_MAX_LIN, GNN_ESHAPE, "%s: %s MLP needs 2..%d Linear layers", fn,
                which, GNN_MAX_LIN);
    GNN_REQUIRE(P.dims[0] == in, GNN_ESHAPE, "%s: %s MLP input width %d, expected %d", fn, which, P.dims[0], in);
    GNN_REQUIRE(P.dims[P.n_lin] == out, GNN_ESHAPE, "%s: %s MLP output width %d, expected %d", fn, which,
                P.dims[P.n_lin], out);
    for (int k = 1; k < P.n_lin; ++k)
        GNN_REQUIRE(hidden <= 0 || P.dims[k] == hidden, GNN_ESHAPE, "%s: %s MLP hidden width %d, expected %d", fn,
                    which, P.dims[k], hidden);
    for (int k = 0; k < P.n_lin; ++k) {
        GNN_REQUIRE(P.dims[k] >= 1 && P.dims[k] <= 1024, GNN_ESHAPE, "%s: %s MLP width out of range", fn, which);
        GNN_REQUIRE(P.W[k] && P.b[k], GNN_EINVAL, "%s: %s MLP layer %d has NULL parameters", fn, which, k);
    }
    if (ln) GNN_REQUIRE(P.gamma && P.beta, GNN_EINVAL, "%s: %s MLP needs LayerNorm parameters", fn, which);
    if (P.gamma) GNN_REQUIRE(P.dims[P.n_lin] <= 256, GNN_ESHAPE, "%s: LayerNorm width > 256", fn);
    return GNN_OK;
}

int check_cfg(const gnn_mp_config* cfg, const gnn_mp_params* W, const char* fn) {
    GNN_REQUIRE(cfg && W, GNN_EINVAL, "%s: NULL config or parameters", fn);
    GNN_REQUIRE(cfg->precision == GNN_PREC_FP32 || cfg->precision == GNN_PREC_BF16, GNN_EDTYPE,
                "%s: unknown precision %d", fn, cfg->precision);
    GNN_REQUIRE(cfg->halo_mode == GNN_HALO_SYNC || cfg->halo_mode == GNN_HALO_NONE, GNN_EINVAL,
                "%s: unknown halo mode %d", fn, cfg->halo_mode);
    GNN_REQUIRE(cfg->ln_eps > 0.f, GNN_EINVAL, "%s: ln_eps must be positive", fn);
    const int H = cfg->hidden;
    GNN_REQUIRE(cfg->edge_fwd_kernel >= GNN_EDGE_FWD_AUTO && cfg->edge_fwd_kernel <= GNN_EDGE_FWD_TM, GNN_EINVAL,
                "%s: unknown edge forward kernel %d", fn, cfg->edge_fwd_kernel);
    GNN_REQUIRE(cfg->precision != GNN_PREC_BF16 || H <= 64 ||
                    (cfg->edge_fwd_kernel != GNN_EDGE_FWD_RT && cfg->edge_fwd_kernel != GNN_EDGE_FWD_WS),
                GNN_EUNSUPPORTED, "%s: edge forward kernel %d needs H <= 64", fn, cfg->edge_fwd_kernel);
    GNN_REQUIRE(cfg->precision != GNN_PREC_BF16 || H == 128 || cfg->edge_fwd_kernel != GNN_EDGE_FWD_TM,
                GNN_EUNSUPPORTED, "%s: edge forward kernel %d needs H = 128", fn, cfg->edge_fwd_kernel);
    GNN_REQUIRE(cfg->ctas_per_sm >= 0 && cfg->ctas_per_sm <= 32, GNN_EINVAL, "%s: ctas_per_sm %d out of range",
                fn, cfg->ctas_per_sm);
    if (cfg->precision == GNN_PREC_FP32)
        GNN_REQUIRE(H >= 1 && H <= 256, GNN_ESHAPE, "%s: FP32 path needs 1 <= H <= 256 (H=%d)", fn, H);
    else
        GNN_REQUIRE(H == 16 || H == 32 || H == 64 || H == 128, GNN_ESHAPE,
                    "%s: BF16 path needs H in {16,32,64,128} (H=%d)", fn, H);
    int rc = check_mlp(W->edge, 3 * H, H, H, true, fn, "edge");
    if (rc) return rc;
    return check_mlp(W->node, 2 * H, H, H, true, fn, "node");
}

}  // namespace

extern "C" {

int gnn_check(void* stream) {
    GNN_CUDA_CHECK(cudaStreamSynchronize((cudaStream_t)stream), "gnn_check: stream synchronize");
    // every translation unit with waiting kernels has its own error word
    cudaError_t (*const take[])(unsigned int*) = {
        gnn::plain::take_device_error, gnn::fused::take_device_error, gnn::fused::take_device_error_bwd,
        gnn::fused::take_device_error_bwd128, gnn::fused::take_device_error_rowmlp,
        gnn::fused::take_device_error_edge128, gnn::fused::take_device_error_rowenc128,
        gnn::fused::take_device_error_rowdec128, gnn::fused::take_device_error_node128,
        gnn::diag::take_device_error};
    const char* const unit[] = {"plain", "fused", "fused_bwd", "bwd128", "rowmlp", "edge128", "rowenc128",
                                "rowdec128", "node128", "diag"};
    static_assert(sizeof(unit) / sizeof(unit[0]) == sizeof(take) / sizeof(take[0]), "one name per unit");
    unsigned int word = 0;
    char where[160] = "";
    size_t n = 0;
    for (size_t i = 0; i < sizeof(take) / sizeof(take[0]); ++i) {
        unsigned int w = 0;
        GNN_CUDA_CHECK(take[i](&w), "gnn_check: read error word");
        word |= w;
        if ((w & GNN_DEVERR_TIMEOUT) && n + 16 < sizeof(where))
            n += (size_t)snprintf(where + n, sizeof(where) - n, "%s%s", n ? ", " : "", unit[i]);
    }
    if (word & GNN_DEVERR_TIMEOUT)
        return set_error(GNN_ETIMEOUT, "gnn_check: a device-side wait timed out (in the kernels of %s)", where);
    return GNN_OK;
}

int gnn_mp_workspace_size(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                          size_t* fwd_bytes, size_t* bwd_bytes) {
    int rc = check_graph(G, "gnn_mp_workspace_size");
    if (rc) return rc;
    if ((rc = check_cfg(cfg, W, "gnn_mp_workspace_size"))) return rc;
    GNN_REQUIRE(fwd_bytes && bwd_bytes, GNN_EINVAL, "gnn_mp_workspace_size: NULL output");
    if (cfg->precision == GNN_PREC_FP32) {
        *fwd_bytes = gnn::plain::mp_forward_ws(*G, *cfg, *W);
        *bwd_bytes = gnn::plain::mp_backward_ws(*G, *cfg, *W);
    } else {
        *fwd_bytes = gnn::fused::mp_forward_ws(*G, *cfg, *W);
        *bwd_bytes = gnn::fused::mp_backward_ws(*G, *cfg, *W);
    }
    return GNN_OK;
}

int gnn_mp_act_size(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W, size_t* bytes) {
    int rc = check_graph(G, "gnn_mp_act_size");
    if (rc) return rc;
    if ((rc = check_cfg(cfg, W, "gnn_mp_act_size"))) return rc;
    GNN_REQUIRE(bytes, GNN_EINVAL, "gnn_mp_act_size: NULL output");
    *bytes = gnn::fused::mp_act_bytes(*G, *cfg, *W);
    return GNN_OK;
}

static int check_act(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W, const void* act,
                     const char* fn) {
    if (gnn::fused::mp_act_bytes(*G, *cfg, *W) == 0 || G->n_edges == 0) return GNN_OK;
    GNN_REQUIRE(act && ((uintptr_t)act & 15) == 0, GNN_EINVAL, "%s: act must be a 16-byte aligned device buffer",
                fn);
    return GNN_OK;
}

int gnn_mp_forward_act(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                       const float* x_in, const void* e_in, float* x_out, void* e_out, float* a_star_out, void* act,
                       void* ws, size_t ws_bytes, void* stream) {
    int rc = check_graph(G, "gnn_mp_forward_act");
    if (rc) return rc;
    if ((rc = check_cfg(cfg, W, "gnn_mp_forward_act"))) return rc;
    if ((rc = check_act(G, cfg, W, act, "gnn_mp_forward_act"))) return rc;
    if (cfg->precision == GNN_PREC_FP32 || gnn::fused::mp_act_bytes(*G, *cfg, *W) == 0)
        return gnn_mp_forward(G, cfg, W, x_in, e_in, x_out, e_out, a_star_out, ws, ws_bytes, stream);
    if (G->n_rows) GNN_REQUIRE(x_in && x_out, GNN_EINVAL, "gnn_mp_forward_act: NULL node buffer");
    if (G->n_edges) GNN_REQUIRE(e_in, GNN_EINVAL, "gnn_mp_forward_act: NULL e_in");
    GNN_REQUIRE(e_out || (cfg->flags & GNN_FLAG_NO_EDGE_OUT) || G->n_edges == 0, GNN_EINVAL,
                "gnn_mp_forward_act: NULL e_out without GNN_FLAG_NO_EDGE_OUT");
    GNN_REQUIRE(x_out != x_in || G->n_rows == 0, GNN_EINVAL, "gnn_mp_forward_act: x_out aliases x_in");
    GNN_REQUIRE(ws || ws_bytes == 0, GNN_EINVAL, "gnn_mp_forward_act: NULL workspace");
    return gnn::fused::mp_forward(*G, *cfg, *W, x_in, (const __nv_bfloat16*)e_in, x_out, (__nv_bfloat16*)e_out,
                                  a_star_out, ws, ws_bytes, (cudaStream_t)stream, (__nv_bfloat16*)act);
}

int gnn_mp_backward_act(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                        const float* x_in, const void* e_in, const float* a_star, const void* act,
                        const float* dx_out, const void* de_out, float* dx_in, void* de_in, const gnn_mp_params* dW,
                        void* ws, size_t ws_bytes, void* stream) {
    int rc = check_graph(G, "gnn_mp_backward_act");
    if (rc) return rc;
    if ((rc = check_cfg(cfg, W, "gnn_mp_backward_act"))) return rc;
    if ((rc = check_act(G, cfg, W, act, "gnn_mp_backward_act"))) return rc;
    if (cfg->precision == GNN_PREC_FP32 || gnn::fused::mp_act_bytes(*G, *cfg, *W) == 0)
        return gnn_mp_backward(G, cfg, W, x_in, e_in, a_star, dx_out, de_out, dx_in, de_in, dW, ws, ws_bytes,
                               stream);
    GNN_REQUIRE(dW, GNN_EINVAL, "gnn_mp_backward_act: NULL gradient struct");
    if ((rc = check_cfg(cfg, dW, "gnn_mp_backward_act(dW)"))) return rc;
    if (G->n_rows) GNN_REQUIRE(x_in && dx_out && dx_in, GNN_EINVAL, "gnn_mp_backward_act: NULL node buffer");
    if (G->n_edges) GNN_REQUIRE(e_in && de_in, GNN_EINVAL, "gnn_mp_backward_act: NULL edge buffer");
    GNN_REQUIRE(ws || ws_bytes == 0, GNN_EINVAL, "gnn_mp_backward_act: NULL workspace");
    return gnn::fused::mp_backward(*G, *cfg, *W, x_in, (const __nv_bfloat16*)e_in, a_star, dx_out,
                                   (const __nv_bfloat16*)de_out, dx_in, (__nv_bfloat16*)de_in, *dW, ws, ws_bytes,
                                   (cudaStream_t)stream, (const __nv_bfloat16*)act);
}

int gnn_mp_forward(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W, const float* x_in,
                   const void* e_in, float* x_out, void* e_out, float* a_star_out, void* ws, size_t ws_bytes,
                   void* stream) {
    int rc = check_graph(G, "gnn_mp_forward");
    if (rc) return rc;
    if ((rc = check_cfg(cfg, W, "gnn_mp_forward"))) return rc;
    if (G->n_rows) GNN_REQUIRE(x_in && x_out, GNN_EINVAL, "gnn_mp_forward: NULL node buffer");
    if (G->n_edges) GNN_REQUIRE(e_in, GNN_EINVAL, "gnn_mp_forward: NULL e_in");
    GNN_REQUIRE(e_out || (cfg->flags & GNN_FLAG_NO_EDGE_OUT) || G->n_edges == 0, GNN_EINVAL,
                "gnn_mp_forward: NULL e_out without GNN_FLAG_NO_EDGE_OUT");
    GNN_REQUIRE(x_out != x_in || G->n_rows == 0, GNN_EINVAL, "gnn_mp_forward: x_out aliases x_in");
    GNN_REQUIRE(ws || ws_bytes == 0, GNN_EINVAL, "gnn_mp_forward: NULL workspace");
    cudaStream_t s = (cudaStream_t)stream;
    if (cfg->precision == GNN_PREC_FP32)
        return gnn::plain::mp_forward(*G, *cfg, *W, x_in, (const float*)e_in, x_out, (float*)e_out, a_star_out, ws,
                                      ws_bytes, s);
    return gnn::fused::mp_forward(*G, *cfg, *W, x_in, (const __nv_bfloat16*)e_in, x_out, (__nv_bfloat16*)e_out,
                                  a_star_out, ws, ws_bytes, s);
}

int gnn_mp_backward(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W, const float* x_in,
                    const void* e_in, const float* a_star, const float* dx_out, const void* de_out, float* dx_in,
                    void* de_in, const gnn_mp_params* dW, void* ws, size_t ws_bytes, void* stream) {
    int rc = check_graph(G, "gnn_mp_backward");
    if (rc) return rc;
    if ((rc = check_cfg(cfg, W, "gnn_mp_backward"))) return rc;
    GNN_REQUIRE(dW, GNN_EINVAL, "gnn_mp_backward: NULL gradient struct");
    if ((rc = check_cfg(cfg, dW, "gnn_mp_backward(dW)"))) return rc;
    if (G->n_rows) GNN_REQUIRE(x_in && dx_out && dx_in, GNN_EINVAL, "gnn_mp_backward: NULL node buffer");
    if (G->n_edges) GNN_REQUIRE(e_in && de_in, GNN_EINVAL, "gnn_mp_backward: NULL edge buffer");
    GNN_REQUIRE(ws || ws_bytes == 0, GNN_EINVAL, "gnn_mp_backward: NULL workspace");
    cudaStream_t s = (cudaStream_t)stream;
    if (cfg->precision == GNN_PREC_FP32)
        return gnn::plain::mp_backward(*G, *cfg, *W, x_in, (const float*)e_in, a_star, dx_out, (const float*)de_out,
                                       dx_in, (float*)de_in, *dW, ws, ws_bytes, s);
    return gnn::fused::mp_backward(*G, *cfg, *W, x_in, (const __nv_bfloat16*)e_in, a_star, dx_out,
                                   (const __nv_bfloat16*)de_out, dx_in, (__nv_bfloat16*)de_in, *dW, ws, ws_bytes, s);
}

int gnn_mp_forward_static(const gnn_graph_dev* G, const gnn_mp_config* cfg, const gnn_mp_params* W,
                          const float* x_in, const void* e_in, float* x_out, void* e_out, float* a_star_out,
                          void* stream) {
    int rc = check_graph(G, "gnn_mp_forward_static");
    if (rc) return rc;
    if ((rc = check_cfg(cfg, W, "gnn_mp_forward_static"))) return rc;
    GNN_REQUIRE(cfg->precision == GNN_PREC_BF16, GNN_EDTYPE,
                "gnn_mp_forward_static: only the BF16 fused path has a built-in scratch area");
    if (G->n_rows) GNN_REQUIRE(x_in && x_out, GNN_EINVAL, "gnn_mp_forward_static: NULL node buffer");
    if (G->n_edges) GNN_REQUIRE(e_in, GNN_EINVAL, "gnn_mp_forward_static: NULL e_in");
    GNN_REQUIRE(e_out || (cfg->flags & GNN_FLAG_NO_EDGE_OUT) || G->n_edges == 0, GNN_EINVAL,
                "gnn_mp_forward_static: NULL e_out without GNN_FLAG_NO_EDGE_OUT");
    GNN_REQUIRE(x_out != x_in || G->n_rows == 0, GNN_EINVAL, "gnn_mp_forward_static: x_out aliases x_in");
    return gnn::fused::mp_forward_static(*G, *cfg, *W, x_in, (const __nv_bfloat16*)e_in, x_out,
                                         (__nv_bfloat16*)e_out, a_star_out, (cudaStream_t)stream);
}

int gnn_halo_exchange(const gnn_graph_dev* G, float* rows, int32_t width, void* stream) {
    int rc = check_graph(G, "gnn_halo_exchange");
    if (rc) return rc;
    GNN_REQUIRE(width >= 0, GNN_EINVAL, "gnn_halo_exchange: negative width");
    GNN_REQUIRE(rows || G->n_rows == 0, GNN_EINVAL, "gnn_halo_exchange: NULL rows");
    return gnn::plain::halo(*G, rows, width, (cudaStream_t)stream);
}

int gnn_mlp_workspace_size(const gnn_mlp* P, int64_t n_rows, size_t* fwd_bytes, size_t* bwd_bytes) {
    GNN_REQUIRE(P && fwd_bytes && bwd_bytes, GNN_EINVAL, "gnn_mlp_workspace_size: NULL argument");
    GNN_REQUIRE(n_rows >= 0, GNN_ESHAPE, "gnn_mlp_workspace_size: negative rows");
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_workspace_size", "row");
    if (rc) return rc;
    *fwd_bytes = gnn::plain::mlp_ws(*P, n_rows, false);
    *bwd_bytes = gnn::plain::mlp_ws(*P, n_rows, true);
    return GNN_OK;
}

int gnn_mlp_forward(const gnn_mlp* P, int64_t n_rows, const float* X, void* Y, int32_t y_bf16, float ln_eps,
                    void* ws, size_t ws_bytes, void* stream) {
    GNN_REQUIRE(P, GNN_EINVAL, "gnn_mlp_forward: NULL parameters");
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_forward", "row");
    if (rc) return rc;
    GNN_REQUIRE(n_rows >= 0, GNN_ESHAPE, "gnn_mlp_forward: negative rows");
    if (n_rows) GNN_REQUIRE(X && Y && ws, GNN_EINVAL, "gnn_mlp_forward: NULL buffer");
    GNN_REQUIRE(ln_eps > 0.f, GNN_EINVAL, "gnn_mlp_forward: ln_eps must be positive");
    return gnn::plain::mlp_forward(*P, n_rows, X, Y, y_bf16, ln_eps, ws, ws_bytes, (cudaStream_t)stream);
}

int gnn_mlp_backward(const gnn_mlp* P, int64_t n_rows, const float* X, const void* dY, int32_t dy_bf16, float* dX,
                     const gnn_mlp* dP, float ln_eps, void* ws, size_t ws_bytes, void* stream) {
    GNN_REQUIRE(P && dP, GNN_EINVAL, "gnn_mlp_backward: NULL parameters");
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_backward", "row");
    if (rc) return rc;
    if ((rc = check_mlp(*dP, P->dims[0], 0, P->dims[P->n_lin], P->gamma != nullptr, "gnn_mlp_backward", "grad")))
        return rc;
    GNN_REQUIRE(n_rows >= 0, GNN_ESHAPE, "gnn_mlp_backward: negative rows");
    if (n_rows) GNN_REQUIRE(X && dY && ws, GNN_EINVAL, "gnn_mlp_backward: NULL buffer");
    GNN_REQUIRE(ln_eps > 0.f, GNN_EINVAL, "gnn_mlp_backward: ln_eps must be positive");
    return gnn::plain::mlp_backward(*P, n_rows, X, dY, dy_bf16, dX, *dP, ln_eps, ws, ws_bytes, (cudaStream_t)stream);
}

int gnn_mlp_workspace_size_bf16(const gnn_mlp* P, int64_t n_rows, size_t* fwd_bytes, size_t* bwd_bytes) {
    GNN_REQUIRE(P && fwd_bytes && bwd_bytes, GNN_EINVAL, "gnn_mlp_workspace_size_bf16: NULL argument");
    GNN_REQUIRE(n_rows >= 0, GNN_ESHAPE, "gnn_mlp_workspace_size_bf16: negative rows");
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_workspace_size_bf16", "row");
    if (rc) return rc;
    GNN_REQUIRE(gnn::fused::rowmlp_supported(*P), GNN_EUNSUPPORTED,
                "gnn_mlp_workspace_size_bf16: shape not covered by the fused row MLP");
    *fwd_bytes = 0;
    *bwd_bytes = gnn::fused::rowmlp_backward_ws(*P, n_rows);
    return GNN_OK;
}

int gnn_mlp_forward_bf16(const gnn_mlp* P, int64_t n_rows, const float* X, void* Y, int32_t y_bf16, float ln_eps,
                         void* ws, size_t ws_bytes, void* stream) {
    GNN_REQUIRE(P, GNN_EINVAL, "gnn_mlp_forward_bf16: NULL parameters");
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_forward_bf16", "row");
    if (rc) return rc;
    GNN_REQUIRE(n_rows >= 0, GNN_ESHAPE, "gnn_mlp_forward_bf16: negative rows");
    if (n_rows) GNN_REQUIRE(X && Y, GNN_EINVAL, "gnn_mlp_forward_bf16: NULL buffer");
    GNN_REQUIRE(ln_eps > 0.f, GNN_EINVAL, "gnn_mlp_forward_bf16: ln_eps must be positive");
    GNN_REQUIRE(n_rows < (int64_t)1 << 31, GNN_ESHAPE, "gnn_mlp_forward_bf16: more than 2^31-1 rows");
    (void)ws;
    (void)ws_bytes;
    return gnn::fused::rowmlp_forward(*P, n_rows, X, Y, y_bf16, ln_eps, (cudaStream_t)stream);
}

int gnn_mlp_backward_bf16(const gnn_mlp* P, int64_t n_rows, const float* X, const void* dY, int32_t dy_bf16,
                          float* dX, const gnn_mlp* dP, float ln_eps, void* ws, size_t ws_bytes, void* stream) {
    GNN_REQUIRE(P && dP, GNN_EINVAL, "gnn_mlp_backward_bf16: NULL parameters");
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_backward_bf16", "row");
    if (rc) return rc;
    if ((rc = check_mlp(*dP, P->dims[0], 0, P->dims[P->n_lin], P->gamma != nullptr, "gnn_mlp_backward_bf16", "grad")))
        return rc;
    GNN_REQUIRE(n_rows >= 0, GNN_ESHAPE, "gnn_mlp_backward_bf16: negative rows");
    if (n_rows) GNN_REQUIRE(X && dY && ws, GNN_EINVAL, "gnn_mlp_backward_bf16: NULL buffer");
    GNN_REQUIRE(ln_eps > 0.f, GNN_EINVAL, "gnn_mlp_backward_bf16: ln_eps must be positive");
    GNN_REQUIRE(n_rows < (int64_t)1 << 31, GNN_ESHAPE, "gnn_mlp_backward_bf16: more than 2^31-1 rows");
    return gnn::fused::rowmlp_backward(*P, n_rows, X, dY, dy_bf16, dX, *dP, ln_eps, ws, ws_bytes,
                                       (cudaStream_t)stream);
}

int gnn_mlp_act_size_bf16(const gnn_mlp* P, int64_t n_rows, size_t* bytes) {
    GNN_REQUIRE(P && bytes, GNN_EINVAL, "gnn_mlp_act_size_bf16: NULL argument");
    GNN_REQUIRE(n_rows >= 0, GNN_ESHAPE, "gnn_mlp_act_size_bf16: negative rows");
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_act_size_bf16", "row");
    if (rc) return rc;
    *bytes = gnn::fused::rowmlp_act_bytes(*P, n_rows);
    return GNN_OK;
}

int gnn_mlp_forward_bf16_act(const gnn_mlp* P, int64_t n_rows, const float* X, void* Y, int32_t y_bf16, float ln_eps,
                             void* act, void* stream) {
    GNN_REQUIRE(P, GNN_EINVAL, "gnn_mlp_forward_bf16_act: NULL parameters");
    if (gnn::fused::rowmlp_act_bytes(*P, n_rows))
        GNN_REQUIRE(act && ((uintptr_t)act & 15) == 0, GNN_EINVAL,
                    "gnn_mlp_forward_bf16_act: act must be a 16-byte aligned device buffer");
    else
        act = nullptr;
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_forward_bf16_act", "row");
    if (rc) return rc;
    GNN_REQUIRE(n_rows >= 0 && n_rows < (int64_t)1 << 31, GNN_ESHAPE, "gnn_mlp_forward_bf16_act: rows out of range");
    if (n_rows) GNN_REQUIRE(X && Y, GNN_EINVAL, "gnn_mlp_forward_bf16_act: NULL buffer");
    GNN_REQUIRE(ln_eps > 0.f, GNN_EINVAL, "gnn_mlp_forward_bf16_act: ln_eps must be positive");
    return gnn::fused::rowmlp_forward(*P, n_rows, X, Y, y_bf16, ln_eps, (cudaStream_t)stream, (__nv_bfloat16*)act);
}

int gnn_mlp_backward_bf16_act(const gnn_mlp* P, int64_t n_rows, const float* X, const void* dY, int32_t dy_bf16,
                              float* dX, const gnn_mlp* dP, float ln_eps, const void* act, void* ws, size_t ws_bytes,
                              void* stream) {
    GNN_REQUIRE(P && dP, GNN_EINVAL, "gnn_mlp_backward_bf16_act: NULL parameters");
    if (gnn::fused::rowmlp_act_bytes(*P, n_rows))
        GNN_REQUIRE(act && ((uintptr_t)act & 15) == 0, GNN_EINVAL,
                    "gnn_mlp_backward_bf16_act: act must be a 16-byte aligned device buffer");
    else
        act = nullptr;
    int rc = check_mlp(*P, P->dims[0], 0, P->dims[P->n_lin], false, "gnn_mlp_backward_bf16_act", "row");
    if (rc) return rc;
    if ((rc = check_mlp(*dP, P->dims[0], 0, P->dims[P->n_lin], P->gamma != nullptr, "gnn_mlp_backward_bf16_act",
                        "grad")))
        return rc;
    GNN_REQUIRE(n_rows >= 0 && n_rows < (int64_t)1 << 31, GNN_ESHAPE, "gnn_mlp_backward_bf16_act: rows out of range");
    if (n_rows) GNN_REQUIRE(X && dY && ws, GNN_EINVAL, "gnn_mlp_backward_bf16_act: NULL buffer");
    GNN_REQUIRE(ln_eps > 0.f, GNN_EINVAL, "gnn_mlp_backward_bf16_act: ln_eps must be positive");
    return gnn::fused::rowmlp_backward(*P, n_rows, X, dY, dy_bf16, dX, *dP, ln_eps, ws, ws_bytes,
                                       (cudaStream_t)stream, (const __nv_bfloat16*)act);
}

int gnn_consistent_loss(const gnn_graph_dev* G, const float* y, const float* t, int32_t F, float* loss, float* dy,
                        void* ws, size_t ws_bytes, void* stream) {
    int rc = check_graph(G, "gnn_consistent_loss");
    if (rc) return rc;
    GNN_REQUIRE(F >= 1, GNN_ESHAPE, "gnn_consistent_loss: F must be >= 1");
    GNN_REQUIRE(loss && ws, GNN_EINVAL, "gnn_consistent_loss: NULL loss or workspace");
    if (G->n_rows) GNN_REQUIRE(y && t, GNN_EINVAL, "gnn_consistent_loss: NULL y or t");
    return gnn::plain::consistent_loss(*G, y, t, F, loss, dy, ws, ws_bytes, (cudaStream_t)stream);
}

int gnn_measure_fp32_fma(double* tflops, int32_t* sm_count, void* stream) {
    GNN_REQUIRE(tflops && sm_count, GNN_EINVAL, "gnn_measure_fp32_fma: NULL output");
    return gnn::diag::measure_fp32_fma(tflops, sm_count, (cudaStream_t)stream);
}

int gnn_selftest_bounded_wait(uint64_t limit_ns, int32_t* status, void* stream) {
    GNN_REQUIRE(status, GNN_EINVAL, "gnn_selftest_bounded_wait: NULL status");
    GNN_REQUIRE(limit_ns >= 1000 && limit_ns <= 1000000000ull, GNN_EINVAL,
                "gnn_selftest_bounded_wait: limit %llu ns outside [1 us, 1 s]", (unsigned long long)limit_ns);
    return gnn::diag::selftest_bounded_wait(limit_ns, status, (cudaStream_t)stream);
}

}  // extern "C"
