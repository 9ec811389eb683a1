// Fused BF16 row MLP of libgnnmp (the node and edge encoders and the node
// decoder of the encode-process-decode network, Sec. III): Y = MLP(X) over
// tiles of 128 rows with the Linear chain on tcgen05 (BF16 operands, FP32
// accumulation in TMEM) and the bias / ELU / LayerNorm epilogues in FP32, and
// its adjoint with per-tile recomputation of the activations.
//
// Two shapes are covered, fixed at compile time, for H in {16, 32, 64}:
//   encoder  in_dim <= 16 (padded to 16), hidden H, out H, LayerNorm;
//   decoder  in_dim = H, hidden H, out_dim <= 16 (padded to 16), no LayerNorm.
// At H = 128 (2..4 Linears) the encoder runs in rowenc128.cu and the decoder in
// rowdec128.cu. Other shapes stay on the plain FP32 path (gnn_mlp_* with
// GNN_PREC_FP32).

#include <algorithm>
#include <cstring>

#include "fused.h"
#include "fused_bwd_common.cuh"
#include "profiler.h"

namespace gnn {
namespace fused {

cudaError_t take_device_error_rowmlp(unsigned int* out) { return take_device_error_word(out); }

using namespace tc;

struct RowMlpArgs {
    const float* X;
    int64_t n_rows;
    int K0;                     // input width (<= KP)
    int N_out;                  // output width (<= NP)
    void* Y;                    // forward output [n_rows x N_out], FP32 or BF16
    int y_bf16;
    const void* dY;             // backward: gradient of Y [n_rows x N_out], FP32 or BF16
    int dy_bf16;
    float* dX;                  // backward: gradient of X [n_rows x K0] or NULL
    float* part;                // backward: per-CTA weight-gradient partials
    int64_t pstride;
    MlpDev mlp;
    float eps;
    int64_t act_rows;           // saved activations: rows of one block of tmap_h (tiles * 128)
};

// ------------------------------------------------------------------ forward

struct RowFwdSmem {
    uint32_t w0, wm, wl, a0, a1, par, red, bar, tm, total;
};

// W0 [H x KP], hidden weights (n_lin-2) x [H x H], last weight [NP x H], the
// input tile [128 x KP], the activation tile [128 x H], biases / LayerNorm
// parameters, LayerNorm row partials.
template <int H, int KP, int NP>
__host__ __device__ inline RowFwdSmem rowmlp_fwd_smem(int n_lin) {
    RowFwdSmem s;
    s.w0 = 0;
    s.wm = align_up(s.w0 + H * KP * 2, 1024);
    s.wl = align_up(s.wm + (n_lin - 2) * H * H * 2, 1024);
    s.a0 = align_up(s.wl + NP * H * 2, 1024);
    s.a1 = align_up(s.a0 + 128 * KP * 2, 1024);
    s.par = s.a1 + 128 * H * 2;
    s.red = s.par + ((n_lin - 1) * H + 3 * NP) * 4;
    s.bar = align_up(s.red + 2 * (H / 16) * 128 * 4, 8);
    s.tm = s.bar + 8;
    s.total = s.tm + 16 + 1024;
    return s;
}

// The X row of this thread's row into the input tile (KP = 16: column group 0
// holds the whole padded row; KP = H: each thread its own columns).
template <int KP, int CW, int CG>
__device__ __forceinline__ void load_input_row(uint8_t* sA0, const float* X, int64_t r, bool valid, int K0, int row,
                                               int cg, int c0) {
    if constexpr (KP == 16) {
        if (cg == 0) {
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = (valid && i < K0) ? __ldg(X + r * K0 + i) : 0.f;
            st_row_tile<16>(sA0, row, 0, 32, v);
        }
    } else {
        float v[CW];
        if (valid) {
            const float4* p = reinterpret_cast<const float4*>(X + r * KP + c0);
#pragma unroll
            for (int i = 0; i < CW / 4; ++i) {
                const float4 u = __ldg(p + i);
                v[4 * i] = u.x; v[4 * i + 1] = u.y; v[4 * i + 2] = u.z; v[4 * i + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < CW; ++i) v[i] = 0.f;
        }
        st_row_tile<CW>(sA0, row, c0, span_of(KP), v);
    }
}

// ASAVE (training forward): each finished BF16 hidden tile also goes to block k
// of tmap_h (row k * act_rows + t * 128 + i) by a TMA store, for the backward.
template <int H, int KP, int NP, bool LN, bool ASAVE = false>
__global__ void __launch_bounds__(Cfg<H>::NT) k_rowmlp_fwd(const __grid_constant__ CUtensorMap tmap_h, RowMlpArgs A) {
    using C = Cfg<H>;
    constexpr int CW = C::CW, CG = C::CG, S = C::S, SKP = span_of(KP);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const RowFwdSmem L = rowmlp_fwd_smem<H, KP, NP>(n_lin);
    uint8_t* sW0 = sm + L.w0;
    uint8_t* sWm = sm + L.wm;
    uint8_t* sWl = sm + L.wl;
    uint8_t* sA0 = sm + L.a0;
    uint8_t* sA1 = sm + L.a1;
    float* sPar = reinterpret_cast<float*>(sm + L.par);   // b_0..b_{n-2} [H], b_last, gamma, beta [NP]
    float* sRed = reinterpret_cast<float*>(sm + L.red);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;
    const int K0 = A.K0, NO = A.N_out;

    if (warp == 0) {
        tmem_alloc(tslot, C::TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    // weights as K-major BF16 tiles, zero-padded to KP inputs / NP outputs
    for (int i = tid; i < H * (KP / 8); i += C::NT) {
        const int n = i / (KP / 8), k = (i % (KP / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = k + j < K0 ? A.mlp.W[0][n * K0 + k + j] : 0.f;
        st_tile8(sW0, n, k, H, SKP, v);
    }
    for (int l = 1; l < n_lin - 1; ++l) load_weight(sWm + (l - 1) * H * H * 2, A.mlp.W[l], H, 0, H, H, tid, C::NT);
    for (int i = tid; i < NP * (H / 8); i += C::NT) {
        const int n = i / (H / 8), k = (i % (H / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = n < NO ? A.mlp.W[n_lin - 1][n * H + k + j] : 0.f;
        st_tile8(sWl, n, k, NP, S, v);
    }
    for (int i = tid; i < (n_lin - 1) * H; i += C::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < NP; i += C::NT) {
        sPar[(n_lin - 1) * H + i] = i < NO ? A.mlp.b[n_lin - 1][i] : 0.f;
        sPar[(n_lin - 1) * H + NP + i] = (LN && i < NO) ? A.mlp.gamma[i] : 0.f;
        sPar[(n_lin - 1) * H + 2 * NP + i] = (LN && i < NO) ? A.mlp.beta[i] : 0.f;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t ph = 0;
    bool ok = true;
    const int64_t n_tiles = (A.n_rows + 127) / 128;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        load_input_row<KP, CW, CG>(sA0, A.X, r, valid, K0, row, g, c0);
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_mma(tmem, sA0, sW0, H, KP);
            mma_commit(bar);
        }
        float v[CW];
        for (int k = 0; k < n_lin - 1 && ok; ++k) {   // hidden layers: Linear -> ELU
            if (ASAVE && tid == 0) bulk_wait_read_all();   // sA1 may be rewritten after the barrier
            ok = block_wait(bar, ph, tid);
            ph ^= 1;
            tc_fence_after();
            if (!ok) break;
            ld_acc<CW>(tmem, q, c0, v);
            add_bias2<CW>(v, sPar + k * H + c0);
            elu_inplace2<CW>(v);
            st_row_tile<CW>(sA1, row, c0, S, v);
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                if (k + 1 < n_lin - 1)
                    issue_mma(tmem, sA1, sWm + k * H * H * 2, H, H);
                else
                    issue_mma(tmem, sA1, sWl, NP, H);
                mma_commit(bar);
                if constexpr (ASAVE) {
                    tma_store_2d(&tmap_h, 0, (int32_t)(k * A.act_rows + t * 128), sA1);
                    bulk_commit();
                }
            }
        }
        if (!ok) break;
        if (ASAVE && tid == 0) bulk_wait_read_all();
        ok = block_wait(bar, ph, tid);   // the last Linear
        ph ^= 1;
        tc_fence_after();
        if (!ok) break;
        const float* bl = sPar + (n_lin - 1) * H;
        if constexpr (LN) {   // NP == H: bias, LayerNorm over the row's H outputs
            ld_acc<CW>(tmem, q, c0, v);
            add_bias2<CW>(v, bl + c0);
            tc_fence_before();
            float mean, rstd;
            row_stats<H, CG, CW>(v, sRed, row, g, A.eps, mean, rstd);
#pragma unroll
            for (int i = 0; i < CW; ++i) v[i] = (v[i] - mean) * rstd * bl[NP + c0 + i] + bl[2 * NP + c0 + i];
            if (A.y_bf16) {   // whole rows per warp, staged in the activation tile (the last MMA has read it)
                st_row_tile<CW>(sA1, row, c0, S, v);
                __syncthreads();
                constexpr int CPR = H / 8;   // 16-byte chunks per row (NO == H)
                const int nrow = (int)(A.n_rows - t * 128 < 128 ? A.n_rows - t * 128 : 128);
                __nv_bfloat16* y = reinterpret_cast<__nv_bfloat16*>(A.Y) + t * 128 * NO;
                for (int i = tid; i < nrow * CPR; i += C::NT) {
                    const int rr = i / CPR, jj = i - rr * CPR;
                    *reinterpret_cast<uint4*>(y + (int64_t)rr * NO + 8 * jj) =
                        *reinterpret_cast<const uint4*>(sA1 + tile_off(rr, 8 * jj, 128, S));
                }
            } else if (valid) {
                float4* y = reinterpret_cast<float4*>(reinterpret_cast<float*>(A.Y) + r * NO + c0);
#pragma unroll
                for (int i = 0; i < CW / 4; ++i) y[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
        } else {              // NP = 16 output columns, held by column group 0
            if (g == 0) {
                float o[16];
                ld_acc<16>(tmem, q, 0, o);
                if (valid) {
                    for (int i = 0; i < NO; ++i) {
                        const float y = o[i] + bl[i];
                        if (A.y_bf16)
                            reinterpret_cast<__nv_bfloat16*>(A.Y)[r * NO + i] = __float2bfloat16_rn(y);
                        else
                            reinterpret_cast<float*>(A.Y)[r * NO + i] = y;
                    }
                }
            }
            tc_fence_before();
        }
        __syncthreads();   // sA0, sA1 and TMEM are reused by the next tile
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, C::TCOLS);
}

// ------------------------------------------------------------------ backward

struct RowBwdSmem {
    uint32_t w0, wm, wl, a0, ones0, g, hb, ones, par, red, bar, tm, total;
};

// TMEM columns: the work accumulator (H), dW_0 (KP + 16), the hidden dW
// ((n_lin-2) x (H + 16)), dW_last (H + 16), then the LayerNorm gradient sums (2H).
template <int H, int KP>
__host__ __device__ inline uint32_t rowmlp_bwd_tcols(int n_lin, bool ln) {
    return H + (KP + 16) + (uint32_t)(n_lin - 1) * (H + 16) + (ln ? 2 * H : 0);
}

// W0 [H x KP], hidden weights, W_last [NP x H], the input tile [128 x KP]
// followed by its ones block (the bias column of dW_0), the gradient tile,
// the recomputed hidden activations (n_lin-1 tiles [128 x H]), the ones block
// of the other layers, parameters, row partials.
template <int H, int KP, int NP>
__host__ __device__ inline RowBwdSmem rowmlp_bwd_smem(int n_lin) {
    constexpr int S = span_of(H), SKP = span_of(KP);
    RowBwdSmem s;
    s.w0 = 0;
    s.wm = align_up(s.w0 + H * KP * 2, 1024);
    s.wl = align_up(s.wm + (n_lin - 2) * H * H * 2, 1024);
    s.a0 = align_up(s.wl + NP * H * 2, 1024);
    s.ones0 = s.a0 + 128 * KP * 2;                 // the next N-block of [a0 ; ones]
    s.g = align_up(s.ones0 + 128 * SKP, 1024);
    s.hb = s.g + 128 * H * 2;
    s.ones = align_up(s.hb + (n_lin - 1) * 128 * H * 2, 1024);
    s.par = s.ones + 128 * S;
    s.red = s.par + ((n_lin - 1) * H + 3 * NP) * 4;
    s.bar = align_up(s.red + 4 * (H / 16) * 128 * 4, 8);   // mma, h[GNN_MAX_LIN]
    s.tm = s.bar + 8 * (1 + GNN_MAX_LIN);
    uint32_t end = s.tm + 16;
    end = end > s.g + 32768 ? end : s.g + 32768;   // M-padded wgrad views read 32 KB from g
    s.total = end + 1024;
    return s;
}

// SAVED: the forward stored the hidden activations (block k, row k * act_rows +
// r, of tmap_h); they arrive by TMA into the activation buffers, each refilled
// with the next tile's rows once its last reader has passed, and only the last
// Linear is recomputed.
template <int H, int KP, int NP, bool LN, bool DX, bool SAVED = false>
__global__ void __launch_bounds__(CfgB<H>::NT, 1) k_rowmlp_bwd(const __grid_constant__ CUtensorMap tmap_h,
                                                              RowMlpArgs A) {
    using C = CfgB<H>;
    constexpr int S = C::S, SKP = span_of(KP), SNP = span_of(NP), CW = C::CW, CG = C::CG;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const RowBwdSmem P = rowmlp_bwd_smem<H, KP, NP>(n_lin);
    uint8_t* sW0 = sm + P.w0;
    uint8_t* sWm = sm + P.wm;
    uint8_t* sWl = sm + P.wl;
    uint8_t* sA0 = sm + P.a0;
    uint8_t* sG = sm + P.g;
    uint8_t* sHB = sm + P.hb;
    uint8_t* sOnes = sm + P.ones;
    float* sPar = reinterpret_cast<float*>(sm + P.par);
    float* sRed = reinterpret_cast<float*>(sm + P.red);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + P.tm);
    const uint32_t NCOLS = pow2_cols(rowmlp_bwd_tcols<H, KP>(n_lin, LN));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;
    const int K0 = A.K0, NO = A.N_out;

    if (warp == 0) {
        tmem_alloc(tslot, NCOLS);
        tmem_relinquish();
    }
    uint64_t* h_full = bar + 1;   // SAVED: h_k of the tile has landed
    if (tid == 0) {
        mbar_init(bar, 1);
        if (SAVED)
            for (int k = 0; k < n_lin - 1; ++k) mbar_init(h_full + k, 1);
        fence_mbar_init();
    }
    for (int i = tid; i < H * (KP / 8); i += C::NT) {
        const int n = i / (KP / 8), k = (i % (KP / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = k + j < K0 ? A.mlp.W[0][n * K0 + k + j] : 0.f;
        st_tile8(sW0, n, k, H, SKP, v);
    }
    for (int l = 1; l < n_lin - 1; ++l) load_weight(sWm + (l - 1) * H * H * 2, A.mlp.W[l], H, 0, H, H, tid, C::NT);
    for (int i = tid; i < NP * (H / 8); i += C::NT) {
        const int n = i / (H / 8), k = (i % (H / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = n < NO ? A.mlp.W[n_lin - 1][n * H + k + j] : 0.f;
        st_tile8(sWl, n, k, NP, S, v);
    }
    fill_ones(sm + P.ones0, SKP, tid, C::NT);
    fill_ones(sOnes, S, tid, C::NT);
    for (int i = tid; i < (n_lin - 1) * H; i += C::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < NP; i += C::NT) {
        sPar[(n_lin - 1) * H + i] = i < NO ? A.mlp.b[n_lin - 1][i] : 0.f;
        sPar[(n_lin - 1) * H + NP + i] = (LN && i < NO) ? A.mlp.gamma[i] : 0.f;
        sPar[(n_lin - 1) * H + 2 * NP + i] = (LN && i < NO) ? A.mlp.beta[i] : 0.f;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tWork = tmem;
    // dW accumulators: layer 0 [H x (KP+16)], layer l >= 1 [out x (H+16)]
    auto tDW = [&](int l) -> uint32_t {
        return tmem + (uint32_t)(H + (l == 0 ? 0 : (KP + 16) + (l - 1) * (H + 16)));
    };
    const uint32_t tLN = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(H + (KP + 16) + (n_lin - 1) * (H + 16)) +
                         (uint32_t)(g * 2 * CW);
    if constexpr (LN) {
        float z[16] = {};
#pragma unroll
        for (int i = 0; i < 2 * CW; i += 16) tmem_st16(tLN + i, z);
        tmem_st_wait();
    }
    uint32_t ph = 0;
    bool ok = true, first = true;
    const int64_t n_tiles = (A.n_rows + 127) / 128;
    const float* bl = sPar + (n_lin - 1) * H;
    auto mma_sync_issue = [&](auto&& issue) {   // operands written -> one thread issues
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue();
            mma_commit(bar);
        }
    };
    constexpr int HT = 128 * H * 2;   // one activation tile
    const uint32_t hmask = SAVED ? ((1u << (n_lin - 1)) - 1u) : 0u;
    // per-thread parity of h_full[k]; thread 0: loads not yet waited for, the phase parity
    // of each (a timeout can end the tile loop between a load and its tile's end)
    uint32_t ph_h = 0, h_pend = 0, ld_par = 0, pend_par = 0;
    auto load_h = [&](int k, int64_t tt) {
        mbar_arrive_expect_tx(h_full + k, HT);
        tma_load_2d(sHB + k * HT, &tmap_h, 0, (int32_t)(k * A.act_rows + tt * 128), h_full + k);
        h_pend |= 1u << k;
        pend_par = (pend_par & ~(1u << k)) | (ld_par & (1u << k));
        ld_par ^= 1u << k;
    };
    auto wait_h = [&](int k) {
        ok = ok && mbar_wait(h_full + k, (ph_h >> k) & 1u);
        h_pend &= ~(1u << k);
    };
    if (SAVED && tid == 0 && (int64_t)blockIdx.x < n_tiles)
        for (int k = 0; k < n_lin - 1; ++k) load_h(k, blockIdx.x);

    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        const bool more = t + gridDim.x < n_tiles;
        load_input_row<KP, CW, CG>(sA0, A.X, r, valid, K0, row, g, c0);
        if constexpr (SAVED) {   // the last Linear from the saved h_{L-2}
            wait_h(n_lin - 2);
            mma_sync_issue([&] { issue_mma(tWork, sHB + (n_lin - 2) * HT, sWl, NP, H); });
        } else {
            mma_sync_issue([&] { issue_mma(tWork, sA0, sW0, H, KP); });
        }
        // ---- recompute: hidden activations into hb, the last pre-activation in registers
        float v[CW];
        for (int k = 0; k < (SAVED ? 0 : n_lin - 1) && ok; ++k) {
            ok = block_wait(bar, ph, tid);
            ph ^= 1;
            tc_fence_after();
            if (!ok) break;
            ld_acc<CW>(tWork, q, c0, v);
            add_bias2<CW>(v, sPar + k * H + c0);
            elu_inplace2<CW>(v);
            st_row_tile<CW>(sHB + k * 128 * H * 2, row, c0, S, v);
            uint8_t* hk = sHB + k * 128 * H * 2;
            if (k + 1 < n_lin - 1)
                mma_sync_issue([&] { issue_mma(tWork, hk, sWm + k * H * H * 2, H, H); });
            else
                mma_sync_issue([&] { issue_mma(tWork, hk, sWl, NP, H); });
        }
        if (!ok) break;
        ok = block_wait(bar, ph, tid);
        ph ^= 1;
        tc_fence_after();
        if (!ok) break;
        // ---- gradient of the last pre-activation, dz, into sG ([128 x NP])
        if constexpr (LN) {   // NP == H
            ld_acc<CW>(tWork, q, c0, v);
            add_bias2<CW>(v, bl + c0);
            tc_fence_before();
            float gv[CW];
            if (valid) {
                if (A.dy_bf16) {
                    ld_bf16x8(reinterpret_cast<const __nv_bfloat16*>(A.dY) + r * NO + c0, gv);
                    ld_bf16x8(reinterpret_cast<const __nv_bfloat16*>(A.dY) + r * NO + c0 + 8, gv + 8);
                } else {
                    const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(A.dY) + r * NO + c0);
#pragma unroll
                    for (int i = 0; i < CW / 4; ++i) {
                        const float4 u = __ldg(p + i);
                        gv[4 * i] = u.x; gv[4 * i + 1] = u.y; gv[4 * i + 2] = u.z; gv[4 * i + 3] = u.w;
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < CW; ++i) gv[i] = 0.f;
            }
            float dz[CW];
#pragma unroll
            for (int i = 0; i < CW; ++i) dz[i] = gv[i] * bl[NP + c0 + i];
            float mean, rstd, s1, s2;
            row_stats_adj<H, CG, CW>(v, dz, sRed, row, g, A.eps, mean, rstd, s1, s2);
#pragma unroll
            for (int i = 0; i < CW; ++i) v[i] = (v[i] - mean) * rstd;   // xhat
#pragma unroll
            for (int i0 = 0; i0 < CW; i0 += 16) {
                float ag[16], ab[16];
                tmem_ld16(tLN + i0, ag);
                tmem_ld16(tLN + CW + i0, ab);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    ag[i] += gv[i0 + i] * v[i0 + i];
                    ab[i] += gv[i0 + i];
                }
                tmem_st16(tLN + i0, ag);
                tmem_st16(tLN + CW + i0, ab);
            }
            tmem_st_wait();
#pragma unroll
            for (int i = 0; i < CW; ++i) dz[i] = rstd * (dz[i] - s1 - v[i] * s2);
            st_row_tile<CW>(sG, row, c0, S, dz);
        } else {              // no LayerNorm: dz = dY, NP = 16 columns held by column group 0
            if (g == 0) {
                float dz[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) dz[i] = 0.f;
                if (valid) {
                    for (int i = 0; i < NO; ++i)
                        dz[i] = A.dy_bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(A.dY)[r * NO + i])
                                          : reinterpret_cast<const float*>(A.dY)[r * NO + i];
                }
                st_row_tile<16>(sG, row, 0, SNP, dz);
            }
        }
        // ---- adjoint of the chain, layer n_lin-1 .. 0
        for (int l = n_lin - 1; l >= 0 && ok; --l) {
            if (SAVED && l > 0) wait_h(l - 1);   // this step's wgrad operand and ELU derivative input
            // SAVED: h_l's last reader (step l + 1) is done once every thread passes the barrier
            // in this step's issue: the next tile's h_l goes there
            auto refill = [&] {
                if (SAVED && l <= n_lin - 2 && more) load_h(l, t + gridDim.x);
            };
            if (l == n_lin - 1) {
                // dh = dz W_last (K = NP), dW_last += dz^T [h ; 1]
                uint8_t* hk = sHB + (l - 1) * 128 * H * 2;
                mma_sync_issue([&] {
                    issue_dgrad(tWork, sG, SNP, sWl, S, NP, (uint32_t)NP * S, H, NP);
                    issue_wgrad(tDW(l), sG, SNP, 128u * SNP, hk, S, (uint32_t)(smem_u32(sOnes) - smem_u32(hk)), H + 16,
                                !first);
                    refill();
                });
            } else if (l > 0) {
                uint8_t* hk = sHB + (l - 1) * 128 * H * 2;
                mma_sync_issue([&] {
                    issue_dgrad(tWork, sG, S, sWm + (l - 1) * H * H * 2, S, H, (uint32_t)H * S, H, H);
                    issue_wgrad(tDW(l), sG, S, 128u * S, hk, S, (uint32_t)(smem_u32(sOnes) - smem_u32(hk)), H + 16,
                                !first);
                    refill();
                });
            } else {
                // dX = dz W0 (N = KP), dW0 += dz^T [x ; 1]
                mma_sync_issue([&] {
                    if (DX) issue_dgrad(tWork, sG, S, sW0, SKP, H, (uint32_t)H * SKP, KP, H);
                    issue_wgrad(tDW(0), sG, S, 128u * S, sA0, SKP, 128u * SKP, KP + 16, !first);
                    refill();
                });
            }
            ok = block_wait(bar, ph, tid);
            ph ^= 1;
            tc_fence_after();
            if (!ok) break;
            if (l > 0) {
                float dh[CW], hv[CW], dz[CW];
                ld_acc<CW>(tWork, q, c0, dh);
                ld_row_tile<CW>(sHB + (l - 1) * 128 * H * 2, row, c0, S, hv);
                elu_bwd2<CW>(dz, dh, hv);
                tc_fence_before();
                st_row_tile<CW>(sG, row, c0, S, dz);   // this step's MMAs, the readers of sG, are complete
            } else if (DX) {
                if (KP == 16) {
                    if (g == 0) {
                        float dx[16];
                        ld_acc<16>(tWork, q, 0, dx);
                        if (valid)
                            for (int i = 0; i < K0; ++i) A.dX[r * K0 + i] = dx[i];
                    }
                } else {
                    float dx[CW];
                    ld_acc<CW>(tWork, q, c0, dx);
                    if (valid) {
                        float4* p = reinterpret_cast<float4*>(A.dX + r * KP + c0);
#pragma unroll
                        for (int i = 0; i < CW / 4; ++i)
                            p[i] = make_float4(dx[4 * i], dx[4 * i + 1], dx[4 * i + 2], dx[4 * i + 3]);
                    }
                }
                tc_fence_before();
            }
        }
        first = false;
        ph_h ^= hmask;
        __syncthreads();
    }
    if (SAVED && tid == 0)   // loads issued before a timeout ended the tile loop
        for (int k = 0; k < n_lin - 1; ++k)
            if ((h_pend >> k) & 1u) mbar_wait(h_full + k, (pend_par >> k) & 1u);
    // ---- flush the CTA's partial gradients
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (ok) {
        int64_t off = 0;
        for (int l = 0; l < n_lin; ++l) {
            const int N = (l == 0 ? KP : H) + 16;
            const int M = l == n_lin - 1 ? NP : H;
            if (!first) flush_acc<CG>(tDW(l), N, M, q, lane, g, part + off);
            else
                for (int i = tid; i < M * N; i += C::NT) part[off + i] = 0.f;
            off += (int64_t)M * N;
        }
        if constexpr (LN) {
            float ag[CW], ab[CW];
#pragma unroll
            for (int i0 = 0; i0 < CW; i0 += 16) {
                tmem_ld16(tLN + i0, ag + i0);
                tmem_ld16(tLN + CW + i0, ab + i0);
            }
            tmem_ld_wait();
            rows_reduce_store<CW>(ag, sRed, q, lane, g, c0, part + off);
            rows_reduce_store<CW>(ab, sRed, q, lane, g, c0, part + off + H);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// =================================================================== host side

namespace {

using namespace host;

int64_t rowmlp_pstride(int H, int KP, int NP, int n_lin, bool ln) {
    int64_t p = (int64_t)H * (KP + 16) + (int64_t)(n_lin - 2) * H * (H + 16) + (int64_t)NP * (H + 16);
    return p + (ln ? 2 * H : 0);
}

// Saved activations of a row MLP: (n_lin - 1) blocks of whole 128-row tiles [R x H].
int64_t rowmlp_act_rows(int64_t n_rows) { return (n_rows + 127) / 128 * 128; }

template <int H, int KP, int NP, bool LN>
int rowmlp_fwd_h(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, float eps, cudaStream_t s,
                 __nv_bfloat16* act) {
    using C = Cfg<H>;
    RowMlpArgs A{};
    A.X = X;
    A.n_rows = n_rows;
    A.K0 = P.dims[0];
    A.N_out = P.dims[P.n_lin];
    A.Y = Y;
    A.y_bf16 = y_bf16;
    A.mlp = mlp_dev(P);
    A.eps = eps;
    const RowFwdSmem L = rowmlp_fwd_smem<H, KP, NP>(P.n_lin);
    A.act_rows = rowmlp_act_rows(n_rows);
    CUtensorMap tmh;
    std::memset(&tmh, 0, sizeof(tmh));
    int rc;
    if (act && (rc = make_row_tmap(&tmh, act, (int64_t)(P.n_lin - 1) * A.act_rows, H))) return rc;
    int grid = 0;
    auto run = [&](auto kern) -> int {
        int r = persistent_grid(kern, C::NT, L.total, C::TCOLS, (n_rows + 127) / 128, &grid);
        if (r) return r;
        {
            ProfScope _ps(s, "k_rowmlp_fwd");
            kern<<<grid, C::NT, L.total, s>>>(tmh, A);
        }
        GNN_LAUNCH_CHECK("k_rowmlp_fwd");
        return GNN_OK;
    };
    return act ? run(k_rowmlp_fwd<H, KP, NP, LN, true>) : run(k_rowmlp_fwd<H, KP, NP, LN, false>);
}

template <int H, int KP, int NP, bool LN, bool DX>
int rowmlp_bwd_h(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                 const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s, const __nv_bfloat16* act) {
    using C = CfgB<H>;
    const int L = P.n_lin, K0 = P.dims[0], NO = P.dims[L];
    const uint32_t tcols = rowmlp_bwd_tcols<H, KP>(L, LN);
    GNN_REQUIRE(tcols <= 512, GNN_EUNSUPPORTED,
                "gnn_mlp_backward_bf16: too many Linear layers (%d) for the tensor memory at H=%d", L, H);
    const int64_t pstride = rowmlp_pstride(H, KP, NP, L, LN);
    const int nsm = num_sms();
    GNN_REQUIRE(ws_bytes >= (size_t)nsm * pstride * 4, GNN_ENOMEM, "gnn_mlp_backward_bf16: workspace too small");
    RowMlpArgs A{};
    A.X = X;
    A.n_rows = n_rows;
    A.K0 = K0;
    A.N_out = NO;
    A.dY = dY;
    A.dy_bf16 = dy_bf16;
    A.dX = dX;
    A.part = reinterpret_cast<float*>(ws);
    A.pstride = pstride;
    A.mlp = mlp_dev(P);
    A.eps = eps;
    const RowBwdSmem Pl = rowmlp_bwd_smem<H, KP, NP>(L);
    A.act_rows = rowmlp_act_rows(n_rows);
    CUtensorMap tmh;
    std::memset(&tmh, 0, sizeof(tmh));
    int rc;
    if (act && (rc = make_row_tmap(&tmh, act, (int64_t)(L - 1) * A.act_rows, H))) return rc;
    int grid = 0;
    auto run = [&](auto kern) -> int {
        int r = persistent_grid(kern, C::NT, Pl.total, pow2_cols(tcols), (n_rows + 127) / 128, &grid);
        if (r) return r;
        grid = std::min(grid, nsm);
        {
            ProfScope _ps(s, "k_rowmlp_bwd");
            kern<<<grid, C::NT, Pl.total, s>>>(tmh, A);
        }
        GNN_LAUNCH_CHECK("k_rowmlp_bwd");
        return GNN_OK;
    };
    rc = act ? run(k_rowmlp_bwd<H, KP, NP, LN, DX, true>) : run(k_rowmlp_bwd<H, KP, NP, LN, DX, false>);
    if (rc) return rc;
    // partial layout: per layer [M x (in + 16)] (bias in column `in`), then gamma, beta
    RedSeg seg[MAX_SEGS];
    int n = 0;
    int64_t off = 0;
    for (int l = 0; l < L; ++l) {
        const int in = l == 0 ? KP : H, N = in + 16, M = l == L - 1 ? NP : H;
        const int in_real = l == 0 ? K0 : H, out_real = l == L - 1 ? NO : H;
        seg[n++] = RedSeg{dP.W[l], in_real, out_real, in_real, off, N};
        seg[n++] = RedSeg{dP.b[l], 1, out_real, 1, off + in, N};
        off += (int64_t)M * N;
    }
    if (LN) {
        seg[n++] = RedSeg{dP.gamma, NO, 1, NO, off, 0};
        seg[n++] = RedSeg{dP.beta, NO, 1, NO, off + H, 0};
    }
    return reduce_grads(seg, n, A.part, pstride, grid, s);
}

// encoder: in <= 16, hidden = out = H, LayerNorm; decoder: in = hidden = H, out <= 16, no LayerNorm
enum { ROW_ENC = 1, ROW_DEC = 2 };

int rowmlp_shape(const gnn_mlp& P, int* H) {
    const int L = P.n_lin;
    if (L < 2 || L > GNN_MAX_LIN) return 0;
    const int h = P.dims[1];
    if (h != 16 && h != 32 && h != 64) return 0;
    for (int l = 1; l < L; ++l)
        if (P.dims[l] != h) return 0;
    *H = h;
    if (P.gamma && P.dims[0] >= 1 && P.dims[0] <= 16 && P.dims[L] == h) return ROW_ENC;
    if (!P.gamma && P.dims[0] == h && P.dims[L] >= 1 && P.dims[L] <= 16) return ROW_DEC;
    return 0;
}

}  // namespace

bool rowmlp_supported(const gnn_mlp& P) {
    int H;
    return rowmlp_shape(P, &H) != 0 || rowenc128_shape(P) || rowdec128_shape(P);
}

size_t rowmlp_backward_ws(const gnn_mlp& P, int64_t n_rows) {
    if (rowenc128_shape(P)) return rowenc128_backward_ws(P, n_rows);
    if (rowdec128_shape(P)) return rowdec128_backward_ws(P, n_rows);
    int H;
    const int k = rowmlp_shape(P, &H);
    if (!k) return 0;
    const bool enc = k == ROW_ENC;
    return (size_t)num_sms() * rowmlp_pstride(H, enc ? 16 : H, enc ? H : 16, P.n_lin, enc) * 4 + 256;
}

size_t rowmlp_act_bytes(const gnn_mlp& P, int64_t n_rows) {
    int H;
    if (!rowmlp_shape(P, &H) || n_rows <= 0) return 0;
    // activation rows are 32-bit TMA coordinates
    if ((int64_t)(P.n_lin - 1) * rowmlp_act_rows(n_rows) >= ((int64_t)1 << 31)) return 0;
    return (size_t)(P.n_lin - 1) * (size_t)rowmlp_act_rows(n_rows) * (size_t)H * 2;
}

int rowmlp_forward(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, float eps,
                   cudaStream_t s, __nv_bfloat16* act) {
    // H = 128: no activations kept (the adjoint recomputes them)
    if (rowenc128_shape(P)) return rowenc128_forward(P, n_rows, X, Y, y_bf16, eps, s);
    if (rowdec128_shape(P)) return rowdec128_forward(P, n_rows, X, Y, y_bf16, s);
    int H;
    const int k = rowmlp_shape(P, &H);
    GNN_REQUIRE(k, GNN_EUNSUPPORTED, "gnn_mlp_forward_bf16: shape not covered by the fused row MLP");
    if (n_rows == 0) return GNN_OK;
    if (!rowmlp_act_bytes(P, n_rows)) act = nullptr;
    if (k == ROW_ENC) {
        switch (H) {
            case 16: return rowmlp_fwd_h<16, 16, 16, true>(P, n_rows, X, Y, y_bf16, eps, s, act);
            case 32: return rowmlp_fwd_h<32, 16, 32, true>(P, n_rows, X, Y, y_bf16, eps, s, act);
            default: return rowmlp_fwd_h<64, 16, 64, true>(P, n_rows, X, Y, y_bf16, eps, s, act);
        }
    }
    switch (H) {
        case 16: return rowmlp_fwd_h<16, 16, 16, false>(P, n_rows, X, Y, y_bf16, eps, s, act);
        case 32: return rowmlp_fwd_h<32, 32, 16, false>(P, n_rows, X, Y, y_bf16, eps, s, act);
        default: return rowmlp_fwd_h<64, 64, 16, false>(P, n_rows, X, Y, y_bf16, eps, s, act);
    }
}

int rowmlp_backward(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                    const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s, const __nv_bfloat16* act) {
    if (rowenc128_shape(P)) return rowenc128_backward(P, n_rows, X, dY, dy_bf16, dX, dP, eps, ws, ws_bytes, s);
    if (rowdec128_shape(P)) return rowdec128_backward(P, n_rows, X, dY, dy_bf16, dX, dP, ws, ws_bytes, s);
    int H;
    const int k = rowmlp_shape(P, &H);
    GNN_REQUIRE(k, GNN_EUNSUPPORTED, "gnn_mlp_backward_bf16: shape not covered by the fused row MLP");
    if (n_rows == 0) return GNN_OK;
    if (!rowmlp_act_bytes(P, n_rows)) act = nullptr;
#define GNN_ROW_BWD(HH, KP, NP, LN)                                                                          \
    return dX ? rowmlp_bwd_h<HH, KP, NP, LN, true>(P, n_rows, X, dY, dy_bf16, dX, dP, eps, ws, ws_bytes, s, act) \
              : rowmlp_bwd_h<HH, KP, NP, LN, false>(P, n_rows, X, dY, dy_bf16, dX, dP, eps, ws, ws_bytes, s, act)
    if (k == ROW_ENC) {
        switch (H) {
            case 16: GNN_ROW_BWD(16, 16, 16, true);
            case 32: GNN_ROW_BWD(32, 16, 32, true);
            default: GNN_ROW_BWD(64, 16, 64, true);
        }
    }
    switch (H) {
        case 16: GNN_ROW_BWD(16, 16, 16, false);
        case 32: GNN_ROW_BWD(32, 32, 16, false);
        default: GNN_ROW_BWD(64, 64, 16, false);
    }
#undef GNN_ROW_BWD
}

}  // namespace fused
}  // namespace gnn
