// Node update of the consistent NMP layer at H = 128 in the two-group
// tensor-memory form (Eq. 5e): x' = x + LN(MLP_N([a*, x])).
//
// Two groups of four warps take alternate tiles of 128 node rows; one thread
// owns one row (its TMEM lane). The FP32 rows of a* and x come in by warps,
// 32 rows x 32 columns at a time, coalesced, through a 4 KB shared-memory
// buffer per warp, and the thread that owns a row writes it as BF16 into its
// group's 128 TMEM operand columns ([a*, x], K = 256). Every Linear reads its A
// operand from TMEM (W_k from shared memory); the LayerNorm statistics are the
// thread's own (FP32); the residual x and the result x' pass through the same
// per-warp buffer, so that every global access of the kernel is a whole
// 128-byte row segment. TMEM: group g uses columns [256 g, 256 g + 128) for the
// accumulator and the next 128 for the operand (h_k uses the first 64).

#include <algorithm>

#include "fused.h"
#include "profiler.h"
#include "tm128_common.cuh"

namespace gnn {
namespace fused {

cudaError_t take_device_error_node128(unsigned int* out) { return take_device_error_word(out); }

namespace {

using namespace tc;
using namespace tm128;

constexpr int kMaxLin = 4;                      // W_0 [128 x 256] and W_1 .. W_3 resident
constexpr uint32_t kW0 = kH * 2 * kH * 2;       // [128 x 256] BF16
constexpr uint32_t kTB = 32 * 32 * 4;           // per-warp buffer: 32 rows x 32 FP32

struct NodeTmArgs {
    const float* a_star;   // [n_rows x 128]
    const float* x;        // [n_rows x 128]
    float* x_out;          // [n_rows x 128]
    int64_t n_rows;
    MlpDev mlp;
    float eps;
};

struct NodeTmSmem {
    uint32_t w0, w, tb, par, bar, tm, total;
};

__host__ __device__ inline NodeTmSmem node_tm_smem(int n_lin) {
    NodeTmSmem s;
    s.w0 = 0;                                                   // W_0 [128 x 256]
    s.w = kW0;                                                  // W_1 .. W_{L-1}
    s.tb = s.w + (uint32_t)(n_lin - 1) * kWT;                   // tb[8]: one per warp
    s.par = s.tb + 8 * kTB;                                     // b_0 .. b_{L-1}, gamma, beta
    s.bar = align_up(s.par + (uint32_t)(n_lin + 2) * kH * 4, 8);   // mma[2]
    s.tm = s.bar + 2 * 8;
    s.total = s.tm + 16 + 1024;
    return s;
}

// Rows [r0, r0 + 32) x columns [c, c + 32) of an FP32 [n x 128] array: lane l
// loads row 4 i + (l >> 3), 16-byte chunk l & 7 (zero past n_rows).
__device__ __forceinline__ void warp_ld_chunk(const float* src, int64_t r0, int64_t n_rows, int c, int lane,
                                              float4* v) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + 4 * i + (lane >> 3);
        v[i] = r < n_rows ? __ldg(reinterpret_cast<const float4*>(src + r * kH + c) + (lane & 7))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// The chunk into the warp's buffer (16-byte chunk k of row rr at rr * 8 + (k ^ (rr & 7))).
__device__ __forceinline__ void warp_st_buf(float4* tb, int lane, const float4* v) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int rr = 4 * i + (lane >> 3), k = lane & 7;
        tb[rr * 8 + (k ^ (rr & 7))] = v[i];
    }
}

// This lane's row of the buffer (32 values).
__device__ __forceinline__ void lane_ld_row(const float4* tb, int lane, float* v) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float4 u = tb[lane * 8 + (k ^ (lane & 7))];
        v[4 * k] = u.x;
        v[4 * k + 1] = u.y;
        v[4 * k + 2] = u.z;
        v[4 * k + 3] = u.w;
    }
}

__device__ __forceinline__ void lane_st_row(float4* tb, int lane, const float* v) {
#pragma unroll
    for (int k = 0; k < 8; ++k)
        tb[lane * 8 + (k ^ (lane & 7))] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

// D = [a*, x] (TMEM, K = 256) * W_0^T.
__device__ __forceinline__ void issue_mma_ts_k256(uint32_t d_tmem, uint32_t a_tmem, const uint8_t* W0) {
    const uint64_t b0 = kmajor_desc(smem_u32(W0), kH, kS, 0);
    const uint32_t id = idesc_bf16(128, kH);
#pragma unroll
    for (int k0 = 0; k0 < 2 * kH; k0 += 16)
        mma_bf16_ts(d_tmem, a_tmem + (uint32_t)(k0 / 2), desc_step(b0, kmajor_off(kH, kS, k0)), id, k0 > 0 ? 1u : 0u);
}

__global__ void __launch_bounds__(kNT, 1) k_node_fwd_tm(NodeTmArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const NodeTmSmem L = node_tm_smem(n_lin);
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = warp >> 2, q = warp & 3;   // the thread's row is 32 q + lane
    const bool leader = (tid & (kGT - 1)) == 0;
    float4* tb = reinterpret_cast<float4*>(sm + L.tb + warp * kTB);

    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_mma + 1, 1);
        fence_mbar_init();
    }
    load_weight(sm + L.w0, A.mlp.W[0], 2 * kH, 0, kH, 2 * kH, tid, kNT);
    for (int k = 1; k < n_lin; ++k) load_weight(sm + L.w + (k - 1) * kWT, A.mlp.W[k], kH, 0, kH, kH, tid, kNT);
    for (int i = tid; i < n_lin * kH; i += kNT) sPar[i] = A.mlp.b[i / kH][i % kH];
    for (int i = tid; i < kH; i += kNT) {
        sPar[n_lin * kH + i] = A.mlp.gamma[i];
        sPar[(n_lin + 1) * kH + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t tAcc = *tslot + (uint32_t)(gi * 256), tA = tAcc + 128;
    const float* gam = sPar + n_lin * kH;
    const float* bet = sPar + (n_lin + 1) * kH;
    const int64_t n_tiles = (A.n_rows + 127) / 128;
    const int64_t step = 2 * (int64_t)gridDim.x;
    uint32_t ph = 0;
    bool ok = true;

    for (int64_t t = (int64_t)blockIdx.x + gi * (int64_t)gridDim.x; t < n_tiles && ok; t += step) {
        const int64_t r0 = t * 128 + 32 * q;   // the warp's 32 rows
        if (leader && t + step < n_tiles) {    // the group's next rows into L2
            const int64_t rn = (t + step) * 128;
            const uint32_t nb = (uint32_t)(std::min<int64_t>(128, A.n_rows - rn) * kH * 4);
            prefetch_l2(A.a_star + rn * kH, nb);
            prefetch_l2(A.x + rn * kH, nb);
        }
        // [a*, x] as BF16 into the TMEM operand, 32 columns at a time; the next chunk's
        // loads are in flight while this one passes through the buffer
        {
            float4 cur[8], nxt[8];
            warp_ld_chunk(A.a_star, r0, A.n_rows, 0, lane, cur);
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) {
                if (ch + 1 < 8)
                    warp_ld_chunk(ch + 1 < 4 ? A.a_star : A.x, r0, A.n_rows, 32 * ((ch + 1) & 3), lane, nxt);
                warp_st_buf(tb, lane, cur);
                __syncwarp();
                float v[32];
                lane_ld_row(tb, lane, v);
                __syncwarp();
                uint32_t hb[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) hb[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
                tmem_st16u(tA + lane_base + (uint32_t)(16 * ch), hb);
#pragma unroll
                for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
            }
        }
        tmem_st_wait();
        tc_fence_before();
        group_sync(gi);
        if (leader) {
            tc_fence_after();
            issue_mma_ts_k256(tAcc, tA, sm + L.w0);
            mma_commit(bar_mma + gi);
        }
        // h_k = ELU(acc + b_k) into TMEM, then acc = h_k W_{k+1}^T
        for (int k = 0; k < n_lin - 1; ++k) {
            const bool w_ok = leader ? mbar_wait(bar_mma + gi, ph) : true;
            ok = group_and(w_ok, gi);
            ph ^= 1;
            if (!ok) break;
            tc_fence_after();
            {
                float v[kH];
                ld_acc_n<kH>(tAcc + lane_base, sPar + k * kH, v);
#pragma unroll
                for (int c = 0; c < kH; c += 32) elu_to_tmem(tA + lane_base + (uint32_t)(c / 2), v + c);
            }
            hand_off(tAcc, tA, sm + L.w + k * kWT, gi, leader, bar_mma);
        }
        if (!ok) break;
        {
            const bool w_ok = leader ? mbar_wait(bar_mma + gi, ph) : true;
            ok = group_and(w_ok, gi);
            ph ^= 1;
            if (!ok) break;
            tc_fence_after();
        }
        // x' = x + LN(acc + b_{L-1}): mean, then the variance about it (FP32, four chains)
        float ev[kH];
        float mean, rstd;
        {
            float sp[4];
            ld_acc_n<kH>(tAcc + lane_base, sPar + (n_lin - 1) * kH, ev);
#pragma unroll
            for (int c = 0; c < kH; c += 32) sp[c / 32] = sum32(ev + c);
            mean = ((sp[0] + sp[1]) + (sp[2] + sp[3])) * (1.f / kH);
#pragma unroll
            for (int c = 0; c < kH; c += 32) sp[c / 32] = sqdev32(ev + c, mean);
            rstd = rsqrtf(((sp[0] + sp[1]) + (sp[2] + sp[3])) * (1.f / kH) + A.eps);
        }
        // the residual comes in and x' goes out through the warp's buffer, 32 columns at a time
        {
            float4 cur[8], nxt[8];
            warp_ld_chunk(A.x, r0, A.n_rows, 0, lane, cur);
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                const int c = 32 * ch;
                if (ch + 1 < 4) warp_ld_chunk(A.x, r0, A.n_rows, c + 32, lane, nxt);
                warp_st_buf(tb, lane, cur);
                __syncwarp();
                float xv[32];
                lane_ld_row(tb, lane, xv);
#pragma unroll
                for (int i = 0; i < 32; i += 4) {
                    const float4 gm = *reinterpret_cast<const float4*>(gam + c + i);
                    const float4 bt = *reinterpret_cast<const float4*>(bet + c + i);
                    const float2 nm = make_float2(-mean, -mean), rs = make_float2(rstd, rstd);
                    const float2 xa = __fmul2_rn(__fadd2_rn(make_float2(ev[c + i], ev[c + i + 1]), nm), rs);
                    const float2 xb = __fmul2_rn(__fadd2_rn(make_float2(ev[c + i + 2], ev[c + i + 3]), nm), rs);
                    const float2 ya = __fadd2_rn(__ffma2_rn(xa, make_float2(gm.x, gm.y), make_float2(bt.x, bt.y)),
                                                 make_float2(xv[i], xv[i + 1]));
                    const float2 yb = __fadd2_rn(__ffma2_rn(xb, make_float2(gm.z, gm.w), make_float2(bt.z, bt.w)),
                                                 make_float2(xv[i + 2], xv[i + 3]));
                    xv[i] = ya.x;
                    xv[i + 1] = ya.y;
                    xv[i + 2] = yb.x;
                    xv[i + 3] = yb.y;
                }
                __syncwarp();
                lane_st_row(tb, lane, xv);
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + (lane >> 3), k = lane & 7;
                    if (r0 + rr < A.n_rows)
                        reinterpret_cast<float4*>(A.x_out + (r0 + rr) * kH + c)[k] = tb[rr * 8 + (k ^ (rr & 7))];
                }
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
            }
        }
        // the accumulator has been read (wait::ld) before the group's next first Linear
        tc_fence_before();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, 512);
}

}  // namespace

using namespace host;

bool node_fwd_tm_supported(const gnn_mp_params& W) { return W.node.n_lin >= 2 && W.node.n_lin <= kMaxLin; }

int node_fwd_tm(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* a,
                const float* x_in, float* x_out, cudaStream_t s) {
    const int64_t NR = G.n_rows;
    GNN_REQUIRE(node_fwd_tm_supported(W), GNN_EUNSUPPORTED,
                "gnn_mp_forward: the tensor-memory node forward needs 2..%d Linear layers", kMaxLin);
    if (NR == 0) return GNN_OK;
    GNN_REQUIRE((((uintptr_t)a | (uintptr_t)x_in | (uintptr_t)x_out) & 15) == 0, GNN_EINVAL,
                "gnn_mp_forward: node rows must be 16-byte aligned");
    NodeTmArgs A{};
    A.a_star = a;
    A.x = x_in;
    A.x_out = x_out;
    A.n_rows = NR;
    A.mlp = mlp_dev(W.node);
    A.eps = cfg.ln_eps;
    const NodeTmSmem L = node_tm_smem(W.node.n_lin);
    int grid;
    int rc = persistent_grid(k_node_fwd_tm, kNT, L.total, 512, ((NR + 127) / 128 + 1) / 2, &grid);
    if (rc) return rc;
    {
        ProfScope _ps(s, "k_node_fwd");
        k_node_fwd_tm<<<grid, kNT, L.total, s>>>(A);
    }
    GNN_LAUNCH_CHECK("k_node_fwd_tm");
    return GNN_OK;
}

}  // namespace fused
}  // namespace gnn
