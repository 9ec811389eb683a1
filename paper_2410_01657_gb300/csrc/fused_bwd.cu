// Fused BF16 backward (adjoint) of the consistent NMP layer, Eq. 3, with
// per-layer recomputation of the MLP activations.
//
// Launch sequence of gnn_mp_backward (BF16):
//   k_proj_fwd    recompute P|Q = x W1a^T | x W1b^T (forward kernel)
//   k_node_bwd    recompute the node MLP from [a*, x], back-propagate dx_out:
//                 da* (FP32) and dx_in = dx_out + d[x part]; dW of the node MLP
//   halo          adjoint of Eq. 5c-5d = the same symmetric copy-sum on da*
//   k_edge_bwd    recompute the edge MLP per receiver-aligned tile; the
//                 gradient of e' is de_out + da_i / d_ij (adjoint of Eq. 5b);
//                 back-propagate to de_in = g + W1c^T dz1, write dz1 (the
//                 gradient of the first pre-activation) per edge, sum it over
//                 each receiver's edges into dP (FP32, fixed edge order); dW
//   k_proj_bwd    dQ_j = sum of dz1 over the edges sent by j (sender CSR,
//                 fixed order); dx_in += dP W1a + dQ W1b; dW1a, dW1b
//   k_reduce      per-CTA weight-gradient partials summed in CTA order into dW
// No atomics anywhere: every sum has a fixed order, so results are bitwise
// reproducible.
//
// Weight gradients accumulate in TMEM across all tiles a CTA processes:
// D_k[out][in] += dz_k^T h_k is one tcgen05.mma per 16 rows with both operands
// MN-major views of the tiles the chain already holds in shared memory; a
// constant block with a column of ones appended to h_k yields the bias
// gradient sum_rows dz_k in column `in = H_in` of the same accumulator.
// Thread layout: 128 rows x H/16 column groups of 16 columns.

#include <algorithm>
#include <cstring>

#include "fused.h"
#include "fused_bwd_common.cuh"
#include "plain.h"
#include "profiler.h"

namespace gnn {
namespace fused {

cudaError_t take_device_error_bwd(unsigned int* out) { return take_device_error_word(out); }

// ------------------------------------------------------------------ shared memory plans

struct EdgeBwdSmem {
    uint32_t w, e0, de, g, hb, ones, slot, par, seg, red, bar, tm, total;
};

// Edge-backward shared memory. g holds the tile's dz rows during the adjoint
// and, during the recompute, the aggregate gradients da of the tile's
// receivers (when they fit: nr * H * 4 <= TILE). hb holds the recomputed
// hidden activations and, once the adjoint no longer reads them, the staging
// of the segmented sum dP. slot: the next tile's P rows [128 x H], then each
// thread's Q columns for it.
template <int H>
__host__ __device__ inline EdgeBwdSmem edge_bwd_smem(int n_lin) {
    using C = CfgB<H>;
    EdgeBwdSmem s;
    s.w = 0;
    s.e0 = align_up(n_lin * C::WT, 1024);         // 2 stages of {e tile, de tile}
    s.de = s.e0 + C::TILE;
    s.seg = s.e0 + 4 * C::TILE;                    // 2 tile records (GNN_TILE_META_BYTES each)
    s.g = align_up(s.seg + 2 * GNN_TILE_META_BYTES, 1024);
    s.hb = s.g + C::TILE;
    const uint32_t hb_min = 128 * H * 4, hb_tiles = (uint32_t)(n_lin - 1) * C::TILE;
    const uint32_t hb_bytes = hb_tiles > hb_min ? hb_tiles : hb_min;
    s.ones = align_up(s.hb + hb_bytes, 1024);
    s.slot = align_up(s.ones + 128 * C::S, 1024);
    s.par = s.slot + 2 * C::TILE;
    s.red = s.par + (n_lin + 2) * H * 4;
    s.bar = align_up(s.red + 4 * C::CG * 128 * 4, 8);   // full[2], mma, ready, da, wgrad, P rows, h[GNN_MAX_LIN]
    s.tm = s.bar + 8 * (7 + GNN_MAX_LIN);
    uint32_t end = s.tm + 16;
    end = end > s.g + 32768 ? end : s.g + 32768;   // M-padded wgrad views read 32 KB from g
    s.total = end + 1024;
    return s;
}

struct NodeBwdSmem {
    uint32_t w0, w, ain, ones2, g, hb, ones, par, red, bar, tm, total;
};

template <int H>
__host__ __device__ inline NodeBwdSmem node_bwd_smem(int n_lin) {
    using C = CfgB<H>;
    NodeBwdSmem s;
    s.w0 = 0;
    s.w = align_up(2 * C::WT, 1024);
    s.ain = align_up(s.w + (n_lin - 1) * C::WT, 1024);
    s.ones2 = s.ain + 2 * C::TILE;                 // contiguous after ain: the next N-block of [ain ; ones]
    s.g = align_up(s.ones2 + 128 * C::S2, 1024);
    s.hb = s.g + C::TILE;
    s.ones = align_up(s.hb + (n_lin - 1) * C::TILE, 1024);
    s.par = align_up(s.ones + 128 * C::S, 16);
    s.red = s.par + (n_lin + 2) * H * 4;
    s.bar = align_up(s.red + 4 * C::CG * 128 * 4, 8);   // mma, wgrad, ready, h[GNN_MAX_LIN], xa
    s.tm = s.bar + 8 * (4 + GNN_MAX_LIN);
    uint32_t end = s.tm + 16;
    end = end > s.g + 32768 ? end : s.g + 32768;
    s.total = end + 1024;
    return s;
}

struct ProjBwdSmem {
    uint32_t w, a, x, bar, tm, total;
};

// H = 128 also stages each tile's sender-edge ids (up to kProjEids of them).
constexpr int kProjEids = 4096;

template <int H>
__host__ __device__ inline ProjBwdSmem proj_bwd_smem() {
    using C = CfgB<H>;
    ProjBwdSmem s;
    s.w = 0;
    s.a = align_up(2 * C::WT, 1024);
    s.x = s.a + 2 * C::TILE;
    s.bar = align_up(s.x + C::TILE + (H == 128 ? kProjEids * 4 : 0), 8);
    s.tm = s.bar + 16;
    uint32_t end = s.tm + 16;
    end = end > s.a + 32768 ? end : s.a + 32768;
    s.total = end + 1024;
    return s;
}

// TMEM column plans
template <int H>
__host__ __device__ inline uint32_t edge_bwd_tcols(int n_lin) { return H + n_lin * (H + 16); }
// ... plus the LayerNorm parameter-gradient accumulators (2H columns) when they fit
template <int H>
__host__ __device__ inline bool edge_bwd_ln_in_tmem(int n_lin) { return edge_bwd_tcols<H>(n_lin) + 2 * H <= 512; }
// Offset of the LayerNorm parameter gradients in a node-adjoint CTA's partials
// (after the weight-gradient blocks [H x (2H+16)] and (n_lin-1) x [H x (H+16)]).
template <int H>
__host__ __device__ inline int64_t node_ln_off(int n_lin) {
    return (int64_t)H * (2 * H + 16) + (int64_t)(n_lin - 1) * H * (H + 16);
}
template <int H>
__host__ __device__ inline uint32_t node_bwd_tcols(int n_lin) {
    return 2 * H + (2 * H + 16) + (n_lin - 1) * (H + 16);
}

// ------------------------------------------------------------------ k_node_bwd

struct NodeBwdArgs {
    const float* a_star;
    const float* x;
    const float* dx_out;
    float* da;          // out: gradient of a* (FP32)
    float* dx_in;       // out: dx_out + x part of the node-MLP input gradient
    float* part;        // per-CTA weight-gradient partials
    int64_t pstride;
    int64_t n_rows;
    MlpDev mlp;
    float eps;
    int64_t act_rows;   // SAVED: rows of one activation block of tmap_h (tiles * 128)
};

// SAVED: the forward stored the node MLP's hidden activations (block k, row
// k * act_rows + r, of tmap_h) and its BF16 input rows [a*, x] (tmap_xa); they
// arrive by TMA into the activation buffers and the input tile, each refilled
// with the next tile's rows once its last reader has passed (as in k_edge_bwd),
// and only the last Linear is recomputed; a* and x are not read.
template <int H, bool SAVED>
__global__ void __launch_bounds__(CfgB<H>::NT, 1) k_node_bwd(const __grid_constant__ CUtensorMap tmap_h,
                                                            const __grid_constant__ CUtensorMap tmap_xa,
                                                            NodeBwdArgs A) {
    using C = CfgB<H>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int L = A.mlp.n_lin;
    const NodeBwdSmem P = node_bwd_smem<H>(L);
    uint8_t* sW0 = sm + P.w0;
    uint8_t* sW = sm + P.w;
    uint8_t* sAin = sm + P.ain;
    uint8_t* sG = sm + P.g;
    uint8_t* sHB = sm + P.hb;
    uint8_t* sOnes = sm + P.ones;
    float* sPar = reinterpret_cast<float*>(sm + P.par);
    float* sRed = reinterpret_cast<float*>(sm + P.red);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.bar);   // MMA completion
    uint64_t* bar_w = bar + 1;                                  // weight-gradient MMAs of an adjoint step
    uint64_t* ready = bar + 2;                                  // one arrival per warp before an MMA
    uint64_t* h_full = bar + 3;                                 // SAVED: h_k of the tile has landed
    uint64_t* xa_full = bar + 3 + GNN_MAX_LIN;                  // SAVED: the tile's [a*, x] rows have landed
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + P.tm);
    constexpr int S = C::S, S2 = C::S2, CW = C::CW;
    const uint32_t NCOLS = pow2_cols(node_bwd_tcols<H>(L));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;

    if (warp == 0) {
        tmem_alloc(tslot, NCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar_w, 1);
        mbar_init(ready, C::NT / 32);
        if (SAVED) {
            for (int k = 0; k < L - 1; ++k) mbar_init(h_full + k, 1);
            mbar_init(xa_full, 1);
        }
        fence_mbar_init();
    }
    load_weight(sW0, A.mlp.W[0], 2 * H, 0, H, 2 * H, tid, C::NT);
    for (int k = 1; k < L; ++k) load_weight(sW + (k - 1) * C::WT, A.mlp.W[k], H, 0, H, H, tid, C::NT);
    fill_ones(sm + P.ones2, S2, tid, C::NT);
    fill_ones(sOnes, S, tid, C::NT);
    for (int i = tid; i < L * H; i += C::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < H; i += C::NT) {
        sPar[L * H + i] = A.mlp.gamma[i];
        sPar[(L + 1) * H + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tWork = tmem;
    auto tDW = [&](int k) -> uint32_t {
        return tmem + (uint32_t)(2 * H + (k == 0 ? 0 : (2 * H + 16) + (k - 1) * (H + 16)));
    };
    // LayerNorm parameter-gradient column sums, per warp (warp_colsum16): one register each
    constexpr int NCH = CW / 16;
    float acc_g[NCH], acc_b[NCH];
#pragma unroll
    for (int i = 0; i < NCH; ++i) acc_g[i] = acc_b[i] = 0.f;
    uint32_t ph = 0, ph_w = 0, ph_rdy = 0;
    bool ok = true, first = true;
    const int64_t n_tiles = (A.n_rows + 127) / 128;
    // MMA hand-off as in k_edge_bwd: warps arrive on `ready` after their operand writes and
    // accumulator reads, thread 0 issues, every thread waits on the completion barrier itself
    auto handoff = [&](auto&& issue, uint64_t* done) {
        fence_proxy_async();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(ready);
        if (tid == 0) {
            ok = ok && mbar_wait(ready, ph_rdy);
            ph_rdy ^= 1;
            tc_fence_after();
            if (ok) {
                issue();
                mma_commit(done);
            }
        }
    };
    auto mma_wait = [&]() {
        ok = ok && mbar_wait(bar, ph);
        ph ^= 1;
        __syncwarp();
        tc_fence_after();
    };
    const uint32_t hmask = SAVED ? ((1u << (L - 1)) - 1u) : 0u;
    uint32_t ph_h = 0, h_pend = 0;   // per-thread parity of h_full[k]; thread 0's loads not yet waited for
    auto load_h = [&](int k, int64_t tt) {
        mbar_arrive_expect_tx(h_full + k, C::TILE);
        tma_load_2d(sHB + k * C::TILE, &tmap_h, 0, (int32_t)(k * A.act_rows + tt * 128), h_full + k);
        h_pend |= 1u << k;
    };
    auto wait_h = [&](int k) {
        ok = ok && mbar_wait(h_full + k, (ph_h >> k) & 1u);
        h_pend &= ~(1u << k);
    };
    uint32_t ph_xa = 0;
    bool xa_pend = false;   // thread 0
    auto load_xa = [&](int64_t tt) {
        mbar_arrive_expect_tx(xa_full, 2 * C::TILE);
#pragma unroll
        for (int kb = 0; kb < 2 * H / (S2 / 2); ++kb)
            tma_load_2d(sAin + kb * 128 * S2, &tmap_xa, kb * (S2 / 2), (int32_t)(tt * 128), xa_full);
        xa_pend = true;
    };
    if (SAVED && tid == 0 && (int64_t)blockIdx.x < n_tiles) {
        for (int k = 0; k < L - 1; ++k) load_h(k, blockIdx.x);
        load_xa(blockIdx.x);
    }

    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        if (tid == 0 && t + gridDim.x < n_tiles) {   // the next tile's input rows into L2
            const int64_t rn = (t + gridDim.x) * 128;
            const uint32_t nb = (uint32_t)(std::min<int64_t>(128, A.n_rows - rn) * H * 4);
            prefetch_l2(A.a_star + rn * H, nb);
            prefetch_l2(A.x + rn * H, nb);
            prefetch_l2(A.dx_out + rn * H, nb);
        }
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        float gv[CW];
        if constexpr (SAVED) {
            if (valid) {
                const float4* pg = reinterpret_cast<const float4*>(A.dx_out + r * H + c0);
#pragma unroll
                for (int i = 0; i < CW / 4; ++i) {
                    const float4 z = __ldg(pg + i);
                    gv[4 * i] = z.x; gv[4 * i + 1] = z.y; gv[4 * i + 2] = z.z; gv[4 * i + 3] = z.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < CW; ++i) gv[i] = 0.f;
            }
        } else {
            float xv[CW], av[CW];
            if (valid) {
                const float4* pa = reinterpret_cast<const float4*>(A.a_star + r * H + c0);
                const float4* px = reinterpret_cast<const float4*>(A.x + r * H + c0);
                const float4* pg = reinterpret_cast<const float4*>(A.dx_out + r * H + c0);
#pragma unroll
                for (int i = 0; i < CW / 4; ++i) {
                    float4 u = __ldg(pa + i), w = __ldg(px + i), z = __ldg(pg + i);
                    av[4 * i] = u.x; av[4 * i + 1] = u.y; av[4 * i + 2] = u.z; av[4 * i + 3] = u.w;
                    xv[4 * i] = w.x; xv[4 * i + 1] = w.y; xv[4 * i + 2] = w.z; xv[4 * i + 3] = w.w;
                    gv[4 * i] = z.x; gv[4 * i + 1] = z.y; gv[4 * i + 2] = z.z; gv[4 * i + 3] = z.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < CW; ++i) av[i] = xv[i] = gv[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < CW; i += 8) {
                st_tile8(sAin, row, c0 + i, 128, S2, av + i);
                st_tile8(sAin, row, H + c0 + i, 128, S2, xv + i);
            }
        }
        // ---- recompute the chain (SAVED: only the last Linear, from the saved h_{L-2})
        float v[CW];
        if constexpr (SAVED) {
            if (tid == 0) {
                wait_h(L - 2);
                ok = ok && mbar_wait(xa_full, ph_xa);   // the input tile of the step-0 weight gradient
                ph_xa ^= 1;
                xa_pend = false;
                tc_fence_after();
                if (ok) {
                    issue_mma(tWork, sHB + (L - 2) * C::TILE, sW + (L - 2) * C::WT, H, H);
                    mma_commit(bar);
                }
            }
            mma_wait();
            ld_acc<CW>(tWork, q, c0, v);
            add_bias2<CW>(v, sPar + (L - 1) * H + c0);
        } else {
            handoff([&] { issue_mma(tWork, sAin, sW0, H, 2 * H); }, bar);
        }
        for (int k = 0; k < (SAVED ? 0 : L); ++k) {
            mma_wait();
            ld_acc<CW>(tWork, q, c0, v);
            add_bias2<CW>(v, sPar + k * H + c0);
            if (k < L - 1) {
                elu_inplace2<CW>(v);
                st_row_tile<CW>(sHB + k * C::TILE, row, c0, S, v);
                handoff([&] { issue_mma(tWork, sHB + k * C::TILE, sW + k * C::WT, H, H); }, bar);
            }
        }
        tc_fence_before();
        // ---- LayerNorm adjoint (statistics and adjoint sums in one exchange)
        float dz[CW];
#pragma unroll
        for (int i = 0; i < CW; ++i) dz[i] = gv[i] * sPar[L * H + c0 + i];
        float mean, rstd, s1, s2;
        row_stats_adj<H, C::CG, CW>(v, dz, sRed, row, g, A.eps, mean, rstd, s1, s2);
#pragma unroll
        for (int i = 0; i < CW; ++i) {
            v[i] = (v[i] - mean) * rstd;   // xhat
            dz[i] = rstd * (dz[i] - s1 - v[i] * s2);
        }
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            float t16[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) t16[i] = gv[16 * j + i] * v[16 * j + i];
            acc_g[j] += warp_colsum16(t16, lane);
            acc_b[j] += warp_colsum16(gv + 16 * j, lane);
        }
        // ---- chain adjoint, layer L-1 .. 0
        for (int k = L - 1; k >= 0; --k) {
            if (k < L - 1) {   // the previous step's wgrad reads sG
                ok = ok && mbar_wait(bar_w, ph_w);
                ph_w ^= 1;
            }
            if (SAVED && k > 0) wait_h(k - 1);   // this step's wgrad operand and ELU derivative input
            st_row_tile<CW>(sG, row, c0, S, dz);
            handoff([&] {
                if (k == 0) {
                    issue_dgrad(tWork, sG, S, sW0, S2, H, (uint32_t)H * S2, 2 * H, H);
                    mma_commit(bar);
                    issue_wgrad(tDW(0), sG, S, 128u * S, sAin, S2, 128u * S2, 2 * H + 16, !first);
                } else {
                    issue_dgrad(tWork, sG, S, sW + (k - 1) * C::WT, S, H, (uint32_t)H * S, H, H);
                    mma_commit(bar);
                    uint8_t* hk = sHB + (k - 1) * C::TILE;
                    issue_wgrad(tDW(k), sG, S, 128u * S, hk, S, (uint32_t)(smem_u32(sOnes) - smem_u32(hk)), H + 16,
                                !first);
                }
            }, bar_w);
            // SAVED: h_k's last reader (step k + 1) is done: the next tile's h_k goes there
            if (SAVED && tid == 0 && ok && k <= L - 2 && t + gridDim.x < n_tiles) load_h(k, t + gridDim.x);
            mma_wait();
            if (k > 0) {
                float dh[CW], hv[CW];
                ld_acc<CW>(tWork, q, c0, dh);
                ld_row_tile<CW>(sHB + (k - 1) * C::TILE, row, c0, S, hv);
                elu_bwd2<CW>(dz, dh, hv);
            } else {
                float da[CW], dxp[CW];
                ld_acc<CW>(tWork, q, c0, da);
                ld_acc<CW>(tWork, q, H + c0, dxp);
                if (valid) {
                    float4* pda = reinterpret_cast<float4*>(A.da + r * H + c0);
                    float4* pdx = reinterpret_cast<float4*>(A.dx_in + r * H + c0);
#pragma unroll
                    for (int i = 0; i < CW / 4; ++i) {
                        pda[i] = make_float4(da[4 * i], da[4 * i + 1], da[4 * i + 2], da[4 * i + 3]);
                        pdx[i] = make_float4(gv[4 * i] + dxp[4 * i], gv[4 * i + 1] + dxp[4 * i + 1],
                                             gv[4 * i + 2] + dxp[4 * i + 2], gv[4 * i + 3] + dxp[4 * i + 3]);
                    }
                }
            }
            tc_fence_before();
        }
        first = false;
        ok = ok && mbar_wait(bar_w, ph_w);   // the last wgrad reads sAin and sG
        ph_w ^= 1;
        ph_h ^= hmask;
        if (SAVED && tid == 0 && ok && t + gridDim.x < n_tiles) load_xa(t + gridDim.x);   // sAin is free
        if (__syncthreads_or(!ok)) break;   // the block leaves together after a timeout
        tc_fence_after();
    }
    if (SAVED && tid == 0) {   // loads issued before a timeout ended the tile loop
        for (int k = 0; k < L - 1; ++k)
            if ((h_pend >> k) & 1u) mbar_wait(h_full + k, (ph_h >> k) & 1u);
        if (xa_pend) mbar_wait(xa_full, ph_xa);
    }
    // ---- flush the CTA's partial gradients
    tc_fence_before();
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (ok) {
        int64_t off = 0;
        for (int k = 0; k < L; ++k) {
            const int N = k == 0 ? 2 * H + 16 : H + 16;
            if (!first) flush_acc<C::CG>(tDW(k), N, H, q, lane, g, part + off);
            else
                for (int i = tid; i < H * N; i += C::NT) part[off + i] = 0.f;
            off += (int64_t)H * N;
        }
    }
    colsum_store<H, NCH>(acc_g, sRed, q, lane, c0, tid, C::NT, part + node_ln_off<H>(L));
    colsum_store<H, NCH>(acc_b, sRed, q, lane, c0, tid, C::NT, part + node_ln_off<H>(L) + H);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ------------------------------------------------------------------ k_edge_bwd

struct EdgeBwdArgs {
    const uint8_t* tile_meta;   // per-tile records (GNN_TILE_META_BYTES each)
    int64_t n_tiles;
    const __nv_bfloat16* pq;    // P rows [n_rows x H]
    const __nv_bfloat16* q;     // Q rows [n_rows x H]
    const float* da;            // gradient of the aggregate after the halo adjoint
    int has_de_out;
    __nv_bfloat16* de_in;
    __nv_bfloat16* dz1;         // per-edge gradient of the first pre-activation
    float* dP;                  // per-row sum of dz1 over the row's received edges
    float* part;
    int64_t pstride;
    MlpDev mlp;
    float eps;
    int64_t act_rows;           // SAVED: rows of one activation block of tmap_h (tiles * 128)
};

// LNT: the per-thread LayerNorm gradient sums live in TMEM columns after the
// weight-gradient accumulators (read, add, write back once per tile) instead
// of 2*CW registers.
// SAVED: the forward stored the hidden activations h_0 .. h_{L-2} of every edge
// (row k * act_rows + t * 128 + i of tmap_h for edge row i of tile t); the tile's rows arrive by TMA into the
// activation buffers and only the last Linear is recomputed (no P|Q gather, no
// ELU chain). Buffer k is refilled with the next tile's rows as soon as the
// adjoint step that reads it last has passed its hand-off, so the loads have
// most of a tile's time to land; the dP staging moves to the P|Q slot area.
template <int H, bool LNT, bool SAVED>
__global__ void __launch_bounds__(CfgB<H>::NT, 1) k_edge_bwd(const __grid_constant__ CUtensorMap tmap_e,
                                                            const __grid_constant__ CUtensorMap tmap_de,
                                                            const __grid_constant__ CUtensorMap tmap_h,
                                                            EdgeBwdArgs A) {
    using C = CfgB<H>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int L = A.mlp.n_lin;
    const EdgeBwdSmem P = edge_bwd_smem<H>(L);
    uint8_t* sW = sm + P.w;
    uint8_t* sStg0 = sm + P.e0;       // stage s: e tile at +2*s*TILE, de tile right after it
    uint8_t* sRec0 = sm + P.seg;      // stage s: tile record at +s*GNN_TILE_META_BYTES
    uint8_t* sG = sm + P.g;
    uint8_t* sHB = sm + P.hb;
    uint8_t* sOnes = sm + P.ones;
    float* sStage = reinterpret_cast<float*>(SAVED ? sm + P.slot : sHB);   // dP staging at the last adjoint step
    float* sPar = reinterpret_cast<float*>(sm + P.par);
    float* sRed = reinterpret_cast<float*>(sm + P.red);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + P.bar);   // full[2]: stage loaded
    uint64_t* bar = full + 2;       // MMA completion
    uint64_t* ready = full + 3;     // one arrival per warp: operands written, accumulator read
    uint64_t* da_full = full + 4;   // the tile's da rows have landed in sG
    uint64_t* bar_w = full + 5;     // weight-gradient MMAs of an adjoint step (complete behind the epilogue)
    uint64_t* p_full = full + 6;    // the tile's P rows have landed in sP
    uint64_t* h_full = full + 7;    // SAVED: h_k of the tile has landed in sHB + k * TILE
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + P.tm);
    constexpr int S = C::S, CW = C::CW;
    const uint32_t NCOLS = pow2_cols(edge_bwd_tcols<H>(L) + (LNT ? 2 * H : 0));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;
    constexpr int NCH = 2 * CW / 16;                               // 16-byte chunks of a Q slot
    uint8_t* sP = sm + P.slot;                                     // P rows of the tile's receivers
    uint8_t* sSlot = sm + P.slot + C::TILE + (g * 128 + row) * (2 * CW);
    auto slot_at = [&](int k) { return sSlot + 16 * (k ^ ((row >> (NCH >= 8 ? 0 : (NCH == 4 ? 1 : 2))) & (NCH - 1))); };

    if (warp == 0) {
        tmem_alloc(tslot, NCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(full, 1);
        mbar_init(full + 1, 1);
        mbar_init(bar, 1);
        mbar_init(ready, C::NT / 32);
        mbar_init(da_full, 1);
        mbar_init(bar_w, 1);
        mbar_init(p_full, 1);
        if (SAVED)
            for (int k = 0; k < L - 1; ++k) mbar_init(h_full + k, 1);
        fence_mbar_init();
    }
    load_weight(sW, A.mlp.W[0], 3 * H, 2 * H, H, H, tid, C::NT);
    for (int k = 1; k < L; ++k) load_weight(sW + k * C::WT, A.mlp.W[k], H, 0, H, H, tid, C::NT);
    fill_ones(sOnes, S, tid, C::NT);
    for (int i = tid; i < L * H; i += C::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < H; i += C::NT) {
        sPar[L * H + i] = A.mlp.gamma[i];
        sPar[(L + 1) * H + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tWork = tmem;
    auto tDW = [&](int k) -> uint32_t { return tmem + (uint32_t)(H + k * (H + 16)); };
    const uint32_t ones_addr = smem_u32(sOnes);
    // LayerNorm gradient sums sum_rows g * xhat and sum_rows g: in TMEM (LNT, one lane per
    // row), else as per-warp column sums (warp_colsum16, one register per 16 columns)
    constexpr int ACW = LNT ? 1 : CW / 16;
    float acc_g[ACW], acc_b[ACW];
#pragma unroll
    for (int i = 0; i < ACW; ++i) acc_g[i] = acc_b[i] = 0.f;
    const uint32_t tLN = tmem + ((uint32_t)(32 * q) << 16) + edge_bwd_tcols<H>(L) + (uint32_t)(g * 2 * CW);
    if constexpr (LNT) {
        float z[16] = {};
#pragma unroll
        for (int i = 0; i < 2 * CW; i += 16) tmem_st16(tLN + i, z);
        tmem_st_wait();
    }
    uint32_t ph = 0, ph_rdy = 0, ph_da = 0, ph_w = 0, ph_p = 0;
    bool ok = true, first = true;
    // MMA hand-off without block barriers: every warp arrives on `ready` once its
    // operand writes and its TMEM reads of the accumulator are done; thread 0
    // waits for all warps, issues and commits to `bar`; every thread waits on
    // `bar` by itself. After a timeout a thread stops waiting and issuing; the
    // block leaves the tile loop together at the tile-end barrier.
    auto handoff = [&](auto&& issue, uint64_t* done) {
        fence_proxy_async();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(ready);
        if (tid == 0) {
            ok = ok && mbar_wait(ready, ph_rdy);
            ph_rdy ^= 1;
            tc_fence_after();
            if (ok) {
                issue();
                mma_commit(done);
            }
        }
    };
    auto mma_wait = [&]() {
        ok = ok && mbar_wait(bar, ph);
        ph ^= 1;
        __syncwarp();
        tc_fence_after();
    };
    const uint32_t tx_bytes = C::TILE * (A.has_de_out ? 2 : 1) + GNN_TILE_META_BYTES;
    // stage s <- tile t: its record by bulk copy, its e (and de_out) rows by TMA
    // (e0: the tile's first edge, read from its global record one tile in advance)
    auto issue_stage = [&](int s, int64_t t, int32_t e0) {
        uint8_t* rec = sRec0 + s * GNN_TILE_META_BYTES;
        uint8_t* se = sStg0 + s * 2 * C::TILE;
        mbar_arrive_expect_tx(full + s, tx_bytes);
        bulk_load(rec, A.tile_meta + t * GNN_TILE_META_BYTES, GNN_TILE_META_BYTES, full + s);
        tma_load_2d(se, &tmap_e, 0, e0, full + s);
        if (A.has_de_out) tma_load_2d(se + C::TILE, &tmap_de, 0, e0, full + s);
    };
    // the receivers' P rows of the tile whose record is in stage s: one bulk copy of the
    // tile's consecutive rows (thread 0); this thread's Q slot <- the Q row of its edge's
    // sender, own columns, by cp.async
    bool p_pending = false;   // thread 0: a P copy not yet consumed (waited for before exit)
    auto fetch_p = [&](int s) {
        p_pending = true;
        const int32_t* hdr = reinterpret_cast<const int32_t*>(sRec0 + s * GNN_TILE_META_BYTES);
        const int32_t nr = min(max(hdr[1] - hdr[0], 0), 128);   // a tile has 1..128 rows
        const uint32_t bytes = (uint32_t)nr * H * 2;
        if (bytes == 0) {
            mbar_arrive(p_full);
            return;
        }
        mbar_arrive_expect_tx(p_full, bytes);
        bulk_load(sP, A.pq + (int64_t)hdr[0] * H, bytes, p_full);
    };
    auto gather = [&](int s) {
        const uint8_t* rec = sRec0 + s * GNN_TILE_META_BYTES;
        if (row < reinterpret_cast<const int32_t*>(rec)[3]) {
            const int64_t snd = reinterpret_cast<const int32_t*>(rec + 800)[row];
#pragma unroll
            for (int k = 0; k < NCH; ++k) cp_async16(slot_at(k), A.q + snd * H + c0 + 8 * k);
        }
        cp_async_commit();
        if (tid == 0) fetch_p(s);
    };
    auto first_edge = [&](int64_t t) { return ld_nc_s32(A.tile_meta + t * GNN_TILE_META_BYTES + 8); };
    // SAVED: h_k rows of the tile starting at edge eh into buffer k (thread 0); per-thread
    // parity bit k of h_full[k] (one phase per tile); thread 0's loads not yet waited for
    const uint32_t hmask = SAVED ? ((1u << (L - 1)) - 1u) : 0u;
    uint32_t ph_h = 0, h_pend = 0;
    auto load_h = [&](int k, int64_t tt) {
        mbar_arrive_expect_tx(h_full + k, C::TILE);
        tma_load_2d(sHB + k * C::TILE, &tmap_h, 0, (int32_t)(k * A.act_rows + tt * 128), h_full + k);
        h_pend |= 1u << k;
    };
    auto wait_h = [&](int k) {
        ok = ok && mbar_wait(h_full + k, (ph_h >> k) & 1u);
        h_pend &= ~(1u << k);
    };
    int32_t e0_next = 0;   // thread 0: first edge of the CTA's next tile
    if (tid == 0 && (int64_t)blockIdx.x < A.n_tiles) {
        issue_stage(0, blockIdx.x, first_edge(blockIdx.x));
        if (SAVED)
            for (int k = 0; k < L - 1; ++k) load_h(k, blockIdx.x);
        if ((int64_t)blockIdx.x + gridDim.x < A.n_tiles) e0_next = first_edge(blockIdx.x + gridDim.x);
    }
    if ((int64_t)blockIdx.x < A.n_tiles) {
        ok = mbar_wait(full, 0);
        if (ok && !SAVED) gather(0);
    }
    int j = 0;

    for (int64_t t = blockIdx.x; t < A.n_tiles; t += gridDim.x, ++j) {
        const int st = j & 1;
        ok = ok && mbar_wait(full + st, (uint32_t)(j >> 1) & 1u);
        __syncwarp();
        const uint8_t* rec = sRec0 + st * GNN_TILE_META_BYTES;
        const int32_t* hdr = reinterpret_cast<const int32_t*>(rec);
        const int32_t* sRp = reinterpret_cast<const int32_t*>(rec + 16);
        const int16_t* sSeg = reinterpret_cast<const int16_t*>(rec + 544);
        const float* sW1d = reinterpret_cast<const float*>(rec + 1312);
        uint8_t* sE0 = sStg0 + st * 2 * C::TILE;
        uint8_t* sDE = sE0 + C::TILE;
        const int32_t r0 = hdr[0], r1 = hdr[1], e0 = hdr[2], ne = hdr[3];
        const bool valid = row < ne;
        const int64_t eg = (int64_t)e0 + row;
        // the receivers' da rows into sG for the LayerNorm adjoint (sG is free until then)
        const bool da_bulk = (r1 - r0) * H * 4 <= C::TILE;
        if (tid == 0 && ok && da_bulk) {
            mbar_arrive_expect_tx(da_full, (uint32_t)(r1 - r0) * H * 4);
            bulk_load(sG, A.da + (int64_t)r0 * H, (uint32_t)(r1 - r0) * H * 4, da_full);
        }
        if (tid == 0 && ok) {
            if (SAVED) wait_h(L - 2);
            tc_fence_after();
            if (ok) {
                if (SAVED) issue_mma(tWork, sHB + (L - 2) * C::TILE, sW + (L - 1) * C::WT, H, H);
                else issue_mma(tWork, sE0, sW, H, H);
                mma_commit(bar);
            }
            // the other stage was released at the end of the previous tile: prefetch the next tile
            if (t + gridDim.x < A.n_tiles) {
                issue_stage(st ^ 1, t + gridDim.x, e0_next);
                if (t + 2 * (int64_t)gridDim.x < A.n_tiles) e0_next = first_edge(t + 2 * (int64_t)gridDim.x);
            }
        }
        // ---- recompute the chain (SAVED: only the last Linear, from the saved h_{L-2})
        float v[CW];
        if constexpr (SAVED) {
            mma_wait();
            ld_acc<CW>(tWork, q, c0, v);
            add_bias2<CW>(v, sPar + (L - 1) * H + c0);
        }
        if constexpr (!SAVED) cp_async_wait_all();   // this thread's P|Q slot for the tile
        for (int k = 0; k < (SAVED ? 0 : L); ++k) {
            mma_wait();
            ld_acc<CW>(tWork, q, c0, v);
            if (k == 0) {
                ok = ok && mbar_wait(p_full, ph_p);   // the tile's P rows
                ph_p ^= 1;
                p_pending = false;
                if (valid) {
                    const uint8_t* prow = sP + (int)sSeg[row] * (2 * H) + 2 * c0;
#pragma unroll
                    for (int kc = 0; kc < NCH; ++kc) {
                        const uint4 up = *reinterpret_cast<const uint4*>(prow + 16 * kc);
                        const uint4 uq = *reinterpret_cast<const uint4*>(slot_at(kc));
                        const uint32_t pw[4] = {up.x, up.y, up.z, up.w}, qw[4] = {uq.x, uq.y, uq.z, uq.w};
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            float p0, p1, q0, q1;
                            unpack_bf16x2(pw[h], p0, p1);
                            unpack_bf16x2(qw[h], q0, q1);
                            const float2 t2 = __fadd2_rn(__fadd2_rn(make_float2(p0, p1), make_float2(q0, q1)),
                                                         *reinterpret_cast<const float2*>(sPar + c0 + 8 * kc + 2 * h));
                            float2* vv = reinterpret_cast<float2*>(v + 8 * kc + 2 * h);
                            *vv = __fadd2_rn(*vv, t2);
                        }
                    }
                } else {
                    add_bias2<CW>(v, sPar + c0);
                }

            } else {
                add_bias2<CW>(v, sPar + k * H + c0);
            }
            if (k < L - 1) {
                elu_inplace2<CW>(v);
                st_row_tile<CW>(sHB + k * C::TILE, row, c0, S, v);
                handoff([&] { issue_mma(tWork, sHB + k * C::TILE, sW + (k + 1) * C::WT, H, H); }, bar);
            }
        }
        tc_fence_before();
        // ---- gradient of e' (adjoint of Eq. 5b plus the upstream edge gradient)
        float gv[CW];
        if (da_bulk) {
            ok = ok && mbar_wait(da_full, ph_da);
            ph_da ^= 1;
        }
        if (valid) {
            float dar[CW];
            const float* src = da_bulk ? reinterpret_cast<const float*>(sG) + (int64_t)sSeg[row] * H + c0
                                       : A.da + (int64_t)(r0 + sSeg[row]) * H + c0;
#pragma unroll
            for (int i = 0; i < CW / 4; ++i) {
                const float4 u = *reinterpret_cast<const float4*>(src + 4 * i);
                dar[4 * i] = u.x; dar[4 * i + 1] = u.y; dar[4 * i + 2] = u.z; dar[4 * i + 3] = u.w;
            }
            const float w = sW1d[row];
            float deo[CW];
            if (A.has_de_out) ld_row_tile<CW>(sDE, row, c0, S, deo);
#pragma unroll
            for (int i = 0; i < CW; ++i) gv[i] = (A.has_de_out ? deo[i] : 0.f) + w * dar[i];
        } else {
#pragma unroll
            for (int i = 0; i < CW; ++i) gv[i] = 0.f;
        }
        // ---- LayerNorm adjoint (statistics and adjoint sums in one exchange)
        float dz[CW];
#pragma unroll
        for (int i = 0; i < CW; ++i) dz[i] = gv[i] * sPar[L * H + c0 + i];
        float mean, rstd, s1, s2;
        row_stats_adj<H, C::CG, CW>(v, dz, sRed, row, g, A.eps, mean, rstd, s1, s2);
#pragma unroll
        for (int i = 0; i < CW; ++i) v[i] = (v[i] - mean) * rstd;   // xhat
        if constexpr (LNT) {
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
        } else {
#pragma unroll
            for (int j = 0; j < ACW; ++j) {
                float t16[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) t16[i] = gv[16 * j + i] * v[16 * j + i];
                acc_g[j] += warp_colsum16(t16, lane);
                acc_b[j] += warp_colsum16(gv + 16 * j, lane);
            }
        }
#pragma unroll
        for (int i = 0; i < CW; ++i) dz[i] = rstd * (dz[i] - s1 - v[i] * s2);
        // ---- chain adjoint
        for (int k = L - 1; k >= 0; --k) {
            if (k < L - 1) {   // the previous step's wgrad reads sG: wait for it (per thread, no barrier)
                ok = ok && mbar_wait(bar_w, ph_w);
                ph_w ^= 1;
            }
            if (SAVED && k > 0) wait_h(k - 1);   // this step's wgrad operand and ELU derivative input
            st_row_tile<CW>(sG, row, c0, S, dz);
            handoff([&] {
                issue_dgrad(tWork, sG, S, sW + k * C::WT, S, H, (uint32_t)H * S, H, H);
                mma_commit(bar);
                uint8_t* hk = (k == 0) ? sE0 : sHB + (k - 1) * C::TILE;
                issue_wgrad(tDW(k), sG, S, 128u * S, hk, S, ones_addr - smem_u32(hk), H + 16, !first);
            }, bar_w);
            // SAVED: every thread has passed its last read of h_k (step k + 1) and its wgrad has
            // completed (bar_w, waited at the top of this step): the next tile's h_k goes there
            if (SAVED && tid == 0 && ok && k <= L - 2 && t + gridDim.x < A.n_tiles) load_h(k, t + gridDim.x);
            if (!SAVED && k == L - 1 && t + gridDim.x < A.n_tiles) {
                // the slot was consumed by the first recompute step and the next tile's stage
                // (issued at this tile's start) has landed by now: request its P|Q rows
                if (mbar_wait(full + (st ^ 1), (uint32_t)((j + 1) >> 1) & 1u)) gather(st ^ 1);
            }
            if (k == 0) {
                // dz1 per edge (for the sender-side sum; from sG, after the barrier below) and its
                // receiver-side segmented sum
                constexpr int NC = H / 4;
                float4* sS4 = reinterpret_cast<float4*>(sStage);
                if (!SAVED) __syncthreads();   // every warp is past its last read of hb, which the staging overwrites
#pragma unroll
                for (int i = 0; i < CW / 4; ++i)
                    sS4[row * NC + stage_chunk<NC>(c0 / 4 + i, row)] =
                        make_float4(dz[4 * i], dz[4 * i + 1], dz[4 * i + 2], dz[4 * i + 3]);
                __syncthreads();
                {   // whole rows per warp: the tile's dz1 rows, as the MMAs read them from sG
                    constexpr int CPR = H / 8;   // 16-byte chunks per row
                    for (int i = tid; i < ne * CPR; i += C::NT) {
                        const int r = i / CPR, jj = i - r * CPR;
                        *reinterpret_cast<uint4*>(A.dz1 + ((int64_t)e0 + r) * H + 8 * jj) =
                            *reinterpret_cast<const uint4*>(sG + tile_off(r, 8 * jj, 128, S));
                    }
                }
                const int nr = r1 - r0;
                for (int it = tid; it < nr * NC; it += C::NT) {
                    const int rr = it / NC, c = it % NC;
                    const int32_t b0 = sRp[rr], b1 = sRp[rr + 1];
                    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                    for (int32_t e = b0; e < b1; ++e) {
                        const float4 u4 = sS4[e * NC + stage_chunk<NC>(c, e)];
                        acc.x += u4.x;
                        acc.y += u4.y;
                        acc.z += u4.z;
                        acc.w += u4.w;
                    }
                    *reinterpret_cast<float4*>(A.dP + (int64_t)(r0 + rr) * H + 4 * c) = acc;
                }
            }
            mma_wait();
            float dh[CW];
            ld_acc<CW>(tWork, q, c0, dh);
            if (k > 0) {
                float hv[CW];
                ld_row_tile<CW>(sHB + (k - 1) * C::TILE, row, c0, S, hv);
                elu_bwd2<CW>(dz, dh, hv);
            } else {
                float o[CW];
#pragma unroll
                for (int i = 0; i < CW; ++i) o[i] = gv[i] + dh[i];      // residual + W1c^T dz1
                st_row_tile<CW>(sDE, row, c0, S, o);   // copied out by whole rows after the next barrier
            }
            tc_fence_before();
        }
        first = false;
        ok = ok && mbar_wait(bar_w, ph_w);   // the last wgrad reads this tile's e stage and sG
        ph_w ^= 1;
        ph_h ^= hmask;
        __syncthreads();   // every row of de_in is in the stage's de tile
        {
            constexpr int CPR = H / 8;
            for (int i = tid; i < ne * CPR; i += C::NT) {
                const int r = i / CPR, jj = i - r * CPR;
                *reinterpret_cast<uint4*>(A.de_in + ((int64_t)e0 + r) * H + 8 * jj) =
                    *reinterpret_cast<const uint4*>(sDE + tile_off(r, 8 * jj, 128, S));
            }
        }
        fence_proxy_async();
        if (__syncthreads_or(!ok)) break;   // stage release; the block leaves together after a timeout
        tc_fence_after();
    }
    if (p_pending) mbar_wait(p_full, ph_p);
    if (SAVED && tid == 0)   // loads issued before a timeout ended the tile loop
        for (int k = 0; k < L - 1; ++k)
            if ((h_pend >> k) & 1u) mbar_wait(h_full + k, (ph_h >> k) & 1u);
    cp_async_wait_all();
    tc_fence_before();
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (ok) {
        int64_t off = 0;
        for (int k = 0; k < L; ++k) {
            const int N = H + 16;
            if (!first) flush_acc<C::CG>(tDW(k), N, H, q, lane, g, part + off);
            else
                for (int i = tid; i < H * N; i += C::NT) part[off + i] = 0.f;
            off += (int64_t)H * N;
        }
        if constexpr (LNT) {
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
    if constexpr (!LNT) {   // after the L weight-gradient blocks [H x (H+16)]
        const int64_t ln_off = (int64_t)L * H * (H + 16);
        colsum_store<H, ACW>(acc_g, sRed, q, lane, c0, tid, C::NT, part + ln_off);
        colsum_store<H, ACW>(acc_b, sRed, q, lane, c0, tid, C::NT, part + ln_off + H);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ------------------------------------------------------------------ k_proj_bwd

struct ProjBwdArgs {
    const float* x;
    const float* dP;
    const __nv_bfloat16* dz1;
    const int32_t* t_ptr;
    const int32_t* t_eid;
    const float* W1;
    float* dx_in;       // += dP W1a + dQ W1b
    float* part;
    int64_t pstride;
    int64_t n_rows;
};

// Thread layout: 128 rows x H/32 column groups of 32 columns (two CTAs per SM).
template <int H>
struct CfgP {
    static constexpr int S = span_of(H);
    static constexpr int S2 = span_of(2 * H);
    static constexpr int CG = H >= 32 ? H / 32 : 1;
    static constexpr int CW = H / CG;
    static constexpr int NT = 128 * CG;
};

// Two CTAs per SM up to H = 64; at H = 128 one (registers and shared memory).
// The weight gradient [dW1a; dW1b] = [dP dQ]^T x is one M = 2H MMA up to
// H = 64 and two M = 128 halves at H = 128.
template <int H>
__global__ void __launch_bounds__(CfgP<H>::NT, H >= 128 ? 1 : 2) k_proj_bwd(ProjBwdArgs A) {
    using C = CfgP<H>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const ProjBwdSmem P = proj_bwd_smem<H>();
    uint8_t* sW = sm + P.w;
    uint8_t* sA = sm + P.a;
    uint8_t* sX = sm + P.x;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + P.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + P.tm);
    constexpr int S = C::S, S2 = C::S2, CW = C::CW;
    constexpr bool MSPLIT = 2 * H > 128;
    constexpr uint32_t NCOLS = pow2_cols(MSPLIT ? 3 * H : 2 * H);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;

    if (warp == 0) {
        tmem_alloc(tslot, NCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    // [W1a; W1b] as a [2H x H] row tile (rows = stacked outputs, contiguous = inputs)
    load_weight(sW, A.W1, 3 * H, 0, H, H, tid, C::NT, 2 * H, 0);
    load_weight(sW, A.W1, 3 * H, H, H, H, tid, C::NT, 2 * H, H);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tWork = tmem, tDW = tmem + H;
    uint32_t ph = 0;
    bool ok = true, first = true;
    const int64_t n_tiles = (A.n_rows + 127) / 128;

    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        if (tid == 0 && t + gridDim.x < n_tiles) {   // the next tile's input rows into L2
            const int64_t rn = (t + gridDim.x) * 128;
            const int64_t nr = std::min<int64_t>(128, A.n_rows - rn);
            prefetch_l2(A.dP + rn * H, (uint32_t)(nr * H * 4));
            prefetch_l2(A.x + rn * H, (uint32_t)(nr * H * 4));
            if constexpr (H == 128) prefetch_l2(A.dx_in + rn * H, (uint32_t)(nr * H * 4));   // its update
        }
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        if constexpr (H == 128) {
            // warp-cooperative rows: warp w fills rows 8w .. 8w+7 of the operand tiles, lane l
            // columns 4l .. 4l+3, so every dz1, dP and x row is one coalesced 256/512-byte read
            // (the sender-side sum of each column still runs over the edges in order)
            constexpr int UE = 4;   // edges per row requested together, for all eight rows at once
            // the tile's sender-edge ids are one contiguous range of t_eid: staged in shared
            // memory by one coalesced read when it fits, so each gather is a single round trip
            int32_t* sTe = reinterpret_cast<int32_t*>(sX + 128 * H * 2);
            const int64_t rt0 = t * 128, rt1 = min(A.n_rows, rt0 + 128);
            const int32_t kt0 = __ldg(A.t_ptr + rt0), kt1 = __ldg(A.t_ptr + rt1);
            const bool staged = kt1 - kt0 <= kProjEids;
            if (staged)
                for (int i = tid; i < kt1 - kt0; i += C::NT) sTe[i] = __ldg(A.t_eid + kt0 + i);
            __syncthreads();
            int32_t k0[8], deg[8];
            int maxdeg = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t rg = t * 128 + 8 * warp + i;
                k0[i] = rg < A.n_rows ? __ldg(A.t_ptr + rg) : 0;
                deg[i] = rg < A.n_rows ? __ldg(A.t_ptr + rg + 1) - k0[i] : 0;
                maxdeg = max(maxdeg, deg[i]);
            }
            float4 dq[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) dq[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int kb = 0; kb < maxdeg; kb += UE) {
                uint2 z[8][UE];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int u = 0; u < UE; ++u) {
                        const int32_t k = k0[i] + kb + u;
                        const int64_t e = kb + u < deg[i] ? (int64_t)(staged ? sTe[k - kt0] : __ldg(A.t_eid + k)) : -1;
                        z[i][u] = e >= 0 ? __ldg(reinterpret_cast<const uint2*>(A.dz1 + e * H) + lane)
                                         : make_uint2(0u, 0u);
                    }
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int u = 0; u < UE; ++u) {
                        if (kb + u < deg[i]) {
                            float f0, f1, f2, f3;
                            unpack_bf16x2(z[i][u].x, f0, f1);
                            unpack_bf16x2(z[i][u].y, f2, f3);
                            dq[i].x += f0;
                            dq[i].y += f1;
                            dq[i].z += f2;
                            dq[i].w += f3;
                        }
                    }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int rr = 8 * warp + i;
                const int64_t rg = t * 128 + rr;
                float4 dp = make_float4(0.f, 0.f, 0.f, 0.f), xv = dp;
                if (rg < A.n_rows) {
                    dp = __ldg(reinterpret_cast<const float4*>(A.dP + rg * H) + lane);
                    xv = __ldg(reinterpret_cast<const float4*>(A.x + rg * H) + lane);
                }
                *reinterpret_cast<uint2*>(sA + tile_off(rr, H + 4 * lane, 128, S2)) =
                    make_uint2(pack_bf16x2(dq[i].x, dq[i].y), pack_bf16x2(dq[i].z, dq[i].w));
                *reinterpret_cast<uint2*>(sA + tile_off(rr, 4 * lane, 128, S2)) =
                    make_uint2(pack_bf16x2(dp.x, dp.y), pack_bf16x2(dp.z, dp.w));
                *reinterpret_cast<uint2*>(sX + tile_off(rr, 4 * lane, 128, S)) =
                    make_uint2(pack_bf16x2(xv.x, xv.y), pack_bf16x2(xv.z, xv.w));
            }
        } else {
            float dq[CW];
#pragma unroll
            for (int i = 0; i < CW; ++i) dq[i] = 0.f;
            if (valid) {
                // sender-side sum in edge order; the edge ids and then the dz1 rows of UB
                // edges are requested together so their latencies overlap
                constexpr int UB = CW >= 32 ? 2 : 4;
                const int32_t k0 = A.t_ptr[r], k1 = A.t_ptr[r + 1];
                for (int32_t kb = k0; kb < k1; kb += UB) {
                    int64_t e[UB];
#pragma unroll
                    for (int u = 0; u < UB; ++u) e[u] = kb + u < k1 ? (int64_t)__ldg(A.t_eid + kb + u) : -1;
                    uint4 z[UB][CW / 8];
#pragma unroll
                    for (int u = 0; u < UB; ++u)
#pragma unroll
                        for (int i = 0; i < CW / 8; ++i)
                            z[u][i] = e[u] >= 0 ? __ldg(reinterpret_cast<const uint4*>(A.dz1 + e[u] * H + c0) + i)
                                                : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                    for (int u = 0; u < UB; ++u) {
                        if (e[u] < 0) break;
#pragma unroll
                        for (int i = 0; i < CW / 8; ++i) {
                            float f[8];
                            unpack_bf16x2(z[u][i].x, f[0], f[1]);
                            unpack_bf16x2(z[u][i].y, f[2], f[3]);
                            unpack_bf16x2(z[u][i].z, f[4], f[5]);
                            unpack_bf16x2(z[u][i].w, f[6], f[7]);
#pragma unroll
                            for (int j = 0; j < 8; ++j) dq[8 * i + j] += f[j];
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < CW; i += 8) st_tile8(sA, row, H + c0 + i, 128, S2, dq + i);
            {
                float dp[CW], xv[CW];
#pragma unroll
                for (int i = 0; i < CW; ++i) dp[i] = xv[i] = 0.f;
                if (valid) {
                    const float4* pp = reinterpret_cast<const float4*>(A.dP + r * H + c0);
                    const float4* px = reinterpret_cast<const float4*>(A.x + r * H + c0);
#pragma unroll
                    for (int i = 0; i < CW / 4; ++i) {
                        float4 u = __ldg(pp + i), w = __ldg(px + i);
                        dp[4 * i] = u.x; dp[4 * i + 1] = u.y; dp[4 * i + 2] = u.z; dp[4 * i + 3] = u.w;
                        xv[4 * i] = w.x; xv[4 * i + 1] = w.y; xv[4 * i + 2] = w.z; xv[4 * i + 3] = w.w;
                    }
                }
#pragma unroll
                for (int i = 0; i < CW; i += 8) st_tile8(sA, row, c0 + i, 128, S2, dp + i);
                st_row_tile<CW>(sX, row, c0, S, xv);
            }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_dgrad(tWork, sA, S2, sW, S, 2 * H, (uint32_t)(2 * H) * S, H, 2 * H);
            if constexpr (MSPLIT) {   // dW1a from the dP columns, dW1b from the dQ columns
                issue_wgrad(tDW, sA, S2, 128u * S2, sX, S, 128u * S, H, !first);
                issue_wgrad(tDW + H, sA + (H / (S2 / 2)) * 128 * S2, S2, 128u * S2, sX, S, 128u * S, H, !first);
            } else {
                issue_wgrad(tDW, sA, S2, 128u * S2, sX, S, 128u * S, H, !first);
            }
            mma_commit(bar);
        }
        ok = block_wait(bar, ph, tid);
        ph ^= 1;
        tc_fence_after();
        if (!ok) break;
        float d[CW];
        ld_acc<CW>(tWork, q, c0, d);
        tc_fence_before();
        if constexpr (H == 128) {
            // dx_in += d as whole rows per warp: the MMAs have read the operand tile, which now
            // stages the FP32 rows [128 x 128] (row r at 512 r bytes, 16-byte chunks swizzled by r)
            float4* sD = reinterpret_cast<float4*>(sA);
#pragma unroll
            for (int i = 0; i < CW / 4; ++i)
                sD[row * 32 + (((c0 / 4) + i) ^ (row & 7))] = make_float4(d[4 * i], d[4 * i + 1], d[4 * i + 2], d[4 * i + 3]);
            __syncthreads();
#pragma unroll 4
            for (int i = 0; i < 8; ++i) {
                const int rr = 8 * warp + i;
                const int64_t rg = t * 128 + rr;
                if (rg < A.n_rows) {
                    float4* po = reinterpret_cast<float4*>(A.dx_in + rg * H) + lane;
                    const float4 v = sD[rr * 32 + (lane ^ (rr & 7))];
                    float4 o = *po;
                    o.x += v.x;
                    o.y += v.y;
                    o.z += v.z;
                    o.w += v.w;
                    *po = o;
                }
            }
        } else if (valid) {
            float4* po = reinterpret_cast<float4*>(A.dx_in + r * H + c0);
#pragma unroll
            for (int i = 0; i < CW / 4; ++i) {
                float4 o = po[i];
                o.x += d[4 * i];
                o.y += d[4 * i + 1];
                o.z += d[4 * i + 2];
                o.w += d[4 * i + 3];
                po[i] = o;
            }
        }
        first = false;
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (ok) {
        if (first) {
            for (int i = tid; i < 2 * H * H; i += C::NT) part[i] = 0.f;
        } else if constexpr (MSPLIT) {
            flush_acc<C::CG>(tDW, H, H, q, lane, g, part);
            flush_acc<C::CG>(tDW + H, H, H, q, lane, g, part + H * H);
        } else {
            flush_acc<C::CG>(tDW, H, 2 * H, q, lane, g, part);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ------------------------------------------------------------------ partial reduction

// dst[r*dst_ld + c] += sum over CTAs b (ascending) of part[b*pstride + src_off + r*src_ld + c]
struct RedArgs {
    RedSeg seg[MAX_SEGS];
    int n_seg;
    int64_t seg_start[MAX_SEGS + 1];   // prefix sums of rows*cols
    const float* part;
    int64_t pstride;
    int n_cta;
};

__global__ void k_reduce_grads(RedArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.seg_start[A.n_seg]) return;
    int s = 0;
    while (i >= A.seg_start[s + 1]) ++s;
    const RedSeg& sg = A.seg[s];
    const int64_t j = i - A.seg_start[s];
    const int r = (int)(j / sg.cols), c = (int)(j % sg.cols);
    float acc = 0.f;
    const float* p = A.part + sg.src_off + (int64_t)r * sg.src_ld + c;
    // CTA partials in ascending order; the loads of 16 CTAs are requested together
    // (the sum is one latency-bound pass over a few tens of MB)
    constexpr int U = 16;
    int b = 0;
    for (; b + U <= A.n_cta; b += U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldg(p + (int64_t)(b + u) * A.pstride);
#pragma unroll
        for (int u = 0; u < U; ++u) acc += v[u];
    }
    for (; b < A.n_cta; ++b) acc += __ldg(p + (int64_t)b * A.pstride);
    sg.dst[(int64_t)r * sg.dst_ld + c] += acc;
}

// =================================================================== host side

int reduce_grads(RedSeg* segs, int n, const float* part, int64_t pstride, int n_cta, cudaStream_t s) {
    RedArgs A{};
    A.n_seg = n;
    A.seg_start[0] = 0;
    for (int i = 0; i < n; ++i) {
        A.seg[i] = segs[i];
        A.seg_start[i + 1] = A.seg_start[i] + (int64_t)segs[i].rows * segs[i].cols;
    }
    A.part = part;
    A.pstride = pstride;
    A.n_cta = n_cta;
    const int64_t tot = A.seg_start[n];
    if (tot == 0) return GNN_OK;
    {
        ProfScope _ps(s, "k_reduce_grads");
        k_reduce_grads<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A);
    }
    GNN_LAUNCH_CHECK("k_reduce_grads");
    return GNN_OK;
}

namespace {

using namespace host;

struct BwdWs {
    __nv_bfloat16* pq;
    float* a;
    float* da;
    float* dP;
    __nv_bfloat16* dz1;
    float* part;
    size_t bytes;
};

int64_t edge_pstride(int H, int L) { return (int64_t)L * H * (H + 16) + 2 * H; }
int64_t node_pstride(int H, int L) { return (int64_t)H * (2 * H + 16) + (int64_t)(L - 1) * H * (H + 16) + 2 * H; }
int64_t proj_pstride(int H) { return (int64_t)2 * H * H; }

BwdWs carve_bwd(void* ws, const gnn_graph_dev& G, int H, int Le, int Ln, bool need_a) {
    BwdWs w{};
    size_t off = 0;
    auto take = [&](size_t n) {
        off = (off + 255) & ~(size_t)255;
        void* p = ws ? (char*)ws + off : nullptr;
        off += n;
        return p;
    };
    const int64_t NR = G.n_rows, E = G.n_edges;
    const int64_t ncta = num_sms();
    w.pq = (__nv_bfloat16*)take((size_t)NR * 2 * H * 2);
    w.a = need_a ? (float*)take((size_t)NR * H * 4) : nullptr;
    w.da = (float*)take((size_t)NR * H * 4);
    w.dP = (float*)take((size_t)NR * H * 4);
    w.dz1 = (__nv_bfloat16*)take((size_t)E * H * 2);
    // per-CTA weight-gradient partials: one CTA per SM for the edge and node kernels,
    // up to two per SM for the projection kernel
    const int64_t ps = std::max(edge_pstride(H, Le), node_pstride(H, Ln));
    w.part = (float*)take((size_t)std::max(ncta * ps, 2 * ncta * proj_pstride(H)) * 4);
    w.bytes = off + 256;
    return w;
}

template <int H>
int proj_backward_h(const gnn_graph_dev& G, const gnn_mp_params& W, const float* x_in, const float* dP,
                    const __nv_bfloat16* dz1, float* dx_in, const gnn_mp_params& dW, float* part, cudaStream_t s) {
    const int64_t NR = G.n_rows;
    if (NR == 0) return GNN_OK;
    ProjBwdArgs A;
    A.x = x_in;
    A.dP = dP;
    A.dz1 = dz1;
    A.t_ptr = G.t_ptr;
    A.t_eid = G.t_eid;
    A.W1 = W.edge.W[0];
    A.dx_in = dx_in;
    A.part = part;
    A.pstride = proj_pstride(H);
    A.n_rows = NR;
    const ProjBwdSmem P = proj_bwd_smem<H>();
    int grid;
    int rc = persistent_grid(k_proj_bwd<H>, CfgP<H>::NT, P.total, pow2_cols(2 * H > 128 ? 3 * H : 2 * H),
                             (NR + 127) / 128, &grid);
    if (rc) return rc;
    grid = std::min(grid, 2 * num_sms());
    {
        ProfScope _ps(s, "k_proj_bwd");
        k_proj_bwd<H><<<grid, CfgP<H>::NT, P.total, s>>>(A);
    }
    GNN_LAUNCH_CHECK("k_proj_bwd");
    RedSeg seg[2];
    seg[0] = RedSeg{dW.edge.W[0], 3 * H, H, H, 0, H};                     // dW1a -> W1[:, 0:H]
    seg[1] = RedSeg{dW.edge.W[0] + H, 3 * H, H, H, (int64_t)H * H, H};    // dW1b -> W1[:, H:2H]
    return reduce_grads(seg, 2, part, A.pstride, grid, s);
}

template <int H>
int backward_h(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
               const __nv_bfloat16* e_in, const float* a_star, const float* dx_out, const __nv_bfloat16* de_out,
               float* dx_in, __nv_bfloat16* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes,
               cudaStream_t s, const __nv_bfloat16* act) {
    using C = CfgB<H>;
    const int Le = W.edge.n_lin, Ln = W.node.n_lin;
    GNN_REQUIRE(edge_bwd_tcols<H>(Le) <= 512 && node_bwd_tcols<H>(Ln) <= 512, GNN_EUNSUPPORTED,
                "gnn_mp_backward: BF16 backward at H=%d supports at most %d Linear layers per MLP", H,
                H == 64 ? 4 : 7);
    BwdWs w = carve_bwd(ws, G, H, Le, Ln, a_star == nullptr);
    GNN_REQUIRE(ws_bytes >= w.bytes, GNN_ENOMEM, "gnn_mp_backward: workspace too small");
    const int64_t NR = G.n_rows, E = G.n_edges;
    if (NR == 0) return GNN_OK;
    int rc;
    // 0. recompute P|Q (and a* when it was not saved); saved activations need no P|Q
    if (!act || !a_star) {
        if ((rc = proj_forward(G, H, W, x_in, w.pq, s))) return rc;
    }
    if (!a_star) {
        if ((rc = aggregate_forward(G, cfg, W, e_in, w.pq, nullptr, w.a, s))) return rc;
    }
    const float* astar = a_star ? a_star : w.a;
    const int nsm = num_sms();
    // 1. node MLP adjoint
    {
        NodeBwdArgs A;
        A.a_star = astar;
        A.x = x_in;
        A.dx_out = dx_out;
        A.da = w.da;
        A.dx_in = dx_in;
        A.part = w.part;
        A.pstride = node_pstride(H, Ln);
        A.n_rows = NR;
        A.mlp = mlp_dev(W.node);
        A.eps = cfg.ln_eps;
        A.act_rows = (NR + 127) / 128 * 128;
        const NodeBwdSmem P = node_bwd_smem<H>(Ln);
        CUtensorMap tm_hn, tm_xa;
        std::memset(&tm_hn, 0, sizeof(tm_hn));
        std::memset(&tm_xa, 0, sizeof(tm_xa));
        if (act) {
            const __nv_bfloat16* an = act + mp_act_elems_edge(G, W, H);
            if ((rc = make_row_tmap(&tm_hn, an, (int64_t)(Ln - 1) * A.act_rows, H))) return rc;
            if ((rc = make_row_tmap(&tm_xa, an + (int64_t)(Ln - 1) * A.act_rows * H, A.act_rows, 2 * H))) return rc;
        }
        int grid = 0;
        auto run = [&](auto kern) -> int {
            int r = persistent_grid(kern, C::NT, P.total, pow2_cols(node_bwd_tcols<H>(Ln)), (NR + 127) / 128, &grid);
            if (r) return r;
            grid = std::min(grid, nsm);
            {
                ProfScope _ps(s, "k_node_bwd");
                kern<<<grid, C::NT, P.total, s>>>(tm_hn, tm_xa, A);
            }
            GNN_LAUNCH_CHECK("k_node_bwd");
            return GNN_OK;
        };
        if ((rc = act ? run(k_node_bwd<H, true>) : run(k_node_bwd<H, false>))) return rc;
        RedSeg seg[MAX_SEGS];
        int n = 0;
        int64_t off = 0;
        for (int k = 0; k < Ln; ++k) {
            const int in = k == 0 ? 2 * H : H;
            const int N = in + 16;
            seg[n++] = RedSeg{dW.node.W[k], in, H, in, off, N};
            seg[n++] = RedSeg{dW.node.b[k], 1, H, 1, off + in, N};
            off += (int64_t)H * N;
        }
        seg[n++] = RedSeg{dW.node.gamma, H, 1, H, off, 0};
        seg[n++] = RedSeg{dW.node.beta, H, 1, H, off + H, 0};
        if ((rc = reduce_grads(seg, n, w.part, A.pstride, grid, s))) return rc;
    }
    // 2. adjoint of the halo swap + sync
    if (cfg.halo_mode == GNN_HALO_SYNC) {
        if ((rc = plain::halo(G, w.da, H, s))) return rc;
    }
    // 3. edge MLP adjoint
    if (E > 0) {
        CUtensorMap tm_e, tm_de, tm_h;
        if ((rc = make_row_tmap(&tm_e, e_in, E, H))) return rc;
        if ((rc = make_row_tmap(&tm_de, de_out ? (const void*)de_out : (const void*)e_in, E, H))) return rc;
        tm_h = tm_e;
        if (act && (rc = make_row_tmap(&tm_h, act, (int64_t)(Le - 1) * G.n_edge_tiles * 128, H))) return rc;
        EdgeBwdArgs A;
        GNN_REQUIRE(G.tile_meta && ((uintptr_t)G.tile_meta & 15) == 0, GNN_EINVAL,
                    "gnn_mp_backward: tile_meta must be a 16-byte aligned device array");
        A.tile_meta = (const uint8_t*)G.tile_meta;
        A.n_tiles = G.n_edge_tiles;
        A.pq = w.pq;
        A.q = w.pq + NR * H;
        A.da = w.da;
        A.has_de_out = de_out != nullptr;
        A.de_in = de_in;
        A.dz1 = w.dz1;
        A.dP = w.dP;
        A.part = w.part;
        A.pstride = edge_pstride(H, Le);
        A.mlp = mlp_dev(W.edge);
        A.eps = cfg.ln_eps;
        A.act_rows = G.n_edge_tiles * 128;
        const EdgeBwdSmem P = edge_bwd_smem<H>(Le);
        int grid = 0;
        const bool lnt = edge_bwd_ln_in_tmem<H>(Le);
        auto run = [&](auto kern, uint32_t cols) -> int {
            int r = persistent_grid(kern, C::NT, P.total, cols, G.n_edge_tiles, &grid);
            if (r) return r;
            grid = std::min(grid, nsm);
            {
                ProfScope _ps(s, "k_edge_bwd");
                kern<<<grid, C::NT, P.total, s>>>(tm_e, tm_de, tm_h, A);
            }
            GNN_LAUNCH_CHECK("k_edge_bwd");
            return GNN_OK;
        };
        const uint32_t cols_l = pow2_cols(edge_bwd_tcols<H>(Le) + 2 * H), cols = pow2_cols(edge_bwd_tcols<H>(Le));
        if (act) rc = lnt ? run(k_edge_bwd<H, true, true>, cols_l) : run(k_edge_bwd<H, false, true>, cols);
        else rc = lnt ? run(k_edge_bwd<H, true, false>, cols_l) : run(k_edge_bwd<H, false, false>, cols);
        if (rc) return rc;
        RedSeg seg[MAX_SEGS];
        int n = 0;
        int64_t off = 0;
        for (int k = 0; k < Le; ++k) {
            const int N = H + 16;
            if (k == 0) seg[n++] = RedSeg{dW.edge.W[0] + 2 * H, 3 * H, H, H, off, N};   // W1c columns of W1
            else seg[n++] = RedSeg{dW.edge.W[k], H, H, H, off, N};
            seg[n++] = RedSeg{dW.edge.b[k], 1, H, 1, off + H, N};
            off += (int64_t)H * N;
        }
        seg[n++] = RedSeg{dW.edge.gamma, H, 1, H, off, 0};
        seg[n++] = RedSeg{dW.edge.beta, H, 1, H, off + H, 0};
        if ((rc = reduce_grads(seg, n, w.part, A.pstride, grid, s))) return rc;
    } else {
        GNN_CUDA_CHECK(cudaMemsetAsync(w.dP, 0, sizeof(float) * NR * H, s), "memset");
    }
    // 4. projection adjoint: sender-side sums, dx_in += [dP dQ] [W1a; W1b], dW1a, dW1b
    return proj_backward_h<H>(G, W, x_in, w.dP, w.dz1, dx_in, dW, w.part, s);
}

}  // namespace

size_t mp_backward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W) {
    if (cfg.hidden == 128) return backward_h128_ws(G, W);
    return carve_bwd(nullptr, G, cfg.hidden, W.edge.n_lin, W.node.n_lin, true).bytes;
}

int proj_backward(const gnn_graph_dev& G, int H, const gnn_mp_params& W, const float* x_in, const float* dP,
                  const __nv_bfloat16* dz1, float* dx_in, const gnn_mp_params& dW, float* part, cudaStream_t s) {
    switch (H) {
        case 16: return proj_backward_h<16>(G, W, x_in, dP, dz1, dx_in, dW, part, s);
        case 32: return proj_backward_h<32>(G, W, x_in, dP, dz1, dx_in, dW, part, s);
        case 64: return proj_backward_h<64>(G, W, x_in, dP, dz1, dx_in, dW, part, s);
        case 128: return proj_backward_h<128>(G, W, x_in, dP, dz1, dx_in, dW, part, s);
        default: return set_error(GNN_EUNSUPPORTED, "proj_backward: H=%d", H);
    }
}

int mp_backward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                const __nv_bfloat16* e_in, const float* a_star, const float* dx_out, const __nv_bfloat16* de_out,
                float* dx_in, __nv_bfloat16* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes,
                cudaStream_t s, const __nv_bfloat16* act) {
    if (!mp_act_bytes(G, cfg, W)) act = nullptr;
    switch (cfg.hidden) {
        case 16: return backward_h<16>(G, cfg, W, x_in, e_in, a_star, dx_out, de_out, dx_in, de_in, dW, ws, ws_bytes, s, act);
        case 32: return backward_h<32>(G, cfg, W, x_in, e_in, a_star, dx_out, de_out, dx_in, de_in, dW, ws, ws_bytes, s, act);
        case 64: return backward_h<64>(G, cfg, W, x_in, e_in, a_star, dx_out, de_out, dx_in, de_in, dW, ws, ws_bytes, s, act);
        case 128: return backward_h128(G, cfg, W, x_in, e_in, a_star, dx_out, de_out, dx_in, de_in, dW, ws, ws_bytes, s);
        default:
            return set_error(GNN_EUNSUPPORTED, "gnn_mp_backward: the BF16 backward covers H in {16, 32, 64, 128}");
    }
}

}  // namespace fused
}  // namespace gnn
