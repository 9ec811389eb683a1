// Fused BF16 path of libgnnmp: tcgen05 / TMEM kernels for the consistent NMP
// layer (Eq. 5a-5e) and its adjoint.
//
// Layer forward = four launches:
//   k_proj_fwd   P|Q = x W1a^T | x W1b^T per node row. The edge MLP's first
//                Linear acts on [x_i, x_j, e_ij]; splitting W1 = [W1a W1b W1c]
//                gives W1 [x_i; x_j; e] = P_i + Q_j + W1c e, so the 2H-wide part
//                is computed once per node instead of once per edge.
//   k_edge_fwd   per tile of <= 128 receiver-aligned edges: TMA load of the
//                edge-state tile, gather of P_i and Q_j, the Linear/ELU chain
//                on tcgen05 with the accumulator in TMEM, LayerNorm + residual
//                (Eq. 5a), e' written once, and the 1/d-weighted segmented sum
//                over each receiver's edges in FP32 in edge order (Eq. 5b): the
//                per-edge MLP activations never leave the SM.
//   halo         Eq. 5c-5d copy-sum on the aggregates (shared with plain.cu).
//   k_node_fwd   per tile of 128 node rows: [a*, x] -> Linear/ELU chain ->
//                LayerNorm + residual (Eq. 5e).
// All kernels are persistent (grid = resident CTAs), loop over tiles with a
// static stride, and keep the layer's weights in shared memory as BF16.
// Thread layout: 128 rows x CG column groups; thread (row, g) owns TMEM lane
// `row` and columns [g*CW, (g+1)*CW) of every accumulator.

#include <algorithm>
#include <cstring>
#include <mutex>

#include "device_common.cuh"
#include "fused.h"
#include "plain.h"
#include "profiler.h"
#include "fused_common.cuh"

namespace gnn {
namespace fused {

cudaError_t take_device_error(unsigned int* out) { return take_device_error_word(out); }

using namespace tc;

// ------------------------------------------------------------------ k_proj_fwd

// One tile = 128 node rows. The FP32 x rows of the CTA's next tile are loaded
// by TMA into the other of two stages while the current tile is converted to
// BF16 and multiplied; the tile's P and Q rows are staged as BF16 in its own
// x stage and leave as whole rows by TMA stores (tmap_p, tmap_q: rows past
// n_rows are clipped).
template <int H>
__global__ void __launch_bounds__(Cfg<H>::NT) k_proj_fwd(const __grid_constant__ CUtensorMap tmap_x,
                                                        const __grid_constant__ CUtensorMap tmap_p,
                                                        const __grid_constant__ CUtensorMap tmap_q, int64_t n_rows,
                                                        const float* __restrict__ W1) {
    using C = Cfg<H>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const ProjSmem L = proj_smem<H>();
    uint8_t* sW = sm + L.w;
    uint8_t* sA = sm + L.a;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint64_t* bar = full + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * C::CW;
    constexpr uint32_t NCOLS = 2 * H < 32 ? 32 : 2 * H;
    constexpr uint32_t XBYTES = 128 * H * 4;
    auto sX = [&](int s) { return sm + L.x + s * XBYTES; };

    if (warp == 0) {
        tmem_alloc(tslot, NCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(full, 1);
        mbar_init(full + 1, 1);
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    // [W1a; W1b] as a [2H x H] K-major tile: row n < H is W1[n][0:H], row H+n is W1[n][H:2H]
    load_weight(sW, W1, 3 * H, 0, H, H, tid, C::NT, 2 * H, 0);
    load_weight(sW, W1, 3 * H, H, H, H, tid, C::NT, 2 * H, H);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    bool ok = true;
    const int64_t n_tiles = (n_rows + 127) / 128;
    if (tid == 0 && (int64_t)blockIdx.x < n_tiles) {
        mbar_arrive_expect_tx(full, XBYTES);
        tma_f32_tile<H>(sX(0), &tmap_x, (int64_t)blockIdx.x * 128, full);
    }
    int j = 0;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++j) {
        const int st = j & 1;
        ok = block_wait(full + st, (uint32_t)(j >> 1) & 1u, tid);
        if (!ok) break;
        // the other stage was read by the previous tile (ordered by its closing barrier) and
        // its P|Q stores have read it
        if (tid == 0 && t + gridDim.x < n_tiles) {
            bulk_wait_read_all();
            mbar_arrive_expect_tx(full + (st ^ 1), XBYTES);
            tma_f32_tile<H>(sX(st ^ 1), &tmap_x, (t + gridDim.x) * 128, full + (st ^ 1));
        }
        float v[C::CW];
#pragma unroll
        for (int i = 0; i < C::CW / 4; ++i) {
            const float4 u = ld_f32x4_tile<H>(sX(st), row, c0 + 4 * i);   // rows past n_rows read as zero
            v[4 * i] = u.x; v[4 * i + 1] = u.y; v[4 * i + 2] = u.z; v[4 * i + 3] = u.w;
        }
        st_row_tile<C::CW>(sA, row, c0, C::S, v);
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_mma(tmem, sA, sW, 2 * H, H);
            mma_commit(bar);
        }
        ok = block_wait(bar, phase, tid);
        phase ^= 1;
        tc_fence_after();
        if (!ok) break;
        float pv[C::CW], qv[C::CW];
        ld_acc<C::CW>(tmem, q, c0, pv);
        ld_acc<C::CW>(tmem, q, H + c0, qv);
        tc_fence_before();
        // every thread read its x rows before the MMA barrier: the stage takes P and Q
        uint8_t* sP = sX(st);
        uint8_t* sQ = sX(st) + 128 * H * 2;
        st_row_tile<C::CW>(sP, row, c0, C::S, pv);
        st_row_tile<C::CW>(sQ, row, c0, C::S, qv);
        fence_proxy_async();   // generic accesses of the stage precede the TMA stores and its next TMA write
        __syncthreads();       // sA, the x stage and TMEM are reused
        if (tid == 0) {
#pragma unroll
            for (int kb = 0; kb < H / (C::S / 2); ++kb) {
                tma_store_2d(&tmap_p, kb * (C::S / 2), (int32_t)(t * 128), sP + kb * 128 * C::S);
                tma_store_2d(&tmap_q, kb * (C::S / 2), (int32_t)(t * 128), sQ + kb * 128 * C::S);
            }
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();   // the P|Q rows are written before the CTA exits
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ------------------------------------------------------------------ k_edge_fwd

struct EdgeFwdArgs {
    const int32_t* row_ptr;
    const int32_t* col;
    const float* edge_w;
    const int32_t* tiles;
    const uint8_t* tile_meta;   // per-tile records (GNN_TILE_META_BYTES each)
    int64_t n_tiles;
    int64_t n_edges;
    const __nv_bfloat16* pq;    // P rows [n_rows x H]
    const __nv_bfloat16* q;     // Q rows [n_rows x H] (pq + n_rows*H)
    const __nv_bfloat16* e_in;  // edge states [n_edges x H] (the residual of Eq. 5a)
    __nv_bfloat16* e_out;
    float* a;
    MlpDev mlp;
    float eps;
    // Backward recomputation (k_edge_fwd<H, true>): tiles [t0, n_tiles); the
    // scratch row of edge row i of tile t is (t - t0) * 128 + i (zero past ne).
    int64_t t0;
    __nv_bfloat16* hs;            // hidden activations h_0 .. h_{L-2}, hs_stride elements apart
    int64_t hs_stride;
    __nv_bfloat16* dz;            // gradient of the last pre-activation (LayerNorm adjoint)
    const float* da;              // gradient of the aggregate after the halo adjoint
    const __nv_bfloat16* de_out;  // upstream gradient of e' (NULL: zero)
    float* part;                  // per-CTA partials: gamma, beta, last bias gradients (3H)
    int64_t pstride;
    // Training forward (k_edge_fwd_rt<H, true>): the hidden activations h_0 .. h_{L-2}
    // of edge row i of tile t go to row k * act_rows + t * 128 + i of tmap_h (whole
    // 128-row tiles, so one TMA store per tile never touches another tile's rows).
    __nv_bfloat16* act;
    int64_t act_rows;
};

// SAVE: the backward's recomputation of the edge MLP (Eq. 5a) over a range of
// tiles: the hidden activations go to scratch instead of the next Linear only,
// and the LayerNorm epilogue is replaced by its adjoint, whose input is the
// gradient of e' (upstream de' plus da_i / d_ij, the adjoint of Eq. 5b).
//
// One tile at a time per CTA. The tile's record (CSR slice, receivers,
// senders, 1/d) and edge-state rows arrive by bulk copy / TMA; as soon as the
// first Linear has read the edge-state rows, the next tile's record and rows
// are requested into the same buffers, so their latency hides behind this
// tile's chain. The residual of Eq. 5a re-reads e from global memory (L2), and
// the 1/d-weighted sums of Eq. 5b are staged in the activation buffer.
// SAVE writes each hidden tile and the tile's dz with TMA stores (tmap_hs: block k at
// row k * hs_stride / H + (t - t0) * 128; tmap_dz: row (t - t0) * 128), rows past
// the tile's edges zero.
template <int H, bool SAVE = false>
__global__ void __launch_bounds__(Cfg<H>::NT) k_edge_fwd(const __grid_constant__ CUtensorMap tmap_e,
                                                        const __grid_constant__ CUtensorMap tmap_hs,
                                                        const __grid_constant__ CUtensorMap tmap_dz, EdgeFwdArgs A) {
    using C = Cfg<H>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const EdgeFwdSmem L = edge_fwd_smem<H>(n_lin, SAVE);
    uint8_t* sW = sm + L.w;
    uint8_t* sA0 = sm + L.a0;
    uint8_t* sA1 = sm + L.a1;
    float* sPar = reinterpret_cast<float*>(sm + L.par);   // bias[n_lin][H], gamma[H], beta[H]
    float* sRed = reinterpret_cast<float*>(sm + L.red);
    uint64_t* bar_ld = reinterpret_cast<uint64_t*>(sm + L.bar);   // a tile's record and edge rows landed
    uint64_t* bar_mma = bar_ld + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);
    auto sRec = [&](int s) { return sm + L.seg + s * GNN_TILE_META_BYTES; };
    constexpr int SC = H / 2;                               // staged columns per pass (fills sA1 in FP32)
    constexpr int NC = SC / 4;                              // 16-byte chunks per staged row

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * C::CW;

    if (warp == 0) {
        tmem_alloc(tslot, C::TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        fence_mbar_init();
    }
    load_weight(sW, A.mlp.W[0], 3 * H, 2 * H, H, H, tid, C::NT);        // W1c: the edge-state columns of W1
    for (int k = 1; k < n_lin; ++k) load_weight(sW + k * C::WT, A.mlp.W[k], H, 0, H, H, tid, C::NT);
    for (int i = tid; i < n_lin * H; i += C::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < H; i += C::NT) {
        sPar[n_lin * H + i] = A.mlp.gamma[i];
        sPar[(n_lin + 1) * H + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t ph_mma = 0;
    bool ok = true;
    constexpr int NCH = C::CW / 16;
    float accG[NCH], accB[NCH], accZ[NCH];   // SAVE: column sums of g*xhat, g, dz
#pragma unroll
    for (int j = 0; j < NCH; ++j) accG[j] = accB[j] = accZ[j] = 0.f;
    const int64_t tb = SAVE ? A.t0 : 0;
    bool ld_pending = false;   // thread 0: a record + edge-row load nobody has waited for
    auto tile_hdr = [&](int64_t t) { return ld_nc_v4s32(A.tile_meta + t * GNN_TILE_META_BYTES); };
    int4 hdr_next = make_int4(0, 0, 0, 0);   // thread 0: the next tile's header, read one tile ahead
    auto issue_ld = [&](int s, int64_t t, int32_t e0) {
        mbar_arrive_expect_tx(bar_ld, C::TILE + GNN_TILE_META_BYTES);
        bulk_load(sRec(s), A.tile_meta + t * GNN_TILE_META_BYTES, GNN_TILE_META_BYTES, bar_ld);
#pragma unroll
        for (int kb = 0; kb < (H + 63) / 64; ++kb) tma_load_2d(sA0 + kb * 128 * 128, &tmap_e, kb * 64, e0, bar_ld);
        ld_pending = true;
    };
    if (tid == 0 && tb + (int64_t)blockIdx.x < A.n_tiles) {
        issue_ld(0, tb + blockIdx.x, tile_hdr(tb + blockIdx.x).z);
        if (tb + (int64_t)blockIdx.x + gridDim.x < A.n_tiles) hdr_next = tile_hdr(tb + blockIdx.x + gridDim.x);
    }
    int j = 0;

    for (int64_t t = tb + blockIdx.x; t < A.n_tiles && ok; t += gridDim.x, ++j) {
        ok = block_wait(bar_ld, (uint32_t)j & 1u, tid);
        if (!ok) break;
        ld_pending = false;
        const uint8_t* rec = sRec(j & 1);
        const int32_t* hdr = reinterpret_cast<const int32_t*>(rec);
        const int32_t* sRp = reinterpret_cast<const int32_t*>(rec + 16);
        const int16_t* sSeg = reinterpret_cast<const int16_t*>(rec + 544);
        const int32_t* sCol = reinterpret_cast<const int32_t*>(rec + 800);
        const float* sWd = reinterpret_cast<const float*>(rec + 1312);
        const int32_t r0 = hdr[0], r1 = hdr[1], e0 = hdr[2], ne = hdr[3];
        if (tid == 0) {
            tc_fence_after();
            issue_mma(tmem, sA0, sW, H, H);
            mma_commit(bar_mma);
        }
        const bool valid = row < ne;
        const int64_t eg = (int64_t)e0 + row;
        float w = 0.f;
        float pq[C::CW];
        if (valid) {
            const int64_t rcv = r0 + sSeg[row];
            const int64_t snd = sCol[row];
            w = sWd[row];
#pragma unroll
            for (int i = 0; i < C::CW; i += 8) {
                float pv[8], qv[8];
                ld_bf16x8(A.pq + rcv * H + c0 + i, pv);
                ld_bf16x8(A.q + snd * H + c0 + i, qv);
#pragma unroll
                for (int k = 0; k < 8; ++k) pq[i + k] = pv[k] + qv[k];
            }
        } else {
#pragma unroll
            for (int i = 0; i < C::CW; ++i) pq[i] = 0.f;
        }
        float v[C::CW];
        uint4 eres[C::CW / 8];   // forward: the residual e row (BF16), requested before the last MMA wait
        for (int k = 0; k < n_lin && ok; ++k) {
            if constexpr (!SAVE) {
                if (k == n_lin - 1 && valid) {
#pragma unroll
                    for (int i = 0; i < C::CW / 8; ++i)
                        eres[i] = __ldg(reinterpret_cast<const uint4*>(A.e_in + eg * H + c0) + i);
                }
            }
            if (SAVE && tid == 0) bulk_wait_read_all();   // sA1 may be rewritten after the barrier
            ok = block_wait(bar_mma, ph_mma, tid);
            ph_mma ^= 1;
            tc_fence_after();
            if (!ok) break;
            if (k == 0 && tid == 0 && t + gridDim.x < A.n_tiles) {
                // the first Linear has read the edge rows: the next tile's record and rows
                issue_ld((j + 1) & 1, t + gridDim.x, hdr_next.z);
                if constexpr (SAVE) {   // and its receivers' da rows into L2 for the LayerNorm adjoint
                    if (hdr_next.y > hdr_next.x)
                        prefetch_l2(A.da + (int64_t)hdr_next.x * H, (uint32_t)(hdr_next.y - hdr_next.x) * H * 4);
                }
                if (t + 2 * (int64_t)gridDim.x < A.n_tiles) hdr_next = tile_hdr(t + 2 * (int64_t)gridDim.x);
            }
            ld_acc<C::CW>(tmem, q, c0, v);
            const float* bk = sPar + k * H + c0;
            if (k == 0) {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) v[i] += pq[i] + bk[i];
            } else {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) v[i] += bk[i];
            }
            if (k < n_lin - 1) {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) v[i] = elu1_fast(v[i]);
                if constexpr (SAVE) {   // the saved rows past the tile's edges are zero
#pragma unroll
                    for (int i = 0; i < C::CW; ++i) v[i] = valid ? v[i] : 0.f;
                }
                st_row_tile<C::CW>(sA1, row, c0, C::S, v);
                fence_proxy_async();
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    issue_mma(tmem, sA1, sW + (k + 1) * C::WT, H, H);
                    mma_commit(bar_mma);
                    if constexpr (SAVE) {   // the hidden tile to scratch while the MMA reads it
#pragma unroll
                        for (int kb = 0; kb < (H + 63) / 64; ++kb)
                            tma_store_2d(&tmap_hs, kb * 64, (int32_t)(k * (A.hs_stride / H) + (t - tb) * 128),
                                         sA1 + kb * 128 * 128);
                        bulk_commit();
                    }
                }
            }
        }
        if (!ok) break;
        tc_fence_before();
        if constexpr (SAVE) {
            // gradient of e': upstream de' plus da_i / d_ij, then the LayerNorm adjoint
            float gv[C::CW];
            if (valid) {
                const float* dar = A.da + (int64_t)(r0 + sSeg[row]) * H + c0;
#pragma unroll
                for (int i = 0; i < C::CW; i += 4) {
                    const float4 u = __ldg(reinterpret_cast<const float4*>(dar + i));
                    gv[i] = w * u.x;
                    gv[i + 1] = w * u.y;
                    gv[i + 2] = w * u.z;
                    gv[i + 3] = w * u.w;
                }
                if (A.de_out) {
#pragma unroll
                    for (int i = 0; i < C::CW; i += 8) {
                        float d8[8];
                        ld_bf16x8(A.de_out + eg * H + c0 + i, d8);
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) gv[i + jj] = d8[jj] + gv[i + jj];
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) gv[i] = 0.f;
            }
            const float* gam = sPar + n_lin * H + c0;
            float mean, rstd, s1, s2;
            row_stats_adj_gamma<H, C::CG, C::CW>(v, gv, gam, sRed, row, g, A.eps, mean, rstd, s1, s2);
            ln_adjoint_row<C::CW>(v, gv, gam, mean, rstd, s1, s2, valid, lane, accG, accB, accZ);
            st_row_tile<C::CW>(sA1, row, c0, C::S, v);   // dz to scratch by TMA (the last MMA has read sA1)
            fence_proxy_async();
            __syncthreads();   // the record of this tile is rewritten two tiles later, sRed next tile
            if (tid == 0) {
#pragma unroll
                for (int kb = 0; kb < (H + 63) / 64; ++kb)
                    tma_store_2d(&tmap_dz, kb * 64, (int32_t)((t - tb) * 128), sA1 + kb * 128 * 128);
                bulk_commit();
            }
            continue;
        }
        // LayerNorm + residual (Eq. 5a)
        float mean, rstd;
        row_stats<H, C::CG, C::CW>(v, sRed, row, g, A.eps, mean, rstd);
        const float* gam = sPar + n_lin * H + c0;
        const float* bet = sPar + (n_lin + 1) * H + c0;
        if (valid) {
#pragma unroll
            for (int i = 0; i < C::CW / 8; ++i) {
                float eo[8];
                unpack_bf16x2(eres[i].x, eo[0], eo[1]);
                unpack_bf16x2(eres[i].y, eo[2], eo[3]);
                unpack_bf16x2(eres[i].z, eo[4], eo[5]);
                unpack_bf16x2(eres[i].w, eo[6], eo[7]);
#pragma unroll
                for (int k = 0; k < 8; ++k) v[8 * i + k] = eo[k] + (v[8 * i + k] - mean) * rstd * gam[8 * i + k] + bet[8 * i + k];
            }
        }
        // e' leaves by whole rows per warp, staged in the activation buffer (its last
        // reader, the final Linear, has completed), before the sums below reuse it
        if (A.e_out) {
            st_row_tile<C::CW>(sA1, row, c0, C::S, v);
            __syncthreads();
            constexpr int CPR = H / 8;   // 16-byte chunks per row
            for (int i = tid; i < ne * CPR; i += C::NT) {
                const int rr = i / CPR, jj = i - rr * CPR;
                *reinterpret_cast<uint4*>(A.e_out + ((int64_t)e0 + rr) * H + 8 * jj) =
                    *reinterpret_cast<const uint4*>(sA1 + tile_off(rr, 8 * jj, 128, C::S));
            }
        }
        // 1/d-weighted segmented sum over each receiver's edges (Eq. 5b), two column
        // passes staged in FP32 in the activation buffer
        float4* sS4 = reinterpret_cast<float4*>(sA1);
        __syncthreads();
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
            for (int i = 0; i < C::CW; i += 4) {
                const int c = c0 + i - pass * SC;
                if (c >= 0 && c < SC)
                    sS4[row * NC + stage_chunk<NC>(c / 4, row)] =
                        valid ? make_float4(w * v[i], w * v[i + 1], w * v[i + 2], w * v[i + 3])
                              : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            const int nr = r1 - r0;
            for (int it = tid; it < nr * NC; it += C::NT) {
                const int rr = it / NC, cc = it % NC;
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int32_t e = sRp[rr]; e < sRp[rr + 1]; ++e) {
                    const float4 u = sS4[e * NC + stage_chunk<NC>(cc, e)];
                    acc.x += u.x;
                    acc.y += u.y;
                    acc.z += u.z;
                    acc.w += u.w;
                }
                *reinterpret_cast<float4*>(A.a + (int64_t)(r0 + rr) * H + pass * SC + 4 * cc) = acc;
            }
            __syncthreads();
        }
        fence_proxy_async();   // generic writes of sA1 precede the next tile's MMA reads
    }
    if (tid == 0 && ld_pending) mbar_wait(bar_ld, (uint32_t)j & 1u);   // after a timeout: bounded
    if (SAVE && tid == 0) bulk_wait_all();   // the scratch tiles are written before the CTA exits
    if constexpr (SAVE) {
        float* part = A.part + (int64_t)blockIdx.x * A.pstride;
        colsum_store<H, NCH>(accG, sRed, q, lane, c0, tid, C::NT, part);
        colsum_store<H, NCH>(accB, sRed, q, lane, c0, tid, C::NT, part + H);
        colsum_store<H, NCH>(accZ, sRed, q, lane, c0, tid, C::NT, part + 2 * H);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, C::TCOLS);
}

// ------------------------------------------------------------------ k_edge_fwd_ws (warp-specialised)
//
// Same arithmetic as k_edge_fwd, reorganised so that no consumer thread waits
// on a global-memory index load: one producer warp walks the CTA's tiles ahead
// of the consumers, writing each tile's CSR slice, receiver/sender indices and
// 1/d into a ring of NS shared-memory stages and starting the TMA load of the
// tile's edge states into the same stage. Two consumer groups take alternate
// tiles, so one group's MMA and barrier latency overlaps the other group's
// epilogue. Stage s is handed over through mbarriers full[s] (32 producer
// arrivals + the TMA bytes) and empty[s] (one consumer arrival).

constexpr int WS_NS = 4;   // stages
constexpr int WS_NG = 2;   // consumer groups

struct StageMeta {
    int32_t r0, r1, e0, ne;
    int32_t rp[132];       // tile CSR slice, local edge offsets
    int32_t seg[128];      // local receiver of each edge
    int32_t col[128];      // sender row of each edge
    float w[128];          // 1/d of each edge
};

struct EdgeFwdWsSmem {
    uint32_t w, st, meta, a1, stg, par, red, bar, tm, total;
};

template <int H>
__host__ __device__ inline EdgeFwdWsSmem edge_fwd_ws_smem(int n_lin) {
    using C = Cfg<H>;
    EdgeFwdWsSmem s;
    s.w = 0;
    s.st = align_up(n_lin * C::WT, 1024);
    s.meta = s.st + WS_NS * C::TILE;
    s.a1 = align_up(s.meta + WS_NS * (uint32_t)sizeof(StageMeta), 1024);
    s.stg = s.a1 + WS_NG * C::TILE;
    s.par = s.stg + WS_NG * 128 * (H / 2 + 4) * 4;
    s.red = s.par + (n_lin + 2) * H * 4;
    s.bar = align_up(s.red + WS_NG * 2 * C::CG * 128 * 4, 8);
    s.tm = s.bar + 8 * (2 * WS_NS + WS_NG);
    s.total = s.tm + 16 + 1024;
    return s;
}

template <int H>
struct WsCfg {
    static constexpr int GT = Cfg<H>::NT;            // threads per consumer group
    static constexpr int NT = WS_NG * GT + 32;       // + one producer warp
};

template <int H, int CG, int CW>
__device__ __forceinline__ void row_stats_named(const float* v, float* red, int row, int g, float eps, int bar_id,
                                                int nthr, float& mean, float& rstd) {
    // one reduction for sum and sum of squares: var = E[v^2] - mean^2 (FP32)
    float s = 0.f, q = 0.f;
#pragma unroll
    for (int i = 0; i < CW; ++i) {
        s += v[i];
        q += v[i] * v[i];
    }
    red[g * 128 + row] = s;
    red[(CG + g) * 128 + row] = q;
    named_sync(bar_id, nthr);
    float ts = 0.f, tq = 0.f;
#pragma unroll
    for (int k = 0; k < CG; ++k) {
        ts += red[k * 128 + row];
        tq += red[(CG + k) * 128 + row];
    }
    mean = ts * (1.f / H);
    rstd = rsqrtf(fmaxf(tq * (1.f / H) - mean * mean, 0.f) + eps);
}

// One elected thread polls the mbarrier; the named-barrier group agrees.
__device__ __forceinline__ bool group_wait(uint64_t* bar, uint32_t parity, bool elected, int bar_id, int nthr) {
    const bool mine = elected ? mbar_wait(bar, parity) : true;
    return named_and(mine, bar_id, nthr);
}

template <int H>
__global__ void __launch_bounds__(WsCfg<H>::NT, 1)
    k_edge_fwd_ws(const __grid_constant__ CUtensorMap tmap_e, EdgeFwdArgs A) {
    using C = Cfg<H>;
    constexpr int GT = WsCfg<H>::GT;
    constexpr int SC = H / 2, SLD = SC + 4;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const EdgeFwdWsSmem L = edge_fwd_ws_smem<H>(n_lin);
    uint8_t* sW = sm + L.w;
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint64_t* empty = full + WS_NS;
    uint64_t* mbar = empty + WS_NS;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);
    auto stage_e = [&](int s) { return sm + L.st + s * C::TILE; };
    auto stage_m = [&](int s) { return reinterpret_cast<StageMeta*>(sm + L.meta + s * sizeof(StageMeta)); };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = tid >= WS_NG * GT;
    const uint32_t TC = C::TCOLS;
    const uint32_t NCOLS = TC * WS_NG < 32 ? 32 : TC * WS_NG;

    if (warp == 0) {
        tmem_alloc(tslot, NCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < WS_NS; ++s) {
            mbar_init(full + s, 32);
            mbar_init(empty + s, 1);
        }
        for (int g = 0; g < WS_NG; ++g) mbar_init(mbar + g, 1);
        fence_mbar_init();
    }
    load_weight(sW, A.mlp.W[0], 3 * H, 2 * H, H, H, tid, WsCfg<H>::NT);
    for (int k = 1; k < n_lin; ++k) load_weight(sW + k * C::WT, A.mlp.W[k], H, 0, H, H, tid, WsCfg<H>::NT);
    for (int i = tid; i < n_lin * H; i += WsCfg<H>::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < H; i += WsCfg<H>::NT) {
        sPar[n_lin * H + i] = A.mlp.gamma[i];
        sPar[(n_lin + 1) * H + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (producer) {
        // ---------------- producer warp: tile metadata + TMA, NS tiles ahead
        int j = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < A.n_tiles && ok; t += gridDim.x, ++j) {
            const int s = j % WS_NS;
            if (j >= WS_NS) {
                ok = mbar_wait(empty + s, (uint32_t)((j / WS_NS) - 1) & 1u);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
            }
            StageMeta* m = stage_m(s);
            const int32_t r0 = A.tiles[t], r1 = A.tiles[t + 1];
            const int32_t e0 = A.row_ptr[r0], ne = A.row_ptr[r1] - e0;
            for (int i = lane; i <= r1 - r0; i += 32) m->rp[i] = A.row_ptr[r0 + i] - e0;
            __syncwarp();
            for (int rr = lane; rr < r1 - r0; rr += 32)
                for (int32_t e = m->rp[rr]; e < m->rp[rr + 1]; ++e) m->seg[e] = rr;
            for (int e = lane; e < ne; e += 32) {
                m->col[e] = A.col[e0 + e];
                m->w[e] = A.edge_w[e0 + e];
            }
            if (lane == 0) {
                m->r0 = r0;
                m->r1 = r1;
                m->e0 = e0;
                m->ne = ne;
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive_expect_tx(full + s, C::TILE);
#pragma unroll
                for (int kb = 0; kb < (H + 63) / 64; ++kb)
                    tma_load_2d(stage_e(s) + kb * 128 * 128, &tmap_e, kb * 64, e0, full + s);
            } else {
                mbar_arrive(full + s);
            }
        }
    } else {
        // ---------------- consumer group g
        const int g = tid / GT, gt = tid % GT, wg = gt >> 5;
        const int q = wg & 3, cg = wg >> 2, row = 32 * q + lane, c0 = cg * C::CW;
        const int bid = 1 + g;
        const bool elected = gt == 0;
        const uint32_t tm = tmem + (uint32_t)g * TC;
        uint8_t* sA1 = sm + L.a1 + g * C::TILE;
        float* sStage = reinterpret_cast<float*>(sm + L.stg + g * 128 * SLD * 4);
        float* sRed = reinterpret_cast<float*>(sm + L.red + g * 2 * C::CG * 128 * 4);
        uint32_t ph_mma = 0;
        bool ok = true;
        int j = 0;
        for (int64_t t = blockIdx.x; t < A.n_tiles && ok; t += gridDim.x, ++j) {
            if (j % WS_NG != g) continue;
            const int s = j % WS_NS;
            ok = group_wait(full + s, (uint32_t)(j / WS_NS) & 1u, elected, bid, GT);
            if (!ok) break;
            const StageMeta* m = stage_m(s);
            uint8_t* sE = stage_e(s);
            const int32_t r0 = m->r0, r1 = m->r1;
            const int64_t e0 = m->e0;
            const int ne = m->ne;
            if (elected) {
                tc_fence_after();
                issue_mma(tm, sE, sW, H, H);
                mma_commit(mbar + g);
            }
            const bool valid = row < ne;
            const int64_t eg = e0 + row;
            float w = 0.f;
            float pq[C::CW];
            if (valid) {
                const int64_t rcv = r0 + m->seg[row];
                const int64_t snd = m->col[row];
                w = m->w[row];
#pragma unroll
                for (int i = 0; i < C::CW; i += 8) {
                    float pv[8], qv[8];
                    ld_bf16x8(A.pq + rcv * H + c0 + i, pv);
                    ld_bf16x8(A.q + snd * H + c0 + i, qv);
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) pq[i + jj] = pv[jj] + qv[jj];
                }
            } else {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) pq[i] = 0.f;
            }
            float v[C::CW];
            for (int k = 0; k < n_lin && ok; ++k) {
                ok = group_wait(mbar + g, ph_mma, elected, bid, GT);
                ph_mma ^= 1;
                tc_fence_after();
                if (!ok) break;
                ld_acc<C::CW>(tm, q, c0, v);
                const float* bk = sPar + k * H + c0;
                if (k == 0) {
#pragma unroll
                    for (int i = 0; i < C::CW; ++i) v[i] += pq[i] + bk[i];
                } else {
#pragma unroll
                    for (int i = 0; i < C::CW; ++i) v[i] += bk[i];
                }
                if (k < n_lin - 1) {
#pragma unroll
                    for (int i = 0; i < C::CW; ++i) v[i] = elu1_fast(v[i]);
                    st_row_tile<C::CW>(sA1, row, c0, C::S, v);
                    fence_proxy_async();
                    tc_fence_before();
                    named_sync(bid, GT);
                    if (elected) {
                        tc_fence_after();
                        issue_mma(tm, sA1, sW + (k + 1) * C::WT, H, H);
                        mma_commit(mbar + g);
                    }
                }
            }
            if (!ok) break;
            tc_fence_before();
            float mean, rstd;
            row_stats_named<H, C::CG, C::CW>(v, sRed, row, cg, A.eps, bid, GT, mean, rstd);
            float eo[C::CW];
            ld_row_tile<C::CW>(sE, row, c0, C::S, eo);
            const float* gam = sPar + n_lin * H + c0;
            const float* bet = sPar + (n_lin + 1) * H + c0;
#pragma unroll
            for (int i = 0; i < C::CW; ++i) v[i] = eo[i] + (v[i] - mean) * rstd * gam[i] + bet[i];
            if (valid && A.e_out) {
#pragma unroll
                for (int i = 0; i < C::CW; i += 8) st_bf16x8(A.e_out + eg * H + c0 + i, v + i);
            }
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) {
                    const int c = c0 + i;
                    if (c >= pass * SC && c < (pass + 1) * SC) sStage[row * SLD + (c - pass * SC)] = w * v[i];
                }
                named_sync(bid, GT);
                const int nr = r1 - r0;
                for (int it = gt; it < nr * SC; it += GT) {
                    const int rr = it / SC, cc = it % SC;
                    const int32_t b0 = m->rp[rr], b1 = m->rp[rr + 1];
                    float acc = 0.f;
                    for (int32_t e = b0; e < b1; ++e) acc += sStage[e * SLD + cc];
                    A.a[(int64_t)(r0 + rr) * H + pass * SC + cc] = acc;
                }
                named_sync(bid, GT);
            }
            fence_proxy_async();           // generic reads of the stage precede its next TMA write
            named_sync(bid, GT);
            if (elected) mbar_arrive(empty + s);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// ------------------------------------------------------------------ k_edge_fwd_rt (record-tiled groups)
//
// Same arithmetic as k_edge_fwd, organised around the host-built per-tile
// records (CSR slice, local receiver, sender and 1/d of every edge). NG
// consumer groups take interleaved tiles of the CTA's share; a group's next
// tile but one is requested (record by bulk copy, edge states by TMA) as soon
// as its stage is free, so no thread builds metadata and the loads have two
// tiles' time to land. After the first epilogue of a tile has consumed them,
// every thread requests the P row of its edge's receiver and the Q row of its
// sender (its own columns) for the group's next tile with cp.async into a
// private slot: no global gather sits on the MMA chain and none occupies
// registers. The segmented sum of Eq. 5b is staged through the activation
// tile, which is free once the last MMA of the tile has completed.

template <int H>
struct RtCfg {
    static constexpr int NG = H >= 64 ? 2 : 4;     // consumer groups
    static constexpr int GT = Cfg<H>::NT;          // threads per group
    static constexpr int NT = NG * GT;
    static constexpr int SC = H / 2;               // columns per segmented-sum pass
    static constexpr int SLOT = 2 * Cfg<H>::CW;    // bytes of a thread's Q slot
    static constexpr int NCH = SLOT / 16;          // 16-byte chunks per slot
    static constexpr int SWZ_SHIFT = NCH >= 8 ? 0 : (NCH == 4 ? 1 : 2);
    static constexpr uint32_t NCOLS = NG * Cfg<H>::TCOLS < 32 ? 32 : NG * Cfg<H>::TCOLS;
};

struct EdgeFwdRtSmem {
    uint32_t w, par, red, grp, gsz, bar, tm, total;
};

// Per group (gsz bytes at grp + g*gsz): e stages [2 x TILE], activation tile
// (TILE), the tile's P rows [128 x H] (TILE), Q slots (TILE), tile records
// [2 x GNN_TILE_META_BYTES].
template <int H>
__host__ __device__ inline EdgeFwdRtSmem edge_fwd_rt_smem(int n_lin) {
    using C = Cfg<H>;
    using R = RtCfg<H>;
    EdgeFwdRtSmem s;
    s.w = 0;
    s.par = align_up(n_lin * C::WT, 16);
    s.red = s.par + (n_lin + 2) * H * 4;
    s.grp = align_up(s.red + R::NG * 2 * C::CG * 128 * 4, 1024);
    s.gsz = 5 * C::TILE + 2 * GNN_TILE_META_BYTES;
    s.bar = s.grp + R::NG * s.gsz;
    s.tm = s.bar + 8 * 4 * R::NG;
    s.total = s.tm + 16 + 1024;
    return s;
}

// Physical 16-byte chunk of logical chunk k in the slot of `row` (rows of one
// 8-thread shared-memory phase land in distinct banks).
template <int H>
__device__ __forceinline__ int slot_chunk(int k, int row) {
    using R = RtCfg<H>;
    return k ^ ((row >> R::SWZ_SHIFT) & (R::NCH - 1));
}



// ASAVE: also store each edge's hidden activations (the BF16 operands of the
// next Linear) to A.act, so that the backward need not recompute them.
template <int H, bool ASAVE = false>
__global__ void __launch_bounds__(RtCfg<H>::NT, 1)
    k_edge_fwd_rt(const __grid_constant__ CUtensorMap tmap_e, const __grid_constant__ CUtensorMap tmap_h,
                  EdgeFwdArgs A) {
    using C = Cfg<H>;
    using R = RtCfg<H>;
    constexpr int GT = R::GT, SC = R::SC, CW = C::CW, CG = C::CG, NCH = R::NCH;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const EdgeFwdRtSmem L = edge_fwd_rt_smem<H>(n_lin);
    uint8_t* sW = sm + L.w;
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = tid / GT, gt = tid % GT, wg = gt >> 5;
    const int q = wg & 3, cg = wg >> 2, row = 32 * q + lane, c0 = cg * CW;
    const int bid = 1 + g;
    const bool elected = gt == 0;
    uint8_t* G = sm + L.grp + g * L.gsz;
    uint8_t* sA1 = G + 2 * C::TILE;
    uint8_t* sP = G + 3 * C::TILE;                                  // P rows of the tile's receivers
    uint8_t* sSlot = G + 4 * C::TILE + (cg * 128 + row) * R::SLOT;   // this thread's Q columns
    uint8_t* sRec = G + 5 * C::TILE;
    float* sRed = reinterpret_cast<float*>(sm + L.red) + g * 2 * CG * 128;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar) + 4 * g;
    uint64_t* mbar = full + 2;
    uint64_t* p_full = full + 3;   // the tile's P rows have landed

    if (warp == 0) {
        tmem_alloc(tslot, R::NCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        uint64_t* b = reinterpret_cast<uint64_t*>(sm + L.bar);
        for (int i = 0; i < 4 * R::NG; ++i) mbar_init(b + i, 1);
        fence_mbar_init();
    }
    load_weight(sW, A.mlp.W[0], 3 * H, 2 * H, H, H, tid, R::NT);
    for (int k = 1; k < n_lin; ++k) load_weight(sW + k * C::WT, A.mlp.W[k], H, 0, H, H, tid, R::NT);
    for (int i = tid; i < n_lin * H; i += R::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < H; i += R::NT) {
        sPar[n_lin * H + i] = A.mlp.gamma[i];
        sPar[(n_lin + 1) * H + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tslot + (uint32_t)g * C::TCOLS;

    // the group's tiles: blockIdx.x + (u*NG + g)*gridDim.x, u = 0, 1, ...; tile u uses stage u & 1
    const int64_t stride = (int64_t)R::NG * gridDim.x;
    const int64_t t_first = blockIdx.x + (int64_t)g * gridDim.x;
    auto issue = [&](int s, int64_t t, int32_t e0) {   // elected thread: record + edge states of tile t
        mbar_arrive_expect_tx(full + s, C::TILE + GNN_TILE_META_BYTES);
        bulk_load(sRec + s * GNN_TILE_META_BYTES, A.tile_meta + t * GNN_TILE_META_BYTES, GNN_TILE_META_BYTES,
                  full + s);
#pragma unroll
        for (int kb = 0; kb < (H + 63) / 64; ++kb) tma_load_2d(G + s * C::TILE + kb * 128 * 128, &tmap_e, kb * 64, e0,
                                                               full + s);
    };
    // the receivers' P rows of the tile whose record is in stage s: one bulk copy of the
    // tile's consecutive rows (elected thread); each thread's Q slot <- the Q row of its
    // edge's sender, own columns, by cp.async
    auto fetch_p = [&](int s) {
        const int32_t* hdr = reinterpret_cast<const int32_t*>(sRec + s * GNN_TILE_META_BYTES);
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
        const uint8_t* rec = sRec + s * GNN_TILE_META_BYTES;
        if (row < reinterpret_cast<const int32_t*>(rec)[3]) {
            const int64_t snd = reinterpret_cast<const int32_t*>(rec + 800)[row];
            const __nv_bfloat16* Q = A.q + snd * H + c0;
#pragma unroll
            for (int k = 0; k < NCH; ++k) cp_async16(sSlot + 16 * slot_chunk<H>(k, row), Q + 8 * k);
        }
        cp_async_commit();
    };
    bool ok = true;
    uint32_t pending = 0;   // elected thread: bit s = a load into stage s not yet consumed, bit 2+s = its parity
    if (elected) {
        for (int u = 0; u < 2; ++u) {
            const int64_t t = t_first + u * stride;
            if (t < A.n_tiles) {
                issue(u, t, ld_nc_s32(A.tile_meta + t * GNN_TILE_META_BYTES + 8));
                pending |= 1u << u;
            }
        }
    }
    if (t_first < A.n_tiles) {
        ok = mbar_wait(full, 0);
        if (ok) {
            gather(0);
            if (elected) fetch_p(0);
        }
    }
    bool p_pending = elected && t_first < A.n_tiles && ok;   // elected: a P copy not yet consumed

    uint32_t ph_mma = 0, ph_p = 0;
    int u = 0;
    for (int64_t t = t_first; t < A.n_tiles && ok; t += stride, ++u) {
        const int s = u & 1;
        const int64_t t_next = t + stride, t_refill = t + 2 * stride;
        const int32_t e0_refill =
            (elected && t_refill < A.n_tiles) ? ld_nc_s32(A.tile_meta + t_refill * GNN_TILE_META_BYTES + 8) : 0;
        ok = group_wait(full + s, (uint32_t)(u >> 1) & 1u, elected, bid, GT);
        if (!ok) break;
        pending &= ~(5u << s);
        uint8_t* sE = G + s * C::TILE;
        const uint8_t* rec = sRec + s * GNN_TILE_META_BYTES;
        if (elected) {
            tc_fence_after();
            issue_mma(tm, sE, sW, H, H);
            mma_commit(mbar);
        }
        const int32_t* hdr = reinterpret_cast<const int32_t*>(rec);
        const int32_t r0 = hdr[0], nr = hdr[1] - hdr[0], ne = hdr[3];
        const int64_t e0 = hdr[2];
        const bool valid = row < ne;
        const float w = valid ? reinterpret_cast<const float*>(rec + 1312)[row] : 0.f;
        cp_async_wait_all();
        bool next_ready = false;   // the next tile's record is in stage s^1
        float v[CW];
        for (int k = 0; k < n_lin && ok; ++k) {
            if (ASAVE && elected) bulk_wait_read_all();   // sA1 may be rewritten after the group barrier
            ok = group_wait(mbar, ph_mma, elected, bid, GT);
            ph_mma ^= 1;
            tc_fence_after();
            if (!ok) break;
            ld_acc<CW>(tm, q, c0, v);
            const float* bk = sPar + k * H + c0;
            if (k == 0) {
                ok = ok && mbar_wait(p_full, ph_p);   // the tile's P rows
                ph_p ^= 1;
                if (elected) p_pending = false;
                if (valid) {
                    const uint8_t* prow = sP + (int)reinterpret_cast<const int16_t*>(rec + 544)[row] * (2 * H) + 2 * c0;
#pragma unroll
                    for (int kc = 0; kc < NCH; ++kc) {
                        float pv[8], qv[8];
                        const uint4 up = *reinterpret_cast<const uint4*>(prow + 16 * kc);
                        const uint4 uq = *reinterpret_cast<const uint4*>(sSlot + 16 * slot_chunk<H>(kc, row));
                        unpack_bf16x2(up.x, pv[0], pv[1]);
                        unpack_bf16x2(up.y, pv[2], pv[3]);
                        unpack_bf16x2(up.z, pv[4], pv[5]);
                        unpack_bf16x2(up.w, pv[6], pv[7]);
                        unpack_bf16x2(uq.x, qv[0], qv[1]);
                        unpack_bf16x2(uq.y, qv[2], qv[3]);
                        unpack_bf16x2(uq.z, qv[4], qv[5]);
                        unpack_bf16x2(uq.w, qv[6], qv[7]);
#pragma unroll
                        for (int jj = 0; jj < 8; jj += 2) {
                            const float2 pq2 = __fadd2_rn(make_float2(pv[jj], pv[jj + 1]), make_float2(qv[jj], qv[jj + 1]));
                            const float2 t2 = __fadd2_rn(pq2, *reinterpret_cast<const float2*>(bk + 8 * kc + jj));
                            float2* vv = reinterpret_cast<float2*>(v + 8 * kc + jj);
                            *vv = __fadd2_rn(*vv, t2);
                        }
                    }
                }
                // this thread's Q slot is consumed: request the group's next tile's (its record
                // landed a tile ago)
                if (t_next < A.n_tiles) {
                    next_ready = mbar_wait(full + (s ^ 1), (uint32_t)((u + 1) >> 1) & 1u);
                    ok = ok && next_ready;
                    if (next_ready) gather(s ^ 1);
                }
            } else {
                if (k == 1 && elected && next_ready && ok) {
                    // every thread has read the P rows (the barrier before this MMA): the next tile's
                    fetch_p(s ^ 1);
                    p_pending = true;
                }
                add_bias2<CW>(v, bk);
            }
            if (k < n_lin - 1) {
                elu_inplace2<CW>(v);
                st_row_tile<CW>(sA1, row, c0, C::S, v);
                fence_proxy_async();
                tc_fence_before();
                named_sync(bid, GT);
                if (elected) {
                    tc_fence_after();
                    issue_mma(tm, sA1, sW + (k + 1) * C::WT, H, H);
                    mma_commit(mbar);
                    if constexpr (ASAVE) {   // the saved copy leaves while the MMA reads the same tile
                        tma_store_2d(&tmap_h, 0, (int32_t)(k * A.act_rows + t * 128), sA1);
                        bulk_commit();
                    }
                }
            }
        }
        if (!ok) break;
        tc_fence_before();
        float mean, rstd;
        if constexpr (CG == 1) {
            float2 su2 = make_float2(0.f, 0.f), sq2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < CW; i += 2) {
                const float2 x2 = make_float2(v[i], v[i + 1]);
                su2 = __fadd2_rn(su2, x2);
                sq2 = __ffma2_rn(x2, x2, sq2);
            }
            mean = (su2.x + su2.y) * (1.f / H);
            rstd = rsqrtf(fmaxf((sq2.x + sq2.y) * (1.f / H) - mean * mean, 0.f) + A.eps);
        } else {
            row_stats_named<H, CG, CW>(v, sRed, row, cg, A.eps, bid, GT, mean, rstd);
        }
        {
            float eo[CW];
            ld_row_tile<CW>(sE, row, c0, C::S, eo);
            const float* gam = sPar + n_lin * H + c0;
            const float* bet = sPar + (n_lin + 1) * H + c0;
            const float2 r2 = make_float2(rstd, rstd), m2 = make_float2(-mean * rstd, -mean * rstd);
#pragma unroll
            for (int i = 0; i < CW; i += 2) {
                const float2 xh = __ffma2_rn(make_float2(v[i], v[i + 1]), r2, m2);
                const float2 y = __ffma2_rn(xh, *reinterpret_cast<const float2*>(gam + i),
                                            *reinterpret_cast<const float2*>(bet + i));
                const float2 o = __fadd2_rn(y, make_float2(eo[i], eo[i + 1]));
                v[i] = o.x;
                v[i + 1] = o.y;
            }
        }
        // e' goes to this tile's e stage (its last reader was the residual above) and leaves
        // by whole rows per warp after the first barrier of the sums below
        if (A.e_out) st_row_tile<CW>(sE, row, c0, C::S, v);
        // Eq. 5b: a_r = sum over the row's edges of w * e' (edge order), in two passes of SC
        // columns staged in sA1 as 16-byte chunks; one thread per (row, chunk) sums a segment
        float4* sS = reinterpret_cast<float4*>(sA1);
        const int32_t* sRp = reinterpret_cast<const int32_t*>(rec + 16);
        constexpr int NC = SC / 4;
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            if constexpr (CG == 2) {
                if (cg == pass) {
#pragma unroll
                    for (int c = 0; c < NC; ++c)
                        sS[row * NC + stage_chunk<NC>(c, row)] =
                            make_float4(w * v[4 * c], w * v[4 * c + 1], w * v[4 * c + 2], w * v[4 * c + 3]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const float* vp = v + pass * SC + 4 * c;
                    sS[row * NC + stage_chunk<NC>(c, row)] = make_float4(w * vp[0], w * vp[1], w * vp[2], w * vp[3]);
                }
            }
            named_sync(bid, GT);
            if (pass == 0 && A.e_out) {
                constexpr int CPR = H / 8;   // 16-byte chunks per row
                for (int i = gt; i < ne * CPR; i += GT) {
                    const int r = i / CPR, jj = i - r * CPR;
                    *reinterpret_cast<uint4*>(A.e_out + (e0 + r) * H + 8 * jj) =
                        *reinterpret_cast<const uint4*>(sE + tile_off(r, 8 * jj, 128, C::S));
                }
            }
            for (int it = gt; it < nr * NC; it += GT) {
                const int rr = it / NC, c = it % NC;
                const int32_t b0 = sRp[rr], b1 = sRp[rr + 1];
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int32_t e = b0; e < b1; ++e) {
                    const float4 u4 = sS[e * NC + stage_chunk<NC>(c, e)];
                    acc.x += u4.x;
                    acc.y += u4.y;
                    acc.z += u4.z;
                    acc.w += u4.w;
                }
                *reinterpret_cast<float4*>(A.a + (int64_t)(r0 + rr) * H + pass * SC + 4 * c) = acc;
            }
            if (pass == 1) fence_proxy_async();   // generic reads of the stage precede its next async write
            named_sync(bid, GT);
        }
        if (elected && t_refill < A.n_tiles) {
            issue(s, t_refill, e0_refill);
            pending |= (1u << s) | ((((uint32_t)(u + 2) >> 1) & 1u) << (2 + s));
        }
    }
    // after an error, let this group's loads in flight land before the CTA exits
    if (elected) {
        for (int s = 0; s < 2; ++s)
            if (pending & (1u << s)) mbar_wait(full + s, (pending >> (2 + s)) & 1u);
    }
    cp_async_wait_all();
    if (p_pending) mbar_wait(p_full, ph_p);
    if (ASAVE && elected) bulk_wait_all();   // the saved tiles are written before the CTA exits
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, R::NCOLS);
}

// ------------------------------------------------------------------ k_node_fwd

struct NodeFwdArgs {
    const float* a_star;
    const float* x;
    float* x_out;
    int64_t n_rows;
    MlpDev mlp;
    float eps;
    // Backward recomputation (k_node_fwd<H, false, true>): tiles [t0, t1); the
    // scratch row of node row t*128 + i is (t - t0) * 128 + i (zero past n_rows).
    int64_t t0, t1;
    __nv_bfloat16* hs;            // hidden activations h_0 .. h_{L-2}, hs_stride elements apart
    int64_t hs_stride;
    __nv_bfloat16* xa;            // the BF16 input rows [a*, x] (2H wide)
    __nv_bfloat16* dz;            // gradient of the last pre-activation (LayerNorm adjoint)
    const float* dx_out;          // upstream gradient of x'
    float* part;                  // per-CTA partials: gamma, beta, last bias gradients (3H)
    int64_t pstride;
    int64_t act_rows;             // ASAVE: rows of one activation block of tmap_h (tiles * 128)
};

// SAVE: the backward's recomputation of the node MLP (Eq. 5e): the BF16 input
// rows and hidden activations go to scratch and the LayerNorm epilogue is
// replaced by its adjoint, whose input is the gradient of x' (the residual
// branch passes it through unchanged).
// ASAVE (training forward): each finished BF16 hidden tile also goes to block k
// of tmap_h (row k * act_rows + t * 128 + i), and the BF16 input tile [a*, x]
// to tmap_xa (row t * 128 + i), by TMA stores, for the backward.
// SAVE (H = 128) stores the BF16 [a*, x] halves, the hidden tiles and dz with TMA
// stores too: tmap_xa row (t - t0) * 128 (2H wide), tmap_h block k at row
// k * hs_stride / H + (t - t0) * 128, tmap_dz row (t - t0) * 128.
template <int H, bool PF, bool SAVE = false, bool ASAVE = false>
__global__ void __launch_bounds__(Cfg<H>::NT) k_node_fwd(const __grid_constant__ CUtensorMap tmap_a,
                                                        const __grid_constant__ CUtensorMap tmap_x,
                                                        const __grid_constant__ CUtensorMap tmap_h,
                                                        const __grid_constant__ CUtensorMap tmap_xa,
                                                        const __grid_constant__ CUtensorMap tmap_dz,
                                                        const __grid_constant__ CUtensorMap tmap_xo, NodeFwdArgs A) {
    static_assert(!(PF && SAVE), "the recomputation reads its inputs directly");
    static_assert(!SAVE || NodeSplit<H>::value, "the recomputation form is the H = 128 one");
    static_assert(!(ASAVE && (SAVE || NodeSplit<H>::value)), "saved activations: the H <= 64 layer forward");
    using C = Cfg<H>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const NodeFwdSmem L = node_fwd_smem<H, PF>(n_lin, SAVE);
    uint8_t* sW0 = sm + L.w0;
    uint8_t* sW = sm + L.w;
    uint8_t* sA0 = sm + L.a0;
    uint8_t* sA1 = sm + L.a1;
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    float* sRed = reinterpret_cast<float*>(sm + L.red);
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint64_t* full = bar_mma + 1;   // full[2]: FP32 input stage landed (prefetch)
    constexpr uint32_t XB = 128 * H * 4;
    auto sXa = [&](int s) { return sm + L.xs + s * 2 * XB; };   // a* rows, then x rows
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);
    constexpr int S2 = span_of(2 * H);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * C::CW;

    if (warp == 0) {
        tmem_alloc(tslot, C::TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(full, 1);
        mbar_init(full + 1, 1);
        fence_mbar_init();
    }
    load_weight(sW0, A.mlp.W[0], 2 * H, 0, H, 2 * H, tid, C::NT);
    for (int k = 1; k < n_lin; ++k) load_weight(sW + (k - 1) * C::WT, A.mlp.W[k], H, 0, H, H, tid, C::NT);
    for (int i = tid; i < n_lin * H; i += C::NT) sPar[i] = A.mlp.b[i / H][i % H];
    for (int i = tid; i < H; i += C::NT) {
        sPar[n_lin * H + i] = A.mlp.gamma[i];
        sPar[(n_lin + 1) * H + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t ph = 0;
    bool ok = true;
    const int64_t n_tiles = (A.n_rows + 127) / 128;
    auto issue = [&](int s, int64_t t) {   // thread 0: the FP32 a* and x rows of tile t
        mbar_arrive_expect_tx(full + s, 2 * XB);
        tma_f32_tile<H>(sXa(s), &tmap_a, t * 128, full + s);
        tma_f32_tile<H>(sXa(s) + XB, &tmap_x, t * 128, full + s);
    };
    if constexpr (PF) {
        if (tid == 0 && (int64_t)blockIdx.x < n_tiles) issue(0, blockIdx.x);
    }
    int j = 0;
    constexpr int NCH = C::CW / 16;
    float accG[NCH], accB[NCH], accZ[NCH];   // SAVE: column sums of g*xhat, g, dz
#pragma unroll
    for (int i = 0; i < NCH; ++i) accG[i] = accB[i] = accZ[i] = 0.f;
    const int64_t tb = SAVE ? A.t0 : 0, te = SAVE ? A.t1 : n_tiles;

    for (int64_t t = tb + blockIdx.x; t < te && ok; t += gridDim.x, ++j) {
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        const int64_t srow = (t - tb) * 128 + row;   // SAVE: scratch row
        (void)srow;
        const int st = j & 1;
        if constexpr (!PF) {   // the next tile's input rows into L2 (they are read per thread)
            if (tid == 0 && t + gridDim.x < te) {
                const int64_t rn = (t + gridDim.x) * 128;
                const uint32_t nb = (uint32_t)(min((int64_t)128, A.n_rows - rn) * H * 4);
                prefetch_l2(A.a_star + rn * H, nb);
                prefetch_l2(A.x + rn * H, nb);
                if constexpr (SAVE) prefetch_l2(A.dx_out + rn * H, nb);
            }
        }
        float xa[C::CW], xv[C::CW];
        if constexpr (PF) {
            ok = block_wait(full + st, (uint32_t)(j >> 1) & 1u, tid);
            if (!ok) break;
            // the other stage was read by the previous tile (ordered by its closing barrier) and
            // its x' tile stored (waited for here)
            if (tid == 0 && t + gridDim.x < n_tiles) {
                bulk_wait_read_all();
                issue(st ^ 1, t + gridDim.x);
            }
#pragma unroll
            for (int i = 0; i < C::CW / 4; ++i) {   // rows past n_rows read as zero
                const float4 u = ld_f32x4_tile<H>(sXa(st), row, c0 + 4 * i);
                const float4 w = ld_f32x4_tile<H>(sXa(st) + XB, row, c0 + 4 * i);
                xa[4 * i] = u.x; xa[4 * i + 1] = u.y; xa[4 * i + 2] = u.z; xa[4 * i + 3] = u.w;
                xv[4 * i] = w.x; xv[4 * i + 1] = w.y; xv[4 * i + 2] = w.z; xv[4 * i + 3] = w.w;
            }
        } else if (NodeSplit<H>::value) {
            // the operand rows are read whole by warps below; the residual x (FP32) is read
            // per thread for the epilogue, requested here so it lands during the MMA chain
            if (!SAVE && valid) {
                const float4* px = reinterpret_cast<const float4*>(A.x + r * H + c0);
#pragma unroll
                for (int i = 0; i < C::CW / 4; ++i) {
                    const float4 w = __ldg(px + i);
                    xv[4 * i] = w.x; xv[4 * i + 1] = w.y; xv[4 * i + 2] = w.z; xv[4 * i + 3] = w.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) xv[i] = 0.f;
            }
        } else if (valid) {
            const float4* pa = reinterpret_cast<const float4*>(A.a_star + r * H + c0);
            const float4* px = reinterpret_cast<const float4*>(A.x + r * H + c0);
#pragma unroll
            for (int i = 0; i < C::CW / 4; ++i) {
                float4 u = __ldg(pa + i), w = __ldg(px + i);
                xa[4 * i] = u.x; xa[4 * i + 1] = u.y; xa[4 * i + 2] = u.z; xa[4 * i + 3] = u.w;
                xv[4 * i] = w.x; xv[4 * i + 1] = w.y; xv[4 * i + 2] = w.z; xv[4 * i + 3] = w.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < C::CW; ++i) xa[i] = xv[i] = 0.f;
        }
        if constexpr (!NodeSplit<H>::value) {
#pragma unroll
            for (int i = 0; i < C::CW; i += 8) {
                st_tile8(sA0, row, c0 + i, 128, S2, xa + i);
                st_tile8(sA0, row, H + c0 + i, 128, S2, xv + i);
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                issue_mma(tmem, sA0, sW0, H, 2 * H);
                mma_commit(bar_mma);
                if constexpr (ASAVE) {   // one box per S2 / 2 columns, as the tile is laid out
#pragma unroll
                    for (int kb = 0; kb < 2 * H / (S2 / 2); ++kb)
                        tma_store_2d(&tmap_xa, kb * (S2 / 2), (int32_t)(t * 128), sA0 + kb * 128 * S2);
                    bulk_commit();
                }
            }
        } else {
            // K half 0 (a*) then K half 1 (x) through the same [128 x H] buffer, each row read
            // whole by one warp (lane l: columns 4l .. 4l+3; warp w: rows 8w .. 8w+7); the x
            // rows wait in registers until the a* half has been multiplied
            static_assert(C::NT == 512 && H == 128, "row-per-warp fill: 16 warps x 8 rows, 32 lanes x 4 columns");
            float4 xr[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int rr = 8 * warp + i;
                const int64_t rg = t * 128 + rr;
                float4 av = make_float4(0.f, 0.f, 0.f, 0.f);
                xr[i] = av;
                if (rg < A.n_rows) {
                    av = __ldg(reinterpret_cast<const float4*>(A.a_star + rg * H) + lane);
                    xr[i] = __ldg(reinterpret_cast<const float4*>(A.x + rg * H) + lane);
                }
                *reinterpret_cast<uint2*>(sA0 + tile_off(rr, 4 * lane, 128, C::S)) =
                    make_uint2(pack_bf16x2(av.x, av.y), pack_bf16x2(av.z, av.w));
            }
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                issue_mma_koff(tmem, sA0, sW0, H, H, 0, 2 * H, false);
                mma_commit(bar_mma);
                if constexpr (SAVE) {   // the a* half of the saved input rows
#pragma unroll
                    for (int kb = 0; kb < H / 64; ++kb)
                        tma_store_2d(&tmap_xa, kb * 64, (int32_t)((t - tb) * 128), sA0 + kb * 128 * 128);
                    bulk_commit();
                }
            }
            if (SAVE && tid == 0) bulk_wait_read_all();   // sA0 is rewritten after the barrier
            ok = block_wait(bar_mma, ph, tid);
            ph ^= 1;
            tc_fence_after();
            if (!ok) break;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                *reinterpret_cast<uint2*>(sA0 + tile_off(8 * warp + i, 4 * lane, 128, C::S)) =
                    make_uint2(pack_bf16x2(xr[i].x, xr[i].y), pack_bf16x2(xr[i].z, xr[i].w));
            fence_proxy_async();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                issue_mma_koff(tmem, sA0, sW0, H, H, H, 2 * H, true);
                mma_commit(bar_mma);
                if constexpr (SAVE) {   // and the x half
#pragma unroll
                    for (int kb = 0; kb < H / 64; ++kb)
                        tma_store_2d(&tmap_xa, H + kb * 64, (int32_t)((t - tb) * 128), sA0 + kb * 128 * 128);
                    bulk_commit();
                }
            }
        }
        float v[C::CW];
        for (int k = 0; k < n_lin && ok; ++k) {
            if ((ASAVE || SAVE) && tid == 0) bulk_wait_read_all();   // sA0 / sA1 may be rewritten after the barrier
            ok = block_wait(bar_mma, ph, tid);
            ph ^= 1;
            tc_fence_after();
            if (!ok) break;
            ld_acc<C::CW>(tmem, q, c0, v);
            add_bias2<C::CW>(v, sPar + k * H + c0);
            if (k < n_lin - 1) {
                elu_inplace2<C::CW>(v);
                if constexpr (SAVE) {   // the saved rows past the graph's rows are zero
#pragma unroll
                    for (int i = 0; i < C::CW; ++i) v[i] = valid ? v[i] : 0.f;
                }
                st_row_tile<C::CW>(sA1, row, c0, C::S, v);
                fence_proxy_async();
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    issue_mma(tmem, sA1, sW + k * C::WT, H, H);
                    mma_commit(bar_mma);
                    if constexpr (ASAVE) {
                        tma_store_2d(&tmap_h, 0, (int32_t)(k * A.act_rows + t * 128), sA1);
                        bulk_commit();
                    }
                    if constexpr (SAVE) {
#pragma unroll
                        for (int kb = 0; kb < H / 64; ++kb)
                            tma_store_2d(&tmap_h, kb * 64, (int32_t)(k * (A.hs_stride / H) + (t - tb) * 128),
                                         sA1 + kb * 128 * 128);
                        bulk_commit();
                    }
                }
            }
        }
        if (!ok) break;
        tc_fence_before();
        if constexpr (SAVE) {
            float gv[C::CW];
            if (valid) {
                const float4* pg = reinterpret_cast<const float4*>(A.dx_out + r * H + c0);
#pragma unroll
                for (int i = 0; i < C::CW / 4; ++i) {
                    const float4 u = __ldg(pg + i);
                    gv[4 * i] = u.x; gv[4 * i + 1] = u.y; gv[4 * i + 2] = u.z; gv[4 * i + 3] = u.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < C::CW; ++i) gv[i] = 0.f;
            }
            const float* gam = sPar + n_lin * H + c0;
            float mean, rstd, s1, s2;
            row_stats_adj_gamma<H, C::CG, C::CW>(v, gv, gam, sRed, row, g, A.eps, mean, rstd, s1, s2);
            ln_adjoint_row<C::CW>(v, gv, gam, mean, rstd, s1, s2, valid, lane, accG, accB, accZ);
            st_row_tile<C::CW>(sA1, row, c0, C::S, v);   // dz to scratch by TMA (the last MMA has read sA1)
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
#pragma unroll
                for (int kb = 0; kb < H / 64; ++kb)
                    tma_store_2d(&tmap_dz, kb * 64, (int32_t)((t - tb) * 128), sA1 + kb * 128 * 128);
                bulk_commit();
            }
            continue;
        }
        float mean, rstd;
        row_stats<H, C::CG, C::CW>(v, sRed, row, g, A.eps, mean, rstd);
        const float* gam = sPar + n_lin * H + c0;
        const float* bet = sPar + (n_lin + 1) * H + c0;
        if constexpr (PF) {
            // x' overwrites the residual x in the stage (each thread its own chunks) and leaves by
            // TMA stores of the tile's boxes (rows past n_rows are not written)
#pragma unroll
            for (int i = 0; i < C::CW / 4; ++i) {
                const float4 w = ld_f32x4_tile<H>(sXa(st) + XB, row, c0 + 4 * i);
                float4 o;
                o.x = w.x + (v[4 * i] - mean) * rstd * gam[4 * i] + bet[4 * i];
                o.y = w.y + (v[4 * i + 1] - mean) * rstd * gam[4 * i + 1] + bet[4 * i + 1];
                o.z = w.z + (v[4 * i + 2] - mean) * rstd * gam[4 * i + 2] + bet[4 * i + 2];
                o.w = w.w + (v[4 * i + 3] - mean) * rstd * gam[4 * i + 3] + bet[4 * i + 3];
                st_f32x4_tile<H>(sXa(st) + XB, row, c0 + 4 * i, o);
            }
            fence_proxy_async();   // generic accesses of the stage precede the TMA store and its next load
            __syncthreads();
            if (tid == 0) {
                constexpr int BW = H < 32 ? H : 32;
#pragma unroll
                for (int b = 0; b < H / BW; ++b)
                    tma_store_2d(&tmap_xo, b * BW, (int32_t)(t * 128), sXa(st) + XB + b * 128 * BW * 4);
                bulk_commit();
            }
        } else {
            if (valid) {
                float4* po = reinterpret_cast<float4*>(A.x_out + r * H + c0);
#pragma unroll
                for (int i = 0; i < C::CW / 4; ++i) {
                    float4 o;
                    o.x = xv[4 * i] + (v[4 * i] - mean) * rstd * gam[4 * i] + bet[4 * i];
                    o.y = xv[4 * i + 1] + (v[4 * i + 1] - mean) * rstd * gam[4 * i + 1] + bet[4 * i + 1];
                    o.z = xv[4 * i + 2] + (v[4 * i + 2] - mean) * rstd * gam[4 * i + 2] + bet[4 * i + 2];
                    o.w = xv[4 * i + 3] + (v[4 * i + 3] - mean) * rstd * gam[4 * i + 3] + bet[4 * i + 3];
                    po[i] = o;
                }
            }
            __syncthreads();
        }
    }
    if constexpr (SAVE) {
        float* part = A.part + (int64_t)blockIdx.x * A.pstride;
        colsum_store<H, NCH>(accG, sRed, q, lane, c0, tid, C::NT, part);
        colsum_store<H, NCH>(accB, sRed, q, lane, c0, tid, C::NT, part + H);
        colsum_store<H, NCH>(accZ, sRed, q, lane, c0, tid, C::NT, part + 2 * H);
    }
    if ((ASAVE || SAVE || PF) && tid == 0) bulk_wait_all();   // the stored tiles are written before the CTA exits
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, C::TCOLS);
}

// =================================================================== host side

namespace {

using namespace host;

struct FwdWs {
    __nv_bfloat16* pq;
    float* a;
    __nv_bfloat16* e_scratch;
    size_t bytes;
};

FwdWs carve_fwd(void* ws, const gnn_graph_dev& G, int H, bool need_a, bool need_e) {
    FwdWs w{};
    size_t off = 0;
    auto take = [&](size_t n) {
        off = (off + 255) & ~(size_t)255;
        void* p = ws ? (char*)ws + off : nullptr;
        off += n;
        return p;
    };
    w.pq = (__nv_bfloat16*)take((size_t)G.n_rows * 2 * H * 2);
    w.a = need_a ? (float*)take((size_t)G.n_rows * H * 4) : nullptr;
    w.e_scratch = need_e ? (__nv_bfloat16*)take(0) : nullptr;
    w.bytes = off + 256;
    return w;
}

template <int H>
int proj_h(const gnn_graph_dev& G, const gnn_mp_params& W, const float* x_in, __nv_bfloat16* pq, cudaStream_t s) {
    using C = Cfg<H>;
    const int64_t NR = G.n_rows;
    if (NR == 0) return GNN_OK;
    const ProjSmem L = proj_smem<H>();
    int grid;
    CUtensorMap tmx, tmp, tmq;
    int rc = make_f32_tmap(&tmx, x_in, NR, H);
    if (rc) return rc;
    if ((rc = make_row_tmap(&tmp, pq, NR, H))) return rc;
    if ((rc = make_row_tmap(&tmq, pq + NR * H, NR, H))) return rc;
    rc = persistent_grid(k_proj_fwd<H>, C::NT, L.total, 2 * H < 32 ? 32 : 2 * H, (NR + 127) / 128, &grid);
    if (rc) return rc;
    {
        ProfScope _ps(s, "k_proj_fwd");
        k_proj_fwd<H><<<grid, C::NT, L.total, s>>>(tmx, tmp, tmq, NR, W.edge.W[0]);
    }
    GNN_LAUNCH_CHECK("k_proj_fwd");
    return GNN_OK;
}

// Edge MLP + residual + weighted segmented sum (Eq. 5a-5b), then Eq. 5c-5d.
template <int H>
int edge_h(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const __nv_bfloat16* e_in,
           const __nv_bfloat16* pq, __nv_bfloat16* e_out, float* a, __nv_bfloat16* act, cudaStream_t s) {
    using C = Cfg<H>;
    const int64_t NR = G.n_rows, E = G.n_edges;
    if (NR == 0) return GNN_OK;
    if (E > 0) {
        CUtensorMap tm;
        int rc = make_row_tmap(&tm, e_in, E, H);
        if (rc) return rc;
        EdgeFwdArgs A;
        A.row_ptr = G.row_ptr;
        A.col = G.col;
        A.edge_w = G.edge_w;
        A.tiles = G.edge_tiles;
        A.tile_meta = static_cast<const uint8_t*>(G.tile_meta);
        A.n_tiles = G.n_edge_tiles;
        A.n_edges = E;
        A.pq = pq;
        A.q = pq + NR * H;
        A.e_in = e_in;
        A.e_out = e_out;
        A.a = a;
        A.mlp = mlp_dev(W.edge);
        A.eps = cfg.ln_eps;
        A.act = act;
        A.act_rows = G.n_edge_tiles * 128;
        CUtensorMap tmh = tm;
        if (act && (rc = make_row_tmap(&tmh, act, (int64_t)(W.edge.n_lin - 1) * A.act_rows, H))) return rc;
        int grid;
        int variant = cfg.edge_fwd_kernel;
        if (variant == GNN_EDGE_FWD_AUTO || act)
            variant = H <= 64 ? GNN_EDGE_FWD_RT : (edge_fwd_tm_supported(W) ? GNN_EDGE_FWD_TM : GNN_EDGE_FWD_ONE);
        if constexpr (H == 128) {
            if (variant == GNN_EDGE_FWD_TM) {
                if ((rc = edge_fwd_tm(G, cfg, W, e_in, pq, e_out, a, s))) return rc;
                return cfg.halo_mode == GNN_HALO_SYNC ? plain::halo(G, a, H, s) : GNN_OK;
            }
        }
        if constexpr (H <= 64) {
            if (variant == GNN_EDGE_FWD_RT) {
                using R = RtCfg<H>;
                GNN_REQUIRE(G.tile_meta && ((uintptr_t)G.tile_meta & 15) == 0, GNN_EINVAL,
                            "gnn_mp_forward: tile_meta must be a 16-byte aligned device array");
                const EdgeFwdRtSmem L = edge_fwd_rt_smem<H>(W.edge.n_lin);
                const int64_t ntile = (G.n_edge_tiles + R::NG - 1) / R::NG;
                if (act) {
                    rc = persistent_grid(k_edge_fwd_rt<H, true>, R::NT, L.total, R::NCOLS, ntile, &grid,
                                         cfg.ctas_per_sm);
                    if (rc) return rc;
                    ProfScope _ps(s, "k_edge_fwd");
                    k_edge_fwd_rt<H, true><<<grid, R::NT, L.total, s>>>(tm, tmh, A);
                } else {
                    rc = persistent_grid(k_edge_fwd_rt<H>, R::NT, L.total, R::NCOLS, ntile, &grid, cfg.ctas_per_sm);
                    if (rc) return rc;
                    ProfScope _ps(s, "k_edge_fwd");
                    k_edge_fwd_rt<H><<<grid, R::NT, L.total, s>>>(tm, tmh, A);
                }
            } else if (variant == GNN_EDGE_FWD_WS) {
                const EdgeFwdWsSmem L = edge_fwd_ws_smem<H>(W.edge.n_lin);
                const uint32_t ncols = C::TCOLS * WS_NG < 32 ? 32 : C::TCOLS * WS_NG;
                rc = persistent_grid(k_edge_fwd_ws<H>, WsCfg<H>::NT, L.total, ncols, G.n_edge_tiles, &grid,
                                     cfg.ctas_per_sm);
                if (rc) return rc;
                ProfScope _ps(s, "k_edge_fwd");
                k_edge_fwd_ws<H><<<grid, WsCfg<H>::NT, L.total, s>>>(tm, A);
            }
        }
        if (variant == GNN_EDGE_FWD_ONE) {
            GNN_REQUIRE(G.tile_meta && ((uintptr_t)G.tile_meta & 15) == 0, GNN_EINVAL,
                        "gnn_mp_forward: tile_meta must be a 16-byte aligned device array");
            const EdgeFwdSmem L = edge_fwd_smem<H>(W.edge.n_lin);
            rc = persistent_grid(k_edge_fwd<H>, C::NT, L.total, C::TCOLS, G.n_edge_tiles, &grid, cfg.ctas_per_sm);
            if (rc) return rc;
            ProfScope _ps(s, "k_edge_fwd");
            k_edge_fwd<H><<<grid, C::NT, L.total, s>>>(tm, tm, tm, A);
        }
        GNN_LAUNCH_CHECK("k_edge_fwd");
    } else {
        GNN_CUDA_CHECK(cudaMemsetAsync(a, 0, sizeof(float) * NR * H, s), "memset");
    }
    if (cfg.halo_mode == GNN_HALO_SYNC) return plain::halo(G, a, H, s);
    return GNN_OK;
}

template <int H>
int node_h(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* a,
           const float* x_in, float* x_out, __nv_bfloat16* act, cudaStream_t s) {
    using C = Cfg<H>;
    const int64_t NR = G.n_rows;
    if (NR == 0) return GNN_OK;
    if constexpr (H == 128) {   // two tile groups per SM, the operands in tensor memory
        if (!act && node_fwd_tm_supported(W)) return node_fwd_tm(G, cfg, W, a, x_in, x_out, s);
    }
    NodeFwdArgs A;
    A.a_star = a;
    A.x = x_in;
    A.x_out = x_out;
    A.n_rows = NR;
    A.mlp = mlp_dev(W.node);
    A.eps = cfg.ln_eps;
    int grid;
    CUtensorMap tma, tmx;
    int rc = make_f32_tmap(&tma, a, NR, H);
    if (rc) return rc;
    if ((rc = make_f32_tmap(&tmx, x_in, NR, H))) return rc;
    // prefetching stages when they fit beside the weights (H <= 64), else one tile at a time
    const NodeFwdSmem Lp = node_fwd_smem<H, true>(W.node.n_lin);
    const bool pf = H <= 64 && Lp.total <= 227 * 1024;
    const NodeFwdSmem L = pf ? Lp : node_fwd_smem<H, false>(W.node.n_lin);
    // saved activations: block k of act holds h_k of tile t at rows k * act_rows + t * 128
    // and the BF16 [a*, x] input tiles after them (row t * 128 + i, 2H wide)
    A.act_rows = (NR + 127) / 128 * 128;
    CUtensorMap tmh = tma, tmxa = tma, tmxo = tma;
    if (pf && (rc = make_f32_tmap(&tmxo, x_out, NR, H))) return rc;   // x' leaves by TMA stores
    if (act && (rc = make_row_tmap(&tmh, act, (int64_t)(W.node.n_lin - 1) * A.act_rows, H))) return rc;
    if (act && (rc = make_row_tmap(&tmxa, act + (int64_t)(W.node.n_lin - 1) * A.act_rows * H, A.act_rows, 2 * H)))
        return rc;
    auto run = [&](auto kern) -> int {
        int r = persistent_grid(kern, C::NT, L.total, C::TCOLS, (NR + 127) / 128, &grid);
        if (r) return r;
        {
            ProfScope _ps(s, "k_node_fwd");
            kern<<<grid, C::NT, L.total, s>>>(tma, tmx, tmh, tmxa, tma, tmxo, A);
        }
        GNN_LAUNCH_CHECK("k_node_fwd");
        return GNN_OK;
    };
    if constexpr (H <= 64) {
        if (act) return pf ? run(k_node_fwd<H, true, false, true>) : run(k_node_fwd<H, false, false, true>);
    }
    return pf ? run(k_node_fwd<H, true>) : run(k_node_fwd<H, false>);
}

}  // namespace

size_t mp_forward_ws(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params&) {
    return carve_fwd(nullptr, G, cfg.hidden, true, false).bytes;
}

#define GNN_H_DISPATCH(H_, CALL)                                                           \
    switch (H_) {                                                                          \
        case 16: { constexpr int HH = 16; return CALL; }                                   \
        case 32: { constexpr int HH = 32; return CALL; }                                   \
        case 64: { constexpr int HH = 64; return CALL; }                                   \
        case 128: { constexpr int HH = 128; return CALL; }                                 \
        default: return set_error(GNN_ESHAPE, "BF16 path needs H in {16,32,64,128} (H=%d)", H_); \
    }

int proj_forward(const gnn_graph_dev& G, int H, const gnn_mp_params& W, const float* x_in, __nv_bfloat16* pq,
                 cudaStream_t s) {
    GNN_H_DISPATCH(H, proj_h<HH>(G, W, x_in, pq, s));
}

int aggregate_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                      const __nv_bfloat16* e_in, const __nv_bfloat16* pq, __nv_bfloat16* e_out, float* a,
                      cudaStream_t s, __nv_bfloat16* act) {
    GNN_H_DISPATCH(cfg.hidden, edge_h<HH>(G, cfg, W, e_in, pq, e_out, a, act, s));
}

size_t mp_act_elems_edge(const gnn_graph_dev& G, const gnn_mp_params& W, int H) {
    return (size_t)(W.edge.n_lin - 1) * (size_t)G.n_edge_tiles * 128 * (size_t)H;
}

size_t mp_act_bytes(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W) {
    if (cfg.precision != GNN_PREC_BF16 || cfg.hidden > 64 || W.edge.n_lin < 2 || W.node.n_lin < 2) return 0;
    // whole 128-row tiles pay only when the tiles are nearly full (the default edge cap); a
    // graph re-tiled to smaller caps would store mostly padding, so it recomputes instead
    if (G.n_edge_tiles * 128 > G.n_edges + G.n_edges / 4 + 128) return 0;
    // activation rows are 32-bit TMA coordinates: edge row k * tiles * 128 + t * 128 + i,
    // node row k * rows + r
    const int64_t rows = (G.n_rows + 127) / 128 * 128;
    if ((int64_t)(W.edge.n_lin - 1) * G.n_edge_tiles * 128 >= ((int64_t)1 << 31) ||
        (int64_t)(W.node.n_lin - 1) * rows >= ((int64_t)1 << 31))
        return 0;
    // node part: (L_n - 1) hidden blocks [rows x H] and the input block [rows x 2H]
    return (mp_act_elems_edge(G, W, cfg.hidden) + (size_t)(W.node.n_lin + 1) * (size_t)rows * cfg.hidden) * 2;
}

int node_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* a,
                 const float* x_in, float* x_out, cudaStream_t s, __nv_bfloat16* act) {
    GNN_H_DISPATCH(cfg.hidden, node_h<HH>(G, cfg, W, a, x_in, x_out, act, s));
}

// ------------------------------------------------------------------ forward with a built-in scratch area
//
// Some callers cannot allocate device memory when they run the layer: code
// that executes while a CUDA stream is being captured without a graph memory
// pool, or a host framework that owns the device allocator and hands the
// library only the tensors it computes on. mp_forward_static serves them with
// a fixed scratch area that is part of this library's device image instead of
// a caller workspace. Every GPU that loads the library holds the area until
// the process exits, and every call shares it: calls whose executions overlap
// on the GPU (two streams, or two host threads) race on it.

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_static_mu;
void* g_static_addr[128] = {};   // device address of g_static_scratch per device ordinal
}  // namespace

size_t static_scratch_bytes() { return kStaticScratchBytes; }

// The device address of the scratch array on the current device; host code
// must not use the array's name as a pointer. Outside stream capture the
// address is looked up on every call (cheap once the module is loaded), so a
// reset device's reloaded module is seen; while `s` is being captured the
// address recorded by the device's last call outside capture is used.
static int static_scratch_address(cudaStream_t s, void** out) {
    int dev = 0;
    GNN_CUDA_CHECK(cudaGetDevice(&dev), "gnn_mp_forward_static: cudaGetDevice");
    GNN_REQUIRE(dev >= 0 && dev < 128, GNN_EUNSUPPORTED, "gnn_mp_forward_static: device ordinal %d", dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GNN_CUDA_CHECK(cudaStreamIsCapturing(s, &cs), "gnn_mp_forward_static: cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        GNN_CUDA_CHECK(cudaGetSymbolAddress(&p, g_static_scratch), "gnn_mp_forward_static: cudaGetSymbolAddress");
        g_static_addr[dev] = p;
    }
    GNN_REQUIRE(g_static_addr[dev], GNN_EINVAL,
                "gnn_mp_forward_static: first call on device %d made during stream capture; make one call "
                "outside capture first", dev);
    *out = g_static_addr[dev];
    return GNN_OK;
}

int mp_forward_static(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                      const __nv_bfloat16* e_in, float* x_out, __nv_bfloat16* e_out, float* a_star_out,
                      cudaStream_t s) {
    // scratch: P|Q rows (and the aggregate when a_star_out is NULL); every byte
    // of it is written before it is read, so nothing needs clearing between calls
    const size_t need = carve_fwd(nullptr, G, cfg.hidden, a_star_out == nullptr, false).bytes;
    GNN_REQUIRE(need <= kStaticScratchBytes, GNN_ESHAPE,
                "gnn_mp_forward_static: this graph needs %zu bytes of scratch, the built-in area holds %zu "
                "(about n_rows * 4H bytes, plus n_rows * 4H more when a_star_out is NULL); "
                "use gnn_mp_forward with a workspace",
                need, kStaticScratchBytes);
    void* scratch = nullptr;
    int rc = static_scratch_address(s, &scratch);
    if (rc) return rc;
    return mp_forward(G, cfg, W, x_in, e_in, x_out, e_out, a_star_out, scratch, kStaticScratchBytes, s);
}

int mp_forward(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
               const __nv_bfloat16* e_in, float* x_out, __nv_bfloat16* e_out, float* a_star_out, void* ws,
               size_t ws_bytes, cudaStream_t s, __nv_bfloat16* act) {
    const int H = cfg.hidden;
    GNN_REQUIRE(H == 16 || H == 32 || H == 64 || H == 128, GNN_ESHAPE, "gnn_mp_forward: BF16 path needs H in {16,32,64,128}");
    GNN_REQUIRE(W.edge.n_lin >= 2 && W.node.n_lin >= 2, GNN_ESHAPE, "MLPs need >= 2 Linear layers");
    FwdWs w = carve_fwd(ws, G, H, a_star_out == nullptr, false);
    GNN_REQUIRE(ws_bytes >= w.bytes, GNN_ENOMEM, "gnn_mp_forward: workspace too small");
    __nv_bfloat16* eo = (cfg.flags & GNN_FLAG_NO_EDGE_OUT) ? nullptr : e_out;
    float* a = a_star_out ? a_star_out : w.a;
    int rc;
    if ((rc = proj_forward(G, H, W, x_in, w.pq, s))) return rc;
    if (!mp_act_bytes(G, cfg, W)) act = nullptr;
    if ((rc = aggregate_forward(G, cfg, W, e_in, w.pq, eo, a, s, act))) return rc;
    return node_forward(G, cfg, W, a, x_in, x_out, s, act ? act + mp_act_elems_edge(G, W, H) : nullptr);
}

// ------------------------------------------------------------------ backward recomputation (H = 128)

int edge_recompute_save(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                        const __nv_bfloat16* e_in, const __nv_bfloat16* pq, RecomputeSave& o, cudaStream_t s) {
    constexpr int H = 128;
    using C = Cfg<H>;
    const int64_t NR = G.n_rows, E = G.n_edges;
    GNN_REQUIRE(cfg.hidden == H, GNN_EUNSUPPORTED, "edge_recompute_save: H=%d", cfg.hidden);
    if (edge_fwd_tm_supported(W) && cfg.edge_fwd_kernel != GNN_EDGE_FWD_ONE)
        return edge_save_tm(G, cfg, W, e_in, pq, o, s);
    GNN_REQUIRE(G.tile_meta && ((uintptr_t)G.tile_meta & 15) == 0, GNN_EINVAL,
                "gnn_mp_backward: tile_meta must be a 16-byte aligned device array");
    CUtensorMap tm;
    int rc = make_row_tmap(&tm, e_in, E, H);
    if (rc) return rc;
    EdgeFwdArgs A{};
    A.row_ptr = G.row_ptr;
    A.col = G.col;
    A.edge_w = G.edge_w;
    A.tiles = G.edge_tiles;
    A.tile_meta = static_cast<const uint8_t*>(G.tile_meta);
    A.n_tiles = o.t1;
    A.n_edges = E;
    A.pq = pq;
    A.q = pq + NR * H;
    A.e_in = e_in;
    A.mlp = mlp_dev(W.edge);
    A.eps = cfg.ln_eps;
    A.t0 = o.t0;
    A.hs = o.hs;
    A.hs_stride = o.hs_stride;
    A.dz = o.dz;
    A.da = o.da;
    A.de_out = o.de_out;
    A.part = o.part;
    A.pstride = o.pstride;
    const EdgeFwdSmem L = edge_fwd_smem<H>(W.edge.n_lin, true);
    CUtensorMap tmhs, tmdz;
    if ((rc = make_row_tmap(&tmhs, o.hs, (int64_t)(W.edge.n_lin - 1) * (o.hs_stride / H), H))) return rc;
    if ((rc = make_row_tmap(&tmdz, o.dz, o.hs_stride / H, H))) return rc;
    if ((rc = persistent_grid(k_edge_fwd<H, true>, C::NT, L.total, C::TCOLS, o.t1 - o.t0, &o.grid))) return rc;
    {
        ProfScope _ps(s, "k_edge_fwd_save");
        k_edge_fwd<H, true><<<o.grid, C::NT, L.total, s>>>(tm, tmhs, tmdz, A);
    }
    GNN_LAUNCH_CHECK("k_edge_fwd_save");
    return GNN_OK;
}

int node_recompute_save(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W,
                        const float* a_star, const float* x_in, RecomputeSave& o, cudaStream_t s) {
    constexpr int H = 128;
    using C = Cfg<H>;
    GNN_REQUIRE(cfg.hidden == H, GNN_EUNSUPPORTED, "node_recompute_save: H=%d", cfg.hidden);
    NodeFwdArgs A{};
    A.a_star = a_star;
    A.x = x_in;
    A.n_rows = G.n_rows;
    A.mlp = mlp_dev(W.node);
    A.eps = cfg.ln_eps;
    A.t0 = o.t0;
    A.t1 = o.t1;
    A.hs = o.hs;
    A.hs_stride = o.hs_stride;
    A.xa = o.xa;
    A.dz = o.dz;
    A.dx_out = o.dx_out;
    A.part = o.part;
    A.pstride = o.pstride;
    CUtensorMap tma, tmx;   // unused by the recomputation (it reads its rows directly)
    int rc = make_f32_tmap(&tma, a_star, G.n_rows, H);
    if (rc) return rc;
    if ((rc = make_f32_tmap(&tmx, x_in, G.n_rows, H))) return rc;
    CUtensorMap tmhs, tmxa, tmdz;   // the scratch tiles, written by TMA stores
    const int64_t cap = o.hs_stride / H;   // scratch rows per block
    if ((rc = make_row_tmap(&tmhs, o.hs, (int64_t)(W.node.n_lin - 1) * cap, H))) return rc;
    if ((rc = make_row_tmap(&tmxa, o.xa, cap, 2 * H))) return rc;
    if ((rc = make_row_tmap(&tmdz, o.dz, cap, H))) return rc;
    const NodeFwdSmem L = node_fwd_smem<H, false>(W.node.n_lin, true);
    if ((rc = persistent_grid(k_node_fwd<H, false, true>, C::NT, L.total, C::TCOLS, o.t1 - o.t0, &o.grid)))
        return rc;
    {
        ProfScope _ps(s, "k_node_fwd_save");
        k_node_fwd<H, false, true><<<o.grid, C::NT, L.total, s>>>(tma, tmx, tmhs, tmxa, tmdz, tma, A);
    }
    GNN_LAUNCH_CHECK("k_node_fwd_save");
    return GNN_OK;
}

}  // namespace fused
}  // namespace gnn
