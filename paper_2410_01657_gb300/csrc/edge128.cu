// Edge forward of the consistent NMP layer at H = 128 with two tiles in
// flight per SM (Eq. 5a-5b): gather, edge MLP, residual, LayerNorm and the
// 1/d-weighted segmented sum, as k_edge_fwd<128> computes them.
//
// At H = 128 the four BF16 weight tiles of the edge MLP take 128 KB of shared
// memory, which leaves no room for the activation tiles of a second tile. This
// kernel keeps each hidden activation h_k in tensor memory instead, as the A
// operand of the next Linear (tcgen05.mma with A in TMEM, B = W_k in shared
// memory), so that shared memory holds only the weights and one edge-state
// tile per group. Two groups of four warps take alternate tiles of the CTA's
// share; while one group waits on its MMA chain the other runs its epilogues.
// One thread owns one edge row (all 128 columns), so the LayerNorm statistics
// need no exchange between threads.
//
// Per group and tile:
//   TMA: tile record (CSR slice, receivers, senders, 1/d) + edge-state rows e
//   MMA 1: acc = e W1c^T (A = e tile in shared memory)
//   gather P_i, Q_j (BF16, the split first Linear's per-node products)
//   epilogue k < L-1: h_k = ELU(acc + [P_i + Q_j] + b_k) -> BF16 into TMEM (A)
//   MMA k+1: acc = h_k W_{k+1}^T (A in TMEM)
//   epilogue L-1: e' = e + LN(acc + b_L) (FP32 statistics, e read from the
//   tile in shared memory), e' staged as BF16 in the e tile and written out as
//   whole rows, then w e' staged in FP32 (two halves of 64 columns) and summed
//   per receiver in edge order into a.
// TMEM: group g uses columns [256 g, 256 g + 128) for the accumulator and the
// next 64 columns for the BF16 activation (two values per 32-bit column).

#include <algorithm>

#include "fused.h"
#include "profiler.h"
#include "tm128_common.cuh"

namespace gnn {
namespace fused {

cudaError_t take_device_error_edge128(unsigned int* out) { return take_device_error_word(out); }

namespace {

using namespace tc;
using namespace tm128;

constexpr int kMaxLin = 4;                     // weights resident in shared memory

struct TmArgs {
    const uint8_t* tile_meta;   // per-tile records (GNN_TILE_META_BYTES each)
    int64_t n_tiles;
    const __nv_bfloat16* pq;    // P rows [n_rows x H]
    const __nv_bfloat16* q;     // Q rows [n_rows x H]
    const __nv_bfloat16* e_in;  // edge states (prefetched into L2 one tile ahead)
    __nv_bfloat16* e_out;       // NULL: no edge-state output (inference, last layer)
    float* a;
    MlpDev mlp;
    float eps;
};

struct TmSmem {
    uint32_t w, e, rec, par, bar, tm, total;
};

__host__ __device__ inline TmSmem tm_smem(int n_lin) {
    TmSmem s;
    s.w = 0;
    s.e = align_up((uint32_t)n_lin * kWT, 1024);             // e[2] (one per group)
    s.rec = s.e + 2 * kTile;                                 // rec[2]
    s.par = s.rec + 2 * GNN_TILE_META_BYTES;                 // b_0..b_{L-1}, gamma, beta
    s.bar = align_up(s.par + (uint32_t)(n_lin + 2) * kH * 4, 8);   // ld[2], mma[2]
    s.tm = s.bar + 4 * 8;
    s.total = s.tm + 16 + 1024;
    return s;
}


__global__ void __launch_bounds__(kNT, 1) k_edge_fwd_tm(const __grid_constant__ CUtensorMap tmap_e, TmArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const TmSmem L = tm_smem(n_lin);
    uint8_t* sW = sm + L.w;
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    uint64_t* bar_ld = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint64_t* bar_mma = bar_ld + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = warp >> 2, q = warp & 3, row = 32 * q + lane;
    const bool leader = (tid & (kGT - 1)) == 0;          // issues the group's loads and MMAs
    uint8_t* sE = sm + L.e + gi * kTile;
    uint8_t* rec = sm + L.rec + gi * GNN_TILE_META_BYTES;

    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(bar_ld + i, 1);
        fence_mbar_init();
    }
    load_weight(sW, A.mlp.W[0], 3 * kH, 2 * kH, kH, kH, tid, kNT);        // W1c: the edge-state columns of W1
    for (int k = 1; k < n_lin; ++k) load_weight(sW + k * kWT, A.mlp.W[k], kH, 0, kH, kH, tid, kNT);
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

    // the group's tiles: j-th tile of the CTA is blockIdx.x + j * gridDim.x, group gi takes j = gi, gi + 2, ...
    const int64_t step = 2 * (int64_t)gridDim.x;
    const int64_t t_first = (int64_t)blockIdx.x + gi * (int64_t)gridDim.x;
    auto tile_hdr = [&](int64_t t) { return ld_nc_v4s32(A.tile_meta + t * GNN_TILE_META_BYTES); };
    bool ld_pending = false;   // leader: a load nobody has waited for
    auto issue_ld = [&](int64_t t, int32_t e0) {
        mbar_arrive_expect_tx(bar_ld + gi, kTile + GNN_TILE_META_BYTES);
        bulk_load(rec, A.tile_meta + t * GNN_TILE_META_BYTES, GNN_TILE_META_BYTES, bar_ld + gi);
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) tma_load_2d(sE + kb * 128 * kS, &tmap_e, kb * 64, e0, bar_ld + gi);
        ld_pending = true;
    };
    if (leader && t_first < A.n_tiles) issue_ld(t_first, tile_hdr(t_first).z);
    uint32_t ph_ld = 0, ph_mma = 0;
    bool ok = true;
    constexpr int NC = 16;   // 16-byte chunks of a staged half row (64 FP32 columns)
    float4* sS4 = reinterpret_cast<float4*>(sE);

    for (int64_t t = t_first; t < A.n_tiles && ok; t += step) {
        bool w_ok = leader ? mbar_wait(bar_ld + gi, ph_ld) : true;
        ok = group_and(w_ok, gi);
        if (!ok) break;
        ph_ld ^= 1;
        if (leader) {
            ld_pending = false;
            tc_fence_after();
            // MMA 1 on the edge-state tile
            const uint64_t a0 = kmajor_desc(smem_u32(sE), 128, kS, 0), b0 = kmajor_desc(smem_u32(sW), kH, kS, 0);
            const uint32_t id = idesc_bf16(128, kH);
#pragma unroll
            for (int k0 = 0; k0 < kH; k0 += 16)
                mma_bf16(tAcc, desc_step(a0, kmajor_off(128, kS, k0)), desc_step(b0, kmajor_off(kH, kS, k0)), id,
                         k0 > 0 ? 1u : 0u);
            mma_commit(bar_mma + gi);
            if (t + step < A.n_tiles) {   // the group's next edge rows into L2 while this tile runs
                const int4 hn = tile_hdr(t + step);
                if (hn.w > 0) prefetch_l2(A.e_in + (int64_t)hn.z * kH, (uint32_t)hn.w * kH * 2);
            }
        }
        const int32_t* hdr = reinterpret_cast<const int32_t*>(rec);
        const int32_t* sRp = reinterpret_cast<const int32_t*>(rec + 16);
        const int16_t* sSeg = reinterpret_cast<const int16_t*>(rec + 544);
        const int32_t* sCol = reinterpret_cast<const int32_t*>(rec + 800);
        const float* sWd = reinterpret_cast<const float*>(rec + 1312);
        const int32_t r0 = hdr[0], r1 = hdr[1], e0 = hdr[2], ne = hdr[3];
        const bool valid = row < ne;
        float w = 0.f;
        uint4 pq[2][16];   // this edge's P (receiver) and Q (sender) rows, BF16
        if (valid) {
            const int64_t rcv = r0 + sSeg[row], snd = sCol[row];
            w = sWd[row];
            const uint4* pp = reinterpret_cast<const uint4*>(A.pq + rcv * kH);
            const uint4* qp = reinterpret_cast<const uint4*>(A.q + snd * kH);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                pq[0][i] = __ldg(pp + i);
                pq[1][i] = __ldg(qp + i);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) pq[0][i] = pq[1][i] = make_uint4(0u, 0u, 0u, 0u);
        }
        // Linear 0: h_0 = ELU(e W1c^T + P_i + Q_j + b_0)
        w_ok = leader ? mbar_wait(bar_mma + gi, ph_mma) : true;
        ok = group_and(w_ok, gi);
        if (!ok) break;
        ph_mma ^= 1;
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < kH; h += 64) {   // two halves, one TMEM wait each
            float v[64];
            ld_acc_n<64>(tAcc + lane_base + h, sPar + h, v);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint4 up = pq[0][h / 8 + i], uq = pq[1][h / 8 + i];
                const uint32_t pw[4] = {up.x, up.y, up.z, up.w}, qw[4] = {uq.x, uq.y, uq.z, uq.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float p0, p1, q0, q1;
                    unpack_bf16x2(pw[j], p0, p1);
                    unpack_bf16x2(qw[j], q0, q1);
                    float2* v2 = reinterpret_cast<float2*>(v + 8 * i + 2 * j);
                    *v2 = __fadd2_rn(*v2, __fadd2_rn(make_float2(p0, p1), make_float2(q0, q1)));
                }
            }
#pragma unroll
            for (int c = 0; c < 64; c += 32) elu_to_tmem(tA + lane_base + (uint32_t)((h + c) / 2), v + c);
        }
        hand_off(tAcc, tA, sW + kWT, gi, leader, bar_mma);
        // hidden Linears 1 .. L-2
        for (int k = 1; k < n_lin - 1 && ok; ++k) {
            w_ok = leader ? mbar_wait(bar_mma + gi, ph_mma) : true;
            ok = group_and(w_ok, gi);
            if (!ok) break;
            ph_mma ^= 1;
            tc_fence_after();
            {
                float v[kH];
                ld_acc_n<kH>(tAcc + lane_base, sPar + k * kH, v);
#pragma unroll
                for (int c = 0; c < kH; c += 32) elu_to_tmem(tA + lane_base + (uint32_t)(c / 2), v + c);
            }
            hand_off(tAcc, tA, sW + (k + 1) * kWT, gi, leader, bar_mma);
        }
        if (!ok) break;
        // the last Linear: LayerNorm + residual (Eq. 5a); mean, then the variance about it
        w_ok = leader ? mbar_wait(bar_mma + gi, ph_mma) : true;
        ok = group_and(w_ok, gi);
        if (!ok) break;
        ph_mma ^= 1;
        tc_fence_after();
        // mean, then the variance about it (FP32, this thread's row, four independent
        // chains); e' = e + LN(z) stays in registers and, as BF16, goes into the e tile
        const float* bk = sPar + (n_lin - 1) * kH;
        const float* gam = sPar + n_lin * kH;
        const float* bet = sPar + (n_lin + 1) * kH;
        float ev[kH];
        float mean, rstd;
        {
            float sp[4];
            ld_acc_n<kH>(tAcc + lane_base, bk, ev);
#pragma unroll
            for (int c = 0; c < kH; c += 32) sp[c / 32] = sum32(ev + c);
            mean = ((sp[0] + sp[1]) + (sp[2] + sp[3])) * (1.f / kH);
#pragma unroll
            for (int c = 0; c < kH; c += 32) sp[c / 32] = sqdev32(ev + c, mean);
            rstd = rsqrtf(((sp[0] + sp[1]) + (sp[2] + sp[3])) * (1.f / kH) + A.eps);
        }
#pragma unroll
        for (int c = 0; c < kH; c += 8) {
            float er[8];
            ld_tile8(sE, row, c, 128, kS, er);   // the residual e
#pragma unroll
            for (int i = 0; i < 8; i += 4) {
                const float4 gm = *reinterpret_cast<const float4*>(gam + c + i);
                const float4 bt = *reinterpret_cast<const float4*>(bet + c + i);
                const float2 xa = __fmul2_rn(__fadd2_rn(make_float2(ev[c + i], ev[c + i + 1]), make_float2(-mean, -mean)),
                                             make_float2(rstd, rstd));
                const float2 xb = __fmul2_rn(__fadd2_rn(make_float2(ev[c + i + 2], ev[c + i + 3]),
                                                        make_float2(-mean, -mean)),
                                             make_float2(rstd, rstd));
                const float2 ya = __fadd2_rn(__ffma2_rn(xa, make_float2(gm.x, gm.y), make_float2(bt.x, bt.y)),
                                             make_float2(er[i], er[i + 1]));
                const float2 yb = __fadd2_rn(__ffma2_rn(xb, make_float2(gm.z, gm.w), make_float2(bt.z, bt.w)),
                                             make_float2(er[i + 2], er[i + 3]));
                ev[c + i] = ya.x;   // rows past the tile's edges are never read back
                ev[c + i + 1] = ya.y;
                ev[c + i + 2] = yb.x;
                ev[c + i + 3] = yb.y;
            }
            st_tile8(sE, row, c, 128, kS, ev + c);
        }
        tc_fence_before();
        group_sync(gi);
        if (A.e_out) {
            constexpr int CPR = kH / 8;   // 16-byte chunks per row
            for (int i = tid & (kGT - 1); i < ne * CPR; i += kGT) {
                const int rr = i / CPR, jj = i - rr * CPR;
                *reinterpret_cast<uint4*>(A.e_out + ((int64_t)e0 + rr) * kH + 8 * jj) =
                    *reinterpret_cast<const uint4*>(sE + tile_off(rr, 8 * jj, 128, kS));
            }
        }
        group_sync(gi);
        // 1/d-weighted segmented sum over each receiver's edges (Eq. 5b), FP32, edge order;
        // two passes of 64 columns staged in the e tile
        const int nr = r1 - r0;
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) {
                const int c = 64 * pass + 4 * cc;
                sS4[row * NC + stage_chunk<NC>(cc, row)] =
                    make_float4(w * ev[c], w * ev[c + 1], w * ev[c + 2], w * ev[c + 3]);
            }
            group_sync(gi);
            for (int it = tid & (kGT - 1); it < nr * NC; it += kGT) {
                const int rr = it / NC, cc = it % NC;
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int32_t e = sRp[rr]; e < sRp[rr + 1]; ++e) {
                    const float4 u = sS4[e * NC + stage_chunk<NC>(cc, e)];
                    acc.x += u.x;
                    acc.y += u.y;
                    acc.z += u.z;
                    acc.w += u.w;
                }
                *reinterpret_cast<float4*>(A.a + (int64_t)(r0 + rr) * kH + 64 * pass + 4 * cc) = acc;
            }
            group_sync(gi);
        }
        // the e tile and the record are free: the group's next tile
        fence_proxy_async();
        tc_fence_before();
        group_sync(gi);
        if (leader && t + step < A.n_tiles) issue_ld(t + step, tile_hdr(t + step).z);
    }
    if (leader && ld_pending) mbar_wait(bar_ld + gi, ph_ld);   // after a timeout: bounded
    __syncwarp();   // reconverged before the aligned block barrier
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, 512);
}

// ------------------------------------------------------------------ recomputation for the layered adjoint
//
// The backward's recomputation of the edge MLP over tiles [t0, t1) in the same
// two-group, tensor-memory form: each hidden activation h_k goes to TMEM as the
// next Linear's operand and, staged as BF16 in the group's edge-state tile (free
// once the first Linear has read it), to scratch by a TMA store (block k, row
// k * hs_rows + (t - t0) * 128 + i; rows past the tile's edges zero). The
// LayerNorm is replaced by its adjoint: g = de' + da_i / d_ij (the adjoint of
// Eq. 5b after the halo adjoint), dz = rstd (g gamma - mean(g gamma) - xhat
// mean(g gamma xhat)), stored the same way (row (t - t0) * 128 + i), and the
// column sums of g xhat and dz (the gamma and last-bias gradients) accumulate
// per warp over its rows by recursive halving across lanes; at the end the
// eight warps' sums are added in warp order into the CTA's partials
// [dgamma | - | db_{L-1}]. The beta gradient (the column sums of g) is left to
// the kernel of the first Linear, which forms g again.

struct TmSaveArgs {
    const uint8_t* tile_meta;
    int64_t t0, t1;
    const __nv_bfloat16* pq;
    const __nv_bfloat16* q;
    const __nv_bfloat16* e_in;
    const float* da;               // aggregate gradient after the halo adjoint [n_rows x H]
    const __nv_bfloat16* de_out;   // upstream gradient of e' (NULL: zero)
    float* part;                   // per-CTA partials, 3H floats at blockIdx.x * pstride
    int64_t pstride;
    int64_t hs_rows;               // rows of one hidden block of the scratch
    MlpDev mlp;
    float eps;
};


__global__ void __launch_bounds__(kNT, 1) k_edge_save_tm(const __grid_constant__ CUtensorMap tmap_e,
                                                         const __grid_constant__ CUtensorMap tmap_hs,
                                                         const __grid_constant__ CUtensorMap tmap_dz, TmSaveArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const TmSmem L = tm_smem(n_lin);
    uint8_t* sW = sm + L.w;
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    uint64_t* bar_ld = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint64_t* bar_mma = bar_ld + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = warp >> 2, q = warp & 3, row = 32 * q + lane;
    const bool leader = (tid & (kGT - 1)) == 0;
    uint8_t* sE = sm + L.e + gi * kTile;
    uint8_t* rec = sm + L.rec + gi * GNN_TILE_META_BYTES;

    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(bar_ld + i, 1);
        fence_mbar_init();
    }
    load_weight(sW, A.mlp.W[0], 3 * kH, 2 * kH, kH, kH, tid, kNT);
    for (int k = 1; k < n_lin; ++k) load_weight(sW + k * kWT, A.mlp.W[k], kH, 0, kH, kH, tid, kNT);
    for (int i = tid; i < n_lin * kH; i += kNT) sPar[i] = A.mlp.b[i / kH][i % kH];
    for (int i = tid; i < kH; i += kNT) sPar[n_lin * kH + i] = A.mlp.gamma[i];
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t tAcc = *tslot + (uint32_t)(gi * 256), tA = tAcc + 128;

    const int64_t step = 2 * (int64_t)gridDim.x;
    const int64_t t_first = A.t0 + (int64_t)blockIdx.x + gi * (int64_t)gridDim.x;
    auto tile_hdr = [&](int64_t t) { return ld_nc_v4s32(A.tile_meta + t * GNN_TILE_META_BYTES); };
    bool ld_pending = false;
    auto issue_ld = [&](int64_t t, int32_t e0) {
        mbar_arrive_expect_tx(bar_ld + gi, kTile + GNN_TILE_META_BYTES);
        bulk_load(rec, A.tile_meta + t * GNN_TILE_META_BYTES, GNN_TILE_META_BYTES, bar_ld + gi);
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) tma_load_2d(sE + kb * 128 * kS, &tmap_e, kb * 64, e0, bar_ld + gi);
        ld_pending = true;
    };
    if (leader && t_first < A.t1) issue_ld(t_first, tile_hdr(t_first).z);
    uint32_t ph_ld = 0, ph_mma = 0;
    bool ok = true;
    // column sums over the warp's rows: lane l holds column 16 j + (l >> 1) of each 16-column block j
    float accG[8], accZ[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) accG[j] = accZ[j] = 0.f;

    for (int64_t t = t_first; t < A.t1 && ok; t += step) {
        bool w_ok = leader ? mbar_wait(bar_ld + gi, ph_ld) : true;
        ok = group_and(w_ok, gi);
        if (!ok) break;
        ph_ld ^= 1;
        if (leader) {
            ld_pending = false;
            tc_fence_after();
            const uint64_t a0 = kmajor_desc(smem_u32(sE), 128, kS, 0), b0 = kmajor_desc(smem_u32(sW), kH, kS, 0);
            const uint32_t id = idesc_bf16(128, kH);
#pragma unroll
            for (int k0 = 0; k0 < kH; k0 += 16)
                mma_bf16(tAcc, desc_step(a0, kmajor_off(128, kS, k0)), desc_step(b0, kmajor_off(kH, kS, k0)), id,
                         k0 > 0 ? 1u : 0u);
            mma_commit(bar_mma + gi);
            if (t + step < A.t1) {   // the group's next edge rows, their de' rows and their receivers' da rows into L2
                const int4 hn = tile_hdr(t + step);
                if (hn.w > 0) prefetch_l2(A.e_in + (int64_t)hn.z * kH, (uint32_t)hn.w * kH * 2);
                if (hn.y > hn.x) prefetch_l2(A.da + (int64_t)hn.x * kH, (uint32_t)(hn.y - hn.x) * kH * 4);
            }
        }
        const int32_t* hdr = reinterpret_cast<const int32_t*>(rec);
        const int16_t* sSeg = reinterpret_cast<const int16_t*>(rec + 544);
        const int32_t* sCol = reinterpret_cast<const int32_t*>(rec + 800);
        const float* sWd = reinterpret_cast<const float*>(rec + 1312);
        const int32_t r0 = hdr[0], e0 = hdr[2], ne = hdr[3];
        const bool valid = row < ne;
        const int64_t rcv = valid ? r0 + sSeg[row] : 0;
        const float w = valid ? sWd[row] : 0.f;
        const int32_t y = (int32_t)((t - A.t0) * 128);
        uint4 pq[2][16];
        if (valid) {
            const uint4* pp = reinterpret_cast<const uint4*>(A.pq + rcv * kH);
            const uint4* qp = reinterpret_cast<const uint4*>(A.q + (int64_t)sCol[row] * kH);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                pq[0][i] = __ldg(pp + i);
                pq[1][i] = __ldg(qp + i);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) pq[0][i] = pq[1][i] = make_uint4(0u, 0u, 0u, 0u);
        }
        // Linear 0
        w_ok = leader ? mbar_wait(bar_mma + gi, ph_mma) : true;
        ok = group_and(w_ok, gi);
        if (!ok) break;
        ph_mma ^= 1;
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < kH; h += 64) {   // two halves, one TMEM wait each
            float v[64];
            ld_acc_n<64>(tAcc + lane_base + h, sPar + h, v);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint4 up = pq[0][h / 8 + i], uq = pq[1][h / 8 + i];
                const uint32_t pw[4] = {up.x, up.y, up.z, up.w}, qw[4] = {uq.x, uq.y, uq.z, uq.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float p0, p1, q0, q1;
                    unpack_bf16x2(pw[j], p0, p1);
                    unpack_bf16x2(qw[j], q0, q1);
                    float2* v2 = reinterpret_cast<float2*>(v + 8 * i + 2 * j);
                    *v2 = __fadd2_rn(*v2, __fadd2_rn(make_float2(p0, p1), make_float2(q0, q1)));
                }
            }
#pragma unroll
            for (int c = 0; c < 64; c += 32)
                elu_to_tmem_and_tile(tA + lane_base + (uint32_t)((h + c) / 2), v + c, sE, row, h + c, valid);
        }
        save_hand_off(tAcc, tA, sW + kWT, gi, leader, bar_mma, &tmap_hs, sE, y);
        // hidden Linears 1 .. L-2
        for (int k = 1; k < n_lin - 1 && ok; ++k) {
            if (leader) bulk_wait_read_all();   // h_{k-1} has left the staging tile
            w_ok = leader ? mbar_wait(bar_mma + gi, ph_mma) : true;
            ok = group_and(w_ok, gi);
            if (!ok) break;
            ph_mma ^= 1;
            tc_fence_after();
            {
                float v[kH];
                ld_acc_n<kH>(tAcc + lane_base, sPar + k * kH, v);
#pragma unroll
                for (int c = 0; c < kH; c += 32)
                    elu_to_tmem_and_tile(tA + lane_base + (uint32_t)(c / 2), v + c, sE, row, c, valid);
            }
            save_hand_off(tAcc, tA, sW + (k + 1) * kWT, gi, leader, bar_mma, &tmap_hs,
                          sE, (int32_t)(k * A.hs_rows) + y);
        }
        if (!ok) break;
        // the gradient of e': g = de' + w da_i, its first half requested before the last
        // Linear completes; g is kept in TMEM columns [128, 256) of the group (the activation
        // operand is not read again in this tile)
        const uint32_t tG = tAcc + 128;
        uint4 ga[16], gd[8];
        auto load_g = [&](int h) {   // columns [64 h, 64 h + 64) of da (FP32) and de' (BF16)
#pragma unroll
            for (int i = 0; i < 16; ++i)
                ga[i] = valid ? __ldg(reinterpret_cast<const uint4*>(A.da + rcv * kH + 64 * h) + i)
                              : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                gd[i] = (valid && A.de_out)
                            ? __ldg(reinterpret_cast<const uint4*>(A.de_out + ((int64_t)e0 + row) * kH + 64 * h) + i)
                            : make_uint4(0u, 0u, 0u, 0u);
        };
        auto store_g = [&](int h) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {   // 16 columns at a time
                float g[16];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint4 a = ga[4 * b + i];
                    g[4 * i] = __uint_as_float(a.x);
                    g[4 * i + 1] = __uint_as_float(a.y);
                    g[4 * i + 2] = __uint_as_float(a.z);
                    g[4 * i + 3] = __uint_as_float(a.w);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const uint4 d = gd[2 * b + i];
                    const uint32_t dw[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float d0, d1;
                        unpack_bf16x2(dw[j], d0, d1);
                        float2* g2 = reinterpret_cast<float2*>(g + 8 * i + 2 * j);
                        *g2 = __ffma2_rn(*g2, make_float2(w, w), make_float2(d0, d1));
                    }
                }
                tmem_st16(tG + lane_base + 64 * h + 16 * b, g);
            }
        };
        load_g(0);
        if (leader) bulk_wait_read_all();
        w_ok = leader ? mbar_wait(bar_mma + gi, ph_mma) : true;
        ok = group_and(w_ok, gi);
        if (!ok) break;
        ph_mma ^= 1;
        tc_fence_after();
        store_g(0);
        load_g(1);
        store_g(1);
        tmem_st_wait();
        {
            // LayerNorm statistics and the adjoint sums of d = g gamma over the row
            const float* bl = sPar + (n_lin - 1) * kH;
            const float* gam = sPar + n_lin * kH;
            float sv[4], sq[4], sd[4], sdv[4];
#pragma unroll
            for (int c = 0; c < kH; c += 32) {
                float z[32], g[32];
                ld_acc32(tAcc + lane_base + c, bl + c, z);
                tmem_ld16(tG + lane_base + c, g);
                tmem_ld16(tG + lane_base + c + 16, g + 16);
                tmem_ld_wait();
                float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll
                for (int i = 0; i < 32; i += 4) {
                    const float4 gm = *reinterpret_cast<const float4*>(gam + c + i);
                    const float2 za = make_float2(z[i], z[i + 1]), zb = make_float2(z[i + 2], z[i + 3]);
                    const float2 da_ = __fmul2_rn(make_float2(g[i], g[i + 1]), make_float2(gm.x, gm.y));
                    const float2 db_ = __fmul2_rn(make_float2(g[i + 2], g[i + 3]), make_float2(gm.z, gm.w));
                    a0 = __fadd2_rn(a0, __fadd2_rn(za, zb));
                    a1 = __ffma2_rn(za, za, __ffma2_rn(zb, zb, a1));
                    a2 = __fadd2_rn(a2, __fadd2_rn(da_, db_));
                    a3 = __ffma2_rn(da_, za, __ffma2_rn(db_, zb, a3));
                }
                sv[c / 32] = a0.x + a0.y;
                sq[c / 32] = a1.x + a1.y;
                sd[c / 32] = a2.x + a2.y;
                sdv[c / 32] = a3.x + a3.y;
            }
            const float tv = (sv[0] + sv[1]) + (sv[2] + sv[3]), tq = (sq[0] + sq[1]) + (sq[2] + sq[3]);
            const float td = (sd[0] + sd[1]) + (sd[2] + sd[3]), tdv = (sdv[0] + sdv[1]) + (sdv[2] + sdv[3]);
            const float mean = tv * (1.f / kH);
            const float rstd = rsqrtf(fmaxf(tq * (1.f / kH) - mean * mean, 0.f) + A.eps);
            const float s1 = td * (1.f / kH);
            const float s2 = rstd * (tdv - mean * td) * (1.f / kH);
            // xhat = (z + b - mean) rstd, dz = (g gamma) rstd + (xhat (-rstd s2) - rstd s1), in
            // pairs; a row past the tile's edges takes rstd = 0, so its xhat and dz are 0 (its g is 0)
            const float r = valid ? rstd : 0.f;
            const float2 r2 = make_float2(r, r), nm2 = make_float2(-mean, -mean);
            const float2 ks2 = make_float2(-r * s2, -r * s2), ks1 = make_float2(-r * s1, -r * s1);
#pragma unroll
            for (int c = 0; c < kH; c += 16) {
                float z[16], g[16], tg[16], dz[16];
                tmem_ld16(tAcc + lane_base + c, z);
                tmem_ld16(tG + lane_base + c, g);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const float2 b2 = *reinterpret_cast<const float2*>(bl + c + i);
                    const float2 gm2 = *reinterpret_cast<const float2*>(gam + c + i);
                    const float2 g2 = make_float2(g[i], g[i + 1]);
                    const float2 xh = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(z[i], z[i + 1]), b2), nm2), r2);
                    const float2 t2 = __fmul2_rn(g2, xh);
                    const float2 d2 = __ffma2_rn(__fmul2_rn(g2, gm2), r2, __ffma2_rn(xh, ks2, ks1));
                    tg[i] = t2.x;
                    tg[i + 1] = t2.y;
                    dz[i] = d2.x;
                    dz[i + 1] = d2.y;
                }
                accG[c / 16] += warp_colsum16(tg, lane);
                accZ[c / 16] += warp_colsum16(dz, lane);
                st_tile8(sE, row, c, 128, kS, dz);
                st_tile8(sE, row, c + 8, 128, kS, dz + 8);
            }
        }
        tc_fence_before();
        fence_proxy_async();
        group_sync(gi);
        if (leader) {   // dz to scratch, then the group's next tile into the staging tile once it is read
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) tma_store_2d(&tmap_dz, kb * 64, y, sE + kb * 128 * kS);
            bulk_commit();
            bulk_wait_read_all();
            if (t + step < A.t1) issue_ld(t + step, tile_hdr(t + step).z);
        }
    }
    if (leader && ld_pending) mbar_wait(bar_ld + gi, ph_ld);   // after a timeout: bounded
    if (leader) bulk_wait_all();                                // the scratch rows are written
    __syncwarp();   // reconverged before the aligned block barrier
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the CTA's partials: the eight warps' column sums in warp order (the staging tiles are free)
    float* red = reinterpret_cast<float*>(sm + L.e);   // [8 warps][2][H]
    if ((lane & 1) == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 16 * j + (lane >> 1);
            red[(warp * 2 + 0) * kH + c] = accG[j];
            red[(warp * 2 + 1) * kH + c] = accZ[j];
        }
    }
    __syncthreads();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    for (int i = tid; i < 2 * kH; i += kNT) {
        const int k = i / kH, c = i % kH;
        float s = 0.f;
        for (int wi = 0; wi < 8; ++wi) s += red[(wi * 2 + k) * kH + c];
        part[k == 0 ? c : 2 * kH + c] = s;   // dgamma, then db_{L-1} (dbeta: the first-Linear kernel)
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, 512);
}

}  // namespace

using namespace host;

bool edge_fwd_tm_supported(const gnn_mp_params& W) { return W.edge.n_lin >= 2 && W.edge.n_lin <= kMaxLin; }

int edge_fwd_tm(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const __nv_bfloat16* e_in,
                const __nv_bfloat16* pq, __nv_bfloat16* e_out, float* a, cudaStream_t s) {
    const int64_t NR = G.n_rows, E = G.n_edges;
    GNN_REQUIRE(edge_fwd_tm_supported(W), GNN_EUNSUPPORTED,
                "gnn_mp_forward: the tensor-memory edge forward needs 2..%d Linear layers", kMaxLin);
    GNN_REQUIRE(G.tile_meta && ((uintptr_t)G.tile_meta & 15) == 0, GNN_EINVAL,
                "gnn_mp_forward: tile_meta must be a 16-byte aligned device array");
    CUtensorMap tm;
    int rc = make_row_tmap(&tm, e_in, E, kH);
    if (rc) return rc;
    TmArgs A{};
    A.tile_meta = static_cast<const uint8_t*>(G.tile_meta);
    A.n_tiles = G.n_edge_tiles;
    A.pq = pq;
    A.q = pq + NR * kH;
    A.e_in = e_in;
    A.e_out = e_out;
    A.a = a;
    A.mlp = mlp_dev(W.edge);
    A.eps = cfg.ln_eps;
    const TmSmem L = tm_smem(W.edge.n_lin);
    int grid;
    // one CTA per SM (all 512 TMEM columns); each CTA's two groups share its tiles
    rc = persistent_grid(k_edge_fwd_tm, kNT, L.total, 512, (G.n_edge_tiles + 1) / 2, &grid);
    if (rc) return rc;
    {
        ProfScope _ps(s, "k_edge_fwd");
        k_edge_fwd_tm<<<grid, kNT, L.total, s>>>(tm, A);
    }
    GNN_LAUNCH_CHECK("k_edge_fwd_tm");
    return GNN_OK;
}

}  // namespace fused
}  // namespace gnn

namespace gnn {
namespace fused {

int edge_save_tm(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const __nv_bfloat16* e_in,
                 const __nv_bfloat16* pq, RecomputeSave& o, cudaStream_t s) {
    const int64_t NR = G.n_rows, E = G.n_edges;
    GNN_REQUIRE(edge_fwd_tm_supported(W), GNN_EUNSUPPORTED,
                "gnn_mp_backward: the tensor-memory edge recomputation needs 2..%d Linear layers", kMaxLin);
    GNN_REQUIRE(G.tile_meta && ((uintptr_t)G.tile_meta & 15) == 0, GNN_EINVAL,
                "gnn_mp_backward: tile_meta must be a 16-byte aligned device array");
    CUtensorMap tm, tmhs, tmdz;
    int rc = make_row_tmap(&tm, e_in, E, kH);
    if (rc) return rc;
    const int64_t hs_rows = o.hs_stride / kH;
    if ((rc = make_row_tmap(&tmhs, o.hs, (int64_t)(W.edge.n_lin - 1) * hs_rows, kH))) return rc;
    if ((rc = make_row_tmap(&tmdz, o.dz, hs_rows, kH))) return rc;
    TmSaveArgs A{};
    A.tile_meta = static_cast<const uint8_t*>(G.tile_meta);
    A.t0 = o.t0;
    A.t1 = o.t1;
    A.pq = pq;
    A.q = pq + NR * kH;
    A.e_in = e_in;
    A.da = o.da;
    A.de_out = o.de_out;
    A.part = o.part;
    A.pstride = o.pstride;
    A.hs_rows = hs_rows;
    A.mlp = mlp_dev(W.edge);
    A.eps = cfg.ln_eps;
    const TmSmem L = tm_smem(W.edge.n_lin);
    if ((rc = persistent_grid(k_edge_save_tm, kNT, L.total, 512, (o.t1 - o.t0 + 1) / 2, &o.grid))) return rc;
    {
        ProfScope _ps(s, "k_edge_fwd_save");
        k_edge_save_tm<<<o.grid, kNT, L.total, s>>>(tm, tmhs, tmdz, A);
    }
    GNN_LAUNCH_CHECK("k_edge_save_tm");
    return GNN_OK;
}

}  // namespace fused
}  // namespace gnn
