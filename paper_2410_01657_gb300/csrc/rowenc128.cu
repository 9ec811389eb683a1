// Fused BF16 encoder row MLP at H = 128 (the node and edge encoders of the
// encode-process-decode network, Sec. III): Y = LN(MLP(X)) with X [n x K0],
// K0 <= 16, hidden and output width 128, 2 to 4 Linear layers, ELU between
// them; and its adjoint with per-layer recomputation of the activations.
//
// Forward, k_rowenc_fwd_tm: the tensor-memory form of the H = 128 edge
// forward without its gather and aggregation. Two groups of four warps take
// alternate tiles of 128 rows, one thread owns one row: the thread's input row
// goes as BF16 into the group's [128 x 16] input tile, the first Linear reads
// it from shared memory, every later Linear reads its predecessor's ELU output
// from TMEM (A operand) and W_k from shared memory; the LayerNorm statistics
// are the thread's own (FP32), and Y is staged in shared memory and written as
// whole rows, FP32 or BF16.
//
// Adjoint, over chunks of tiles (at most kChunkTiles, fewer when the caller's
// workspace is smaller; scratch rows (t - t0) * 128 + i, zero past the last row):
//   k_rowenc_save_tm  recompute the MLP, save h_0 .. h_{L-2} (BF16), apply the
//                     LayerNorm adjoint to dY: dz_{L-1}, and the column sums
//                     for dgamma, dbeta, db_{L-1}
//   k_bwd_chain2 / k_bwd_chain  k = L-1 .. 1: dz_{k-1} = (dz_k W_k) ELU'(h_{k-1}),
//                     dW_k, db_{k-1} (the layer adjoint's per-Linear kernels)
//   k_rowenc_w0       dW_0 = dz_0^T X, and dX = dz_0 W_0 when asked (db_0 comes
//                     from the chain's last pass)
// Every gradient is a fixed-order sum: per thread in row order, per CTA in
// warp order, then k_reduce_grads over the CTAs in CTA order.

#include <algorithm>

#include "fused.h"
#include "fused_bwd_common.cuh"
#include "profiler.h"
#include "tm128_common.cuh"

namespace gnn {
namespace fused {

cudaError_t take_device_error_rowenc128(unsigned int* out) { return take_device_error_word(out); }

namespace {

using namespace tc;
using namespace tm128;

constexpr int kKP = 16;                         // padded input width
constexpr int kSX = 32;                         // swizzle span of a [128 x 16] BF16 tile
constexpr uint32_t kXT = 128 * kKP * 2;         // [128 x 16] BF16 tile
constexpr int kMaxLin = 4;                      // W_1 .. W_3 resident in shared memory
constexpr int64_t kChunkTiles = 32768;          // tiles per scratch chunk
constexpr int64_t kPstride = 2 * (int64_t)kH * kH + 2 * kH;   // per-CTA partial floats (k_bwd_chain2)
constexpr int kW0PerSm = 4;                     // k_rowenc_w0 CTAs per SM

struct EncArgs {
    const float* X;        // [n_rows x K0]
    int64_t n_rows;
    int K0;
    void* Y;               // forward: [n_rows x 128], FP32 or BF16
    int y_bf16;
    const void* dY;        // recomputation: gradient of Y [n_rows x 128], FP32 or BF16
    int dy_bf16;
    int64_t t0, t1;        // recomputation: tiles [t0, t1)
    int64_t hs_rows;       // recomputation: rows of one hidden block of the scratch
    float* part;           // recomputation: per-CTA partials [dgamma | dbeta | db_{L-1}]
    int64_t pstride;
    MlpDev mlp;
    float eps;
};

struct EncSmem {
    uint32_t w0, w, x, st, par, bar, tm, total;
};

__host__ __device__ inline EncSmem enc_smem(int n_lin) {
    EncSmem s;
    s.w0 = 0;                                                   // W_0 [128 x 16]
    s.w = align_up(kXT, 1024);                                  // W_1 .. W_{L-1}
    s.x = align_up(s.w + (uint32_t)(n_lin - 1) * kWT, 1024);    // x[2]: input tiles, one per group
    s.st = align_up(s.x + 2 * kXT, 1024);                       // st[2]: staging tiles, one per group
    s.par = s.st + 2 * kTile;                                   // b_0 .. b_{L-1}, gamma, beta
    s.bar = align_up(s.par + (uint32_t)(n_lin + 2) * kH * 4, 8);   // mma[2]
    s.tm = s.bar + 2 * 8;
    s.total = s.tm + 16 + 1024;
    return s;
}

// TMEM, barriers, the weights as BF16 K-major tiles (W_0 zero-padded to 16
// inputs) and the FP32 biases / LayerNorm parameters; ends with the block in sync.
__device__ __forceinline__ void enc_prologue(const EncArgs& A, uint8_t* sm, const EncSmem& L, int tid, int warp) {
    const int n_lin = A.mlp.n_lin, K0 = A.K0;
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + L.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L.tm);
    if (warp == 0) {
        tmem_alloc(tslot, 512);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(bar_mma, 1);
        mbar_init(bar_mma + 1, 1);
        fence_mbar_init();
    }
    const float* W0 = A.mlp.W[0];
    for (int i = tid; i < kH * (kKP / 8); i += kNT) {
        const int n = i / (kKP / 8), k = (i % (kKP / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (k + j < K0) ? __ldg(W0 + (int64_t)n * K0 + k + j) : 0.f;
        st_tile8(sm + L.w0, n, k, kH, kSX, v);
    }
    for (int k = 1; k < n_lin; ++k) load_weight(sm + L.w + (k - 1) * kWT, A.mlp.W[k], kH, 0, kH, kH, tid, kNT);
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    for (int i = tid; i < n_lin * kH; i += kNT) sPar[i] = A.mlp.b[i / kH][i % kH];
    for (int i = tid; i < kH; i += kNT) {
        sPar[n_lin * kH + i] = A.mlp.gamma[i];
        sPar[(n_lin + 1) * kH + i] = A.mlp.beta[i];
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// This thread's input row (K0 <= 16 FP32, zero past K0 and past the last row)
// as BF16 into the group's input tile, then the first Linear once the group's
// rows are in: acc = x W_0^T.
__device__ __forceinline__ void enc_first_linear(const EncArgs& A, uint8_t* sX, const uint8_t* sW0, int64_t r,
                                                 bool valid, int row, int gi, bool leader, uint32_t tAcc,
                                                 uint64_t* bar_mma) {
    float v[kKP];
    const float* xr = A.X + r * A.K0;
#pragma unroll
    for (int i = 0; i < kKP; ++i) v[i] = (valid && i < A.K0) ? __ldg(xr + i) : 0.f;
    st_row_tile<kKP>(sX, row, 0, kSX, v);
    fence_proxy_async();
    tc_fence_before();
    group_sync(gi);
    if (leader) {
        tc_fence_after();
        issue_mma(tAcc, sX, sW0, kH, kKP);
        mma_commit(bar_mma + gi);
    }
}

// The group's leader waits for its MMA chain (bounded); the group agrees.
__device__ __forceinline__ bool enc_wait_mma(uint64_t* bar_mma, int gi, bool leader, uint32_t& ph) {
    const bool w_ok = leader ? mbar_wait(bar_mma + gi, ph) : true;
    const bool ok = group_and(w_ok, gi);
    ph ^= 1;
    tc_fence_after();
    return ok;
}

// ------------------------------------------------------------------ forward

__global__ void __launch_bounds__(kNT, 1) k_rowenc_fwd_tm(EncArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const EncSmem L = enc_smem(n_lin);
    const float* sPar = reinterpret_cast<const float*>(sm + L.par);
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + L.bar);
    const uint32_t* tslot = reinterpret_cast<const uint32_t*>(sm + L.tm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = warp >> 2, q = warp & 3, row = 32 * q + lane;
    const bool leader = (tid & (kGT - 1)) == 0;
    uint8_t* sX = sm + L.x + gi * kXT;
    uint8_t* sSt = sm + L.st + gi * kTile;
    enc_prologue(A, sm, L, tid, warp);
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t tAcc = *tslot + (uint32_t)(gi * 256), tA = tAcc + 128;
    const float* gam = sPar + n_lin * kH;
    const float* bet = sPar + (n_lin + 1) * kH;
    const int64_t n_tiles = (A.n_rows + 127) / 128;
    const int64_t step = 2 * (int64_t)gridDim.x;
    uint32_t ph = 0;
    bool ok = true;

    for (int64_t t = (int64_t)blockIdx.x + gi * (int64_t)gridDim.x; t < n_tiles && ok; t += step) {
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        const int nv = A.n_rows - t * 128 < 128 ? (int)(A.n_rows - t * 128) : 128;
        enc_first_linear(A, sX, sm + L.w0, r, valid, row, gi, leader, tAcc, bar_mma);
        // h_k = ELU(acc + b_k) into TMEM, then acc = h_k W_{k+1}^T
        for (int k = 0; k < n_lin - 1; ++k) {
            if (!(ok = enc_wait_mma(bar_mma, gi, leader, ph))) break;
            {
                float v[kH];
                ld_acc_n<kH>(tAcc + lane_base, sPar + k * kH, v);
#pragma unroll
                for (int c = 0; c < kH; c += 32) elu_to_tmem(tA + lane_base + (uint32_t)(c / 2), v + c);
            }
            hand_off(tAcc, tA, sm + L.w + k * kWT, gi, leader, bar_mma);
        }
        if (!ok || !(ok = enc_wait_mma(bar_mma, gi, leader, ph))) break;
        // Y = LN(acc + b_{L-1}): mean, then the variance about it (FP32, four chains)
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
#pragma unroll
        for (int c = 0; c < kH; c += 4) {
            const float4 gm = *reinterpret_cast<const float4*>(gam + c);
            const float4 bt = *reinterpret_cast<const float4*>(bet + c);
            const float2 nm = make_float2(-mean, -mean), rs = make_float2(rstd, rstd);
            const float2 xa = __fmul2_rn(__fadd2_rn(make_float2(ev[c], ev[c + 1]), nm), rs);
            const float2 xb = __fmul2_rn(__fadd2_rn(make_float2(ev[c + 2], ev[c + 3]), nm), rs);
            const float2 ya = __ffma2_rn(xa, make_float2(gm.x, gm.y), make_float2(bt.x, bt.y));
            const float2 yb = __ffma2_rn(xb, make_float2(gm.z, gm.w), make_float2(bt.z, bt.w));
            ev[c] = ya.x;
            ev[c + 1] = ya.y;
            ev[c + 2] = yb.x;
            ev[c + 3] = yb.y;
        }
        // the tile's rows through the staging tile, written as whole rows
        if (A.y_bf16) {
#pragma unroll
            for (int c = 0; c < kH; c += 8) st_tile8(sSt, row, c, 128, kS, ev + c);
            group_sync(gi);
            __nv_bfloat16* Y = static_cast<__nv_bfloat16*>(A.Y) + t * 128 * kH;
            constexpr int CPR = kH / 8;
            for (int i = tid & (kGT - 1); i < nv * CPR; i += kGT) {
                const int rr = i / CPR, jj = i - rr * CPR;
                *reinterpret_cast<uint4*>(Y + (int64_t)rr * kH + 8 * jj) =
                    *reinterpret_cast<const uint4*>(sSt + tile_off(rr, 8 * jj, 128, kS));
            }
            group_sync(gi);
        } else {
            constexpr int NC = 16;   // 16-byte chunks of a staged half row (64 FP32 columns)
            float4* sS4 = reinterpret_cast<float4*>(sSt);
            float* Y = static_cast<float*>(A.Y) + t * 128 * kH;
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    const int c = 64 * pass + 4 * cc;
                    sS4[row * NC + stage_chunk<NC>(cc, row)] = make_float4(ev[c], ev[c + 1], ev[c + 2], ev[c + 3]);
                }
                group_sync(gi);
                for (int it = tid & (kGT - 1); it < nv * NC; it += kGT) {
                    const int rr = it / NC, cc = it % NC;
                    *reinterpret_cast<float4*>(Y + (int64_t)rr * kH + 64 * pass + 4 * cc) =
                        sS4[rr * NC + stage_chunk<NC>(cc, rr)];
                }
                group_sync(gi);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, 512);
}

// ------------------------------------------------------------------ recomputation for the adjoint
//
// The forward over tiles [t0, t1) with each h_k, staged as BF16 in the group's
// staging tile, also going to block k of the scratch by a TMA store (row
// k * hs_rows + (t - t0) * 128 + i; zero past the last row). The LayerNorm is
// replaced by its adjoint: with g = dY and d = g gamma, dz = rstd (d - mean(d) -
// xhat mean(d xhat)), stored the same way; the column sums of g xhat, g and dz
// (the gamma, beta and last-bias gradients) accumulate per warp over its rows
// by recursive halving across lanes, and at the end the eight warps' sums are
// added in warp order into the CTA's partials.

__global__ void __launch_bounds__(kNT, 1) k_rowenc_save_tm(const __grid_constant__ CUtensorMap tmap_hs,
                                                           const __grid_constant__ CUtensorMap tmap_dz, EncArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin;
    const EncSmem L = enc_smem(n_lin);
    const float* sPar = reinterpret_cast<const float*>(sm + L.par);
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + L.bar);
    const uint32_t* tslot = reinterpret_cast<const uint32_t*>(sm + L.tm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = warp >> 2, q = warp & 3, row = 32 * q + lane;
    const bool leader = (tid & (kGT - 1)) == 0;
    uint8_t* sX = sm + L.x + gi * kXT;
    uint8_t* sSt = sm + L.st + gi * kTile;
    enc_prologue(A, sm, L, tid, warp);
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t tAcc = *tslot + (uint32_t)(gi * 256), tA = tAcc + 128;
    const uint32_t tG = tAcc + 128;   // g, once the last Linear has read the activation operand
    const float* bl = sPar + (n_lin - 1) * kH;
    const float* gam = sPar + n_lin * kH;
    const int64_t step = 2 * (int64_t)gridDim.x;
    uint32_t ph = 0;
    bool ok = true;
    float accG[8], accB[8], accZ[8];   // lane l: column 16 j + (l >> 1) of 16-column block j
#pragma unroll
    for (int j = 0; j < 8; ++j) accG[j] = accB[j] = accZ[j] = 0.f;

    for (int64_t t = A.t0 + (int64_t)blockIdx.x + gi * (int64_t)gridDim.x; t < A.t1 && ok; t += step) {
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        const int32_t y = (int32_t)((t - A.t0) * 128);
        enc_first_linear(A, sX, sm + L.w0, r, valid, row, gi, leader, tAcc, bar_mma);
        for (int k = 0; k < n_lin - 1; ++k) {
            if (leader) bulk_wait_read_all();   // the staging tile's last store has read it
            if (!(ok = enc_wait_mma(bar_mma, gi, leader, ph))) break;
            {
                float v[kH];
                ld_acc_n<kH>(tAcc + lane_base, sPar + k * kH, v);
#pragma unroll
                for (int c = 0; c < kH; c += 32)
                    elu_to_tmem_and_tile(tA + lane_base + (uint32_t)(c / 2), v + c, sSt, row, c, valid);
            }
            save_hand_off(tAcc, tA, sm + L.w + k * kWT, gi, leader, bar_mma, &tmap_hs, sSt,
                          (int32_t)(k * A.hs_rows) + y);
        }
        if (!ok) break;
        // g = dY, requested before the last Linear completes, kept in TMEM [tG, tG + 128)
        uint4 gv[16];
        auto load_g = [&](int h) {   // columns [64 h, 64 h + 64)
            if (A.dy_bf16) {
                const uint4* p = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(A.dY) + r * kH + 64 * h);
#pragma unroll
                for (int i = 0; i < 8; ++i) gv[i] = valid ? __ldg(p + i) : make_uint4(0u, 0u, 0u, 0u);
            } else {
                const uint4* p = reinterpret_cast<const uint4*>(static_cast<const float*>(A.dY) + r * kH + 64 * h);
#pragma unroll
                for (int i = 0; i < 16; ++i) gv[i] = valid ? __ldg(p + i) : make_uint4(0u, 0u, 0u, 0u);
            }
        };
        auto store_g = [&](int h) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {   // 16 columns at a time
                float g[16];
                if (A.dy_bf16) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const uint4 d = gv[2 * b + i];
                        unpack_bf16x2(d.x, g[8 * i], g[8 * i + 1]);
                        unpack_bf16x2(d.y, g[8 * i + 2], g[8 * i + 3]);
                        unpack_bf16x2(d.z, g[8 * i + 4], g[8 * i + 5]);
                        unpack_bf16x2(d.w, g[8 * i + 6], g[8 * i + 7]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const uint4 a = gv[4 * b + i];
                        g[4 * i] = __uint_as_float(a.x);
                        g[4 * i + 1] = __uint_as_float(a.y);
                        g[4 * i + 2] = __uint_as_float(a.z);
                        g[4 * i + 3] = __uint_as_float(a.w);
                    }
                }
                tmem_st16(tG + lane_base + 64 * h + 16 * b, g);
            }
        };
        load_g(0);
        if (leader) bulk_wait_read_all();   // h_{L-2} has left the staging tile
        if (!(ok = enc_wait_mma(bar_mma, gi, leader, ph))) break;
        store_g(0);
        load_g(1);
        store_g(1);
        tmem_st_wait();
        {
            // LayerNorm statistics and the adjoint sums of d = g gamma over the row
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
#pragma unroll
            for (int c = 0; c < kH; c += 16) {
                float z[16], g[16], tg[16], dz[16];
                tmem_ld16(tAcc + lane_base + c, z);
                tmem_ld16(tG + lane_base + c, g);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float xh = valid ? (z[i] + bl[c + i] - mean) * rstd : 0.f;
                    tg[i] = g[i] * xh;
                    dz[i] = valid ? rstd * (g[i] * gam[c + i] - s1 - xh * s2) : 0.f;
                }
                accG[c / 16] += warp_colsum16(tg, lane);
                accB[c / 16] += warp_colsum16(g, lane);
                accZ[c / 16] += warp_colsum16(dz, lane);
                st_tile8(sSt, row, c, 128, kS, dz);
                st_tile8(sSt, row, c + 8, 128, kS, dz + 8);
            }
        }
        tc_fence_before();
        fence_proxy_async();
        group_sync(gi);
        if (leader) {   // dz to scratch; the staging tile is free again once the store has read it
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) tma_store_2d(&tmap_dz, kb * 64, y, sSt + kb * 128 * kS);
            bulk_commit();
            bulk_wait_read_all();
        }
    }
    if (leader) bulk_wait_all();   // the scratch rows are written
    __syncwarp();   // reconverged before the aligned block barrier
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the CTA's partials: the eight warps' column sums in warp order (the staging tiles are free)
    float* red = reinterpret_cast<float*>(sm + L.st);   // [8 warps][3][H]
    if ((lane & 1) == 0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 16 * j + (lane >> 1);
            red[(warp * 3 + 0) * kH + c] = accG[j];
            red[(warp * 3 + 1) * kH + c] = accB[j];
            red[(warp * 3 + 2) * kH + c] = accZ[j];
        }
    }
    __syncthreads();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    for (int i = tid; i < 3 * kH; i += kNT) {
        const int k = i / kH, c = i % kH;
        float s = 0.f;
        for (int wi = 0; wi < 8; ++wi) s += red[(wi * 3 + k) * kH + c];
        part[i] = s;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, 512);
}

// ------------------------------------------------------------------ k_rowenc_w0

struct W0Args {
    const __nv_bfloat16* dz;   // dz_0 rows of the chunk, tile-padded [(t1 - t0) * 128 x 128]
    const float* X;            // [n_rows x K0]
    const float* W0;           // [128 x K0]
    float* dX;                 // [n_rows x K0], NULL: not wanted
    int64_t n_rows, t0, t1;
    int K0;
    float* part;               // per-CTA: dW_0 [128 x 16]
    int64_t pstride;
};

constexpr int kW0NT = 256;
constexpr int kDzLd = kH + 8;   // BF16 per staged dz row: 272-byte rows, 16-byte reads of 8 rows hit distinct banks
struct W0Smem {
    static constexpr uint32_t dz = 0;                         // [128][kDzLd] BF16
    static constexpr uint32_t x = 128 * kDzLd * 2;            // [128][16] FP32
    static constexpr uint32_t w = x + 128 * kKP * 4;          // [128][16] FP32 (W_0, zero-padded)
    static constexpr uint32_t total = w + kH * kKP * 4;
};

// Thread (c, kh): row c of dW_0 for inputs 8 kh .. 8 kh + 7 over the CTA's rows;
// for dX, thread (row = c, kh) the same inputs of its row.
__global__ void __launch_bounds__(kW0NT) k_rowenc_w0(W0Args A) {
    extern __shared__ __align__(16) uint8_t w0_smem[];
    __nv_bfloat16* sDz = reinterpret_cast<__nv_bfloat16*>(w0_smem + W0Smem::dz);
    float* sX = reinterpret_cast<float*>(w0_smem + W0Smem::x);
    float* sW = reinterpret_cast<float*>(w0_smem + W0Smem::w);
    const int tid = threadIdx.x, c = tid & (kH - 1), kh = tid >> 7, K0 = A.K0;
    if (A.dX)
        for (int i = tid; i < kH * kKP; i += kW0NT) sW[i] = (i % kKP) < K0 ? A.W0[(i / kKP) * K0 + i % kKP] : 0.f;
    float2 acc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int64_t t = A.t0 + blockIdx.x; t < A.t1; t += gridDim.x) {
        __syncthreads();   // the previous tile's reads are done
        const uint4* src = reinterpret_cast<const uint4*>(A.dz + (t - A.t0) * 128 * kH);
        for (int i = tid; i < 128 * (kH / 8); i += kW0NT) {
            const int rr = i / (kH / 8), j = i % (kH / 8);
            *reinterpret_cast<uint4*>(sDz + rr * kDzLd + 8 * j) = __ldg(src + i);
        }
        const int64_t rbase = t * 128;
        for (int i = tid; i < 128 * kKP; i += kW0NT) {
            const int rr = i / kKP, k = i % kKP;
            sX[i] = (k < K0 && rbase + rr < A.n_rows) ? __ldg(A.X + (rbase + rr) * K0 + k) : 0.f;
        }
        __syncthreads();
        const float4* sX4 = reinterpret_cast<const float4*>(sX);
#pragma unroll 4
        for (int rr = 0; rr < 128; ++rr) {
            const float d = __bfloat162float(sDz[rr * kDzLd + c]);
            const float2 d2 = make_float2(d, d);
            const float4 x0 = sX4[rr * 4 + 2 * kh], x1 = sX4[rr * 4 + 2 * kh + 1];
            acc[0] = __ffma2_rn(d2, make_float2(x0.x, x0.y), acc[0]);
            acc[1] = __ffma2_rn(d2, make_float2(x0.z, x0.w), acc[1]);
            acc[2] = __ffma2_rn(d2, make_float2(x1.x, x1.y), acc[2]);
            acc[3] = __ffma2_rn(d2, make_float2(x1.z, x1.w), acc[3]);
        }
        if (A.dX && rbase + c < A.n_rows) {   // thread (row = c, kh)
            float2 o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = make_float2(0.f, 0.f);
            const float4* sW4 = reinterpret_cast<const float4*>(sW);
            for (int c0 = 0; c0 < kH; c0 += 8) {
                float d[8];
                const uint4 u = *reinterpret_cast<const uint4*>(sDz + c * kDzLd + c0);
                unpack_bf16x2(u.x, d[0], d[1]);
                unpack_bf16x2(u.y, d[2], d[3]);
                unpack_bf16x2(u.z, d[4], d[5]);
                unpack_bf16x2(u.w, d[6], d[7]);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float2 d2 = make_float2(d[j], d[j]);
                    const float4 w0 = sW4[(c0 + j) * 4 + 2 * kh], w1 = sW4[(c0 + j) * 4 + 2 * kh + 1];
                    o[0] = __ffma2_rn(d2, make_float2(w0.x, w0.y), o[0]);
                    o[1] = __ffma2_rn(d2, make_float2(w0.z, w0.w), o[1]);
                    o[2] = __ffma2_rn(d2, make_float2(w1.x, w1.y), o[2]);
                    o[3] = __ffma2_rn(d2, make_float2(w1.z, w1.w), o[3]);
                }
            }
            const float ov[8] = {o[0].x, o[0].y, o[1].x, o[1].y, o[2].x, o[2].y, o[3].x, o[3].y};
            float* dst = A.dX + (rbase + c) * K0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (8 * kh + k < K0) dst[8 * kh + k] = ov[k];
        }
    }
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    const float av[8] = {acc[0].x, acc[0].y, acc[1].x, acc[1].y, acc[2].x, acc[2].y, acc[3].x, acc[3].y};
#pragma unroll
    for (int k = 0; k < 8; ++k) part[c * kKP + 8 * kh + k] = av[k];
}

// =================================================================== host side

using namespace host;

struct EncWs {
    float* part;             // kW0PerSm * num_sms CTAs x kPstride floats
    __nv_bfloat16* hs;       // (L-1) x [chunk rows x H]
    int64_t hs_stride;
    __nv_bfloat16* dzs[2];   // [chunk rows x H] each
    size_t bytes;
};

EncWs carve_enc(void* ws, int n_lin, int64_t chunk) {
    EncWs w{};
    size_t off = 0;
    auto take = [&](size_t n) {
        off = (off + 255) & ~(size_t)255;
        void* p = ws ? (char*)ws + off : nullptr;
        off += n;
        return p;
    };
    const int64_t rows = chunk * 128;
    w.part = (float*)take((size_t)kW0PerSm * num_sms() * kPstride * 4);
    w.hs_stride = rows * kH;
    w.hs = (__nv_bfloat16*)take((size_t)(n_lin - 1) * rows * kH * 2);
    w.dzs[0] = (__nv_bfloat16*)take((size_t)rows * kH * 2);
    w.dzs[1] = (__nv_bfloat16*)take((size_t)rows * kH * 2);
    w.bytes = off + 256;
    return w;
}

int64_t enc_chunk(int64_t n_rows) { return std::max<int64_t>(1, std::min<int64_t>(kChunkTiles, (n_rows + 127) / 128)); }

EncArgs enc_args(const gnn_mlp& P, int64_t n_rows, const float* X, float eps) {
    EncArgs A{};
    A.X = X;
    A.n_rows = n_rows;
    A.K0 = P.dims[0];
    A.mlp = mlp_dev(P);
    A.eps = eps;
    return A;
}

}  // namespace

bool rowenc128_shape(const gnn_mlp& P) {
    const int L = P.n_lin;
    if (L < 2 || L > kMaxLin || !P.gamma) return false;
    if (P.dims[0] < 1 || P.dims[0] > kKP) return false;
    for (int l = 1; l <= L; ++l)
        if (P.dims[l] != kH) return false;
    return true;
}

size_t rowenc128_backward_ws(const gnn_mlp& P, int64_t n_rows) {
    return carve_enc(nullptr, P.n_lin, enc_chunk(n_rows)).bytes;
}

int rowenc128_forward(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, float eps,
                      cudaStream_t s) {
    GNN_REQUIRE(rowenc128_shape(P), GNN_EUNSUPPORTED, "gnn_mlp_forward_bf16: not an H=128 encoder of 2..%d Linears",
                kMaxLin);
    if (n_rows == 0) return GNN_OK;
    GNN_REQUIRE(((uintptr_t)Y & 15) == 0, GNN_EINVAL, "gnn_mlp_forward_bf16: Y must be 16-byte aligned at H=128");
    EncArgs A = enc_args(P, n_rows, X, eps);
    A.Y = Y;
    A.y_bf16 = y_bf16;
    const EncSmem L = enc_smem(P.n_lin);
    int grid;
    int rc = persistent_grid(k_rowenc_fwd_tm, kNT, L.total, 512, ((n_rows + 127) / 128 + 1) / 2, &grid);
    if (rc) return rc;
    {
        ProfScope _ps(s, "k_rowmlp_fwd");
        k_rowenc_fwd_tm<<<grid, kNT, L.total, s>>>(A);
    }
    GNN_LAUNCH_CHECK("k_rowenc_fwd_tm");
    return GNN_OK;
}

int rowenc128_backward(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                       const gnn_mlp& dP, float eps, void* ws, size_t ws_bytes, cudaStream_t s) {
    GNN_REQUIRE(rowenc128_shape(P), GNN_EUNSUPPORTED, "gnn_mlp_backward_bf16: not an H=128 encoder of 2..%d Linears",
                kMaxLin);
    if (n_rows == 0) return GNN_OK;
    GNN_REQUIRE(((uintptr_t)dY & 15) == 0, GNN_EINVAL, "gnn_mlp_backward_bf16: dY must be 16-byte aligned at H=128");
    const int Lw = P.n_lin, K0 = P.dims[0];
    const int64_t n_tiles = (n_rows + 127) / 128;
    // the largest chunk of tiles whose scratch fits the workspace given
    int64_t chunk = enc_chunk(n_rows);
    if (ws_bytes < carve_enc(nullptr, Lw, chunk).bytes) {
        const size_t fixed = carve_enc(nullptr, Lw, 0).bytes;
        const size_t per_tile = carve_enc(nullptr, Lw, 2).bytes - carve_enc(nullptr, Lw, 1).bytes;
        chunk = ws_bytes > fixed ? (int64_t)((ws_bytes - fixed) / per_tile) : 0;
        while (chunk > 0 && carve_enc(nullptr, Lw, chunk).bytes > ws_bytes) --chunk;
        GNN_REQUIRE(chunk >= 1, GNN_ENOMEM, "gnn_mlp_backward_bf16: workspace too small (%zu bytes)", ws_bytes);
    }
    EncWs w = carve_enc(ws, Lw, chunk);
    const EncSmem L = enc_smem(Lw);
    int rc;
    for (int64_t t0 = 0; t0 < n_tiles; t0 += chunk) {
        const int64_t t1 = std::min(n_tiles, t0 + chunk);
        const int64_t rows = (t1 - t0) * 128;
        // 1. recomputation: h_0 .. h_{L-2}, dz_{L-1}, LayerNorm and last-bias partials
        CUtensorMap tmhs, tmdz;
        if ((rc = make_row_tmap(&tmhs, w.hs, (int64_t)(Lw - 1) * (w.hs_stride / kH), kH))) return rc;
        if ((rc = make_row_tmap(&tmdz, w.dzs[0], rows, kH))) return rc;
        EncArgs A = enc_args(P, n_rows, X, eps);
        A.dY = dY;
        A.dy_bf16 = dy_bf16;
        A.t0 = t0;
        A.t1 = t1;
        A.hs_rows = w.hs_stride / kH;
        A.part = w.part;
        A.pstride = kPstride;
        int grid;
        if ((rc = persistent_grid(k_rowenc_save_tm, kNT, L.total, 512, (t1 - t0 + 1) / 2, &grid))) return rc;
        {
            ProfScope _ps(s, "k_rowmlp_save");
            k_rowenc_save_tm<<<grid, kNT, L.total, s>>>(tmhs, tmdz, A);
        }
        GNN_LAUNCH_CHECK("k_rowenc_save_tm");
        {
            RedSeg seg[3];
            seg[0] = RedSeg{dP.gamma, kH, 1, kH, 0, 0};
            seg[1] = RedSeg{dP.beta, kH, 1, kH, kH, 0};
            seg[2] = RedSeg{dP.b[Lw - 1], kH, 1, kH, 2 * kH, 0};
            if ((rc = reduce_grads(seg, 3, w.part, kPstride, grid, s))) return rc;
        }
        // 2. Linears L-1 .. 1
        int cur = 0;
        if ((rc = chain_backward_h128(P, dP, w.hs, w.hs_stride, w.dzs, w.part, kPstride, t1 - t0, &cur, s)))
            return rc;
        // 3. the first Linear: dW_0, dX
        W0Args B{};
        B.dz = w.dzs[cur];
        B.X = X;
        B.W0 = P.W[0];
        B.dX = dX;
        B.n_rows = n_rows;
        B.t0 = t0;
        B.t1 = t1;
        B.K0 = K0;
        B.part = w.part;
        B.pstride = kPstride;
        GNN_CUDA_CHECK(cudaFuncSetAttribute(k_rowenc_w0, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)W0Smem::total),
                       "cudaFuncSetAttribute");
        const int g0 = (int)std::min<int64_t>(t1 - t0, (int64_t)kW0PerSm * num_sms());
        {
            ProfScope _ps(s, "k_rowmlp_w0");
            k_rowenc_w0<<<g0, kW0NT, W0Smem::total, s>>>(B);
        }
        GNN_LAUNCH_CHECK("k_rowenc_w0");
        RedSeg seg[1] = {RedSeg{dP.W[0], K0, kH, K0, 0, kKP}};
        if ((rc = reduce_grads(seg, 1, w.part, kPstride, g0, s))) return rc;
    }
    return GNN_OK;
}

}  // namespace fused
}  // namespace gnn
