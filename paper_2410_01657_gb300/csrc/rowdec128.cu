// Fused BF16 decoder row MLP at H = 128 (the node decoder of the
// encode-process-decode network, Sec. III): Y = MLP(X) with X [n x 128],
// hidden width 128, output width <= 16, 2 to 4 Linear layers, ELU between
// them, no LayerNorm; and its adjoint with per-layer recomputation.
//
// Forward, k_rowdec_fwd_tm: two groups of four warps take alternate tiles of
// 128 rows, one thread owns one row. The thread converts its input row to BF16
// straight into the group's TMEM operand columns, so every Linear reads its A
// operand from TMEM (W_k from shared memory); the last Linear is an N = 16 MMA
// (outputs zero-padded to 16) and the thread writes its row's outputs.
//
// Adjoint, over chunks of tiles (at most kChunkTiles, fewer when the caller's
// workspace is smaller; scratch rows (t - t0) * 128 + i, zero past the last row):
//   k_rowdec_save_tm  recompute the MLP up to h_{L-2}, saving X (BF16) and
//                     h_0 .. h_{L-3}; with dz_{L-1} = dY (no LayerNorm), one
//                     N = 128, K = 16 MMA gives dh_{L-2} = dY W_{L-1} and one
//                     M = 128, N = 16 MMA accumulates dW_{L-1}^T = h_{L-2}^T dY
//                     over the group's tiles; dz_{L-2} = dh_{L-2} ELU'(h_{L-2})
//                     to scratch, and the column sums for db_{L-1}, db_{L-2}
//   k_bwd_chain2 / k_bwd_chain  k = L-2 .. 1 (the layer adjoint's per-Linear kernels)
//   k_bwd_chain<INPUT> dX = dz_0 W_0 and dW_0 = dz_0^T X
// Every gradient is a fixed-order sum (per thread in row order, per CTA in
// warp and group order, then over the CTAs in CTA order).

#include <algorithm>

#include "fused.h"
#include "fused_bwd_common.cuh"
#include "profiler.h"
#include "tm128_common.cuh"

namespace gnn {
namespace fused {

cudaError_t take_device_error_rowdec128(unsigned int* out) { return take_device_error_word(out); }

namespace {

using namespace tc;
using namespace tm128;

constexpr int kNO = 16;                         // padded output width
constexpr int kSY = 32;                         // swizzle span of a [128 x 16] BF16 tile
constexpr uint32_t kYT = 128 * kNO * 2;         // [128 x 16] BF16 tile
constexpr uint32_t kWL = kNO * kH * 2;          // [16 x 128] BF16 last weight tile
constexpr int kMaxLin = 4;                      // W_0 .. W_2 resident in shared memory
constexpr int64_t kChunkTiles = 32768;          // tiles per scratch chunk
constexpr int64_t kPstride = 2 * (int64_t)kH * kH + 2 * kH;   // per-CTA partial floats (k_bwd_chain2)
// the recomputation's partials: dW_{L-1} [16 x 128], db_{L-1} [16], db_{L-2} [128]
constexpr int64_t kPdW = 0, kPdbL = kNO * kH, kPdbH = kPdbL + kNO;

struct DecArgs {
    const float* X;        // [n_rows x 128]
    int64_t n_rows;
    int NO;                // output width (<= 16)
    void* Y;               // forward: [n_rows x NO], FP32 or BF16
    int y_bf16;
    const void* dY;        // recomputation: gradient of Y [n_rows x NO], FP32 or BF16
    int dy_bf16;
    int64_t t0, t1;        // recomputation: tiles [t0, t1)
    int64_t hs_rows;       // recomputation: rows of one block of the scratch
    float* part;           // recomputation: per-CTA partials (kPdW, kPdbL, kPdbH)
    int64_t pstride;
    MlpDev mlp;
};

struct DecSmem {
    uint32_t w, wl, dy, st, par, bar, tm, total;
};

__host__ __device__ inline DecSmem dec_smem(int n_lin) {
    DecSmem s;
    s.w = 0;                                                    // W_0 .. W_{L-2}
    s.wl = align_up((uint32_t)(n_lin - 1) * kWT, 1024);        // W_{L-1} [16 x 128], rows past NO zero
    s.dy = align_up(s.wl + kWL, 1024);                          // dy[2]: [128 x 16] per group
    s.st = align_up(s.dy + 2 * kYT, 1024);                      // st[2]: staging tiles, one per group
    s.par = s.st + 2 * kTile;                                   // b_0 .. b_{L-2} [128], b_{L-1} [16]
    s.bar = align_up(s.par + (uint32_t)((n_lin - 1) * kH + kNO) * 4, 8);   // mma[2]
    s.tm = s.bar + 2 * 8;
    s.total = s.tm + 16 + 1024;
    return s;
}

// TMEM, barriers, the weights as BF16 K-major tiles and the FP32 biases; ends
// with the block in sync.
__device__ __forceinline__ void dec_prologue(const DecArgs& A, uint8_t* sm, const DecSmem& L, int tid, int warp) {
    const int n_lin = A.mlp.n_lin, NO = A.NO;
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
    for (int k = 0; k < n_lin - 1; ++k) load_weight(sm + L.w + k * kWT, A.mlp.W[k], kH, 0, kH, kH, tid, kNT);
    const float* Wl = A.mlp.W[n_lin - 1];
    for (int i = tid; i < kNO * (kH / 8); i += kNT) {
        const int n = i / (kH / 8), k = (i % (kH / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = n < NO ? __ldg(Wl + (int64_t)n * kH + k + j) : 0.f;
        st_tile8(sm + L.wl, n, k, kNO, kS, v);
    }
    float* sPar = reinterpret_cast<float*>(sm + L.par);
    for (int i = tid; i < (n_lin - 1) * kH; i += kNT) sPar[i] = A.mlp.b[i / kH][i % kH];
    for (int i = tid; i < kNO; i += kNT) sPar[(n_lin - 1) * kH + i] = i < NO ? A.mlp.b[n_lin - 1][i] : 0.f;
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Columns [c, c + 32) of this thread's input row (zero for rows past the end):
// FP32 from global memory into v.
__device__ __forceinline__ void ld_x32(const float* xr, bool valid, int c, float* v) {
    const float4* p = reinterpret_cast<const float4*>(xr + c);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 u = valid ? __ldg(p + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * i] = u.x;
        v[4 * i + 1] = u.y;
        v[4 * i + 2] = u.z;
        v[4 * i + 3] = u.w;
    }
}

// 32 values as BF16 pairs into 16 TMEM columns of this thread's lane.
__device__ __forceinline__ void bf16_to_tmem(uint32_t taddr, const float* v) {
    uint32_t hb[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) hb[i] = pack_bf16x2(v[2 * i], v[2 * i + 1]);
    tmem_st16u(taddr, hb);
}

// D = A[128 x 128] (TMEM) * W^T with W the [16 x 128] K-major last weight tile.
__device__ __forceinline__ void issue_mma_ts_n16(uint32_t d_tmem, uint32_t a_tmem, const uint8_t* Wt) {
    const uint64_t b0 = kmajor_desc(smem_u32(Wt), kNO, kS, 0);
    const uint32_t id = idesc_bf16(128, kNO);
#pragma unroll
    for (int k0 = 0; k0 < kH; k0 += 16)
        mma_bf16_ts(d_tmem, a_tmem + (uint32_t)(k0 / 2), desc_step(b0, kmajor_off(kNO, kS, k0)), id,
                    k0 > 0 ? 1u : 0u);
}

// The group's leader waits for its MMA chain (bounded); the group agrees.
__device__ __forceinline__ bool dec_wait_mma(uint64_t* bar_mma, int gi, bool leader, uint32_t& ph) {
    const bool w_ok = leader ? mbar_wait(bar_mma + gi, ph) : true;
    const bool ok = group_and(w_ok, gi);
    ph ^= 1;
    tc_fence_after();
    return ok;
}

// ------------------------------------------------------------------ forward

__global__ void __launch_bounds__(kNT, 1) k_rowdec_fwd_tm(DecArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin, NO = A.NO;
    const DecSmem L = dec_smem(n_lin);
    const float* sPar = reinterpret_cast<const float*>(sm + L.par);
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + L.bar);
    const uint32_t* tslot = reinterpret_cast<const uint32_t*>(sm + L.tm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = warp >> 2, q = warp & 3, row = 32 * q + lane;
    const bool leader = (tid & (kGT - 1)) == 0;
    dec_prologue(A, sm, L, tid, warp);
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t tAcc = *tslot + (uint32_t)(gi * 256), tA = tAcc + 128;
    const int64_t n_tiles = (A.n_rows + 127) / 128;
    const int64_t step = 2 * (int64_t)gridDim.x;
    uint32_t ph = 0;
    bool ok = true;

    for (int64_t t = (int64_t)blockIdx.x + gi * (int64_t)gridDim.x; t < n_tiles && ok; t += step) {
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        const float* xr = A.X + (valid ? r : 0) * kH;
#pragma unroll
        for (int c = 0; c < kH; c += 32) {
            float v[32];
            ld_x32(xr, valid, c, v);
            bf16_to_tmem(tA + lane_base + (uint32_t)(c / 2), v);
        }
        hand_off(tAcc, tA, sm + L.w, gi, leader, bar_mma);
        // h_k = ELU(acc + b_k) into TMEM, then the next Linear (the last one N = 16)
        for (int k = 0; k < n_lin - 1; ++k) {
            if (!(ok = dec_wait_mma(bar_mma, gi, leader, ph))) break;
            {
                float v[kH];
                ld_acc_n<kH>(tAcc + lane_base, sPar + k * kH, v);
#pragma unroll
                for (int c = 0; c < kH; c += 32) elu_to_tmem(tA + lane_base + (uint32_t)(c / 2), v + c);
            }
            if (k + 1 < n_lin - 1) {
                hand_off(tAcc, tA, sm + L.w + (k + 1) * kWT, gi, leader, bar_mma);
            } else {
                tmem_st_wait();
                tc_fence_before();
                group_sync(gi);
                if (leader) {
                    tc_fence_after();
                    issue_mma_ts_n16(tAcc, tA, sm + L.wl);
                    mma_commit(bar_mma + gi);
                }
            }
        }
        if (!ok || !(ok = dec_wait_mma(bar_mma, gi, leader, ph))) break;
        float y[kNO];
        ld_acc_n<kNO>(tAcc + lane_base, sPar + (n_lin - 1) * kH, y);
        if (valid) {
            if (A.y_bf16) {
                __nv_bfloat16* yr = static_cast<__nv_bfloat16*>(A.Y) + r * NO;
#pragma unroll
                for (int o = 0; o < kNO; ++o)
                    if (o < NO) yr[o] = __float2bfloat16_rn(y[o]);
            } else {
                float* yr = static_cast<float*>(A.Y) + r * NO;
#pragma unroll
                for (int o = 0; o < kNO; ++o)
                    if (o < NO) yr[o] = y[o];
            }
        }
        // the accumulator is read (wait::ld inside ld_acc_n) before the group's next MMA
        tc_fence_before();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, 512);
}

// ------------------------------------------------------------------ recomputation for the adjoint

// ELU of 32 pre-activations as BF16 into the staging tile at (row, c..c+31);
// rows past the tile's edges stage zeros.
__device__ __forceinline__ void elu_to_tile(const float* v, uint8_t* tile, int row, int c, bool valid) {
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
        float h[8];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const float2 e = elu1_fast2(make_float2(v[i + j], v[i + j + 1]));
            h[j] = valid ? e.x : 0.f;
            h[j + 1] = valid ? e.y : 0.f;
        }
        st_tile8(tile, row, c + i, 128, kS, h);
    }
}

__global__ void __launch_bounds__(kNT, 1) k_rowdec_save_tm(const __grid_constant__ CUtensorMap tmap_hs,
                                                           const __grid_constant__ CUtensorMap tmap_dz, DecArgs A) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    const int n_lin = A.mlp.n_lin, NO = A.NO;
    const DecSmem L = dec_smem(n_lin);
    const float* sPar = reinterpret_cast<const float*>(sm + L.par);
    uint64_t* bar_mma = reinterpret_cast<uint64_t*>(sm + L.bar);
    const uint32_t* tslot = reinterpret_cast<const uint32_t*>(sm + L.tm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gi = warp >> 2, q = warp & 3, row = 32 * q + lane;
    const bool leader = (tid & (kGT - 1)) == 0;
    uint8_t* sDy = sm + L.dy + gi * kYT;
    uint8_t* sSt = sm + L.st + gi * kTile;
    dec_prologue(A, sm, L, tid, warp);
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t tAcc = *tslot + (uint32_t)(gi * 256), tA = tAcc + 128;
    const uint32_t tDW = tAcc + 192;   // the group's dW_{L-1}^T [128 x 16], summed over its tiles
    const int64_t step = 2 * (int64_t)gridDim.x;
    uint32_t ph = 0;
    bool ok = true, dw_live = false;
    float accY = 0.f, accZ[8];   // lane l: column 16 j + (l >> 1) of 16-column block j
#pragma unroll
    for (int j = 0; j < 8; ++j) accZ[j] = 0.f;

    for (int64_t t = A.t0 + (int64_t)blockIdx.x + gi * (int64_t)gridDim.x; t < A.t1 && ok; t += step) {
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        const int32_t y = (int32_t)((t - A.t0) * 128);
        // X: the first Linear's operand in TMEM and, as BF16, block 0 of the scratch
        const float* xr = A.X + (valid ? r : 0) * kH;
#pragma unroll
        for (int c = 0; c < kH; c += 32) {
            float v[32];
            ld_x32(xr, valid, c, v);
            bf16_to_tmem(tA + lane_base + (uint32_t)(c / 2), v);
#pragma unroll
            for (int i = 0; i < 32; i += 8) st_tile8(sSt, row, c + i, 128, kS, v + i);
        }
        save_hand_off(tAcc, tA, sm + L.w, gi, leader, bar_mma, &tmap_hs, sSt, y);
        // h_0 .. h_{L-3}: operand of the next Linear and block k + 1 of the scratch
        for (int k = 0; k < n_lin - 2; ++k) {
            if (leader) bulk_wait_read_all();
            if (!(ok = dec_wait_mma(bar_mma, gi, leader, ph))) break;
            {
                float v[kH];
                ld_acc_n<kH>(tAcc + lane_base, sPar + k * kH, v);
#pragma unroll
                for (int c = 0; c < kH; c += 32)
                    elu_to_tmem_and_tile(tA + lane_base + (uint32_t)(c / 2), v + c, sSt, row, c, valid);
            }
            save_hand_off(tAcc, tA, sm + L.w + (k + 1) * kWT, gi, leader, bar_mma, &tmap_hs, sSt,
                          (int32_t)((k + 1) * A.hs_rows) + y);
        }
        if (!ok) break;
        // h_{L-2} into the staging tile (the weight gradient's operand), dY into the dY tile
        if (leader) bulk_wait_read_all();
        if (!(ok = dec_wait_mma(bar_mma, gi, leader, ph))) break;
        {
            float v[kH];
            ld_acc_n<kH>(tAcc + lane_base, sPar + (n_lin - 2) * kH, v);
#pragma unroll
            for (int c = 0; c < kH; c += 32) elu_to_tile(v + c, sSt, row, c, valid);
        }
        {
            float dy[kNO];
#pragma unroll
            for (int o = 0; o < kNO; ++o) {
                float g = 0.f;
                if (valid && o < NO)
                    g = A.dy_bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(A.dY)[r * NO + o])
                                  : static_cast<const float*>(A.dY)[r * NO + o];
                dy[o] = g;
            }
            st_row_tile<kNO>(sDy, row, 0, kSY, dy);
            accY += warp_colsum16(dy, lane);
        }
        fence_proxy_async();
        tc_fence_before();
        group_sync(gi);
        if (leader) {   // dh_{L-2} = dY W_{L-1}; dW_{L-1}^T += h_{L-2}^T dY
            tc_fence_after();
            issue_dgrad(tAcc, sDy, kSY, sm + L.wl, kS, kNO, (uint32_t)kNO * kS, kH, kNO);
            issue_wgrad(tDW, sSt, kS, 128u * kS, sDy, kSY, 128u * kSY, kNO, dw_live);
            mma_commit(bar_mma + gi);
        }
        dw_live = true;
        if (!(ok = dec_wait_mma(bar_mma, gi, leader, ph))) break;
        // dz_{L-2} = dh_{L-2} ELU'(h_{L-2}) (from h's BF16 copy), over the staging tile, to scratch
#pragma unroll
        for (int c = 0; c < kH; c += 16) {
            float dh[16], h[16];
            tmem_ld16(tAcc + lane_base + c, dh);
            ld_tile8(sSt, row, c, 128, kS, h);
            ld_tile8(sSt, row, c + 8, 128, kS, h + 8);
            tmem_ld_wait();
#pragma unroll
            for (int i = 0; i < 16; ++i) dh[i] = valid ? elu1_bwd_from_out(dh[i], h[i]) : 0.f;
            accZ[c / 16] += warp_colsum16(dh, lane);
            st_tile8(sSt, row, c, 128, kS, dh);
            st_tile8(sSt, row, c + 8, 128, kS, dh + 8);
        }
        tc_fence_before();
        fence_proxy_async();
        group_sync(gi);
        if (leader) {
#pragma unroll
            for (int kb = 0; kb < 2; ++kb) tma_store_2d(&tmap_dz, kb * 64, y, sSt + kb * 128 * kS);
            bulk_commit();
            bulk_wait_read_all();
        }
        group_sync(gi);   // the staging tile is free for the next tile's X
    }
    if (leader) bulk_wait_all();   // the scratch rows are written
    __syncwarp();   // reconverged before the aligned block barrier
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the CTA's partials: dW_{L-1} (group 0's sum + group 1's), then the column sums in warp order
    float* red = reinterpret_cast<float*>(sm + L.st);
    float dw[kNO];
    if (dw_live) {   // uniform over the group (the group's tile count)
        tmem_ld16(tDW + lane_base, dw);
        tmem_ld_wait();
    } else {
#pragma unroll
        for (int o = 0; o < kNO; ++o) dw[o] = 0.f;
    }
    if (gi == 1)
#pragma unroll
        for (int o = 0; o < kNO; ++o) red[o * kH + row] = dw[o];
    __syncthreads();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (gi == 0)
#pragma unroll
        for (int o = 0; o < kNO; ++o) part[kPdW + o * kH + row] = dw[o] + red[o * kH + row];
    __syncthreads();
    constexpr int NS = kNO + kH;   // [db_{L-1} | db_{L-2}] per warp
    if ((lane & 1) == 0) {
        red[warp * NS + (lane >> 1)] = accY;
#pragma unroll
        for (int j = 0; j < 8; ++j) red[warp * NS + kNO + 16 * j + (lane >> 1)] = accZ[j];
    }
    __syncthreads();
    for (int i = tid; i < NS; i += kNT) {
        float s = 0.f;
        for (int wi = 0; wi < 8; ++wi) s += red[wi * NS + i];
        part[kPdbL + i] = s;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(*tslot, 512);
}

// =================================================================== host side

using namespace host;

struct DecWs {
    float* part;             // num_sms CTAs x kPstride floats
    __nv_bfloat16* hs;       // (L-1) x [chunk rows x H]: X, h_0 .. h_{L-3}
    int64_t hs_stride;
    __nv_bfloat16* dzs[2];   // [chunk rows x H] each
    size_t bytes;
};

DecWs carve_dec(void* ws, int n_lin, int64_t chunk) {
    DecWs w{};
    size_t off = 0;
    auto take = [&](size_t n) {
        off = (off + 255) & ~(size_t)255;
        void* p = ws ? (char*)ws + off : nullptr;
        off += n;
        return p;
    };
    const int64_t rows = chunk * 128;
    w.part = (float*)take((size_t)num_sms() * kPstride * 4);
    w.hs_stride = rows * kH;
    w.hs = (__nv_bfloat16*)take((size_t)(n_lin - 1) * rows * kH * 2);
    w.dzs[0] = (__nv_bfloat16*)take((size_t)rows * kH * 2);
    w.dzs[1] = (__nv_bfloat16*)take((size_t)rows * kH * 2);
    w.bytes = off + 256;
    return w;
}

int64_t dec_chunk(int64_t n_rows) { return std::max<int64_t>(1, std::min<int64_t>(kChunkTiles, (n_rows + 127) / 128)); }

DecArgs dec_args(const gnn_mlp& P, int64_t n_rows, const float* X) {
    DecArgs A{};
    A.X = X;
    A.n_rows = n_rows;
    A.NO = P.dims[P.n_lin];
    A.mlp = mlp_dev(P);
    return A;
}

}  // namespace

bool rowdec128_shape(const gnn_mlp& P) {
    const int L = P.n_lin;
    if (L < 2 || L > kMaxLin || P.gamma) return false;
    for (int l = 0; l < L; ++l)
        if (P.dims[l] != kH) return false;
    return P.dims[L] >= 1 && P.dims[L] <= kNO;
}

size_t rowdec128_backward_ws(const gnn_mlp& P, int64_t n_rows) {
    return carve_dec(nullptr, P.n_lin, dec_chunk(n_rows)).bytes;
}

int rowdec128_forward(const gnn_mlp& P, int64_t n_rows, const float* X, void* Y, int y_bf16, cudaStream_t s) {
    GNN_REQUIRE(rowdec128_shape(P), GNN_EUNSUPPORTED, "gnn_mlp_forward_bf16: not an H=128 decoder of 2..%d Linears",
                kMaxLin);
    if (n_rows == 0) return GNN_OK;
    GNN_REQUIRE(((uintptr_t)X & 15) == 0, GNN_EINVAL, "gnn_mlp_forward_bf16: X must be 16-byte aligned at H=128");
    DecArgs A = dec_args(P, n_rows, X);
    A.Y = Y;
    A.y_bf16 = y_bf16;
    const DecSmem L = dec_smem(P.n_lin);
    int grid;
    int rc = persistent_grid(k_rowdec_fwd_tm, kNT, L.total, 512, ((n_rows + 127) / 128 + 1) / 2, &grid);
    if (rc) return rc;
    {
        ProfScope _ps(s, "k_rowmlp_fwd");
        k_rowdec_fwd_tm<<<grid, kNT, L.total, s>>>(A);
    }
    GNN_LAUNCH_CHECK("k_rowdec_fwd_tm");
    return GNN_OK;
}

int rowdec128_backward(const gnn_mlp& P, int64_t n_rows, const float* X, const void* dY, int dy_bf16, float* dX,
                       const gnn_mlp& dP, void* ws, size_t ws_bytes, cudaStream_t s) {
    GNN_REQUIRE(rowdec128_shape(P), GNN_EUNSUPPORTED, "gnn_mlp_backward_bf16: not an H=128 decoder of 2..%d Linears",
                kMaxLin);
    if (n_rows == 0) return GNN_OK;
    GNN_REQUIRE(((uintptr_t)X & 15) == 0 && ((uintptr_t)dX & 15) == 0, GNN_EINVAL,
                "gnn_mlp_backward_bf16: X and dX must be 16-byte aligned at H=128");
    const int Lw = P.n_lin, NO = P.dims[Lw];
    const int64_t n_tiles = (n_rows + 127) / 128;
    // the largest chunk of tiles whose scratch fits the workspace given
    int64_t chunk = dec_chunk(n_rows);
    if (ws_bytes < carve_dec(nullptr, Lw, chunk).bytes) {
        const size_t fixed = carve_dec(nullptr, Lw, 0).bytes;
        const size_t per_tile = carve_dec(nullptr, Lw, 2).bytes - carve_dec(nullptr, Lw, 1).bytes;
        chunk = ws_bytes > fixed ? (int64_t)((ws_bytes - fixed) / per_tile) : 0;
        while (chunk > 0 && carve_dec(nullptr, Lw, chunk).bytes > ws_bytes) --chunk;
        GNN_REQUIRE(chunk >= 1, GNN_ENOMEM, "gnn_mlp_backward_bf16: workspace too small (%zu bytes)", ws_bytes);
    }
    DecWs w = carve_dec(ws, Lw, chunk);
    const DecSmem L = dec_smem(Lw);
    // the hidden Linears 1 .. L-2 as an MLP of L-1 Linears for the chain kernel
    gnn_mlp Ph = P, dPh = dP;
    Ph.n_lin = dPh.n_lin = Lw - 1;
    int rc;
    for (int64_t t0 = 0; t0 < n_tiles; t0 += chunk) {
        const int64_t t1 = std::min(n_tiles, t0 + chunk);
        const int64_t rows = (t1 - t0) * 128;
        // 1. recomputation and the last Linear's adjoint: X, h_0 .. h_{L-3}, dz_{L-2},
        //    dW_{L-1}, db_{L-1}, db_{L-2}
        CUtensorMap tmhs, tmdz;
        if ((rc = make_row_tmap(&tmhs, w.hs, (int64_t)(Lw - 1) * (w.hs_stride / kH), kH))) return rc;
        if ((rc = make_row_tmap(&tmdz, w.dzs[0], rows, kH))) return rc;
        DecArgs A = dec_args(P, n_rows, X);
        A.dY = dY;
        A.dy_bf16 = dy_bf16;
        A.t0 = t0;
        A.t1 = t1;
        A.hs_rows = w.hs_stride / kH;
        A.part = w.part;
        A.pstride = kPstride;
        int grid;
        if ((rc = persistent_grid(k_rowdec_save_tm, kNT, L.total, 512, (t1 - t0 + 1) / 2, &grid))) return rc;
        {
            ProfScope _ps(s, "k_rowmlp_save");
            k_rowdec_save_tm<<<grid, kNT, L.total, s>>>(tmhs, tmdz, A);
        }
        GNN_LAUNCH_CHECK("k_rowdec_save_tm");
        {
            RedSeg seg[3];
            seg[0] = RedSeg{dP.W[Lw - 1], kH, NO, kH, kPdW, kH};
            seg[1] = RedSeg{dP.b[Lw - 1], NO, 1, NO, kPdbL, 0};
            seg[2] = RedSeg{dP.b[Lw - 2], kH, 1, kH, kPdbH, 0};
            if ((rc = reduce_grads(seg, 3, w.part, kPstride, grid, s))) return rc;
        }
        // 2. Linears L-2 .. 1 (h_{k-1} in block k of the scratch)
        int cur = 0;
        if ((rc = chain_backward_h128(Ph, dPh, w.hs + w.hs_stride, w.hs_stride, w.dzs, w.part, kPstride, t1 - t0,
                                      &cur, s)))
            return rc;
        // 3. the first Linear: dX = dz_0 W_0, dW_0 = dz_0^T X (X in block 0)
        if ((rc = chain_input_h128(P.W[0], dP.W[0], w.dzs[cur], w.hs, dX, t0 * 128, n_rows, w.part, kPstride,
                                   t1 - t0, s)))
            return rc;
    }
    return GNN_OK;
}

}  // namespace fused
}  // namespace gnn
