// Pieces of the two-group tensor-memory kernels at H = 128 (the edge forward
// and its recomputation for the adjoint, the encoder row MLP): each group of
// four warps owns 256 TMEM columns, the accumulator of the running Linear in
// the first 128 and the BF16 activation that the next Linear reads as its A
// operand in the next 64; one thread owns one row (TMEM lane) of a 128-row tile.
#pragma once

#include "fused_common.cuh"

namespace gnn {
namespace fused {
namespace tm128 {

using namespace tc;

constexpr int kH = 128;
constexpr int kNT = 256;                       // two groups of four warps
constexpr int kGT = 128;                       // threads per group
constexpr uint32_t kTile = 128 * kH * 2;       // [128 x 128] BF16 row tile
constexpr uint32_t kWT = kH * kH * 2;          // [128 x 128] BF16 weight tile
constexpr int kS = 128;                        // swizzle span of a 128-wide BF16 tile

// D[tmem] (+)= A[tmem] * B[smem desc]: A is M x K BF16 in tensor memory, lane =
// row, two consecutive K values per 32-bit column.
__device__ __forceinline__ void mma_bf16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D = A[128 x 128] (TMEM) * W^T, W a K-major [128 x 128] row tile.
__device__ __forceinline__ void issue_mma_ts(uint32_t d_tmem, uint32_t a_tmem, const uint8_t* Wt) {
    const uint64_t b0 = kmajor_desc(smem_u32(Wt), kH, kS, 0);
    const uint32_t id = idesc_bf16(128, kH);
#pragma unroll
    for (int k0 = 0; k0 < kH; k0 += 16)
        mma_bf16_ts(d_tmem, a_tmem + (uint32_t)(k0 / 2), desc_step(b0, kmajor_off(kH, kS, k0)), id, k0 > 0 ? 1u : 0u);
}

// 16 packed BF16 pairs into 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st16u(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// 32 accumulator columns [c, c + 32) of this thread's lane, plus bias (16-byte
// aligned, read as float4).
__device__ __forceinline__ void ld_acc32(uint32_t taddr, const float* bias, float* v) {
    tmem_ld16(taddr, v);
    tmem_ld16(taddr + 16, v + 16);
    tmem_ld_wait();
    const float4* b4 = reinterpret_cast<const float4*>(bias);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 b = b4[i];
        float2* v2 = reinterpret_cast<float2*>(v + 4 * i);
        v2[0] = __fadd2_rn(v2[0], make_float2(b.x, b.y));
        v2[1] = __fadd2_rn(v2[1], make_float2(b.z, b.w));
    }
}

// N accumulator columns [0, N) of this thread's lane with a single wait (the loads
// overlap each other), plus bias.
template <int N>
__device__ __forceinline__ void ld_acc_n(uint32_t taddr, const float* bias, float* v) {
#pragma unroll
    for (int i = 0; i < N; i += 16) tmem_ld16(taddr + i, v + i);
    tmem_ld_wait();
    const float4* b4 = reinterpret_cast<const float4*>(bias);
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
        const float4 b = b4[i];
        float2* v2 = reinterpret_cast<float2*>(v + 4 * i);
        v2[0] = __fadd2_rn(v2[0], make_float2(b.x, b.y));
        v2[1] = __fadd2_rn(v2[1], make_float2(b.z, b.w));
    }
}

// 32 FP32 columns of this thread's lane from registers into TMEM.
__device__ __forceinline__ void st_tmem32(uint32_t taddr, const float* v) {
    tmem_st16(taddr, v);
    tmem_st16(taddr + 16, v + 16);
}

// Sum of 32 values in four independent chains (latency), then combined.
__device__ __forceinline__ float sum32(const float* v) {
    float2 a = make_float2(v[0], v[1]), b = make_float2(v[2], v[3]);
    float2 c = make_float2(v[4], v[5]), d = make_float2(v[6], v[7]);
#pragma unroll
    for (int i = 8; i < 32; i += 8) {
        a = __fadd2_rn(a, make_float2(v[i], v[i + 1]));
        b = __fadd2_rn(b, make_float2(v[i + 2], v[i + 3]));
        c = __fadd2_rn(c, make_float2(v[i + 4], v[i + 5]));
        d = __fadd2_rn(d, make_float2(v[i + 6], v[i + 7]));
    }
    a = __fadd2_rn(__fadd2_rn(a, b), __fadd2_rn(c, d));
    return a.x + a.y;
}

// Sum of (v - m)^2 over 32 values, four independent chains.
__device__ __forceinline__ float sqdev32(const float* v, float m) {
    const float2 nm = make_float2(-m, -m);
    float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
        const float2 d = __fadd2_rn(make_float2(v[i], v[i + 1]), nm);
        acc[(i / 2) & 3] = __ffma2_rn(d, d, acc[(i / 2) & 3]);
    }
    const float2 a = __fadd2_rn(__fadd2_rn(acc[0], acc[1]), __fadd2_rn(acc[2], acc[3]));
    return a.x + a.y;
}

// ELU of 32 pre-activations, BF16-packed into 16 TMEM columns (the next Linear's A operand).
__device__ __forceinline__ void elu_to_tmem(uint32_t taddr, const float* v) {
    uint32_t hb[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float2 h = elu1_fast2(make_float2(v[2 * i], v[2 * i + 1]));
        hb[i] = pack_bf16x2(h.x, h.y);
    }
    tmem_st16u(taddr, hb);
}

// One group's named barrier (ids 1, 2), optionally AND-ing a predicate.
__device__ __forceinline__ void group_sync(int gi) { named_sync(1 + gi, kGT); }
__device__ __forceinline__ bool group_and(bool v, int gi) { return named_and(v, 1 + gi, kGT); }

// The group's activation is in TMEM: order the stores before the MMA that reads
// them, then the leader issues acc = h W^T.
__device__ __forceinline__ void hand_off(uint32_t tAcc, uint32_t tA, const uint8_t* Wt, int gi, bool leader,
                                         uint64_t* bar_mma) {
    tmem_st_wait();
    tc_fence_before();
    group_sync(gi);
    if (leader) {
        tc_fence_after();
        issue_mma_ts(tAcc, tA, Wt);
        mma_commit(bar_mma + gi);
    }
}

// ELU of 32 pre-activations into TMEM (the next operand) and, as BF16, into the
// staging tile at (row, c..c+31); rows past the tile's edges stage zeros.
__device__ __forceinline__ void elu_to_tmem_and_tile(uint32_t taddr, const float* v, uint8_t* tile, int row, int c,
                                                     bool valid) {
    uint32_t hb[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float2 h = elu1_fast2(make_float2(v[2 * i], v[2 * i + 1]));
        hb[i] = pack_bf16x2(h.x, h.y);
    }
    tmem_st16u(taddr, hb);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 u = valid ? make_uint4(hb[4 * i], hb[4 * i + 1], hb[4 * i + 2], hb[4 * i + 3])
                              : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(tile + tile_off(row, c + 8 * i, 128, kS)) = u;
    }
}

// After an epilogue that wrote h_k to TMEM and the staging tile: the leader
// issues the next Linear and the TMA store of h_k (both read what the group wrote).
__device__ __forceinline__ void save_hand_off(uint32_t tAcc, uint32_t tA, const uint8_t* Wt, int gi, bool leader,
                                              uint64_t* bar_mma, const CUtensorMap* tmap, const uint8_t* tile,
                                              int32_t y) {
    tmem_st_wait();
    fence_proxy_async();
    tc_fence_before();
    group_sync(gi);
    if (leader) {
        tc_fence_after();
        issue_mma_ts(tAcc, tA, Wt);
        mma_commit(bar_mma + gi);
#pragma unroll
        for (int kb = 0; kb < 2; ++kb) tma_store_2d(tmap, kb * 64, y, tile + kb * 128 * kS);
        bulk_commit();
    }
}

}  // namespace tm128
}  // namespace fused
}  // namespace gnn
