// Pieces shared by the fused BF16 backward kernels (layer adjoint and row
// MLP adjoint): per-H thread layout, weight- and input-gradient MMAs on the
// operand tiles the recompute already holds, the ones block that yields bias
// gradients, row reductions, and the per-CTA partial-gradient reduction.
#pragma once

#include "fused_common.cuh"

namespace gnn {
namespace fused {

template <int H>
struct CfgB {
    static constexpr int S = span_of(H);
    static constexpr int S2 = span_of(2 * H);
    static constexpr int CG = H >= 16 ? H / 16 : 1;
    static constexpr int CW = H / CG;         // 16
    static constexpr int NT = 128 * CG;
    static constexpr int TILE = 128 * H * 2;
    static constexpr int WT = H * H * 2;
    static constexpr int NW = H + 16;         // wgrad N: H inputs + the ones block
};

__host__ __device__ constexpr uint32_t pow2_cols(uint32_t n) {
    uint32_t c = 32;
    while (c < n) c <<= 1;
    return c;
}

// ------------------------------------------------------------------ device helpers

// D[128 x N] (+)= A[128 x K] (K-major row tile, span Sa) * B where B is a
// K x N MN-major row tile (rows = K, contiguous = N, span Sb, N-blocks lbo apart).
__device__ __forceinline__ void issue_dgrad(uint32_t d, const uint8_t* A, int Sa, const uint8_t* Bt, int Sb,
                                            int b_rows, uint32_t lbo, int N, int K) {
    const uint64_t a0 = kmajor_desc(smem_u32(A), 128, Sa, 0);
    const uint64_t b0 = sdesc(smem_u32(Bt), lbo, 8 * Sb, swz_code(Sb));
    const uint32_t id = idesc_bf16(128, N, 0, 1);
    (void)b_rows;
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16)
        mma_bf16(d, desc_step(a0, kmajor_off(128, Sa, k0)), desc_step(b0, (uint32_t)k0 * Sb), id, k0 > 0 ? 1u : 0u);
}

// D[128 x N] (+)= A^T B over the 128 rows of two MN-major row tiles:
// A: rows = K (=128), contiguous = M features (span Sa, M-blocks lbo_a apart);
// B: rows = K, contiguous = N features (span Sb, N-blocks lbo_b apart).
__device__ __forceinline__ void issue_wgrad(uint32_t d, const uint8_t* A, int Sa, uint32_t lbo_a, const uint8_t* Bt,
                                            int Sb, uint32_t lbo_b, int N, bool accumulate) {
    const uint64_t a0 = sdesc(smem_u32(A), lbo_a, 8 * Sa, swz_code(Sa));
    const uint64_t b0 = sdesc(smem_u32(Bt), lbo_b, 8 * Sb, swz_code(Sb));
    const uint32_t id = idesc_bf16(128, N, 1, 1);
#pragma unroll
    for (int k0 = 0; k0 < 128; k0 += 16)
        mma_bf16(d, desc_step(a0, (uint32_t)k0 * Sa), desc_step(b0, (uint32_t)k0 * Sb), id,
                 (accumulate || k0 > 0) ? 1u : 0u);
}

// Ones block: a [128 x S/2] row tile whose column 0 is 1 and the rest 0.
__device__ __forceinline__ void fill_ones(uint8_t* dst, int S, int tid, int nt) {
    const int per = S / 2;
    for (int i = tid; i < 128 * (per / 8); i += nt) {
        const int r = i / (per / 8), c = (i % (per / 8)) * 8;
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (c == 0) v[0] = 1.f;
        st_tile8(dst, r, c, 128, S, v);
    }
}

// Row sums of two per-thread partial vectors over the CG threads of a row.
template <int CG>
__device__ __forceinline__ void row_sum2(float a, float b, float* red, int row, int g, float& sa, float& sb) {
    red[g * 128 + row] = a;
    red[(CG + g) * 128 + row] = b;
    __syncthreads();
    sa = 0.f;
    sb = 0.f;
#pragma unroll
    for (int k = 0; k < CG; ++k) {
        sa += red[k * 128 + row];
        sb += red[(CG + k) * 128 + row];
    }
    __syncthreads();
}

// LayerNorm statistics and adjoint sums of a row split over CG threads, in
// one exchange: with d = g * gamma, the forward's mean and rstd come from
// sum v and sum v^2, and the adjoint's (1/H) sum d and (1/H) sum d * xhat
// from sum d and sum d * v, since sum d * xhat = rstd (sum d v - mean sum d).
template <int H, int CG, int CW>
__device__ __forceinline__ void row_stats_adj(const float* v, const float* d, float* red, int row, int g, float eps,
                                              float& mean, float& rstd, float& s1, float& s2) {
    float sv = 0.f, sq = 0.f, sd = 0.f, sdv = 0.f;
#pragma unroll
    for (int i = 0; i < CW; ++i) {
        sv += v[i];
        sq += v[i] * v[i];
        sd += d[i];
        sdv += d[i] * v[i];
    }
    red[(0 * CG + g) * 128 + row] = sv;
    red[(1 * CG + g) * 128 + row] = sq;
    red[(2 * CG + g) * 128 + row] = sd;
    red[(3 * CG + g) * 128 + row] = sdv;
    __syncthreads();
    sv = sq = sd = sdv = 0.f;
#pragma unroll
    for (int k = 0; k < CG; ++k) {
        sv += red[(0 * CG + k) * 128 + row];
        sq += red[(1 * CG + k) * 128 + row];
        sd += red[(2 * CG + k) * 128 + row];
        sdv += red[(3 * CG + k) * 128 + row];
    }
    mean = sv * (1.f / H);
    rstd = rsqrtf(fmaxf(sq * (1.f / H) - mean * mean, 0.f) + eps);
    s1 = sd * (1.f / H);
    s2 = rstd * (sdv - mean * sd) * (1.f / H);
}

// Reduce per-thread column accumulators acc[CW] over the 128 rows of the CTA
// (lanes by shuffle, then the 4 lane quarters in order) into out[c0..c0+CW).
template <int CW>
__device__ __forceinline__ void rows_reduce_store(float* acc, float* red, int q, int lane, int g, int c0, float* out) {
#pragma unroll
    for (int i = 0; i < CW; ++i) {
#pragma unroll
        for (int o = 16; o; o >>= 1) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    }
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < CW; ++i) red[(g * 4 + q) * CW + i] = acc[i];
    }
    __syncthreads();
    if (q == 0 && lane < CW) {
        float s = 0.f;
        for (int k = 0; k < 4; ++k) s += red[(g * 4 + k) * CW + lane];
        out[c0 + lane] = s;
    }
    __syncthreads();
}

// Flush a TMEM accumulator [128 lanes x N cols] (rows < m_valid) into dst[m*N + n].
template <int CG>
__device__ __forceinline__ void flush_acc(uint32_t tmem, int N, int m_valid, int q, int lane, int g, float* dst) {
    const int m = 32 * q + lane;
    for (int c = g * 16; c < N; c += CG * 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c, v);
        tmem_ld_wait();
        if (m < m_valid) {
#pragma unroll
            for (int i = 0; i < 16; ++i) dst[(int64_t)m * N + c + i] = v[i];
        }
    }
}


// Per-CTA weight-gradient partials: segment s of the result is rows x cols of
// dst (leading dimension dst_ld), read from the partials at src_off with
// leading dimension src_ld; k_reduce_grads sums the CTAs' partials in CTA order.
struct RedSeg {
    float* dst;
    int dst_ld, rows, cols;
    int64_t src_off, src_ld;
};

constexpr int MAX_SEGS = 2 * GNN_MAX_LIN + 4;

int reduce_grads(RedSeg* segs, int n, const float* part, int64_t pstride, int n_cta, cudaStream_t s);

}  // namespace fused
}  // namespace gnn
