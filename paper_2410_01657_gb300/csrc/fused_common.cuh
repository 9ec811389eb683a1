// Shared pieces of the fused BF16 kernels (forward and backward translation
// units): per-H configuration, shared-memory plans, operand staging helpers
// and the host-side launch helpers (TMA descriptors, persistent grids).
#pragma once

#include <algorithm>
#include <mutex>

#include "device_common.cuh"
#include "tc_common.cuh"

namespace gnn {
namespace fused {

using namespace tc;

template <int H>
struct Cfg {
    static constexpr int S = (2 * H >= 128) ? 128 : 2 * H;   // swizzle span of a K=H tile
    static constexpr int CG = H >= 32 ? H / 32 : 1;          // column groups
    static constexpr int CW = H / CG;                        // columns per thread
    static constexpr int NT = 128 * CG;                      // threads per CTA
    static constexpr int TILE = 128 * H * 2;                 // [128 x H] BF16 row tile
    static constexpr int WT = H * H * 2;                     // [H x H] BF16 weight tile
    static constexpr uint32_t TCOLS = H < 32 ? 32 : H;       // TMEM columns of one accumulator
};

__host__ __device__ constexpr int span_of(int K) { return 2 * K >= 128 ? 128 : 2 * K; }
__host__ __device__ constexpr uint32_t align_up(uint32_t v, uint32_t a) { return (v + a - 1) / a * a; }

struct MlpDev {
    const float* W[GNN_MAX_LIN];
    const float* b[GNN_MAX_LIN];
    const float* gamma;
    const float* beta;
    int n_lin;
};

// ------------------------------------------------------------------ device helpers

// One thread polls the mbarrier (bounded), the block agrees on the outcome.
// The barrier also orders the observed completion before every thread's
// subsequent tcgen05/shared-memory accesses.
__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t parity, int tid) {
    const int mine = (tid == 0) ? (mbar_wait(bar, parity) ? 1 : 0) : 1;
    __syncwarp();   // warp 0 reconverged before the aligned block barrier
    return __syncthreads_and(mine) != 0;
}

// 2^x on the special-function unit (approximate, denormals flushed).
__device__ __forceinline__ float ex2_sfu(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ELU (alpha 1): z for z > 0, e^z - 1 otherwise, with e^z = 2^(z log2 e).
// Evaluating the exponential at min(z, 0) keeps it in (0, 1], and since
// e^z - 1 >= z everywhere one max selects the branch. The result is rounded
// to BF16 next, far coarser than the absolute error of the SFU exponential.
__device__ __forceinline__ float elu1_fast(float z) {
    return fmaxf(z, ex2_sfu(fminf(z, 0.f) * 1.4426950408889634f) - 1.f);
}

// Paired forms on the packed FP32 pipe (two lanes per instruction).
__device__ __forceinline__ float2 elu1_fast2(float2 z) {
    const float2 m = make_float2(fminf(z.x, 0.f), fminf(z.y, 0.f));
    const float2 t = __fmul2_rn(m, make_float2(1.4426950408889634f, 1.4426950408889634f));
    const float2 e = __fadd2_rn(make_float2(ex2_sfu(t.x), ex2_sfu(t.y)), make_float2(-1.f, -1.f));
    return make_float2(fmaxf(z.x, e.x), fmaxf(z.y, e.y));
}

// v[i] += b[i] for CW values (CW even, b 8-byte aligned).
template <int CW>
__device__ __forceinline__ void add_bias2(float* v, const float* b) {
    float2* v2 = reinterpret_cast<float2*>(v);
    const float2* b2 = reinterpret_cast<const float2*>(b);
#pragma unroll
    for (int i = 0; i < CW / 2; ++i) v2[i] = __fadd2_rn(v2[i], b2[i]);
}

// v = ELU(v) for CW values.
template <int CW>
__device__ __forceinline__ void elu_inplace2(float* v) {
    float2* v2 = reinterpret_cast<float2*>(v);
#pragma unroll
    for (int i = 0; i < CW / 2; ++i) v2[i] = elu1_fast2(v2[i]);
}

// dz = dL/dz of h = ELU(z) from dh and the output h, in pairs (see elu1_bwd_from_out).
template <int CW>
__device__ __forceinline__ void elu_bwd2(float* dz, const float* dh, const float* h) {
#pragma unroll
    for (int i = 0; i < CW; i += 2) {
        const float2 d = make_float2(dh[i], dh[i + 1]);
        const float2 r = __ffma2_rn(d, make_float2(fminf(h[i], 0.f), fminf(h[i + 1], 0.f)), d);
        dz[i] = r.x;
        dz[i + 1] = r.y;
    }
}

// dL/dz of h = ELU(z) from the output: dh for h > 0, dh (h + 1) = dh e^z otherwise.
__device__ __forceinline__ float elu1_bwd_from_out(float dh, float h) { return fmaf(dh, fminf(h, 0.f), dh); }

// Convert W[n][c_off + k] (FP32, row stride ld, n < N, k < K) into rows
// row_off.. of a K-major BF16 row tile with rows_total rows.
__device__ __forceinline__ void load_weight(uint8_t* dst, const float* __restrict__ W, int ld, int c_off, int N,
                                            int K, int tid, int nt, int rows_total = -1, int row_off = 0) {
    const int S = span_of(K);
    if (rows_total < 0) rows_total = N;
    for (int i = tid; i < N * (K / 8); i += nt) {
        const int n = i / (K / 8), k = (i % (K / 8)) * 8;
        float v[8];
        const float4* p = reinterpret_cast<const float4*>(W + (int64_t)n * ld + c_off + k);
        float4 a = __ldg(p), b = __ldg(p + 1);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        st_tile8(dst, row_off + n, k, rows_total, S, v);
    }
}

// The MMA issue loops below build each operand's descriptor once and step
// its start-address field (16-byte units, bits 0..13) by the K-step's byte
// offset: the issuing thread's work per MMA is two adds, which keeps the
// block's wait for the issue short. Shared-memory offsets stay below 256 KB,
// so the field never carries into the next one.
__device__ __forceinline__ uint64_t desc_step(uint64_t d, uint32_t bytes) { return d + (uint64_t)(bytes >> 4); }

// Byte offset of the K-step at column k0 of a K-major row tile (rows, span S).
__host__ __device__ __forceinline__ uint32_t kmajor_off(int rows, int S, int k0) {
    return (uint32_t)(k0 / (S / 2)) * rows * S + (uint32_t)(k0 % (S / 2)) * 2;
}

// Issue D = A[128 x K] * B[N x K]^T (both K-major row tiles) from one thread.
__device__ __forceinline__ void issue_mma(uint32_t d_tmem, const uint8_t* A, const uint8_t* Bt, int N, int K) {
    const int S = span_of(K);
    const uint64_t a0 = kmajor_desc(smem_u32(A), 128, S, 0), b0 = kmajor_desc(smem_u32(Bt), N, S, 0);
    const uint32_t id = idesc_bf16(128, N);
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16)
        mma_bf16(d_tmem, desc_step(a0, kmajor_off(128, S, k0)), desc_step(b0, kmajor_off(N, S, k0)), id,
                 k0 > 0 ? 1u : 0u);
}

// D (+)= A[128 x K] * B[N x (b_k0 .. b_k0+K)]^T where B is a K-major row tile
// whose full K extent is b_ktot (its swizzle span follows b_ktot).
__device__ __forceinline__ void issue_mma_koff(uint32_t d_tmem, const uint8_t* A, const uint8_t* Bt, int N, int K,
                                               int b_k0, int b_ktot, bool accumulate) {
    const int Sa = span_of(K), Sb = span_of(b_ktot);
    const uint64_t a0 = kmajor_desc(smem_u32(A), 128, Sa, 0), b0 = kmajor_desc(smem_u32(Bt), N, Sb, 0);
    const uint32_t id = idesc_bf16(128, N);
#pragma unroll
    for (int k0 = 0; k0 < K; k0 += 16)
        mma_bf16(d_tmem, desc_step(a0, kmajor_off(128, Sa, k0)), desc_step(b0, kmajor_off(N, Sb, b_k0 + k0)), id,
                 (accumulate || k0 > 0) ? 1u : 0u);
}

// Thread's CW accumulator columns starting at c0 of TMEM lane 32*q + laneid.
template <int CW>
__device__ __forceinline__ void ld_acc(uint32_t tmem, int q, int c0, float* v) {
#pragma unroll
    for (int i = 0; i < CW / 16; ++i) tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(c0 + 16 * i), v + 16 * i);
    tmem_ld_wait();
}

// FP32 node-row tile loaded by make_f32_tmap boxes (128 rows x BW columns
// each, BW = min(H, 32), swizzled over BW*4 bytes): four floats at (r, c..c+3).
template <int H>
__device__ __forceinline__ float4 ld_f32x4_tile(const uint8_t* tile, int r, int c) {
    constexpr int BW = H < 32 ? H : 32, SB = BW * 4;
    const uint32_t o = (uint32_t)r * SB + (uint32_t)(c % BW) * 4;
    const uint32_t sw = o ^ (((o >> 7) & (uint32_t)(SB / 16 - 1)) << 4);
    return *reinterpret_cast<const float4*>(tile + (uint32_t)(c / BW) * 128 * SB + sw);
}

// Four floats at (r, c..c+3) of an FP32 node-row tile in the layout of
// make_f32_tmap boxes (the store counterpart of ld_f32x4_tile).
template <int H>
__device__ __forceinline__ void st_f32x4_tile(uint8_t* tile, int r, int c, float4 v) {
    constexpr int BW = H < 32 ? H : 32, SB = BW * 4;
    const uint32_t o = (uint32_t)r * SB + (uint32_t)(c % BW) * 4;
    const uint32_t sw = o ^ (((o >> 7) & (uint32_t)(SB / 16 - 1)) << 4);
    *reinterpret_cast<float4*>(tile + (uint32_t)(c / BW) * 128 * SB + sw) = v;
}

// Issue the TMA loads of the FP32 node-row tile starting at row r0 (H/BW boxes).
template <int H>
__device__ __forceinline__ void tma_f32_tile(uint8_t* dst, const CUtensorMap* map, int64_t r0, uint64_t* bar) {
    constexpr int BW = H < 32 ? H : 32;
#pragma unroll
    for (int b = 0; b < H / BW; ++b) tma_load_2d(dst + b * 128 * BW * 4, map, b * BW, (int32_t)r0, bar);
}

// Physical 16-byte chunk of staging chunk c of edge row e (NC chunks of four
// FP32 per row): the rows of one 8-thread shared-memory phase hit distinct banks.
template <int NC>
__device__ __forceinline__ int stage_chunk(int c, int e) {
    constexpr int SH = NC >= 8 ? 0 : (NC == 4 ? 1 : 2);
    constexpr int M = (NC >= 8 ? 8 : NC) - 1;
    return c ^ ((e >> SH) & M);
}

template <int CW>
__device__ __forceinline__ void st_row_tile(uint8_t* tile, int row, int c0, int S, const float* v) {
#pragma unroll
    for (int i = 0; i < CW; i += 8) st_tile8(tile, row, c0 + i, 128, S, v + i);
}

template <int CW>
__device__ __forceinline__ void ld_row_tile(const uint8_t* tile, int row, int c0, int S, float* v) {
#pragma unroll
    for (int i = 0; i < CW; i += 8) ld_tile8(tile, row, c0 + i, 128, S, v + i);
}

// Row mean / rstd of a row split over CG threads (two-pass, FP32), via red[2][CG][128].
template <int H, int CG, int CW>
__device__ __forceinline__ void row_stats(const float* v, float* red, int row, int g, float eps, float& mean,
                                          float& rstd) {
    // one reduction for sum and sum of squares: var = E[v^2] - mean^2 (FP32)
    float s = 0.f, q = 0.f;
#pragma unroll
    for (int i = 0; i < CW; ++i) {
        s += v[i];
        q += v[i] * v[i];
    }
    red[g * 128 + row] = s;
    red[(CG + g) * 128 + row] = q;
    __syncthreads();
    float ts = 0.f, tq = 0.f;
#pragma unroll
    for (int k = 0; k < CG; ++k) {
        ts += red[k * 128 + row];
        tq += red[(CG + k) * 128 + row];
    }
    mean = ts * (1.f / H);
    rstd = rsqrtf(fmaxf(tq * (1.f / H) - mean * mean, 0.f) + eps);
}

// LayerNorm statistics of v and the adjoint sums of d = g * gamma over a row
// split over CG threads, in one exchange through red[4][CG][128]: mean, rstd,
// s1 = (1/H) sum d and s2 = (1/H) sum d * xhat = rstd (sum d v - mean sum d) / H.
template <int H, int CG, int CW>
__device__ __forceinline__ void row_stats_adj_gamma(const float* v, const float* gv, const float* gam, float* red,
                                                    int row, int g, float eps, float& mean, float& rstd, float& s1,
                                                    float& s2) {
    float sv = 0.f, sq = 0.f, sd = 0.f, sdv = 0.f;
#pragma unroll
    for (int i = 0; i < CW; ++i) {
        const float d = gv[i] * gam[i];
        sv += v[i];
        sq += v[i] * v[i];
        sd += d;
        sdv += d * v[i];
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
    __syncthreads();   // red is reused by the caller
    mean = sv * (1.f / H);
    rstd = rsqrtf(fmaxf(sq * (1.f / H) - mean * mean, 0.f) + eps);
    s1 = sd * (1.f / H);
    s2 = rstd * (sdv - mean * sd) * (1.f / H);
}

// Sum of v[0..15] over the 32 lanes of a warp by recursive halving: at each
// step a lane keeps half of its values and adds its partner's copy of that
// half. Lane l returns the total of value (l >> 1); lanes l and l^1 agree.
__device__ __forceinline__ float warp_colsum16(const float* v, int lane) {
    float a[8], b[4], c[2];
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        a[i] = (b4 ? v[i + 8] : v[i]) + __shfl_xor_sync(0xffffffffu, b4 ? v[i] : v[i + 8], 16);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        b[i] = (b3 ? a[i + 4] : a[i]) + __shfl_xor_sync(0xffffffffu, b3 ? a[i] : a[i + 4], 8);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        c[i] = (b2 ? b[i + 2] : b[i]) + __shfl_xor_sync(0xffffffffu, b2 ? b[i] : b[i + 2], 4);
    float d = (b1 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b1 ? c[0] : c[1], 2);
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

// Column sums accumulated per warp by warp_colsum16 (acc[j]: column
// c0 + 16 j + (lane >> 1) over the warp's 32 rows) summed over the four row
// quarters in ascending order into out[0..H); red holds 4*H floats.
template <int H, int NCH>
__device__ __forceinline__ void colsum_store(const float* acc, float* red, int q, int lane, int c0, int tid, int nt,
                                             float* out) {
    __syncthreads();
    if ((lane & 1) == 0) {
#pragma unroll
        for (int j = 0; j < NCH; ++j) red[q * H + c0 + 16 * j + (lane >> 1)] = acc[j];
    }
    __syncthreads();
    for (int c = tid; c < H; c += nt) out[c] = ((red[c] + red[H + c]) + red[2 * H + c]) + red[3 * H + c];
    __syncthreads();
}

// LayerNorm adjoint of one row's CW columns (the thread's share), given the
// statistics of row_stats_adj_gamma: v (the pre-LayerNorm values) is replaced
// by dz = rstd (g gamma - s1 - xhat s2); the column sums of g * xhat, g and
// dz over the warp's rows are added to accG, accB, accZ (one per 16 columns).
// Rows that are not valid contribute zeros.
template <int CW>
__device__ __forceinline__ void ln_adjoint_row(float* v, const float* gv, const float* gam, float mean, float rstd,
                                               float s1, float s2, bool valid, int lane, float* accG, float* accB,
                                               float* accZ) {
#pragma unroll
    for (int j = 0; j < CW / 16; ++j) {
        float t[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = 16 * j + i;
            const float xh = valid ? (v[c] - mean) * rstd : 0.f;
            t[i] = gv[c] * xh;
            v[c] = valid ? rstd * (gv[c] * gam[c] - s1 - xh * s2) : 0.f;
        }
        accG[j] += warp_colsum16(t, lane);
        accB[j] += warp_colsum16(gv + 16 * j, lane);
        accZ[j] += warp_colsum16(v + 16 * j, lane);
    }
}

__device__ __forceinline__ void ld_bf16x8(const __nv_bfloat16* p, float* v) {
    uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    unpack_bf16x2(u.x, v[0], v[1]);
    unpack_bf16x2(u.y, v[2], v[3]);
    unpack_bf16x2(u.z, v[4], v[5]);
    unpack_bf16x2(u.w, v[6], v[7]);
}

__device__ __forceinline__ void st_bf16x8(__nv_bfloat16* p, const float* v) {
    uint4 u;
    u.x = pack_bf16x2(v[0], v[1]);
    u.y = pack_bf16x2(v[2], v[3]);
    u.z = pack_bf16x2(v[4], v[5]);
    u.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(p) = u;
}

// ------------------------------------------------------------------ shared memory plans

struct EdgeFwdSmem {
    uint32_t w, a0, a1, par, seg, red, bar, tm, total;
};

// adj: the backward's recomputation (SAVE mode), whose LayerNorm adjoint
// exchanges four row sums instead of two.
template <int H>
__host__ __device__ inline EdgeFwdSmem edge_fwd_smem(int n_lin, bool adj = false) {
    using C = Cfg<H>;
    EdgeFwdSmem s;
    s.w = 0;
    s.a0 = align_up(s.w + n_lin * C::WT, 1024);
    s.a1 = s.a0 + C::TILE;
    s.par = align_up(s.a1 + C::TILE, 16);
    s.seg = align_up(s.par + (n_lin + 2) * H * 4, 128);   // two tile records (GNN_TILE_META_BYTES each)
    s.red = s.seg + 2 * GNN_TILE_META_BYTES;
    s.bar = align_up(s.red + (adj ? 4 : 2) * C::CG * 128 * 4, 8);   // record/rows landed, MMA done
    s.tm = s.bar + 16;
    s.total = s.tm + 16 + 1024;      // + slack for 1024-byte alignment of the base
    return s;
}

struct NodeFwdSmem {
    uint32_t w0, w, a0, a1, par, red, xs, bar, tm, total;
};

// Node-forward input staging (PF): two stages of the FP32 [a* | x] rows of a
// tile ([128 x H] each), loaded by TMA one tile ahead; used when they fit.

// H = 128 streams the [a*, x] input through one [128 x H] buffer in two K
// halves (the whole 2H-wide tile would not fit next to the weights).
template <int H>
struct NodeSplit {
    static constexpr bool value = H >= 128;
};

template <int H, bool PF = false>
__host__ __device__ inline NodeFwdSmem node_fwd_smem(int n_lin, bool adj = false) {
    using C = Cfg<H>;
    constexpr bool split = NodeSplit<H>::value;
    NodeFwdSmem s;
    s.w0 = 0;                                         // W1 of the node MLP: [H x 2H]
    s.w = align_up(s.w0 + 2 * C::WT, 1024);           // W2.. : (n_lin-1) x [H x H]
    s.a0 = align_up(s.w + (n_lin - 1) * C::WT, 1024); // [128 x 2H] input tile (or [128 x H] when split)
    s.a1 = split ? s.a0 : s.a0 + 2 * C::TILE;          // split: the chain reuses the input buffer
    s.par = align_up(s.a1 + C::TILE, 16);
    s.red = s.par + (n_lin + 2) * H * 4;
    s.xs = align_up(s.red + (adj ? 4 : 2) * C::CG * 128 * 4, 1024);
    s.bar = align_up(s.xs + (PF ? 2 * 2 * 128 * H * 4 : 0), 8);   // mma, full[2]
    s.tm = s.bar + 24;
    s.total = s.tm + 16 + 1024;
    return s;
}

struct ProjSmem {
    uint32_t w, a, x, bar, tm, total;
};

template <int H>
__host__ __device__ inline ProjSmem proj_smem() {
    using C = Cfg<H>;
    ProjSmem s;
    s.w = 0;                                          // [2H x H]: W1a rows then W1b rows
    s.a = align_up(s.w + 2 * C::WT, 1024);
    s.x = align_up(s.a + C::TILE, 1024);              // 2 stages of FP32 x rows [128 x H]
    s.bar = align_up(s.x + 2 * 128 * H * 4, 8);       // full[2], mma
    s.tm = s.bar + 24;
    s.total = s.tm + 16 + 1024;
    return s;
}

__device__ __forceinline__ uint8_t* aligned_smem(uint8_t* raw) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
}


// ------------------------------------------------------------------ host helpers

namespace host {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map over a [rows x H] BF16 row-major matrix, box = 128 rows x one swizzle span.
inline int make_row_tmap(CUtensorMap* m, const void* base, int64_t rows, int H) {
    EncodeTiledFn enc = encode_fn();
    GNN_REQUIRE(enc, GNN_ECUDA, "cuTensorMapEncodeTiled is not available");
    GNN_REQUIRE(((uintptr_t)base & 15) == 0, GNN_EINVAL, "edge buffer must be 16-byte aligned for TMA");
    const int S = span_of(H);
    cuuint64_t dims[2] = {(cuuint64_t)H, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)H * 2};
    cuuint32_t box[2] = {(cuuint32_t)(S / 2), 128};
    cuuint32_t estr[2] = {1, 1};
    CUtensorMapSwizzle sw = S == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                     : (S == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    GNN_REQUIRE(r == CUDA_SUCCESS, GNN_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GNN_OK;
}

// Tensor map over a [rows x H] FP32 row-major matrix for node-row tiles:
// box = 128 rows x min(H, 32) columns, swizzled over the box width (128 or
// 64 bytes), so that one thread per row reads its columns without bank
// conflicts (ld_f32x4_tile).
inline int make_f32_tmap(CUtensorMap* m, const void* base, int64_t rows, int H) {
    EncodeTiledFn enc = encode_fn();
    GNN_REQUIRE(enc, GNN_ECUDA, "cuTensorMapEncodeTiled is not available");
    GNN_REQUIRE(((uintptr_t)base & 15) == 0, GNN_EINVAL, "node buffer must be 16-byte aligned for TMA");
    const int bw = H < 32 ? H : 32;
    cuuint64_t dims[2] = {(cuuint64_t)H, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)H * 4};
    cuuint32_t box[2] = {(cuuint32_t)bw, 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, bw == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    GNN_REQUIRE(r == CUDA_SUCCESS, GNN_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GNN_OK;
}

inline int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

// Persistent grid: resident CTAs (by shared memory / registers and by TMEM
// columns) times SMs, capped by the number of tiles.
template <class K>
int persistent_grid(K kernel, int threads, uint32_t smem, uint32_t tmem_cols, int64_t tiles, int* out,
                    int max_per_sm = 0) {
    GNN_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "cudaFuncSetAttribute");
    GNN_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared),
                   "cudaFuncSetAttribute(carveout)");
    int per_sm = 0;
    GNN_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem),
                   "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    GNN_REQUIRE(per_sm >= 1, GNN_EUNSUPPORTED, "fused kernel does not fit on an SM (smem %u)", smem);
    per_sm = std::min<int>(per_sm, (int)(512 / tmem_cols));
    if (max_per_sm > 0) per_sm = std::min(per_sm, max_per_sm);
    *out = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)per_sm * num_sms()));
    return GNN_OK;
}

inline MlpDev mlp_dev(const gnn_mlp& P) {
    MlpDev d;
    for (int k = 0; k < GNN_MAX_LIN; ++k) {
        d.W[k] = k < P.n_lin ? P.W[k] : nullptr;
        d.b[k] = k < P.n_lin ? P.b[k] : nullptr;
    }
    d.gamma = P.gamma;
    d.beta = P.beta;
    d.n_lin = P.n_lin;
    return d;
}

}  // namespace host

}  // namespace fused
}  // namespace gnn
