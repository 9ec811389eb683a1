// Layered BF16 backward of the consistent NMP layer at H = 128 (Eq. 3 with
// per-layer recomputation of the MLP activations).
//
// At H = 128 one SM cannot hold the single-kernel edge adjoint of the smaller
// widths: every 128 x 128 FP32 weight-gradient accumulator takes a quarter of
// TMEM and every BF16 activation tile 32 KB of shared memory. The adjoint
// therefore runs one Linear at a time over tiles of 128 rows, with the
// recomputed activations in an HBM scratch of tile-padded rows (the rows past
// a tile's end are zero, so they add nothing to any product or sum):
//   k_node_fwd<128, false, true> / k_edge_save_tm   (forward units)
//       recompute the MLP, save h_0 .. h_{L-2} (and a node tile's BF16
//       [a*, x] rows), apply the LayerNorm adjoint: dz_{L-1}, dgamma,
//       db_{L-1}, and (nodes) dbeta
//   k_bwd_chain2 / k_bwd_chain, k = L-1 .. 1, two Linears per pass while two remain
//       dh_{k-1} = dz_k W_k, dz_{k-1} = dh_{k-1} ELU'(h_{k-1}),
//       dW_k += dz_k^T h_{k-1} (TMEM, over the CTA's tiles), db_{k-1}
//   k_bwd_node0   [da*, dx] = dz_0 W_0, dW_0 += dz_0^T [a*, x], dx_in = dx' + dx
//   k_halo        adjoint of Eq. 5c-5d on da*
//   k_bwd_edge0   de_in = g + dz_0 W1c with g = de' + da_i / d_ij, dW1c += dz_0^T e,
//                 dbeta (the column sums of g), dz_0 per edge and its sum over each
//                 receiver's edges (dP)
//   k_bwd_chain_edge0   the edge MLP's Linear 1 and k_bwd_edge0 in one pass, when
//                 the pairs leave Linear 1 alone (dz_0 stays in shared memory)
//   k_proj_bwd    dQ, dx_in += dP W1a + dQ W1b, dW1a, dW1b
// Tiles are processed in chunks of at most kChunkTiles (fewer when the
// caller's workspace is smaller) so that the scratch stays bounded; each
// kernel's per-CTA partials are summed (CTA order) into dW right after it, so
// every gradient has a fixed summation order.

#include <algorithm>

#include "fused.h"
#include "fused_bwd_common.cuh"
#include "plain.h"
#include "profiler.h"

namespace gnn {
namespace fused {

cudaError_t take_device_error_bwd128(unsigned int* out) { return take_device_error_word(out); }

namespace {

constexpr int H128 = 128;
constexpr int kTile = 128 * H128 * 2;        // [128 x 128] BF16 row tile
constexpr int kS = 128;                       // swizzle span of a 128-wide BF16 tile
constexpr int64_t kChunkTiles = 32768;        // tiles per scratch chunk
constexpr int64_t kPstride = 2 * H128 * H128 + 2 * H128;   // per-CTA partial floats (largest: k_bwd_chain2)

// ------------------------------------------------------------------ k_bwd_chain

struct ChainArgs {
    const float* W;              // W_k [H x H] (FP32)
    __nv_bfloat16* dz_out;       // dz_{k-1} rows (tile-padded)
    int64_t n_tiles;
    float* part;                 // per-CTA: dW_k [H x H], then db_{k-1} [H]
    int64_t pstride;
    float* dx;                   // INPUT: dX rows [n_rows x H] (FP32); scratch row i is row row0 + i
    int64_t row0, n_rows;
};

// One CTA per SM, 128 rows x 4 column groups of 32 columns. Three stages of
// {dz_k rows, h_{k-1} rows} keep two tiles' loads in flight, and two TMEM
// accumulators let thread 0 issue tile j+1's MMAs while the block runs tile
// j's epilogue (the weight gradient accumulates in a third region).
// INPUT: the first Linear of a row MLP whose input X is no activation: h_{k-1}
// is the BF16 copy of X, and the epilogue writes dX = dz_0 W_0 in FP32 instead
// of an ELU adjoint (no bias gradient).
constexpr int kChainNT = 512;
constexpr int kChainNS = 3;
struct ChainSmem {
    static constexpr uint32_t w = 0, st = kTile;                      // stage s: dz, then h, at st + s * 2 * kTile
    static constexpr uint32_t red = st;                               // 4 x H floats, after the tile loop
    static constexpr uint32_t bar = st + kChainNS * 2 * kTile;        // full[NS], done_d[2], done_w[2], TMEM slot
    static constexpr uint32_t total = bar + 64 + 1024;
};
static_assert(ChainSmem::total <= 227 * 1024, "k_bwd_chain shared memory");

template <bool INPUT>
__global__ void __launch_bounds__(kChainNT, 1) k_bwd_chain(const __grid_constant__ CUtensorMap tm_dz,
                                                          const __grid_constant__ CUtensorMap tm_h, ChainArgs A) {
    constexpr int H = H128, S = kS, CG = 4, CW = 32, NT = kChainNT, NCH = CW / 16, NS = kChainNS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    uint8_t* sW = sm + ChainSmem::w;
    float* sRed = reinterpret_cast<float*>(sm + ChainSmem::red);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + ChainSmem::bar);   // full[NS]: stage loaded
    uint64_t* done_d = full + NS;     // done_d[b]: dgrad into accumulator b complete
    uint64_t* done_w = done_d + 2;    // done_w[b]: that tile's wgrad complete (its stage is free)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done_w + 2);
    auto sDz = [&](int s) { return sm + ChainSmem::st + s * 2 * kTile; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;
    if (warp == 0) {
        tmem_alloc(tslot, 4 * H);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(full + i, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(done_d + i, 1);
            mbar_init(done_w + i, 1);
        }
        fence_mbar_init();
    }
    load_weight(sW, A.W, H, 0, H, H, tid, NT);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot, tDW = tmem + 2 * H;
    auto tWork = [&](int b) { return tmem + (uint32_t)(b * H); };
    const int64_t n_mine = A.n_tiles > (int64_t)blockIdx.x
                               ? (A.n_tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](int64_t j) { return (int64_t)blockIdx.x + j * gridDim.x; };
    // thread 0 only: loads issued / MMAs issued so far, and whether it is still well
    int64_t n_ld = 0, n_mma = 0;
    bool ok0 = true;
    auto issue_load = [&]() {   // next tile of this CTA into stage n_ld % NS
        const int s = (int)(n_ld % NS);
        const int32_t y = (int32_t)(tile_of(n_ld) * 128);
        mbar_arrive_expect_tx(full + s, 2 * kTile);
        for (int kb = 0; kb < 2; ++kb) {
            tma_load_2d(sDz(s) + kb * 128 * S, &tm_dz, kb * 64, y, full + s);
            tma_load_2d(sDz(s) + kTile + kb * 128 * S, &tm_h, kb * 64, y, full + s);
        }
        ++n_ld;
    };
    auto issue_mma = [&]() {    // MMAs of tile n_mma once its stage has landed
        const int s = (int)(n_mma % NS), b = (int)(n_mma & 1);
        ok0 = ok0 && mbar_wait(full + s, (uint32_t)(n_mma / NS) & 1u);
        if (!ok0) return;
        tc_fence_after();
        issue_dgrad(tWork(b), sDz(s), S, sW, S, H, (uint32_t)H * S, H, H);
        mma_commit(done_d + b);
        issue_wgrad(tDW, sDz(s), S, 128u * S, sDz(s) + kTile, S, 128u * S, H, n_mma > 0);
        mma_commit(done_w + b);
        ++n_mma;
    };
    if (tid == 0) {
        while (n_ld < n_mine && n_ld < NS) issue_load();
        if (n_mine > 0) issue_mma();
    }
    float acc[NCH];
#pragma unroll
    for (int j = 0; j < NCH; ++j) acc[j] = 0.f;
    bool ok = true;

    for (int64_t j = 0; j < n_mine; ++j) {
        const int s = (int)(j % NS), b = (int)(j & 1);
        const uint32_t par = (uint32_t)(j >> 1) & 1u;
        // tile j+1's MMAs run during this epilogue (its accumulator was read in iteration j-1)
        if (tid == 0 && j + 1 < n_mine) issue_mma();
        ok = ok && mbar_wait(done_d + b, par);
        __syncwarp();
        tc_fence_after();
        const int64_t t = tile_of(j);
        if constexpr (INPUT) {
            const int64_t gr = A.row0 + t * 128 + row;
#pragma unroll
            for (int jj = 0; jj < NCH; ++jj) {
                float dh[16];
                tmem_ld16(tWork(b) + ((uint32_t)(32 * q) << 16) + (uint32_t)(c0 + 16 * jj), dh);
                tmem_ld_wait();
                if (A.dx && gr < A.n_rows) {
                    float4* d4 = reinterpret_cast<float4*>(A.dx + gr * H + c0 + 16 * jj);
#pragma unroll
                    for (int i = 0; i < 4; ++i) d4[i] = make_float4(dh[4 * i], dh[4 * i + 1], dh[4 * i + 2], dh[4 * i + 3]);
                }
            }
        } else {
            __nv_bfloat16* zrow = A.dz_out + (t * 128 + row) * H + c0;
            const uint8_t* hT = sDz(s) + kTile;
#pragma unroll
            for (int jj = 0; jj < NCH; ++jj) {
                float dh[16], hv[16];
                tmem_ld16(tWork(b) + ((uint32_t)(32 * q) << 16) + (uint32_t)(c0 + 16 * jj), dh);
                ld_tile8(hT, row, c0 + 16 * jj, 128, S, hv);
                ld_tile8(hT, row, c0 + 16 * jj + 8, 128, S, hv + 8);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) dh[i] = elu1_bwd_from_out(dh[i], hv[i]);
                st_bf16x8(zrow + 16 * jj, dh);
                st_bf16x8(zrow + 16 * jj + 8, dh + 8);
                acc[jj] += warp_colsum16(dh, lane);
            }
        }
        tc_fence_before();
        fence_proxy_async();
        __syncwarp();   // reconverged before the aligned block barrier
        ok = __syncthreads_and(ok && (tid != 0 || ok0)) != 0;   // every thread is past its reads of stage s
        if (!ok) break;
        if (tid == 0) {   // stage s is free once tile j's wgrad is done: the CTA's tile j+NS goes there
            ok0 = mbar_wait(done_w + b, par);
            if (ok0 && n_ld < n_mine) issue_load();
        }
    }
    if (tid == 0) {   // bounded waits for what this CTA started and nobody waited for
        if (n_mma > 0) mbar_wait(done_w + ((n_mma - 1) & 1), (uint32_t)((n_mma - 1) >> 1) & 1u);
        for (int64_t i = n_mma; i < n_ld; ++i) mbar_wait(full + (i % NS), (uint32_t)(i / NS) & 1u);
    }
    __syncwarp();   // reconverged before the aligned block barrier
    ok = __syncthreads_and(ok && (tid != 0 || ok0)) != 0;
    tc_fence_after();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (ok) {
        if (n_mine > 0) flush_acc<CG>(tDW, H, H, q, lane, g, part);
        else
            for (int i = tid; i < H * H; i += NT) part[i] = 0.f;
    }
    if constexpr (!INPUT) colsum_store<H, NCH>(acc, sRed, q, lane, c0, tid, NT, part + H * H);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 4 * H);
}

// ------------------------------------------------------------------ k_bwd_chain2
//
// Two consecutive Linears k and k-1 of the per-Linear adjoint in one pass, so
// that dz_{k-1} never travels through HBM: per tile, MMA pair 1 (D1 = dz_k W_k,
// dW_k += dz_k^T h_{k-1}), epilogue 1 (dz_{k-1} = D1 ELU'(h_{k-1}) as BF16 into
// the shared-memory slot dz_k came in, which pair 1 has finished reading, and
// its column sums), MMA pair 2 (D2 = dz_{k-1} W_{k-1}, dW_{k-1} += dz_{k-1}^T
// h_{k-2}), epilogue 2 (dz_{k-2} = D2 ELU'(h_{k-2}), its column sums, staged in
// the stage's h_{k-1} slot and written to HBM as whole rows by a TMA store).
// The operands and roundings are those of two k_bwd_chain passes, so the
// results are the same bit for bit. TMEM: D1, D2, dW_k, dW_{k-1} (128 columns
// each). Two stages of {dz_k, h_{k-1}} rows; h_{k-2} has one stage, reloaded as
// soon as epilogue 2 has read it into registers and pair 2's weight gradient
// has read it.
// The two epilogues run on two warp groups, so that epilogue 2 of tile j runs
// beside epilogue 1 of tile j + 1: group X (warps 0-7) waits for pair 1, writes
// dz_{k-1}, tells group Y's leader through an mbarrier (zr) that the stage is
// ready for pair 2 and no longer read by X, and issues the next tile's pair 1;
// group Y (warps 8-15) issues pair 2, runs epilogue 2, reloads h_{k-2} and,
// after the TMA store of dz_{k-2}, the stage. Each warp covers 64 columns of
// its 32 rows (TMEM lane quarter).

struct Chain2Args {
    const float* Wa;             // W_k [H x H] (FP32)
    const float* Wb;             // W_{k-1}
    const __nv_bfloat16* hb;     // h_{k-2} rows (prefetched into L2 two tiles ahead)
    int64_t n_tiles;             // dz_{k-2} leaves through the tm_out tensor map (tile-padded rows)
    float* part;                 // per-CTA: dW_k, dW_{k-1} [H x H], then db_{k-1}, db_{k-2} [H]
    int64_t pstride;
};

constexpr int kC2NT = 512;
struct Chain2Smem {
    static constexpr uint32_t wa = 0, wb = kTile;
    static constexpr uint32_t a = 2 * kTile;          // stage s: dz_k (then dz_{k-1}), h_{k-1} (then dz_{k-2}), at a + s * 2 * kTile
    static constexpr uint32_t b = a + 4 * kTile;      // h_{k-2}
    static constexpr uint32_t red = a;                // 8 x H floats, after the tile loop
    static constexpr uint32_t bar = b + kTile;        // fullA[2], fullB, c1, c2d, c2w, zr[2], hbf, n1, TMEM slot
    static constexpr uint32_t total = bar + 128 + 1024;
};
static_assert(Chain2Smem::total <= 227 * 1024, "k_bwd_chain2 shared memory");

// One warp group's named barrier (X: 1, Y: 2; 256 threads), AND-ing a predicate.
__device__ __forceinline__ bool wg_and(bool v, bool isX) { return named_and(v, isX ? 1 : 2, 256); }

__global__ void __launch_bounds__(kC2NT, 1) k_bwd_chain2(const __grid_constant__ CUtensorMap tm_dz,
                                                         const __grid_constant__ CUtensorMap tm_ha,
                                                         const __grid_constant__ CUtensorMap tm_hb,
                                                         const __grid_constant__ CUtensorMap tm_out, Chain2Args A) {
    constexpr int H = H128, S = kS, CG = 4, CW = 64, NT = kC2NT, NCH = CW / 16, GT = 256;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    uint8_t* sWa = sm + Chain2Smem::wa;
    uint8_t* sWb = sm + Chain2Smem::wb;
    uint8_t* sHb = sm + Chain2Smem::b;
    float* sRed = reinterpret_cast<float*>(sm + Chain2Smem::red);
    uint64_t* fullA = reinterpret_cast<uint64_t*>(sm + Chain2Smem::bar);   // fullA[2]: stage landed
    uint64_t* fullB = fullA + 2;   // h_{k-2} landed
    uint64_t* c1 = fullA + 3;      // MMA pair 1 complete
    uint64_t* c2d = fullA + 4;     // pair 2's dgrad complete
    uint64_t* c2w = fullA + 5;     // pair 2's wgrad complete
    uint64_t* zr = fullA + 6;      // zr[j % 2]: group X has written tile j's dz_{k-1} and is done with its stage
    uint64_t* hbf = fullA + 8;     // every group-Y thread has read the tile's h_{k-2} (256 arrivals)
    int64_t* sN1 = reinterpret_cast<int64_t*>(fullA + 9);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fullA + 10);
    auto sDz = [&](int st) { return sm + Chain2Smem::a + st * 2 * kTile; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool isX = warp < 8;
    const int q = warp & 3, row = 32 * q + lane, c0 = 64 * ((warp >> 2) & 1), gt = tid & (GT - 1);
    const bool leader = gt == 0;   // X: thread 0, Y: thread 256
    if (warp == 0) {
        tmem_alloc(tslot, 4 * H);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 8; ++i) mbar_init(fullA + i, 1);
        mbar_init(hbf, GT);
        fence_mbar_init();
    }
    load_weight(sWa, A.Wa, H, 0, H, H, tid, NT);
    load_weight(sWb, A.Wb, H, 0, H, H, tid, NT);
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot, tD1 = tmem, tD2 = tmem + H, tWa = tmem + 2 * H, tWb = tmem + 3 * H;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const int64_t n_mine = A.n_tiles > (int64_t)blockIdx.x
                               ? (A.n_tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](int64_t j) { return (int64_t)blockIdx.x + j * gridDim.x; };
    // leaders only: X issues pair 1 (n1); Y issues the loads (nA, nB), pair 2 (n2) and the stores
    int64_t nA = 0, nB = 0, n1 = 0, n2 = 0;
    bool ok0 = true;
    auto issue_A = [&]() {   // dz_k and h_{k-1} rows of tile nA into stage nA % 2 (and its h_{k-2} into L2)
        const int st = (int)(nA & 1);
        const int32_t y = (int32_t)(tile_of(nA) * 128);
        mbar_arrive_expect_tx(fullA + st, 2 * kTile);
        for (int kb = 0; kb < 2; ++kb) {
            tma_load_2d(sDz(st) + kb * 128 * S, &tm_dz, kb * 64, y, fullA + st);
            tma_load_2d(sDz(st) + kTile + kb * 128 * S, &tm_ha, kb * 64, y, fullA + st);
        }
        prefetch_l2(A.hb + (int64_t)y * H, kTile);
        ++nA;
    };
    auto issue_B = [&]() {   // h_{k-2} rows of tile nB
        const int32_t y = (int32_t)(tile_of(nB) * 128);
        mbar_arrive_expect_tx(fullB, kTile);
        for (int kb = 0; kb < 2; ++kb) tma_load_2d(sHb + kb * 128 * S, &tm_hb, kb * 64, y, fullB);
        ++nB;
    };
    auto issue_pair1 = [&]() {   // tile n1's first MMA pair once its stage has landed
        const int st = (int)(n1 & 1);
        ok0 = ok0 && mbar_wait(fullA + st, (uint32_t)(n1 >> 1) & 1u);
        if (!ok0) return;
        tc_fence_after();
        issue_dgrad(tD1, sDz(st), S, sWa, S, H, (uint32_t)H * S, H, H);
        issue_wgrad(tWa, sDz(st), S, 128u * S, sDz(st) + kTile, S, 128u * S, H, n1 > 0);
        mma_commit(c1);
        ++n1;
    };
    if (tid == 256 && n_mine > 0) {
        while (nA < n_mine && nA < 2) issue_A();
        issue_B();
    }
    if (tid == 0 && n_mine > 0) issue_pair1();
    float acc[NCH];   // X: column sums of dz_{k-1} (db_{k-1}); Y: of dz_{k-2} (db_{k-2})
#pragma unroll
    for (int j = 0; j < NCH; ++j) acc[j] = 0.f;
    bool ok = true;

    if (isX) {
        for (int64_t j = 0; j < n_mine; ++j) {
            const int st = (int)(j & 1);
            const uint32_t par = (uint32_t)j & 1u;   // c1 completes once per tile
            // epilogue 1: dz_{k-1} into the dz_k slot of the stage, column sums for db_{k-1}
            ok = wg_and(leader ? mbar_wait(c1, par) : true, true);
            if (!ok) break;
            tc_fence_after();
            uint8_t* z = sDz(st);
            const uint8_t* hT = z + kTile;
#pragma unroll
            for (int jj = 0; jj < NCH; ++jj) {
                float dh[16], hv[16];
                tmem_ld16(tD1 + lane_base + (uint32_t)(c0 + 16 * jj), dh);
                ld_tile8(hT, row, c0 + 16 * jj, 128, S, hv);
                ld_tile8(hT, row, c0 + 16 * jj + 8, 128, S, hv + 8);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) dh[i] = elu1_bwd_from_out(dh[i], hv[i]);
                st_tile8(z, row, c0 + 16 * jj, 128, S, dh);
                st_tile8(z, row, c0 + 16 * jj + 8, 128, S, dh + 8);
                acc[jj] += warp_colsum16(dh, lane);
            }
            tc_fence_before();
            fence_proxy_async();
            ok = wg_and(!leader || ok0, true);   // every X thread is done with the stage
            if (!ok) break;
            if (leader) {   // dz_{k-1} is in place for pair 2; then the next tile's pair 1 (D1 has been read)
                mbar_arrive(zr + st);
                if (j + 1 < n_mine) issue_pair1();
            }
        }
        if (leader) *sN1 = n1;
    } else {
        for (int64_t j = 0; j < n_mine; ++j) {
            const int st = (int)(j & 1);
            const uint32_t par = (uint32_t)j & 1u;   // fullB, c2d, c2w complete once per tile
            if (leader) {   // pair 2 once group X has written dz_{k-1} and h_{k-2} has landed (zr alternates
                            // between two barriers, so group X, at most two tiles ahead, cannot alias a phase)
                ok0 = ok0 && mbar_wait(zr + st, (uint32_t)(j >> 1) & 1u) && mbar_wait(fullB, par);
                if (ok0) {
                    tc_fence_after();
                    uint8_t* z = sDz(st);
                    issue_dgrad(tD2, z, S, sWb, S, H, (uint32_t)H * S, H, H);
                    mma_commit(c2d);
                    issue_wgrad(tWb, z, S, 128u * S, sHb, S, 128u * S, H, n2 > 0);
                    mma_commit(c2w);
                    ++n2;
                }
            }
            ok = wg_and(leader ? (ok0 && mbar_wait(c2d, par)) : true, false);
            if (!ok) break;
            tc_fence_after();
            // this thread's h_{k-2} (64 columns, BF16 pairs), read before h_{k-2} is reloaded. The
            // reads are released through an mbarrier that the leader acquires before the TMA
            // reload: a block barrier does not order loads still in flight against the async
            // proxy's writes (measured: with one, some rows took the next tile's h_{k-2})
            uint4 hbw[CW / 8];
#pragma unroll
            for (int i = 0; i < CW / 8; ++i)
                hbw[i] = *reinterpret_cast<const uint4*>(sHb + tile_off(row, c0 + 8 * i, 128, S));
            fence_proxy_async();
            mbar_arrive(hbf);
            if (leader) {   // every Y thread has read h_{k-2} and the wgrad of pair 2 has too: the next tile's
                ok0 = ok0 && mbar_wait(hbf, par) && mbar_wait(c2w, par);
                if (ok0 && nB < n_mine) issue_B();
            }
            __syncwarp();   // the leader's warp reconverged before the aligned TMEM loads
            // epilogue 2: dz_{k-2} staged in the stage's h_{k-1} slot (pair 1 and group X have read it)
            uint8_t* zt = sDz(st) + kTile;
#pragma unroll
            for (int jj = 0; jj < NCH; ++jj) {
                float dh[16], hv[16];
                tmem_ld16(tD2 + lane_base + (uint32_t)(c0 + 16 * jj), dh);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const uint4 u = hbw[2 * jj + i];
                    unpack_bf16x2(u.x, hv[8 * i], hv[8 * i + 1]);
                    unpack_bf16x2(u.y, hv[8 * i + 2], hv[8 * i + 3]);
                    unpack_bf16x2(u.z, hv[8 * i + 4], hv[8 * i + 5]);
                    unpack_bf16x2(u.w, hv[8 * i + 6], hv[8 * i + 7]);
                }
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) dh[i] = elu1_bwd_from_out(dh[i], hv[i]);
                st_tile8(zt, row, c0 + 16 * jj, 128, S, dh);
                st_tile8(zt, row, c0 + 16 * jj + 8, 128, S, dh + 8);
                acc[jj] += warp_colsum16(dh, lane);
            }
            tc_fence_before();
            fence_proxy_async();   // the staged rows precede their TMA store and the stage's refill
            ok = wg_and(!leader || ok0, false);   // D2 read, dz_{k-2} staged
            if (!ok) break;
            if (leader) {   // dz_{k-2} leaves as whole rows; tile j + 2 into stage st once the store has read it
#pragma unroll
                for (int kb = 0; kb < 2; ++kb)
                    tma_store_2d(&tm_out, kb * 64, (int32_t)(tile_of(j) * 128), zt + kb * 128 * S);
                bulk_commit();
                if (nA < n_mine) {
                    bulk_wait_read_all();
                    issue_A();
                }
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (tid == 256) {   // bounded waits for what this CTA started and nobody waited for
        const int64_t m1 = *sN1;
        if (m1 > 0) mbar_wait(c1, (uint32_t)(m1 - 1) & 1u);
        if (n2 > 0) {
            mbar_wait(c2d, (uint32_t)(n2 - 1) & 1u);
            mbar_wait(c2w, (uint32_t)(n2 - 1) & 1u);
        }
        for (int64_t i = m1; i < nA; ++i) mbar_wait(fullA + (i & 1), (uint32_t)(i >> 1) & 1u);
        for (int64_t i = n2; i < nB; ++i) mbar_wait(fullB, (uint32_t)i & 1u);
        bulk_wait_all();   // the stored dz rows are written
    }
    __syncwarp();
    const bool all_ok = __syncthreads_and(ok && (!leader || ok0)) != 0;
    tc_fence_after();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (all_ok) {
        if (n_mine > 0) {
            flush_acc<CG>(tWa, H, H, q, lane, warp >> 2, part);
            flush_acc<CG>(tWb, H, H, q, lane, warp >> 2, part + H * H);
        } else {
            for (int i = tid; i < 2 * H * H; i += NT) part[i] = 0.f;
        }
    }
    // column sums: warp (q, half) of a group holds columns c0 + 16 j + (lane >> 1) over its 32 rows;
    // the four row quarters are added in order, db_{k-1} from group X, db_{k-2} from group Y
    __syncthreads();
    if ((lane & 1) == 0) {
#pragma unroll
        for (int jj = 0; jj < NCH; ++jj) sRed[(isX ? 0 : 4 * H) + q * H + c0 + 16 * jj + (lane >> 1)] = acc[jj];
    }
    __syncthreads();
    for (int c = tid; c < 2 * H; c += NT) {
        const float* r = sRed + (c < H ? 0 : 4 * H) + (c % H);
        part[2 * H * H + c] = ((r[0] + r[H]) + r[2 * H]) + r[3 * H];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 4 * H);
}

// ------------------------------------------------------------------ k_bwd_edge0

// The gradient of e' from the edge's side of Eq. 5b and the upstream gradient:
// g = de' + w da_i (w = 1/d_ij), one rounding.
__device__ __forceinline__ float edge_g(float w, float da, float de) { return __fmaf_rn(w, da, de); }

struct Edge0Args {
    const uint8_t* tile_meta;    // per-tile records (GNN_TILE_META_BYTES each)
    int64_t t0, t1;              // tile range; the scratch rows of tile t start at (t - t0) * 128
    const float* W1;             // W1 [H x 3H]; W1c = columns 2H .. 3H
    const __nv_bfloat16* de_out; // NULL: zero
    const float* da;             // aggregate gradient after the halo adjoint
    __nv_bfloat16* de_in;
    __nv_bfloat16* dz1;          // per-edge dz_0 [E x H]
    float* dP;                   // [n_rows x H]
    float* part;                 // per-CTA: dW1c [H x H]
    int64_t pstride;
};

// 128 rows x 4 column groups of 32 columns, one CTA per SM, two stages of
// {tile record, dz_0 rows, e rows}.
constexpr int kE0NT = 512;
struct Edge0Smem {
    static constexpr uint32_t w = 0, st = kTile;          // stage s: dz tile, then e tile, at st + s * 2 * kTile
    static constexpr uint32_t rec = st + 4 * kTile;       // stage s: record at rec + s * GNN_TILE_META_BYTES
    static constexpr uint32_t bar = rec + 2 * GNN_TILE_META_BYTES;
    static constexpr uint32_t total = bar + 64 + 1024;
};

__global__ void __launch_bounds__(kE0NT, 1) k_bwd_edge0(const __grid_constant__ CUtensorMap tm_dz,
                                                       const __grid_constant__ CUtensorMap tm_e, Edge0Args A) {
    constexpr int H = H128, S = kS, CG = 4, CW = 32, NT = kE0NT, NCH = CW / 16;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    uint8_t* sW = sm + Edge0Smem::w;
    float* sRed = reinterpret_cast<float*>(sm + Edge0Smem::st);   // 4 x H floats, after the tile loop
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + Edge0Smem::bar);   // full[2]
    uint64_t* bar = full + 2;     // dgrad done
    uint64_t* bar_w = full + 3;   // wgrad done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 4);
    auto sDz = [&](int s) { return sm + Edge0Smem::st + s * 2 * kTile; };
    auto sRec = [&](int s) { return sm + Edge0Smem::rec + s * GNN_TILE_META_BYTES; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;
    if (warp == 0) {
        tmem_alloc(tslot, 2 * H);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(full, 1);
        mbar_init(full + 1, 1);
        mbar_init(bar, 1);
        mbar_init(bar_w, 1);
        fence_mbar_init();
    }
    load_weight(sW, A.W1, 3 * H, 2 * H, H, H, tid, NT);   // W1c as a K-major [H x H] tile
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot, tWork = tmem, tDW = tmem + H;
    int64_t n_issued = 0;   // thread 0: loads issued (stage i & 1, phase (i >> 1) & 1)
    auto tile_hdr = [&](int64_t t) { return ld_nc_v4s32(A.tile_meta + t * GNN_TILE_META_BYTES); };
    int4 hdr_next = make_int4(0, 0, 0, 0);   // thread 0: the next tile's header, read one tile ahead
    auto issue = [&](int s, int64_t t, int32_t e0) {   // thread 0: record, dz_0 rows and e rows of tile t
        ++n_issued;
        mbar_arrive_expect_tx(full + s, 2 * kTile + GNN_TILE_META_BYTES);
        bulk_load(sRec(s), A.tile_meta + t * GNN_TILE_META_BYTES, GNN_TILE_META_BYTES, full + s);
        for (int kb = 0; kb < 2; ++kb) {
            tma_load_2d(sDz(s) + kb * 128 * S, &tm_dz, kb * 64, (int32_t)((t - A.t0) * 128), full + s);
            tma_load_2d(sDz(s) + kTile + kb * 128 * S, &tm_e, kb * 64, e0, full + s);
        }
    };
    const int64_t tfirst = A.t0 + blockIdx.x;
    if (tid == 0 && tfirst < A.t1) {
        issue(0, tfirst, tile_hdr(tfirst).z);
        if (tfirst + gridDim.x < A.t1) hdr_next = tile_hdr(tfirst + gridDim.x);
    }
    uint32_t ph = 0;
    bool ok = true, first = true, mp = false;
    int j = 0;
    int64_t n_consumed = 0;
    float accb[NCH];   // column sums of g: the LayerNorm beta gradient
#pragma unroll
    for (int jj = 0; jj < NCH; ++jj) accb[jj] = 0.f;

    for (int64_t t = tfirst; t < A.t1; t += gridDim.x, ++j) {
        const int st = j & 1;
        ok = block_wait(full + st, (uint32_t)(j >> 1) & 1u, tid);
        if (!ok) break;
        ++n_consumed;
        uint8_t* dzt = sDz(st);
        uint8_t* et = dzt + kTile;
        if (tid == 0) {
            tc_fence_after();
            issue_dgrad(tWork, dzt, S, sW, S, H, (uint32_t)H * S, H, H);
            mma_commit(bar);
            issue_wgrad(tDW, dzt, S, 128u * S, et, S, 128u * S, H, !first);
            mma_commit(bar_w);
            mp = true;
            // the other stage was released at the end of the previous tile
            if (t + gridDim.x < A.t1) {
                issue(st ^ 1, t + gridDim.x, hdr_next.z);
                if (hdr_next.y > hdr_next.x)   // its receivers' da rows into L2
                    prefetch_l2(A.da + (int64_t)hdr_next.x * H, (uint32_t)(hdr_next.y - hdr_next.x) * H * 4);
                if (t + 2 * (int64_t)gridDim.x < A.t1) hdr_next = tile_hdr(t + 2 * (int64_t)gridDim.x);
            }
        }
        const uint8_t* rec = sRec(st);
        const int32_t* hdr = reinterpret_cast<const int32_t*>(rec);
        const int32_t* sRp = reinterpret_cast<const int32_t*>(rec + 16);
        const int16_t* sSeg = reinterpret_cast<const int16_t*>(rec + 544);
        const float* sWd = reinterpret_cast<const float*>(rec + 1312);
        const int32_t r0 = hdr[0], r1 = hdr[1], e0 = hdr[2], ne = hdr[3];
        const bool valid = row < ne;
        const int64_t eg = (int64_t)e0 + row;
        // gradient of e' (Eq. 5b adjoint plus the upstream de'), requested before the MMA wait
        float gv[CW];
        if (valid) {
            const float w = sWd[row];
            const float* dar = A.da + (int64_t)(r0 + sSeg[row]) * H + c0;
            float dv[CW];
            if (A.de_out) {
#pragma unroll
                for (int i = 0; i < CW; i += 8) ld_bf16x8(A.de_out + eg * H + c0 + i, dv + i);
            } else {
#pragma unroll
                for (int i = 0; i < CW; ++i) dv[i] = 0.f;
            }
#pragma unroll
            for (int i = 0; i < CW; i += 4) {
                const float4 u = __ldg(reinterpret_cast<const float4*>(dar + i));
                gv[i] = edge_g(w, u.x, dv[i]);
                gv[i + 1] = edge_g(w, u.y, dv[i + 1]);
                gv[i + 2] = edge_g(w, u.z, dv[i + 2]);
                gv[i + 3] = edge_g(w, u.w, dv[i + 3]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < CW; ++i) gv[i] = 0.f;
        }
#pragma unroll
        for (int jj = 0; jj < NCH; ++jj) accb[jj] += warp_colsum16(gv + 16 * jj, lane);
        {   // dz_0 per edge, for the sender-side sums of the projection adjoint: whole rows per
            // warp from the stage's dz tile (TMA-loaded, complete since the stage barrier)
            constexpr int CPR = H / 8;
            for (int i = tid; i < ne * CPR; i += NT) {
                const int rr = i / CPR, jj = i - rr * CPR;
                *reinterpret_cast<uint4*>(A.dz1 + ((int64_t)e0 + rr) * H + 8 * jj) =
                    *reinterpret_cast<const uint4*>(dzt + tile_off(rr, 8 * jj, 128, S));
            }
        }
        // receiver-side sums of dz_0 over each receiver's edges (dP, fixed edge order)
        for (int it = tid; it < (r1 - r0) * (H / 8); it += NT) {
            const int rr = it / (H / 8), c = (it % (H / 8)) * 8;
            float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int32_t e = sRp[rr]; e < sRp[rr + 1]; ++e) {
                float z8[8];
                ld_tile8(dzt, e, c, 128, S, z8);
#pragma unroll
                for (int k = 0; k < 8; ++k) s8[k] += z8[k];
            }
            float4* dp = reinterpret_cast<float4*>(A.dP + (int64_t)(r0 + rr) * H + c);
            dp[0] = make_float4(s8[0], s8[1], s8[2], s8[3]);
            dp[1] = make_float4(s8[4], s8[5], s8[6], s8[7]);
        }
        ok = block_wait(bar, ph, tid);
        tc_fence_after();
        if (!ok) break;
        float dh[CW];
        ld_acc<CW>(tWork, q, c0, dh);
        tc_fence_before();
#pragma unroll
        for (int i = 0; i < CW; ++i) dh[i] = __fadd_rn(gv[i], dh[i]);   // residual branch plus W1c^T dz_0
        fence_proxy_async();
        ok = block_wait(bar_w, ph, tid);   // the stage is free: wgrad done, every thread past its reads
        if (!ok) break;
        mp = false;
        ph ^= 1;
        tc_fence_after();
        first = false;
        // de_in by whole rows per warp, staged in the stage's e tile (the wgrad has read it); the
        // stage is refilled only after the next tile's stage barrier
        st_row_tile<CW>(et, row, c0, S, dh);
        __syncthreads();
        {
            constexpr int CPR = H / 8;
            for (int i = tid; i < ne * CPR; i += NT) {
                const int rr = i / CPR, jj = i - rr * CPR;
                *reinterpret_cast<uint4*>(A.de_in + ((int64_t)e0 + rr) * H + 8 * jj) =
                    *reinterpret_cast<const uint4*>(et + tile_off(rr, 8 * jj, 128, S));
            }
        }
        fence_proxy_async();   // generic accesses of the stage precede its TMA refill
    }
    if (tid == 0 && !ok) {   // after a timeout: wait (bounded) for what this CTA started
        if (mp) mbar_wait(bar_w, ph);
        if (n_issued > n_consumed) {   // at most the last load is outstanding
            const int64_t i = n_issued - 1;
            mbar_wait(full + (i & 1), (uint32_t)(i >> 1) & 1u);
        }
    }
    __syncwarp();   // reconverged before the aligned block barrier
    ok = __syncthreads_and(ok) != 0;
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (ok) {
        if (!first) flush_acc<CG>(tDW, H, H, q, lane, g, part);
        else
            for (int i = tid; i < H * H; i += NT) part[i] = 0.f;
    }
    colsum_store<H, NCH>(accb, sRed, q, lane, c0, tid, NT, part + H * H);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 2 * H);
}

// ------------------------------------------------------------------ k_bwd_chain_edge0
//
// The edge MLP's last two adjoint steps in one pass when Linear 1 is the one
// left for the chain: the work of k_bwd_chain (k = 1) and of k_bwd_edge0, so
// that dz_0 never travels through the scratch. Per tile: MMA pair 1 (D1 =
// dz_1 W_1, dW_1 += dz_1^T h_0), epilogue 1 (dz_0 = D1 ELU'(h_0) as BF16 into
// the shared-memory slot dz_1 came in, its column sums for db_0), MMA pair 2
// (D2 = dz_0 W1c, dW1c += dz_0^T e), dz_0 per edge (whole rows) and its sums
// over each receiver's edges (dP), epilogue 2 (de_in = g + D2 with g = de' +
// da_i / d_ij, staged in the stage's h_0 slot and written as whole rows, the
// column sums of g for the LayerNorm beta gradient).
//
// Two warp groups split the epilogues, so that epilogue 2 of tile j runs beside
// epilogue 1 of tile j + 1: group X (warps 0-7) waits for pair 1, writes dz_0,
// tells group Y's leader through an mbarrier (zr) that dz_0 is in place, issues
// the next tile's pair 1 and then writes dz_0 per edge and dP; group Y (warps
// 8-15) issues pair 2, runs epilogue 2, reloads the e tile once pair 2 has read
// it and the stage once group X has said (mbarrier xd) that it has read it.
// Each warp covers 64 columns of its 32 rows (TMEM lane quarter). Operands,
// roundings and summation orders are those of the two separate kernels, so the
// results are the same bit for bit. TMEM: D1, D2, dW_1, dW1c (128 columns
// each). Two stages of {dz_1, h_0} rows; one stage of e rows. The tile records
// stay in global memory (brought into L2 two tiles ahead).

struct ChainE0Args {
    const float* Wa;             // W_1 [H x H] (FP32)
    const float* W1;             // W_0 = W1 [H x 3H]; W1c = columns 2H .. 3H
    const uint8_t* tile_meta;    // per-tile records (GNN_TILE_META_BYTES each)
    int64_t t0, n_tiles;         // the chunk: tiles t0 .. t0 + n_tiles; scratch row of tile t0 + i is 128 i
    const __nv_bfloat16* de_out; // NULL: zero
    const float* da;             // aggregate gradient after the halo adjoint
    __nv_bfloat16* de_in;
    __nv_bfloat16* dz1;          // per-edge dz_0 [E x H]
    float* dP;                   // [n_rows x H]
    float* part;                 // per-CTA: dW_1, dW1c [H x H], then db_0 and dbeta [H]
    int64_t pstride;
};

constexpr int kCE0NT = 512;
struct ChainE0Smem {
    static constexpr uint32_t wa = 0, wb = kTile;
    static constexpr uint32_t a = 2 * kTile;          // stage s: dz_1 (then dz_0), h_0 (then de_in), at a + s * 2 * kTile
    static constexpr uint32_t e = a + 4 * kTile;      // e rows
    static constexpr uint32_t red = a;                // 8 x H floats, after the tile loop
    static constexpr uint32_t bar = e + kTile;        // fullA[2], fullB, c1, c2d, c2w, zr[2], xd, n1, TMEM slot
    static constexpr uint32_t total = bar + 128 + 1024;
};
static_assert(ChainE0Smem::total <= 227 * 1024, "k_bwd_chain_edge0 shared memory");

__global__ void __launch_bounds__(kCE0NT, 1) k_bwd_chain_edge0(const __grid_constant__ CUtensorMap tm_dz,
                                                              const __grid_constant__ CUtensorMap tm_h,
                                                              const __grid_constant__ CUtensorMap tm_e,
                                                              ChainE0Args A) {
    constexpr int H = H128, S = kS, CG = 4, CW = 64, NT = kCE0NT, NCH = CW / 16, CPR = H / 8, GT = 256;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    uint8_t* sWa = sm + ChainE0Smem::wa;
    uint8_t* sWb = sm + ChainE0Smem::wb;
    uint8_t* sE = sm + ChainE0Smem::e;
    float* sRed = reinterpret_cast<float*>(sm + ChainE0Smem::red);
    uint64_t* fullA = reinterpret_cast<uint64_t*>(sm + ChainE0Smem::bar);   // fullA[2]: stage landed
    uint64_t* fullB = fullA + 2;   // e rows landed
    uint64_t* c1 = fullA + 3;      // MMA pair 1 complete
    uint64_t* c2d = fullA + 4;     // pair 2's dgrad complete
    uint64_t* c2w = fullA + 5;     // pair 2's wgrad complete
    uint64_t* zr = fullA + 6;      // zr[j % 2]: group X has written tile j's dz_0
    uint64_t* xd = fullA + 8;      // group X has read the tile's stage
    int64_t* sN1 = reinterpret_cast<int64_t*>(fullA + 9);   // pair 1 issues (for the final waits)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fullA + 10);
    auto sDz = [&](int st) { return sm + ChainE0Smem::a + st * 2 * kTile; };

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool isX = warp < 8;
    const int q = warp & 3, row = 32 * q + lane, c0 = 64 * ((warp >> 2) & 1), gt = tid & (GT - 1);
    const bool leader = gt == 0;   // X: thread 0, Y: thread 256
    if (warp == 0) {
        tmem_alloc(tslot, 4 * H);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 9; ++i) mbar_init(fullA + i, 1);
        fence_mbar_init();
    }
    load_weight(sWa, A.Wa, H, 0, H, H, tid, NT);
    load_weight(sWb, A.W1, 3 * H, 2 * H, H, H, tid, NT);   // W1c as a K-major [H x H] tile
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot, tD1 = tmem, tD2 = tmem + H, tWa = tmem + 2 * H, tWb = tmem + 3 * H;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const int64_t n_mine = A.n_tiles > (int64_t)blockIdx.x
                               ? (A.n_tiles - 1 - (int64_t)blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](int64_t j) { return (int64_t)blockIdx.x + j * gridDim.x; };   // chunk-relative
    auto rec_of = [&](int64_t j) { return A.tile_meta + (A.t0 + tile_of(j)) * GNN_TILE_META_BYTES; };
    // leaders only: X issues pair 1 (n1); Y issues the loads (nA, nB) and pair 2 (n2)
    int64_t nA = 0, nB = 0, n1 = 0, n2 = 0;
    bool ok0 = true;
    int4 hB = make_int4(0, 0, 0, 0);   // Y: the header of the tile whose e rows load next
    auto issue_A = [&]() {   // dz_1 and h_0 rows of tile nA into stage nA % 2, its record into L2
        const int st = (int)(nA & 1);
        const int32_t y = (int32_t)(tile_of(nA) * 128);
        mbar_arrive_expect_tx(fullA + st, 2 * kTile);
        for (int kb = 0; kb < 2; ++kb) {
            tma_load_2d(sDz(st) + kb * 128 * S, &tm_dz, kb * 64, y, fullA + st);
            tma_load_2d(sDz(st) + kTile + kb * 128 * S, &tm_h, kb * 64, y, fullA + st);
        }
        prefetch_l2(rec_of(nA), GNN_TILE_META_BYTES);
        ++nA;
    };
    auto issue_B = [&]() {   // e rows of tile nB; its receivers' da rows and its de' rows into L2
        mbar_arrive_expect_tx(fullB, kTile);
        for (int kb = 0; kb < 2; ++kb) tma_load_2d(sE + kb * 128 * S, &tm_e, kb * 64, hB.z, fullB);
        if (hB.y > hB.x) prefetch_l2(A.da + (int64_t)hB.x * H, (uint32_t)(hB.y - hB.x) * H * 4);
        if (A.de_out && hB.w > 0) prefetch_l2(A.de_out + (int64_t)hB.z * H, (uint32_t)hB.w * H * 2);
        ++nB;
        if (nB < n_mine) hB = ld_nc_v4s32(rec_of(nB));
    };
    auto issue_pair1 = [&]() {   // tile n1's first MMA pair once its stage has landed
        const int st = (int)(n1 & 1);
        ok0 = ok0 && mbar_wait(fullA + st, (uint32_t)(n1 >> 1) & 1u);
        if (!ok0) return;
        tc_fence_after();
        issue_dgrad(tD1, sDz(st), S, sWa, S, H, (uint32_t)H * S, H, H);
        issue_wgrad(tWa, sDz(st), S, 128u * S, sDz(st) + kTile, S, 128u * S, H, n1 > 0);
        mma_commit(c1);
        ++n1;
    };
    if (tid == 256 && n_mine > 0) {
        hB = ld_nc_v4s32(rec_of(0));
        while (nA < n_mine && nA < 2) issue_A();
        issue_B();
    }
    if (tid == 0 && n_mine > 0) issue_pair1();
    float acc[NCH];   // X: column sums of dz_0 (db_0); Y: of g (the LayerNorm beta gradient)
#pragma unroll
    for (int j = 0; j < NCH; ++j) acc[j] = 0.f;
    bool ok = true;

    if (isX) {
        for (int64_t j = 0; j < n_mine; ++j) {
            const int st = (int)(j & 1);
            const uint32_t par = (uint32_t)j & 1u;   // c1 and xd complete once per tile
            const uint8_t* rec = rec_of(j);
            const int4 hd = ld_nc_v4s32(rec);
            const int32_t* rp = reinterpret_cast<const int32_t*>(rec + 16);
            // epilogue 1: dz_0 into the dz_1 slot of the stage, column sums for db_0
            ok = wg_and(leader ? mbar_wait(c1, par) : true, true);
            if (!ok) break;
            tc_fence_after();
            uint8_t* z = sDz(st);
            const uint8_t* hT = z + kTile;
#pragma unroll
            for (int jj = 0; jj < NCH; ++jj) {
                float dh[16], hv[16];
                tmem_ld16(tD1 + lane_base + (uint32_t)(c0 + 16 * jj), dh);
                ld_tile8(hT, row, c0 + 16 * jj, 128, S, hv);
                ld_tile8(hT, row, c0 + 16 * jj + 8, 128, S, hv + 8);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) dh[i] = elu1_bwd_from_out(dh[i], hv[i]);
                st_tile8(z, row, c0 + 16 * jj, 128, S, dh);
                st_tile8(z, row, c0 + 16 * jj + 8, 128, S, dh + 8);
                acc[jj] += warp_colsum16(dh, lane);
            }
            tc_fence_before();
            fence_proxy_async();
            wg_and(true, true);
            if (leader) {   // dz_0 is in place for pair 2; then the next tile's pair 1 (D1 has been read)
                mbar_arrive(zr + st);
                if (j + 1 < n_mine) issue_pair1();
            }
            // dz_0 per edge, for the sender-side sums of the projection adjoint (whole rows per warp)
            const int32_t r0 = hd.x, nr = hd.y - hd.x, e0 = hd.z, ne = hd.w;
            for (int i = gt; i < ne * CPR; i += GT) {
                const int rr = i / CPR, jj = i - rr * CPR;
                *reinterpret_cast<uint4*>(A.dz1 + ((int64_t)e0 + rr) * H + 8 * jj) =
                    *reinterpret_cast<const uint4*>(z + tile_off(rr, 8 * jj, 128, S));
            }
            // receiver-side sums of dz_0 over each receiver's edges (dP, fixed edge order)
            for (int it = gt; it < nr * CPR; it += GT) {
                const int rr = it / CPR, c = (it % CPR) * 8;
                const int32_t ea = __ldg(rp + rr), eb = __ldg(rp + rr + 1);
                float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int32_t e = ea; e < eb; ++e) {
                    float z8[8];
                    ld_tile8(z, e, c, 128, S, z8);
#pragma unroll
                    for (int k = 0; k < 8; ++k) s8[k] += z8[k];
                }
                float4* dp = reinterpret_cast<float4*>(A.dP + (int64_t)(r0 + rr) * H + c);
                dp[0] = make_float4(s8[0], s8[1], s8[2], s8[3]);
                dp[1] = make_float4(s8[4], s8[5], s8[6], s8[7]);
            }
            ok = wg_and(!leader || ok0, true);   // every X thread is past its reads of the stage
            if (!ok) break;
            if (leader) mbar_arrive(xd);
        }
        if (leader) *sN1 = n1;
    } else {
        for (int64_t j = 0; j < n_mine; ++j) {
            const int st = (int)(j & 1);
            const uint32_t par = (uint32_t)j & 1u;   // fullB, c2d, c2w complete once per tile
            const uint8_t* rec = rec_of(j);
            const int4 hd = ld_nc_v4s32(rec);
            const int seg = __ldg(reinterpret_cast<const int16_t*>(rec + 544) + row);
            const float w = __ldg(reinterpret_cast<const float*>(rec + 1312) + row);
            const int32_t e0 = hd.z, ne = hd.w;
            const bool valid = row < ne;
            if (leader) {   // pair 2 once group X has written dz_0 and the e rows have landed (zr alternates
                            // between two barriers, so group X, at most two tiles ahead, cannot alias a phase)
                ok0 = ok0 && mbar_wait(zr + st, (uint32_t)(j >> 1) & 1u) && mbar_wait(fullB, par);
                if (ok0) {
                    tc_fence_after();
                    uint8_t* z = sDz(st);
                    issue_dgrad(tD2, z, S, sWb, S, H, (uint32_t)H * S, H, H);
                    mma_commit(c2d);
                    issue_wgrad(tWb, z, S, 128u * S, sE, S, 128u * S, H, n2 > 0);
                    mma_commit(c2w);
                    ++n2;
                }
            }
            // the inputs of g, 16 columns at a time, one chunk ahead
            const float4* dar = reinterpret_cast<const float4*>(A.da + (int64_t)(hd.x + (valid ? seg : 0)) * H + c0);
            const bool has_de = valid && A.de_out;
            const uint4* der = has_de ? reinterpret_cast<const uint4*>(A.de_out + ((int64_t)e0 + row) * H + c0) : nullptr;
            float4 ga[2][4];
            uint4 gd[2][2];
            auto load_chunk = [&](int jj, int b) {
#pragma unroll
                for (int i = 0; i < 4; ++i) ga[b][i] = valid ? __ldg(dar + 4 * jj + i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 2; ++i) gd[b][i] = has_de ? __ldg(der + 2 * jj + i) : make_uint4(0u, 0u, 0u, 0u);
            };
            load_chunk(0, 0);
            ok = wg_and(leader ? (ok0 && mbar_wait(c2d, par)) : true, false);
            if (!ok) break;
            tc_fence_after();
            // epilogue 2: de_in = g + D2, staged in the stage's h_0 slot (pair 1 and epilogue 1 have read it)
            uint8_t* hT = sDz(st) + kTile;
#pragma unroll
            for (int jj = 0; jj < NCH; ++jj) {
                if (jj + 1 < NCH) load_chunk(jj + 1, (jj + 1) & 1);
                const int b = jj & 1;
                float gv[16], dh[16];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const uint32_t dw[4] = {gd[b][i].x, gd[b][i].y, gd[b][i].z, gd[b][i].w};
                    const float4 u0 = ga[b][2 * i], u1 = ga[b][2 * i + 1];
                    const float av[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float d0, d1;
                        unpack_bf16x2(dw[k], d0, d1);
                        gv[8 * i + 2 * k] = edge_g(w, av[2 * k], d0);
                        gv[8 * i + 2 * k + 1] = edge_g(w, av[2 * k + 1], d1);
                    }
                }
                acc[jj] += warp_colsum16(gv, lane);
                tmem_ld16(tD2 + lane_base + (uint32_t)(c0 + 16 * jj), dh);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 16; ++i) dh[i] = __fadd_rn(gv[i], dh[i]);
                st_tile8(hT, row, c0 + 16 * jj, 128, S, dh);
                st_tile8(hT, row, c0 + 16 * jj + 8, 128, S, dh + 8);
            }
            tc_fence_before();
            wg_and(true, false);   // D2 read, de_in staged
            if (leader) {   // pair 2's wgrad has read dz_0 and e: the next tile's e rows
                ok0 = ok0 && mbar_wait(c2w, par);
                if (ok0 && nB < n_mine) issue_B();
            }
            for (int i = gt; i < ne * CPR; i += GT) {
                const int rr = i / CPR, jj = i - rr * CPR;
                *reinterpret_cast<uint4*>(A.de_in + ((int64_t)e0 + rr) * H + 8 * jj) =
                    *reinterpret_cast<const uint4*>(hT + tile_off(rr, 8 * jj, 128, S));
            }
            fence_proxy_async();   // generic accesses of the stage precede its TMA refill
            ok = wg_and(!leader || ok0, false);   // every Y thread is past its accesses of the stage
            if (!ok) break;
            if (leader && nA < n_mine) {   // tile j + 2 into stage st once group X has read it
                ok0 = mbar_wait(xd, par);
                if (ok0) issue_A();
            }
        }
    }
    __syncwarp();
    __syncthreads();
    if (tid == 256) {   // bounded waits for what this CTA started and nobody waited for
        const int64_t m1 = *sN1;
        if (m1 > 0) mbar_wait(c1, (uint32_t)(m1 - 1) & 1u);
        if (n2 > 0) {
            mbar_wait(c2d, (uint32_t)(n2 - 1) & 1u);
            mbar_wait(c2w, (uint32_t)(n2 - 1) & 1u);
        }
        for (int64_t i = m1; i < nA; ++i) mbar_wait(fullA + (i & 1), (uint32_t)(i >> 1) & 1u);
        for (int64_t i = n2; i < nB; ++i) mbar_wait(fullB, (uint32_t)i & 1u);
    }
    __syncwarp();
    const bool all_ok = __syncthreads_and(ok && (!leader || ok0)) != 0;
    tc_fence_after();
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (all_ok) {
        if (n_mine > 0) {
            flush_acc<CG>(tWa, H, H, q, lane, warp >> 2, part);
            flush_acc<CG>(tWb, H, H, q, lane, warp >> 2, part + H * H);
        } else {
            for (int i = tid; i < 2 * H * H; i += NT) part[i] = 0.f;
        }
    }
    // column sums: warp (q, half) of a group holds columns c0 + 16 j + (lane >> 1) over its 32 rows;
    // the four row quarters are added in order, db_0 from group X, dbeta from group Y
    __syncthreads();
    if ((lane & 1) == 0) {
#pragma unroll
        for (int jj = 0; jj < NCH; ++jj) sRed[(isX ? 0 : 4 * H) + q * H + c0 + 16 * jj + (lane >> 1)] = acc[jj];
    }
    __syncthreads();
    for (int c = tid; c < 2 * H; c += NT) {
        const float* r = sRed + (c < H ? 0 : 4 * H) + (c % H);
        part[2 * H * H + c] = ((r[0] + r[H]) + r[2 * H]) + r[3 * H];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 4 * H);
}

// ------------------------------------------------------------------ k_bwd_node0

struct Node0Args {
    int64_t t0, t1;              // tile range; the scratch rows of tile t start at (t - t0) * 128
    int64_t n_rows;
    const float* W0;             // W_0 of the node MLP [H x 2H]
    const float* dx_out;
    float* da;                   // out: gradient of a*
    float* dx_in;                // out: dx_out + the x part
    float* part;                 // per-CTA: dW_0 [H x 2H]
    int64_t pstride;
};

// 128 rows x 4 column groups, one CTA per SM (TMEM: a 256-column input
// gradient and the 256-column dW_0 accumulator). The epilogue reads only TMEM,
// the dx' rows and its own FP32 staging tile, so the next tile's rows load while
// it runs; da* and then dx_in pass through the staging tile and leave as whole
// rows by TMA stores (rows past n_rows are clipped).
constexpr int kN0NT = 512;
struct Node0Smem {
    static constexpr uint32_t w = 0, dz = 2 * kTile, xa = 3 * kTile, f = 5 * kTile;   // f: [128 x H] FP32
    static constexpr uint32_t bar = f + 128 * H128 * 4;
    static constexpr uint32_t total = bar + 64 + 1024;
};
static_assert(Node0Smem::total <= 227 * 1024, "k_bwd_node0 shared memory");

__global__ void __launch_bounds__(kN0NT, 1) k_bwd_node0(const __grid_constant__ CUtensorMap tm_dz,
                                                       const __grid_constant__ CUtensorMap tm_xa,
                                                       const __grid_constant__ CUtensorMap tm_da,
                                                       const __grid_constant__ CUtensorMap tm_dxi, Node0Args A) {
    constexpr int H = H128, S = kS, CG = 4, CW = 32, NT = kN0NT;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = aligned_smem(smem_raw);
    uint8_t* sW0 = sm + Node0Smem::w;
    uint8_t* sDz = sm + Node0Smem::dz;
    uint8_t* sXa = sm + Node0Smem::xa;
    uint8_t* sF = sm + Node0Smem::f;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + Node0Smem::bar);
    uint64_t* bar = full + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, g = warp >> 2, row = 32 * q + lane, c0 = g * CW;
    if (warp == 0) {
        tmem_alloc(tslot, 4 * H);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(full, 1);
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    load_weight(sW0, A.W0, 2 * H, 0, H, 2 * H, tid, NT);   // [H x 2H], K-major over the 2H inputs
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot, tWork = tmem, tDW = tmem + 2 * H;
    bool lp = false, mp = false;
    auto issue = [&](int64_t t) {   // thread 0: dz_0 rows and [a*, x] rows of tile t
        lp = true;
        const int32_t y = (int32_t)((t - A.t0) * 128);
        mbar_arrive_expect_tx(full, 3 * kTile);
        for (int kb = 0; kb < 2; ++kb) tma_load_2d(sDz + kb * 128 * S, &tm_dz, kb * 64, y, full);
        for (int kb = 0; kb < 4; ++kb) tma_load_2d(sXa + kb * 128 * S, &tm_xa, kb * 64, y, full);
    };
    const int64_t tfirst = A.t0 + blockIdx.x;
    if (tid == 0 && tfirst < A.t1) issue(tfirst);
    uint32_t ph = 0;
    bool ok = true, first = true;

    for (int64_t t = tfirst; t < A.t1; t += gridDim.x) {
        if (tid == 0 && t + gridDim.x < A.t1) {   // the next tile's dx' rows into L2
            const int64_t rn = (t + gridDim.x) * 128;
            if (rn < A.n_rows)
                prefetch_l2(A.dx_out + rn * H, (uint32_t)(min((int64_t)128, A.n_rows - rn) * H * 4));
        }
        ok = block_wait(full, ph, tid);
        if (!ok) break;
        lp = false;
        if (tid == 0) {
            tc_fence_after();
            issue_dgrad(tWork, sDz, S, sW0, S, H, (uint32_t)H * S, 2 * H, H);
            issue_wgrad(tDW, sDz, S, 128u * S, sXa, S, 128u * S, 2 * H, !first);
            mma_commit(bar);
            mp = true;
        }
        const int64_t r = t * 128 + row;
        const bool valid = r < A.n_rows;
        float gx[CW];
        if (valid) {
            const float4* pg = reinterpret_cast<const float4*>(A.dx_out + r * H + c0);
#pragma unroll
            for (int i = 0; i < CW / 4; ++i) {
                const float4 u = __ldg(pg + i);
                gx[4 * i] = u.x; gx[4 * i + 1] = u.y; gx[4 * i + 2] = u.z; gx[4 * i + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < CW; ++i) gx[i] = 0.f;
        }
        if (tid == 0) bulk_wait_read_all();   // the previous tile's dx_in store has read the staging tile
        ok = block_wait(bar, ph, tid);
        if (!ok) break;
        mp = false;
        ph ^= 1;
        tc_fence_after();
        first = false;
        // both MMAs are done: the stage takes the next tile while the epilogue runs
        if (tid == 0 && t + gridDim.x < A.t1) issue(t + gridDim.x);
        __syncwarp();   // warp 0 reconverged before the aligned TMEM loads
        float d[CW];
        ld_acc<CW>(tWork, q, c0, d);   // gradient of a* (first H inputs)
#pragma unroll
        for (int i = 0; i < CW / 4; ++i)
            st_f32x4_tile<H>(sF, row, c0 + 4 * i, make_float4(d[4 * i], d[4 * i + 1], d[4 * i + 2], d[4 * i + 3]));
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int b = 0; b < H / 32; ++b) tma_store_2d(&tm_da, 32 * b, (int32_t)(t * 128), sF + b * 128 * 128);
            bulk_commit();
        }
        __syncwarp();   // warp 0 reconverged before the aligned TMEM loads
        ld_acc<CW>(tWork + H, q, c0, d);   // gradient of x (last H inputs) plus the residual branch
        tc_fence_before();
#pragma unroll
        for (int i = 0; i < CW; ++i) d[i] = gx[i] + d[i];
        if (tid == 0) bulk_wait_read_all();   // the da* store has read the staging tile
        __syncwarp();
        __syncthreads();
#pragma unroll
        for (int i = 0; i < CW / 4; ++i)
            st_f32x4_tile<H>(sF, row, c0 + 4 * i, make_float4(d[4 * i], d[4 * i + 1], d[4 * i + 2], d[4 * i + 3]));
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int b = 0; b < H / 32; ++b) tma_store_2d(&tm_dxi, 32 * b, (int32_t)(t * 128), sF + b * 128 * 128);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();   // the stored rows are written before the CTA exits
    if (tid == 0 && !ok) {   // after a timeout: wait (bounded) for what this CTA started
        if (mp) mbar_wait(bar, ph);
        if (lp) mbar_wait(full, mp ? ph ^ 1 : ph);
    }
    __syncwarp();   // reconverged before the aligned block barrier
    ok = __syncthreads_and(ok) != 0;
    float* part = A.part + (int64_t)blockIdx.x * A.pstride;
    if (ok) {
        if (!first) flush_acc<CG>(tDW, 2 * H, H, q, lane, g, part);
        else
            for (int i = tid; i < 2 * H * H; i += NT) part[i] = 0.f;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 4 * H);
}

// =================================================================== host side

using namespace host;

struct B128Ws {
    __nv_bfloat16* pq;
    float* a;
    float* da;
    float* dP;
    __nv_bfloat16* dz1;
    float* part;
    __nv_bfloat16* hs;       // (L-1) x [chunk rows x H]
    int64_t hs_stride;
    __nv_bfloat16* dzs[2];   // [chunk rows x H] each
    __nv_bfloat16* xa;       // [chunk rows x 2H]
    int64_t chunk;           // tiles per chunk
    size_t bytes;
};

// Tiles per chunk when the workspace is not limiting.
int64_t default_chunk(const gnn_graph_dev& G) {
    const int64_t node_tiles = (G.n_rows + 127) / 128;
    return std::max<int64_t>(1, std::min<int64_t>(kChunkTiles, std::max<int64_t>(node_tiles, G.n_edge_tiles)));
}

B128Ws carve_b128(void* ws, const gnn_graph_dev& G, int Le, int Ln, bool need_a, int64_t chunk) {
    constexpr int H = H128;
    B128Ws w{};
    size_t off = 0;
    auto take = [&](size_t n) {
        off = (off + 255) & ~(size_t)255;
        void* p = ws ? (char*)ws + off : nullptr;
        off += n;
        return p;
    };
    const int64_t NR = G.n_rows, E = G.n_edges;
    w.chunk = chunk;
    const int64_t rows = w.chunk * 128;
    const int L = std::max(Le, Ln);
    w.pq = (__nv_bfloat16*)take((size_t)NR * 2 * H * 2);
    w.a = need_a ? (float*)take((size_t)NR * H * 4) : nullptr;
    w.da = (float*)take((size_t)NR * H * 4);
    w.dP = (float*)take((size_t)NR * H * 4);
    w.dz1 = (__nv_bfloat16*)take((size_t)E * H * 2);
    w.part = (float*)take((size_t)2 * num_sms() * kPstride * 4);
    w.hs_stride = rows * H;
    w.hs = (__nv_bfloat16*)take((size_t)(L - 1) * rows * H * 2);
    w.dzs[0] = (__nv_bfloat16*)take((size_t)rows * H * 2);
    w.dzs[1] = (__nv_bfloat16*)take((size_t)rows * H * 2);
    w.xa = (__nv_bfloat16*)take((size_t)rows * 2 * H * 2);
    w.bytes = off + 256;
    return w;
}

// dz_{k-1} and the gradients of W_k, b_{k-1} for k = L-1 .. 1 over a chunk of
// n_tiles tiles; returns the buffer that holds dz_0.
int chain_backward(const gnn_mlp& W, const gnn_mlp& dW, B128Ws& w, int64_t n_tiles, int* cur, bool pairs,
                   cudaStream_t s, int k_last = 1) {
    return chain_backward_h128(W, dW, w.hs, w.hs_stride, w.dzs, w.part, kPstride, n_tiles, cur, s, pairs, k_last);
}

// gamma, beta and the last bias of an MLP from the recomputation's partials
// [dgamma | dbeta | db_{L-1}]; without `beta` the beta gradient is left to the
// kernel of the first Linear (the edge MLP's, which forms g again)
int reduce_ln(const gnn_mlp& dW, const B128Ws& w, int grid, cudaStream_t s, bool beta = true) {
    constexpr int H = H128;
    RedSeg seg[3];
    int n = 0;
    seg[n++] = RedSeg{dW.gamma, H, 1, H, 0, 0};
    if (beta) seg[n++] = RedSeg{dW.beta, H, 1, H, H, 0};
    seg[n++] = RedSeg{dW.b[dW.n_lin - 1], H, 1, H, 2 * H, 0};
    return reduce_grads(seg, n, w.part, kPstride, grid, s);
}

// Linear 1 and the first Linear's edge part of the edge MLP adjoint over tiles
// [t0, t1) of a chunk (k_bwd_chain_edge0): dz_1 is in w.dzs[cur], h_0 in block 0
// of w.hs.
int chain_edge0(const gnn_graph_dev& G, const gnn_mp_params& W, const gnn_mp_params& dW, B128Ws& w, int64_t t0,
                int64_t t1, int cur, const CUtensorMap& tm_e, const __nv_bfloat16* de_out, __nv_bfloat16* de_in,
                cudaStream_t s) {
    constexpr int H = H128;
    const int64_t rows = (t1 - t0) * 128;
    CUtensorMap tm_dz, tm_h;
    int rc = make_row_tmap(&tm_dz, w.dzs[cur], rows, H);
    if (rc) return rc;
    if ((rc = make_row_tmap(&tm_h, w.hs, rows, H))) return rc;
    ChainE0Args A{};
    A.Wa = W.edge.W[1];
    A.W1 = W.edge.W[0];
    A.tile_meta = static_cast<const uint8_t*>(G.tile_meta);
    A.t0 = t0;
    A.n_tiles = t1 - t0;
    A.de_out = de_out;
    A.da = w.da;
    A.de_in = de_in;
    A.dz1 = w.dz1;
    A.dP = w.dP;
    A.part = w.part;
    A.pstride = kPstride;
    int grid;
    if ((rc = persistent_grid(k_bwd_chain_edge0, kCE0NT, ChainE0Smem::total, 4 * H, t1 - t0, &grid))) return rc;
    {
        ProfScope _ps(s, "k_bwd_chain_edge0");
        k_bwd_chain_edge0<<<grid, kCE0NT, ChainE0Smem::total, s>>>(tm_dz, tm_h, tm_e, A);
    }
    GNN_LAUNCH_CHECK("k_bwd_chain_edge0");
    RedSeg seg[4];
    seg[0] = RedSeg{dW.edge.W[1], H, H, H, 0, H};
    seg[1] = RedSeg{dW.edge.W[0] + 2 * H, 3 * H, H, H, (int64_t)H * H, H};   // W1c columns of W1
    seg[2] = RedSeg{dW.edge.b[0], H, 1, H, 2 * (int64_t)H * H, 0};
    seg[3] = RedSeg{dW.edge.beta, H, 1, H, 2 * (int64_t)H * H + H, 0};
    return reduce_grads(seg, 4, w.part, kPstride, grid, s);
}

}  // namespace

int chain_backward_h128(const gnn_mlp& W, const gnn_mlp& dW, __nv_bfloat16* hs, int64_t hs_stride,
                        __nv_bfloat16* const dzs[2], float* part, int64_t pstride, int64_t n_tiles, int* cur,
                        cudaStream_t s, bool pairs, int k_last) {
    constexpr int H = H128;
    GNN_REQUIRE(pstride >= 2 * H * H + 2 * H, GNN_EINVAL, "chain adjoint: partial stride too small");
    GNN_REQUIRE(k_last >= 1, GNN_EINVAL, "chain adjoint: k_last %d", k_last);
    const int L = W.n_lin;
    int grid, grid2;
    int rc = persistent_grid(k_bwd_chain<false>, kChainNT, ChainSmem::total, 4 * H, n_tiles, &grid);
    if (rc) return rc;
    if ((rc = persistent_grid(k_bwd_chain2, kC2NT, Chain2Smem::total, 4 * H, n_tiles, &grid2))) return rc;
    const int64_t rows = n_tiles * 128;
    for (int k = L - 1; k >= k_last;) {
        CUtensorMap tm_dz, tm_h;
        if ((rc = make_row_tmap(&tm_dz, dzs[*cur], rows, H))) return rc;
        if ((rc = make_row_tmap(&tm_h, hs + (int64_t)(k - 1) * hs_stride, rows, H))) return rc;
        if (pairs && k - 1 >= k_last) {   // Linears k and k-1 in one pass
            CUtensorMap tm_hb, tm_out;
            if ((rc = make_row_tmap(&tm_hb, hs + (int64_t)(k - 2) * hs_stride, rows, H))) return rc;
            if ((rc = make_row_tmap(&tm_out, dzs[*cur ^ 1], rows, H))) return rc;
            Chain2Args A{};
            A.Wa = W.W[k];
            A.Wb = W.W[k - 1];
            A.hb = hs + (int64_t)(k - 2) * hs_stride;
            A.n_tiles = n_tiles;
            A.part = part;
            A.pstride = pstride;
            {
                ProfScope _ps(s, "k_bwd_chain2");
                k_bwd_chain2<<<grid2, kC2NT, Chain2Smem::total, s>>>(tm_dz, tm_h, tm_hb, tm_out, A);
            }
            GNN_LAUNCH_CHECK("k_bwd_chain2");
            RedSeg seg[4];
            seg[0] = RedSeg{dW.W[k], H, H, H, 0, H};
            seg[1] = RedSeg{dW.W[k - 1], H, H, H, (int64_t)H * H, H};
            seg[2] = RedSeg{dW.b[k - 1], H, 1, H, 2 * (int64_t)H * H, 0};
            seg[3] = RedSeg{dW.b[k - 2], H, 1, H, 2 * (int64_t)H * H + H, 0};
            if ((rc = reduce_grads(seg, 4, part, pstride, grid2, s))) return rc;
            *cur ^= 1;
            k -= 2;
            continue;
        }
        ChainArgs A{};
        A.W = W.W[k];
        A.dz_out = dzs[*cur ^ 1];
        A.n_tiles = n_tiles;
        A.part = part;
        A.pstride = pstride;
        {
            ProfScope _ps(s, "k_bwd_chain");
            k_bwd_chain<false><<<grid, kChainNT, ChainSmem::total, s>>>(tm_dz, tm_h, A);
        }
        GNN_LAUNCH_CHECK("k_bwd_chain");
        RedSeg seg[2];
        seg[0] = RedSeg{dW.W[k], H, H, H, 0, H};
        seg[1] = RedSeg{dW.b[k - 1], H, 1, H, (int64_t)H * H, 0};
        if ((rc = reduce_grads(seg, 2, part, pstride, grid, s))) return rc;
        *cur ^= 1;
        --k;
    }
    return GNN_OK;
}

int chain_input_h128(const float* W0, float* dW0, const __nv_bfloat16* dz, const __nv_bfloat16* xb, float* dx,
                     int64_t row0, int64_t n_rows, float* part, int64_t pstride, int64_t n_tiles, cudaStream_t s) {
    constexpr int H = H128;
    const uint32_t smem = ChainSmem::total;
    int grid;
    int rc = persistent_grid(k_bwd_chain<true>, kChainNT, smem, 4 * H, n_tiles, &grid);
    if (rc) return rc;
    CUtensorMap tm_dz, tm_h;
    if ((rc = make_row_tmap(&tm_dz, dz, n_tiles * 128, H))) return rc;
    if ((rc = make_row_tmap(&tm_h, xb, n_tiles * 128, H))) return rc;
    ChainArgs A{};
    A.W = W0;
    A.n_tiles = n_tiles;
    A.part = part;
    A.pstride = pstride;
    A.dx = dx;
    A.row0 = row0;
    A.n_rows = n_rows;
    {
        ProfScope _ps(s, "k_bwd_chain");
        k_bwd_chain<true><<<grid, kChainNT, smem, s>>>(tm_dz, tm_h, A);
    }
    GNN_LAUNCH_CHECK("k_bwd_chain");
    RedSeg seg[1] = {RedSeg{dW0, H, H, H, 0, H}};
    return reduce_grads(seg, 1, part, pstride, grid, s);
}

size_t backward_h128_ws(const gnn_graph_dev& G, const gnn_mp_params& W) {
    return carve_b128(nullptr, G, W.edge.n_lin, W.node.n_lin, true, default_chunk(G)).bytes;
}

int backward_h128(const gnn_graph_dev& G, const gnn_mp_config& cfg, const gnn_mp_params& W, const float* x_in,
                  const __nv_bfloat16* e_in, const float* a_star, const float* dx_out, const __nv_bfloat16* de_out,
                  float* dx_in, __nv_bfloat16* de_in, const gnn_mp_params& dW, void* ws, size_t ws_bytes,
                  cudaStream_t s) {
    constexpr int H = H128;
    const int Le = W.edge.n_lin, Ln = W.node.n_lin;
    GNN_REQUIRE(Le >= 2 && Le <= 4 && Ln >= 2 && Ln <= 4, GNN_EUNSUPPORTED,
                "gnn_mp_backward: BF16 backward at H=128 supports 2 to 4 Linear layers per MLP");
    // the largest chunk of tiles whose scratch fits the workspace given
    const bool need_a = a_star == nullptr;
    int64_t chunk = default_chunk(G);
    if (ws_bytes < carve_b128(nullptr, G, Le, Ln, need_a, chunk).bytes) {
        const size_t fixed = carve_b128(nullptr, G, Le, Ln, need_a, 0).bytes;
        const size_t per_tile = carve_b128(nullptr, G, Le, Ln, need_a, 2).bytes - carve_b128(nullptr, G, Le, Ln, need_a, 1).bytes;
        chunk = ws_bytes > fixed ? (int64_t)((ws_bytes - fixed) / per_tile) : 0;
        while (chunk > 0 && carve_b128(nullptr, G, Le, Ln, need_a, chunk).bytes > ws_bytes) --chunk;
        GNN_REQUIRE(chunk >= 1, GNN_ENOMEM, "gnn_mp_backward: workspace too small (%zu bytes)", ws_bytes);
    }
    B128Ws w = carve_b128(ws, G, Le, Ln, need_a, chunk);
    const bool pairs = !(cfg.flags & GNN_FLAG_ADJ_ONE_LINEAR);
    const int64_t NR = G.n_rows, E = G.n_edges;
    if (NR == 0) return GNN_OK;
    int rc;
    // 0. recompute P|Q (and a* when it was not saved)
    if ((rc = proj_forward(G, H, W, x_in, w.pq, s))) return rc;
    if (!a_star) {
        if ((rc = aggregate_forward(G, cfg, W, e_in, w.pq, nullptr, w.a, s))) return rc;
    }
    const float* astar = a_star ? a_star : w.a;
    // 1. node MLP adjoint, chunk by chunk
    const int64_t node_tiles = (NR + 127) / 128;
    for (int64_t t0 = 0; t0 < node_tiles; t0 += w.chunk) {
        const int64_t t1 = std::min(node_tiles, t0 + w.chunk);
        RecomputeSave o{};
        o.t0 = t0;
        o.t1 = t1;
        o.hs = w.hs;
        o.hs_stride = w.hs_stride;
        o.xa = w.xa;
        o.dz = w.dzs[0];
        o.dx_out = dx_out;
        o.part = w.part;
        o.pstride = kPstride;
        if ((rc = node_recompute_save(G, cfg, W, astar, x_in, o, s))) return rc;
        if ((rc = reduce_ln(dW.node, w, o.grid, s))) return rc;
        int cur = 0;
        if ((rc = chain_backward(W.node, dW.node, w, t1 - t0, &cur, pairs, s))) return rc;
        CUtensorMap tm_dz, tm_xa;
        const int64_t rows = (t1 - t0) * 128;
        if ((rc = make_row_tmap(&tm_dz, w.dzs[cur], rows, H))) return rc;
        if ((rc = make_row_tmap(&tm_xa, w.xa, rows, 2 * H))) return rc;
        Node0Args A;
        A.t0 = t0;
        A.t1 = t1;
        A.n_rows = NR;
        A.W0 = W.node.W[0];
        A.dx_out = dx_out;
        A.da = w.da;
        A.dx_in = dx_in;
        A.part = w.part;
        A.pstride = kPstride;
        int grid;
        if ((rc = persistent_grid(k_bwd_node0, kN0NT, Node0Smem::total, 4 * H, t1 - t0, &grid))) return rc;
        CUtensorMap tm_da, tm_dxi;
        if ((rc = make_f32_tmap(&tm_da, w.da, NR, H))) return rc;
        if ((rc = make_f32_tmap(&tm_dxi, dx_in, NR, H))) return rc;
        {
            ProfScope _ps(s, "k_bwd_node0");
            k_bwd_node0<<<grid, kN0NT, Node0Smem::total, s>>>(tm_dz, tm_xa, tm_da, tm_dxi, A);
        }
        GNN_LAUNCH_CHECK("k_bwd_node0");
        RedSeg seg[1] = {RedSeg{dW.node.W[0], 2 * H, H, 2 * H, 0, 2 * H}};
        if ((rc = reduce_grads(seg, 1, w.part, kPstride, grid, s))) return rc;
    }
    // 2. adjoint of the halo swap + sync
    if (cfg.halo_mode == GNN_HALO_SYNC) {
        if ((rc = plain::halo(G, w.da, H, s))) return rc;
    }
    // 3. edge MLP adjoint, chunk by chunk
    if (E > 0) {
        GNN_REQUIRE(G.tile_meta && ((uintptr_t)G.tile_meta & 15) == 0, GNN_EINVAL,
                    "gnn_mp_backward: tile_meta must be a 16-byte aligned device array");
        CUtensorMap tm_e;
        if ((rc = make_row_tmap(&tm_e, e_in, E, H))) return rc;
        // with an odd number of Linears after the first, the pairs leave Linear 1 alone: it
        // runs with the first Linear's edge part in one pass (k_bwd_chain_edge0)
        const bool merge_e0 = pairs && (Le - 1) % 2 == 1;
        for (int64_t t0 = 0; t0 < G.n_edge_tiles; t0 += w.chunk) {
            const int64_t t1 = std::min<int64_t>(G.n_edge_tiles, t0 + w.chunk);
            RecomputeSave o{};
            o.t0 = t0;
            o.t1 = t1;
            o.hs = w.hs;
            o.hs_stride = w.hs_stride;
            o.dz = w.dzs[0];
            o.da = w.da;
            o.de_out = de_out;
            o.part = w.part;
            o.pstride = kPstride;
            if ((rc = edge_recompute_save(G, cfg, W, e_in, w.pq, o, s))) return rc;
            if ((rc = reduce_ln(dW.edge, w, o.grid, s, false))) return rc;
            int cur = 0;
            if (merge_e0) {   // Linears L-1 .. 2 in pairs, then Linear 1 with the first Linear's edge part
                if ((rc = chain_backward(W.edge, dW.edge, w, t1 - t0, &cur, pairs, s, 2))) return rc;
                if ((rc = chain_edge0(G, W, dW, w, t0, t1, cur, tm_e, de_out, de_in, s))) return rc;
                continue;
            }
            if ((rc = chain_backward(W.edge, dW.edge, w, t1 - t0, &cur, pairs, s))) return rc;
            CUtensorMap tm_dz;
            if ((rc = make_row_tmap(&tm_dz, w.dzs[cur], (t1 - t0) * 128, H))) return rc;
            Edge0Args A;
            A.tile_meta = static_cast<const uint8_t*>(G.tile_meta);
            A.t0 = t0;
            A.t1 = t1;
            A.W1 = W.edge.W[0];
            A.de_out = de_out;
            A.da = w.da;
            A.de_in = de_in;
            A.dz1 = w.dz1;
            A.dP = w.dP;
            A.part = w.part;
            A.pstride = kPstride;
            int grid;
            if ((rc = persistent_grid(k_bwd_edge0, kE0NT, Edge0Smem::total, 2 * H, t1 - t0, &grid))) return rc;
            {
                ProfScope _ps(s, "k_bwd_edge0");
                k_bwd_edge0<<<grid, kE0NT, Edge0Smem::total, s>>>(tm_dz, tm_e, A);
            }
            GNN_LAUNCH_CHECK("k_bwd_edge0");
            RedSeg seg[2] = {RedSeg{dW.edge.W[0] + 2 * H, 3 * H, H, H, 0, H},   // W1c columns of W1
                             RedSeg{dW.edge.beta, H, 1, H, (int64_t)H * H, 0}};
            if ((rc = reduce_grads(seg, 2, w.part, kPstride, grid, s))) return rc;
        }
    } else {
        GNN_CUDA_CHECK(cudaMemsetAsync(w.dP, 0, sizeof(float) * NR * H, s), "memset");
    }
    // 4. projection adjoint: sender-side sums, dx_in += [dP dQ] [W1a; W1b], dW1a, dW1b
    return proj_backward(G, H, W, x_in, w.dP, w.dz1, dx_in, dW, w.part, s);
}

}  // namespace fused
}  // namespace gnn
