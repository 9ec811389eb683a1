// sm_103a building blocks for the fused kernels: mbarriers with bounded waits,
// TMA tile loads, tcgen05 (TMEM allocation, BF16 MMA, TMEM loads) and the
// shared-memory operand layouts the tensor core reads.
//
// Operand layout ("row tile"): a [rows x K] BF16 matrix is stored as K/(S/2)
// column blocks of S bytes per row (S = swizzle span, 32/64/128 bytes); inside
// a block, row r occupies bytes [r*S, r*S+S) and its 16-byte chunks are
// permuted by the hardware swizzle: byte offset o within the 1024-byte-aligned
// block goes to o ^ (((o >> 7) & (S/16 - 1)) << 4). Eight rows form one
// swizzle atom of 8*S bytes. The same bytes serve as a K-major operand
// (rows = M or N, contiguous = K) and as an MN-major operand (rows = K,
// contiguous = M or N), which is how the backward kernels reuse forward tiles.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "device_common.cuh"

namespace gnn {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------------ mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Default limit of every device-side wait: 1 s of %globaltimer.
constexpr uint64_t kWaitLimitNs = 1000000000ull;

// Waits for the phase with the given parity to complete, for at most
// limit_ns; on timeout latches GNN_DEVERR_TIMEOUT and returns false (the caller
// skips its remaining work instead of hanging the GPU).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitLimitNs) {
    const uint32_t b = smem_u32(bar);
    if (mbar_try_wait(b, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
        if (mbar_try_wait(b, parity)) return true;
        __nanosleep(64);   // yield issue slots to the warps doing work
        if (globaltimer_ns() - t0 > limit_ns) {
            raise_device_error(GNN_DEVERR_TIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Named barrier over `n` threads (a multiple of 32) of the CTA. bar.sync is an
// aligned barrier: every warp must reach it converged, so the warp is
// reconverged first (a thread may come from code only it ran: a wait, an issue).
__device__ __forceinline__ void named_sync(int id, int n) {
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Named barrier that also ANDs a predicate over the participating threads
// (reconverged first, as named_sync).
__device__ __forceinline__ bool named_and(bool v, int id, int n) {
    uint32_t r;
    __syncwarp();
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// ------------------------------------------------------------------ TMA

// 2-D tiled load of box {x..x+bx, y..y+by} into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t x, int32_t y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Contiguous global -> shared copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared -> global tile store through a tensor map (x a multiple of 16 bytes,
// y >= 0; rows past the tensor's extent are not written), tracked by the
// issuing thread's bulk async-groups: commit, then wait until the shared
// source may be overwritten (read) or the writes are done (all).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int32_t x, int32_t y, const void* src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)map),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Hint: bring `bytes` (multiple of 16, 16-byte aligned) of global memory into L2.
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"((uint64_t)src), "r"(bytes) : "memory");
}

// Per-thread asynchronous 16-byte global -> shared copy (both addresses
// 16-byte aligned); completion is tracked per thread by commit/wait groups,
// and only the issuing thread may read the bytes after its wait.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Non-coherent 32-bit global load (read-only data).
__device__ __forceinline__ int32_t ld_nc_s32(const void* p) { return __ldg(reinterpret_cast<const int32_t*>(p)); }
// Non-coherent 16-byte global load (read-only, 16-byte aligned): e.g. a tile record's
// header {first row, end row, first edge, edge count}.
__device__ __forceinline__ int4 ld_nc_v4s32(const void* p) { return __ldg(reinterpret_cast<const int4*>(p)); }

// ------------------------------------------------------------------ tcgen05

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem desc] * B[smem desc], BF16 inputs, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on bar once every previously issued tcgen05.mma of this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns: thread i of the warp receives lane (base lane + i).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 lanes x 16 consecutive 32-bit columns from registers: thread i writes lane (base lane + i).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------------ descriptors

// Swizzle code of the shared-memory descriptor for a span of S bytes.
__host__ __device__ constexpr uint32_t swz_code(int S) { return S == 128 ? 2u : (S == 64 ? 4u : 6u); }

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (16-byte units), descriptor version 1, swizzle mode.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)swz << 61;
    return d;
}

// Instruction descriptor of kind::f16 with BF16 A/B, FP32 D; a_mn / b_mn
// select MN-major operands.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn = 0, int b_mn = 0) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (r, c) of a row tile with `rows` rows and span S.
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int c, int rows, int S) {
    const int per = S / 2;                       // BF16 elements per block row
    const int blk = c / per;
    const uint32_t o = (uint32_t)r * S + (uint32_t)(c % per) * 2;
    const uint32_t sw = o ^ (((o >> 7) & (uint32_t)(S / 16 - 1)) << 4);
    return (uint32_t)blk * rows * S + sw;
}

// K-major descriptor of a row tile for the K-step starting at column k0
// (a multiple of 16): rows = M (or N), 8-row atoms S*8 bytes apart.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t base, int rows, int S, int k0) {
    const int per = S / 2;
    const uint32_t start = base + (uint32_t)(k0 / per) * rows * S + (uint32_t)(k0 % per) * 2;
    return sdesc(start, 16, 8 * S, swz_code(S));
}

// MN-major descriptor of a row tile whose rows are the K index, for the
// K-step of rows k0..k0+15 and the MN block starting at column n0 (a multiple
// of S/2): consecutive MN blocks are `rows*S` bytes apart (LBO), 8-row K
// groups are 8*S bytes apart (SBO).
__device__ __forceinline__ uint64_t mnmajor_desc(uint32_t base, int rows, int S, int k0, int n0) {
    const int per = S / 2;
    const uint32_t start = base + (uint32_t)(n0 / per) * rows * S + (uint32_t)k0 * S;
    return sdesc(start, (uint32_t)rows * S, 8 * S, swz_code(S));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void unpack_bf16x2(uint32_t u, float& lo, float& hi) {
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&u);
    float2 f = __bfloat1622float2(v);
    lo = f.x;
    hi = f.y;
}

// Store 8 FP32 values as BF16 at (r, c..c+7) of a row tile (c a multiple of 8).
__device__ __forceinline__ void st_tile8(uint8_t* tile, int r, int c, int rows, int S, const float* v) {
    uint4 u;
    u.x = pack_bf16x2(v[0], v[1]);
    u.y = pack_bf16x2(v[2], v[3]);
    u.z = pack_bf16x2(v[4], v[5]);
    u.w = pack_bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(tile + tile_off(r, c, rows, S)) = u;
}

// Load 8 BF16 values at (r, c..c+7) of a row tile as FP32.
__device__ __forceinline__ void ld_tile8(const uint8_t* tile, int r, int c, int rows, int S, float* v) {
    uint4 u = *reinterpret_cast<const uint4*>(tile + tile_off(r, c, rows, S));
    unpack_bf16x2(u.x, v[0], v[1]);
    unpack_bf16x2(u.y, v[2], v[3]);
    unpack_bf16x2(u.z, v[4], v[5]);
    unpack_bf16x2(u.w, v[6], v[7]);
}

}  // namespace tc
}  // namespace gnn
