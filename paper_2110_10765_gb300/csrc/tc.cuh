// Blackwell (sm_103a) fifth-generation tensor-core helpers in inline PTX:
// tensor-memory (TMEM) allocation, tcgen05.mma from shared-memory operand
// descriptors, completion through an mbarrier with a bounded wait, and
// TMEM -> register loads.
//
// Operand tiles are stored without swizzling in the canonical K-major
// layout: an R x K tile (R rows of the M or N dimension, K contiguous) is a
// grid of 8-row x 16-byte "core matrices" of 128 contiguous bytes (row r of a
// core matrix at byte 16 r); core matrices adjacent along K are LBO bytes
// apart and those adjacent along R are SBO bytes apart.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace ci {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (R-direction) byte offsets, the fixed descriptor version bit, no
// swizzle.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16 with FP16 A and B, FP32 accumulator,
// both operands K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[adesc] B[bdesc], issued by one thread.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        bool accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate));
}

// The mbarrier arrives once every MMA issued so far by this thread is done.
__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
        smem_addr(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// One arrival of this thread (release: its earlier shared-memory writes are
// visible to whoever waits on the phase).
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(mbar)) : "memory");
}

// One arrival that also announces `bytes` of bulk copies completing on the
// current phase.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// Tensor (TMA) copy of the box at column x (x * element size a multiple of
// 16 bytes), row y of a 2-D tensor map into shared memory, completing on the
// mbarrier; elements outside the tensor are filled with zeros.
__device__ __forceinline__ void tma_2d(void *dst_smem, const void *map, int x, int y, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_addr(dst_smem)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(mbar))
        : "memory");
}

// Barrier `id` (1..15) over `nthreads` threads (whole warps) of the CTA.
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// Wait for phase `parity` of the mbarrier to complete, at most max_iter
// polls; returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int max_iter) {
    uint32_t done = 0;
    for (int it = 0; it < max_iter && !done; ++it) {
        asm volatile(
            "{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.b32 %0, 1, 0, q;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
    }
    return done != 0;
}

// TMEM allocation by one whole warp: the base address goes to *dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(dst)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(base), "r"(ncols));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Generic-proxy stores to shared memory become visible to the tensor core.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// NV (2 or 4) consecutive columns at each of taddr + 8 t (t = 0..7) of this
// thread's lane, waited for: v[NV t + c] = column taddr + 8 t + c.
template <int NV>
__device__ __forceinline__ void ld8xN(uint32_t taddr, float v[8 * NV]) {
    static_assert(NV == 2 || NV == 4, "two or four columns");
    uint32_t r[8 * NV];
    if constexpr (NV == 4) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%32 + 0];\n"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%32 + 8];\n"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%32 + 16];\n"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%12,%13,%14,%15}, [%32 + 24];\n"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%16,%17,%18,%19}, [%32 + 32];\n"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%20,%21,%22,%23}, [%32 + 40];\n"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%24,%25,%26,%27}, [%32 + 48];\n"
            "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%28,%29,%30,%31}, [%32 + 56];\n"
            "tcgen05.wait::ld.sync.aligned;\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%16 + 0];\n"
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%2,%3}, [%16 + 8];\n"
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4,%5}, [%16 + 16];\n"
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%6,%7}, [%16 + 24];\n"
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%8,%9}, [%16 + 32];\n"
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%10,%11}, [%16 + 40];\n"
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%12,%13}, [%16 + 48];\n"
            "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%14,%15}, [%16 + 56];\n"
            "tcgen05.wait::ld.sync.aligned;\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
    }
#pragma unroll
    for (int i = 0; i < 8 * NV; ++i) v[i] = __uint_as_float(r[i]);
}

// Eight consecutive columns at each of taddr + 64 p (p = 0..3) of this
// thread's lane, waited for: v[8 p + c] = column taddr + 64 p + c.
__device__ __forceinline__ void ld4x8(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%32 + 0];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%32 + 64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%32 + 128];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24,%25,%26,%27,%28,%29,%30,%31}, [%32 + 192];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace ci
