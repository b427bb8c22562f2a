// Small tcgen05, mbarrier and TMA helpers shared by the tensor-core kernels and
// the double-float contraction: shared-memory matrix descriptors (K-major, no
// swizzle), instruction descriptors, barrier set-up and a bounded wait, and a
// three-dimensional tensor-map load.
#pragma once
#include <cstdint>

namespace fbc {
namespace tc {

constexpr int kWaitLimit = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K-direction core
// matrix) byte offset, stride (8-row group) byte offset, fixed version bits,
// no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = bf16, 2 = tf32),
// both K-major, N >> 3 and M >> 4.
__device__ __forceinline__ uint32_t idesc(int fmt, int M, int N) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) of a bf16 operand stored K-major in 8-row x
// 16-byte core matrices: rows of a core matrix 16 bytes apart, core matrices
// along K 128 bytes apart (LBO), 8-row groups sbo bytes apart (SBO).
__device__ __forceinline__ uint32_t canon_bf16(int row, int k, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count));
}

// One arrival that also announces `bytes` of asynchronous copies to come.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(m)),
                 "r"(bytes)
                 : "memory");
}

// Tiled tensor-map load of one box at coordinates (c0, c1, c2), innermost
// first, into shared memory at `dst` (128-byte aligned); completion is counted
// on the barrier `m` in bytes.  `map` is the generic address of a tensor map in
// kernel-parameter (__grid_constant__), constant or global memory.  Coordinates
// outside the tensor read the map's fill value (zero).  c0 times the element
// size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* map, uint64_t* m, int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(m))
        : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t phase) {
    for (int it = 0; it < kWaitLimit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(m)), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t id, uint32_t accum) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(id), "r"(accum));
}

__device__ __forceinline__ void commit(uint64_t* m) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m)));
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
          "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(u[i]);
}

// Pipeline wait: bounded by `limit` polls, and gives up as soon as another role has set *abort.
__device__ __forceinline__ bool wait_or_abort(uint64_t* m, uint32_t parity, volatile int* abort, int limit) {
    for (int it = 0; it < limit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(m)), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 255 && *abort) return false;
    }
    return false;
}

// wait_or_abort for a role thread that has nothing else to do meanwhile: each poll may suspend the
// thread for up to about hint_ns nanoseconds (it resumes as soon as the phase completes), so a waiting
// thread takes no issue slots from the warps that work.  Bounded by `limit` polls.
__device__ __forceinline__ bool wait_or_abort_sleep(uint64_t* m, uint32_t parity, volatile int* abort, int limit,
                                                    uint32_t hint_ns) {
    for (int it = 0; it < limit; it++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(m)), "r"(parity), "r"(hint_ns)
            : "memory");
        if (ok) return true;
        if ((it & 15) == 15 && *abort) return false;
    }
    return false;
}

// Named barrier 1 among the NT threads of the builder warps that also returns,
// to every one of them, whether any passed flag != 0: a decision all of them
// take alike.
template <int NT = 256>
__device__ __forceinline__ bool builders_sync_any(int flag) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.s32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(flag), "n"(NT)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// 4 bytes, or zero when src_bytes is 0
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// 16 bytes, of which the first src_bytes (0 or 16) come from global memory and the rest are zero
__device__ __forceinline__ void cp_async16z(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}

// 8 consecutive FP32 accumulator columns of this thread's TMEM lane (no wait: follow with tcgen05.wait::ld)
__device__ __forceinline__ void ld8_nowait(uint32_t taddr, uint32_t (&u)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(m))
        : "memory");
}

}  // namespace tc
}  // namespace fbc
