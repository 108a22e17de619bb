// tc.cuh -- 5th-generation tensor core (tcgen05) building blocks for sm_103a, in inline PTX:
// tensor-memory allocation, shared-memory matrix descriptors, the single-thread MMA issue,
// completion through an mbarrier, and accumulator read-back.
//
// Operand layout used throughout: K-major, no swizzle. A matrix of R rows (the M or N index)
// and K columns (the reduction index) is stored as "core matrices" of 8 rows x 16 bytes
// (8 rows x 4 tf32 values); core matrix (r / 8, k4) with k4 = k * elem / 16 sits at byte
//     (r / 8) * SBO + k4 * LBO,     row r % 8 at +16 * (r % 8) inside it.
// With LBO = 128 (K-adjacent core matrices contiguous) and SBO = (K * elem / 16) * 128, one
// MMA with K = 32 bytes (8 tf32 or 16 bf16 values) starts at +256 bytes per K step.
//
// Every wait on an mbarrier is bounded in time (the call's limit); a wait that gives up
// records MPJSVD_STATUS_TIMEOUT and returns false.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace mpj {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- shared-memory matrix descriptor (K-major, no swizzle)
__device__ __forceinline__ uint64_t tc_desc(const void* smem_tile, uint32_t lbo, uint32_t sbo)
{
    const uint32_t a = smem_u32(smem_tile);
    uint64_t d = 0;
    d |= (uint64_t)((a & 0x3FFFFu) >> 4);          // bits 0-13: start address >> 4
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;   // bits 16-29: leading-dimension byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;   // bits 32-45: stride-dimension byte offset
    d |= (uint64_t)1 << 46;                        // bits 46-47: descriptor version 1
    // base offset 0, absolute LBO mode 0, layout (bits 61-63) 0 = no swizzle
    return d;
}

// ---- instruction descriptors (dense, D = F32, A and B K-major)
// kind::tf32: A, B = TF32 (format 2); kind::f16 with bf16 operands: format 1.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, uint32_t ab_format)
{
    return (1u << 4)                       // bits 4-5: D format F32
           | (ab_format << 7)              // bits 7-9: A format
           | (ab_format << 10)             // bits 10-12: B format
           | ((uint32_t)(N >> 3) << 17)    // bits 17-22: N >> 3
           | ((uint32_t)(M >> 4) << 24);   // bits 24-28: M >> 4
}
constexpr uint32_t kTcFmtTF32 = 2;
constexpr uint32_t kTcFmtBF16 = 1;

// ---- tensor memory (one warp allocates / frees; the address is written to shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(smem_dst)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Asynchronous global -> shared copies of one thread (cp.async): `bytes` of the 16 (or 4)
// are read from src, the rest of the destination is zero-filled; completion is per thread,
// by commit groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---- MMA: D[tmem] (+)= A[smem] * B[smem]^T (both K-major), issued by one thread
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                           uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate) : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(mbar)) : "memory");
}

// ---- accumulator read-back: lanes 32 * (warp % 4) .. + 31, 16 consecutive 32-bit columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- mbarrier (one arrival per phase: the commit)
__device__ __forceinline__ void mbar_init(uint64_t* mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(smem_u32(mbar)), "r"(parity) : "memory");
    return ok != 0;
}
// Every thread waits (bounded) for the completion of the phase with this parity. Returns false
// (all threads) if the wait gave up or the call failed elsewhere; a wait that ran out of time
// records MPJSVD_STATUS_TIMEOUT. All threads of the CTA must call it.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, DevState* st)
{
    const uint64_t t0 = globaltimer_ns(), lim = spin_limit_ns(st);
    unsigned spins = 0;
    int ok = 1;
    while (!mbar_test(mbar, parity)) {
        if ((++spins & 1023u) == 0) {
            if (call_failed(st)) { ok = 0; break; }
            if (globaltimer_ns() - t0 > lim) {
                atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                ok = 0;
                break;
            }
        }
    }
    ok = __syncthreads_and(ok);
    if (ok) tc_fence_after();
    return ok != 0;
}

// One thread waits (bounded) for the phase with this parity; false if it gave up (a wait that
// ran out of time records MPJSVD_STATUS_TIMEOUT) or the call failed elsewhere.
__device__ __forceinline__ bool mbar_wait1(uint64_t* mbar, uint32_t parity, DevState* st)
{
    const uint64_t t0 = globaltimer_ns(), lim = spin_limit_ns(st);
    unsigned spins = 0;
    while (!mbar_test(mbar, parity)) {
        if ((++spins & 1023u) == 0) {
            if (call_failed(st)) return false;
            if (globaltimer_ns() - t0 > lim) {
                atomicOr(&st->status, MPJSVD_STATUS_TIMEOUT);
                return false;
            }
        }
    }
    return true;
}

// TF32 rounding (round to nearest, ties away) of a binary32 value: hi part of the 3-term split
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace mpj
