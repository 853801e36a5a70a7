// Fifth-generation tensor core (tcgen05) building blocks, inline PTX for
// sm_100a / sm_103a: tensor-memory (TMEM) allocation, shared-memory matrix
// descriptors, single-CTA MMA issue and completion, TMEM loads.
//
// Conventions measured on GB300 with dedicated probes (descriptor fields,
// data-path layouts), as used by the normalisation-matrix kernels:
//   * operands in shared memory without swizzling are tiled by "core
//     matrices" of 8 rows x 16 bytes (128 contiguous bytes); the
//     descriptor's leading-dimension offset (LBO) is the byte distance
//     between core matrices adjacent along K, the stride-dimension offset
//     (SBO) the distance between core matrices adjacent along M (or N), for
//     K-major and MN-major operands alike; in an MN-major core matrix the
//     16 contiguous bytes are 8 consecutive M (N) elements of one k;
//   * an M = 128 accumulator has row r in TMEM lane r; an M = 64 one has
//     rows 16q .. 16q + 15 in lanes 32q .. 32q + 15 (q = 0..3); column n
//     is TMEM column (base + n), 32 bits each;
//   * the fp32 accumulation of the MMA is not rounded to nearest (sums are
//     truncated and small addends can lose bits at alignment), so exact
//     results need every partial sum to be an integer below 2^24 in a
//     common unit (see the normalisation-matrix kernel).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "async_copy.cuh"

namespace tdmix {

// Allocates `ncols` TMEM columns (a power of two >= 32) for this CTA and
// writes the base address to *dst (shared memory).  Executed by one whole
// warp; the permit is relinquished so later allocations cannot block.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Frees what tmem_alloc took (the same whole warp).
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of tcgen05 operations across a thread barrier.
__device__ __forceinline__ void tc_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Makes this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor without swizzling: start address,
// LBO (K-direction core-matrix stride) and SBO (M/N-direction stride), all
// in bytes and multiples of 16; bits 46-48 hold the fixed value 0b001.
__device__ __forceinline__ uint64_t smem_matrix_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t(lbo >> 4) << 16;
  d |= uint64_t(sbo >> 4) << 32;
  d |= 1ull << 46;
  return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B, fp32 accumulator,
// both operands MN-major, shape M x N (K = 16 per instruction).
__host__ __device__ constexpr uint32_t idesc_bf16_mn_major(int M, int N) {
  return (1u << 4)                    // D format: f32
         | (1u << 7) | (1u << 10)     // A, B format: bf16
         | (1u << 15) | (1u << 16)    // A, B MN-major
         | (uint32_t(N >> 3) << 17)   // N / 8
         | (uint32_t(M >> 4) << 24);  // M / 16
}

// D (TMEM) = A B (+ D if accumulate), issued by one thread.
__device__ __forceinline__ void tc_mma_bf16(uint32_t d_taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_taddr),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u)
      : "memory");
}

// The mbarrier `bar` completes one phase when every tcgen05 operation this
// thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane (lane quarter of
// the warp, warp-collective); complete after tmem_wait_ld.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tdmix
