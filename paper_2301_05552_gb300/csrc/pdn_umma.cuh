// Blackwell (sm_100 family) tensor-core building blocks of the learned
// surrogate, in inline PTX: tcgen05.mma issued by one thread of the CTA,
// operands in shared memory (no-swizzle K-major core-matrix layout), the
// FP32 accumulator in tensor memory (TMEM), read back with tcgen05.ld.
//
// The network of the surrogate (10 -> 64 -> 64 -> 64 -> 10, ReLU, BF16
// operands, FP32 accumulation) is evaluated for 128 points at once, one point
// per thread of a 128-thread CTA: the activations of the 128 points form the
// A operand (M = 128 rows), the layer's weights W [out][in] the B operand
// (K-major: each output's input weights contiguous), and the layer's
// pre-activations land in TMEM lane t (= row t = thread t), columns 0..N-1.
//
// Core-matrix layout (no swizzle): a K-major operand of R rows and K columns
// of bf16 is stored as 8-row x 8-column core matrices of 128 contiguous bytes
// (row r of a core at byte 16 r); core (i, j) (rows 8i.., columns 8j..) sits
// at byte i * sbo + j * lbo with lbo = 128 (K-adjacent cores next to each
// other) and sbo = 16 K (one row band of K / 8 cores).  One MMA consumes
// K = 16 (two K-adjacent cores); the next K step starts 2 * lbo bytes on.
//
// Every wait on the MMA completion barrier is bounded; a wait that gives up
// reports it to the caller, which stops issuing work and raises an error
// status instead of hanging.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace pdn {
namespace umma {

// Byte offset of element (r, c) of a K-major bf16 operand with K columns in
// the core-matrix layout above.
__host__ __device__ constexpr uint32_t core_offset(int r, int c, int K) {
  return (uint32_t)((r >> 3) * (16 * K) + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between K-adjacent core matrices) and stride byte offset (between
// row-adjacent core matrices), all in 16-byte units; bits 46-48 hold the
// fixed value 0b001; base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D in FP32 (bits 4-5 = 1), A and B in
// BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at
// bits 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// TMEM allocation of ncols columns (a power of two >= 32) by one whole warp;
// the base address is written to shared memory at dst.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory writes of this thread become visible to the tensor core (the
// async proxy); each writing thread fences before the CTA barrier.
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait until the barrier's phase with the given parity has completed, for at
// most max_tries polls; false when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t max_tries) {
  const uint32_t a = saddr(bar);
  for (uint32_t k = 0; k < max_tries; ++k) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// D[tmem] (+)= A B with A, B given by shared-memory descriptors (one thread).
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
  const uint32_t acc = accumulate ? 1u : 0u;
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// The barrier receives one arrival when every MMA issued so far by this
// thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes
// 32 w .. 32 w + 31: taddr carries the lane in bits 16-31).  The load and
// its wait are one asm statement, so no use of the registers can be
// scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace umma
}  // namespace pdn
