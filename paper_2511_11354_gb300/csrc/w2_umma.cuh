// Building blocks of the 5th-generation tensor core path (tcgen05, sm_103a):
// the shared-memory matrix descriptor, the instruction descriptor of
// kind::f16, tensor-memory (TMEM) allocation, MMA issue and completion,
// TMEM loads and stores, and mbarrier waits with a time bound.
//
// Operand layout used throughout (the "no swizzle" canonical layout of the
// PTX ISA's tcgen05 matrix descriptors): a 16-bit matrix is cut into core
// matrices of 8 rows x 16 bytes (8 x 8 elements), each stored as 128
// contiguous bytes (row r at byte 16 r).  For a K-major operand the rows of
// a core matrix run along M (or N) and its 8 elements along K; for an
// MN-major operand the rows run along K and the elements along M (or N).
// The descriptor gives the byte distance between core matrices adjacent
// along K (leading-dimension byte offset) and along M or N (stride-dimension
// byte offset).
#pragma once
#include <stdint.h>

namespace w2 {
namespace umma {

// Shared-memory matrix descriptor, 64 bits:
//   bits  0-13  start address >> 4
//   bits 16-29  leading-dimension byte offset >> 4 (K-direction core-matrix stride)
//   bits 32-45  stride-dimension byte offset >> 4  (M/N-direction core-matrix stride)
//   bits 46-48  fixed value 0b001
//   bits 49-51  matrix base offset (0: no swizzle)
//   bit  52     leading-dimension offset mode (0: byte offset)
//   bits 61-63  swizzling mode (0: none)
// Addresses and offsets are multiples of 16 bytes below 256 KB.
__host__ __device__ constexpr uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Instruction descriptor of tcgen05.mma kind::f16, 32 bits, for BF16 A and B
// and an FP32 accumulator:
//   bits  0-1  sparsity selector (0)      bit 2  sparsity (0: dense)
//   bit   3    saturate (0)               bits 4-5  D format (1: F32)
//   bits  7-9  A format (1: BF16)         bits 10-12  B format (1: BF16)
//   bit  13    negate A (0)               bit 14  negate B (0)
//   bit  15    A major (0: K, 1: MN)      bit 16  B major (0: K, 1: MN)
//   bits 17-22 N >> 3                     bits 24-28  M >> 4
//   bits 30-31 maximum shift (0; weight-stationary form only)
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shapes a cta_group::1 kind::f16 MMA accepts: M = 64 with N a multiple of
// 8, or M = 128 with N a multiple of 16, N in [8 or 16, 256].
__host__ __device__ constexpr bool shape_ok(int M, int N) {
  return (M == 64 && N >= 8 && N <= 256 && N % 8 == 0) || (M == 128 && N >= 16 && N <= 256 && N % 16 == 0);
}

// Byte offset of element (r, c) in a tiled 16-bit matrix of `ncol` columns
// (core matrix (r / 8, c / 8) at ((r / 8) (ncol / 8) + c / 8) 128 bytes,
// element at row r % 8, column c % 8 inside it).
__host__ __device__ constexpr uint32_t tile_off(int r, int c, int ncol) {
  return (uint32_t)((((r >> 3) * (ncol >> 3) + (c >> 3)) << 7) + ((r & 7) << 4) + ((c & 7) << 1));
}

#if defined(__CUDACC__)
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// TMEM allocation by one whole warp: `ncols` columns (a power of two, at
// least 32) of all 128 lanes; the TMEM address is written to *slot (shared
// memory).  The same warp releases them with tmem_dealloc before the CTA ends.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of tensor-core work around thread synchronisation.
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Shared-memory writes of this thread made visible to the tensor core's operand reads.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// D[tmem] (+)= A B, A and B described by shared-memory descriptors; issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// One arrival on *mbar once every MMA this thread has issued is complete.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// One arrival on *mbar (release: this thread's earlier shared-memory writes,
// with fence_proxy_async before it also to the tensor core, happen before
// the phase completes).
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(mbar)) : "memory");
}
// Wait for the phase with parity `parity` of *mbar to complete, for at most
// `limit` SM clock cycles; false if it did not.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(mbar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// 32 lanes x 16 columns of 32-bit TMEM words: thread t of the warp receives
// lane (lane of taddr) + t, columns (column of taddr) .. + 15.  A warp may
// touch only the 32 lanes of its quarter (warp index mod 4).  The load and
// its completion wait are one statement, so the values are ready on return.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
// The same for 32 columns.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
// The store counterpart (same lanes and columns), with its completion wait.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
#endif  // __CUDACC__

}  // namespace umma
}  // namespace w2
