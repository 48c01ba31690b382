// Fifth-generation tensor core (tcgen05) helpers for TF32 contractions with FP32
// accumulators in tensor memory (TMEM), issued by one thread of the CTA.
//
// Operands live in shared memory in the canonical K-major layout without
// swizzle: the matrix is cut into core matrices of 8 rows x 16 bytes (8 x 4
// TF32 values), each stored as 128 contiguous bytes (row r of the core matrix
// at byte 16 r).  Core matrices that are neighbours along K are LBO = 128 bytes
// apart, neighbours along M (or N) SBO = 32 Kp bytes apart (Kp = K padded to a
// multiple of 8), so element (r, k) sits at byte
//   (r / 8) SBO + (k / 4) LBO + 16 (r % 8) + 4 (k % 4).
// One MMA consumes K = 8 (two core matrices along K); the K-step s starts at
// byte 256 s.  The accumulator of an M = 128 MMA occupies TMEM lanes 0..127
// (row i in lane i) and N consecutive columns (one FP32 value each); warp w of
// the CTA may read lanes 32 (w % 4) .. 32 (w % 4) + 31.
#pragma once
#include <cstdint>

namespace ttiga {
namespace tc {

constexpr int kLBO = 128;  // bytes between core matrices adjacent along K

__host__ __device__ constexpr int sbo_bytes(int kp) { return 32 * kp; }
// Byte offset of element (r, k) of a K-major operand with Kp (multiple of 8) padded columns.
__host__ __device__ constexpr int operand_offset(int r, int k, int kp) {
  return (r >> 3) * sbo_bytes(kp) + (k >> 2) * kLBO + 16 * (r & 7) + 4 * (k & 3);
}
// Bytes of an operand with `rows` (multiple of 8) rows and Kp padded columns.
__host__ __device__ constexpr int operand_bytes(int rows, int kp) { return rows * kp * 4; }

__device__ __forceinline__ uint32_t smem_u32addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets, descriptor version 1 (bits 46-48 = 0b001), base offset 0, relative LBO,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of tcgen05.mma kind::tf32: dense, D in FP32, A and B in
// TF32, both K-major, no negation, shape M x N (M = 64 or 128; N a multiple of 8
// for M = 64, of 16 for M = 128, up to 256).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TF32 value of x rounded to nearest (ties away), as the 32-bit pattern the MMA reads.
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// TMEM allocation by one whole warp: ncols (power of two, >= 32) columns; the TMEM
// address is written to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32addr(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A B^T (+ D when accumulate), one K = 8 step; issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}

// Arrive once on the mbarrier when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32addr(mbar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Make generic-proxy shared-memory stores visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init1(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval1(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32addr(bar)) : "memory");
}
// Wait for the phase with the given parity; false when `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity, long long limit) {
  const uint32_t addr = smem_u32addr(bar);
  for (long long spin = 0; spin < limit; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of the warp's 32 TMEM lanes: lane l of the warp gets
// row (lane base + l), columns col .. col + 15 of the address taddr (lane << 16 | col).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace tc
}  // namespace ttiga
