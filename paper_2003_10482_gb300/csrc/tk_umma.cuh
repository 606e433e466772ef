// Building blocks of the 5th-generation tensor-core path (tcgen05): the
// shared-memory matrix descriptor of a K-major operand with the 128-byte
// swizzle, the instruction descriptor of kind::tf32 with FP32 accumulation,
// MMA issue and commit, tensor-memory (TMEM) allocation and loads, and the
// FP32 -> TF32 split that keeps FP32-level accuracy from TF32 products.
//
// Operand layout (K-major, 128-byte swizzle).  A tile of R rows and 32 FP32 /
// TF32 values per row (128 bytes) is stored as R/8 atoms of 8 rows x 128 bytes
// (1024 bytes each, 1024-byte aligned), atoms contiguous along the rows; the
// 16-byte chunk j of row r sits at chunk position j ^ (r mod 8) of its row.
// One MMA consumes K = 8 TF32 values (32 bytes) per row; the k-th group of 8
// is addressed by adding 32 k bytes to the descriptor's start address (the
// swizzle is a function of the address bits, so the atom stays aligned).
//
// Accumulator layout (cta_group::1, M = 128): row i of D is TMEM lane i,
// column j of D is TMEM column (base + j), one 32-bit column per FP32 value.
// Warp w of the CTA may read lanes 32 (w mod 4) .. 32 (w mod 4) + 31.
#pragma once
#include <stdint.h>

#include "tk_contract_impl.cuh"

namespace tk {
namespace umma {

// Byte offset of value k (0..31) of row r inside a 128-byte-swizzled K-major tile.
__host__ __device__ constexpr uint32_t sw128_offset(uint32_t r, uint32_t k) {
  return (r >> 3) * 1024u + (r & 7u) * 128u + ((((k >> 2) ^ r) & 7u) << 4) + (k & 3u) * 4u;
}

// Shared-memory matrix descriptor: start address, leading byte offset (not
// used by a swizzled K-major operand whose K per MMA fits one swizzle row),
// stride byte offset (distance between 8-row atoms: 1024 bytes), the
// descriptor version of tcgen05 (bit 46) and the swizzle mode (2 = 128 bytes).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t smem_addr) {
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: D in FP32 (bits 4-5 = 1), A and B in
// TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.  Valid shapes for cta_group::1: M = 64
// with N a multiple of 8, or M = 128 with N a multiple of 16, 16 <= N <= 256.
__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t M, uint32_t N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// D (TMEM) = A B^T (+ D when accumulate != 0); issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on `bar` when every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// TMEM allocation of `ncols` columns (a power of two >= 32) by one whole warp;
// the address is written to shared memory at `dst`.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane (warp-collective);
// the registers are valid after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  tmem_ld16_async(taddr, r);
  tmem_wait_ld();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Round an FP32 value to TF32 (10 explicit mantissa bits, nearest, ties away).
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// x = hi + lo + e with hi, lo TF32 and |e| <= 2^-11 |lo| <= 2^-22 |x|: the
// products hi*hi' + hi*lo' + lo*hi' then carry x*x' to about 2^-21 relative.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - hi);
}

}  // namespace umma
}  // namespace tk
