// Fifth-generation tensor-core primitives for sm_103a (inline PTX): tensor
// memory (TMEM) allocation, shared-memory matrix descriptors for the K-major
// 128-byte-swizzled operand layout, tcgen05.mma of kind::tf32 with the A
// operand in shared memory or in TMEM, completion through an mbarrier, and
// tcgen05.ld of accumulator rows. Used by the tensor-core segment sweep.
//
// Operand layout (K-major, 128-byte swizzle). An R x Kc tile of 32-bit
// elements (Kc a multiple of 32) is stored as Kc/32 K-blocks; K-block kb holds
// row r's elements kb*32 .. kb*32+31 in one 128-byte line at byte offset
// kb*R*128 + r*128, with its eight 16-byte chunks permuted by chunk ^ (r % 8).
// Eight consecutive rows form one 1024-byte swizzle atom; tiles start on a
// 1024-byte boundary. A descriptor for the 8-element K step s of a tile
// points at K-block s/4, byte (s%4)*32 inside the line, with the atom stride
// (1024 bytes) as its stride byte offset.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lqr {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) in an R-row swizzled K-major tile.
__host__ __device__ __forceinline__ uint32_t sw_off(int R, int r, int k) {
  const uint32_t kb = (uint32_t)k >> 5, kin = (uint32_t)k & 31;
  const uint32_t chunk = (kin >> 2) ^ ((uint32_t)r & 7);
  return kb * (uint32_t)R * 128u + (uint32_t)r * 128u + chunk * 16u + (kin & 3) * 4u;
}
__device__ __forceinline__ float& sw_at(float* tile, int R, int r, int k) {
  return *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(tile) + sw_off(R, r, k));
}
__device__ __forceinline__ float sw_get(const float* tile, int R, int r, int k) {
  return *reinterpret_cast<const float*>(reinterpret_cast<const unsigned char*>(tile) + sw_off(R, r, k));
}

// Shared-memory matrix descriptor: start address, stride byte offset 1024
// (one swizzle atom of 8 rows), fixed field 0b001 at bits 46-48, 128-byte
// swizzle (layout type 2 in bits 61-63). The leading byte offset is unused
// for K-major swizzled operands whose K step stays inside one 128-byte line.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused), 16 bytes
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}
// Descriptor of K step s (8 TF32 elements) of an R-row tile at saddr.
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr, int R, int s) {
  return sdesc(saddr + (uint32_t)(s >> 2) * (uint32_t)R * 128u + (uint32_t)(s & 3) * 32u);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M x N (M = 128: N a multiple of 16 up to 256), optional negated A.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N, bool neg_a) {
  return (1u << 4)                        // accumulator format F32
         | (2u << 7)                      // A format TF32
         | (2u << 10)                     // B format TF32
         | ((neg_a ? 1u : 0u) << 13)      // negate A
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

// D[tmem] (+)= A[smem] B[smem]'  (accumulate when acc != 0); one thread issues.
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc)
      : "memory");
}
// The same with A read from TMEM (lane = row of A, column = K index).
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(acc)
      : "memory");
}
// The mbarrier at bar receives one arrival when every tcgen05.mma this thread
// issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// Generic-proxy shared-memory writes made visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// TMEM allocation by one whole warp; the base address lands in *dst (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane (warp w reads
// lanes 32 (w % 4) .. +31; taddr carries that lane base in bits 31:16).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// mbarrier helpers
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
// One arrival that also expects `bytes` of asynchronous copies on the barrier.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// Bulk asynchronous copy global -> shared, completion counted in bytes on bar;
// bytes a multiple of 16, both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Waits for the phase with the given parity to complete; false when `limit`
// polls (non-blocking tests, 32 ns apart) pass without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_test_wait(bar, parity)) return true;
    __nanosleep(32);
  }
  return false;
}

}  // namespace tc
}  // namespace lqr
