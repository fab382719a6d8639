// Fifth-generation tensor-core primitives (tcgen05, sm_103a) as inline PTX: tensor-memory allocation,
// one-thread MMA issue with shared-memory matrix descriptors, completion through an mbarrier with a
// bounded wait, and tensor-memory loads for the epilogue.
//
// Operand layout used by every caller: K-major, no swizzle, in blocks of one MMA K step (16 BF16 =
// 32 bytes of K) by 128 rows.  Inside a block, the 8-row x 16-byte core matrices of rows 8g..8g+7
// sit at 256 g bytes (stride between core matrices along M/N: SBO = 256) and the two core matrices
// of the K step at +0 and +128 bytes (stride along K: LBO = 128); a row's 16 bytes are contiguous.
// One block is 4,096 bytes; the MMA of K step s reads block s only.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace srbe {
namespace tc {

constexpr int kRows = 128;            // rows of an operand block (the MMA's M, or N of the B operand)
constexpr int kKstep = 16;            // BF16 elements of K per MMA
constexpr int kBlockBytes = 4096;     // one K step of a 128-row operand
constexpr int kBlockElems = kBlockBytes / 2;

// BF16 element index of (row r, k) in a blocked operand
__device__ __forceinline__ int off(int r, int k) {
  return (k >> 4) * kBlockElems + (r >> 3) * 128 + ((k >> 3) & 1) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, LBO, SBO (bytes, multiples of 16), descriptor
// version 1, base offset 0, no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint64_t block_desc(const void *block) { return desc(smem_addr(block), 128, 256); }

// instruction descriptor of kind::f16 with BF16 A and B (K-major), FP32 accumulator, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (tensor memory) (+)= A B^T, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate ? 1u : 0u)
      : "memory");
}

// the mbarrier arrives once every MMA this thread issued before has completed
__device__ __forceinline__ void commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

// waits for the phase with the given parity to complete; false after max_tries polls
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, int max_tries) {
  uint32_t done = 0;
  for (int i = 0; i < max_tries && !done; ++i)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
  return done != 0;
}

// tensor-memory allocation by one whole warp: ncols (a power of 2, >= 32) columns, base written to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's tensor-memory lane (warp w reads lanes 32w..32w+31)
__device__ __forceinline__ void ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// x = hi + lo with hi = bf16(x) (round to nearest) and lo = bf16(x - hi).  The product of two split
// operands taken as hi hi + hi lo + lo hi (lo lo dropped) keeps about 16 significand bits.
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// eight consecutive K values of one row (k0 a multiple of 8) split into BF16 (hi, lo) and stored as
// two 16-byte chunks: the row's contiguous 16 bytes of the blocked layout in each operand
__device__ __forceinline__ void store8_split(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int r, int k0, const float *v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(v[2 * q], h0, l0);
    split_bf16(v[2 * q + 1], h1, l1);
    h[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  *reinterpret_cast<uint4 *>(hi + off(r, k0)) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4 *>(lo + off(r, k0)) = make_uint4(l[0], l[1], l[2], l[3]);
}

}  // namespace tc
}  // namespace srbe
