// Helpers shared by the tensor-core kernels with FP64-class accuracy (Fourier stage of the row
// analysis, degree-block rotations): digit splitting of double-float values into bfloat16
// integers, K-major canonical shared-memory planes, tcgen05 descriptors, bounded mbarrier waits
// and bulk copies.
//
// A value x with |x| < 2^e is represented as X = round(x 2^(42 - e)) = sum_j d_j 128^j with
// d_0..d_4 in [-64, 63] (balanced base 2^7) and the top digit d_5 the rest (|d_5| <= 128); every
// digit is an integer that bfloat16 holds exactly. Of the 36 digit products of a matrix product
// the 21 with j_a + j_b >= 5 are kept; products of equal j_a + j_b share one FP32 accumulator in
// tensor memory, exact because every sum stays below 2^24 (Ozaki-style error-free splitting).
#pragma once

#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "dfloat.cuh"
#include "tc_digits.cuh"

namespace shbim {
namespace tc {

constexpr int kMT = 128;         // rows per tile (MMA M = tensor-memory lanes)
constexpr int kKS = 16;          // K per MMA

// element (row n, k) of one K-major canonical plane of K = 16: 8-row x 16-byte core matrices,
// [row group][k chunk][row % 8][k % 8]
__host__ __device__ inline int canon16(int n, int k) { return ((n >> 3) * 2 + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory descriptor of a K = 16 canonical plane (no swizzle)
__device__ __forceinline__ uint64_t desc_k16(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(128u >> 4) << 16;   // leading-dimension byte offset: next 8-element k chunk
  d |= (uint64_t)(256u >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version; no swizzle
  return d;
}

// instruction descriptor of kind::f16 with bf16 A and B (K-major), f32 D, M = 128
__host__ __device__ inline uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kMT >> 4) << 24);
}

// nanoseconds of the device's global timer
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of parity `parity` of an mbarrier to complete, for at most limit_ns
// nanoseconds (the limit is the launching context's wait limit); false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  uint32_t done = 0;
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
    if (done) return true;
    const uint64_t t = global_ns();
    if (it == 0) t0 = t;
    else if (t - t0 > limit_ns) return false;
  }
}

// limit of the waits that drain a CTA's own copies and products after a timeout, before it frees
// its shared and tensor memory: long enough for any operation in flight to land
constexpr uint64_t kDrainNs = 2000000000ull;

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ uint32_t pack_bf16f(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // small integers: exact
  return *reinterpret_cast<const uint32_t*>(&v);
}

// untiled bulk copy global -> shared completing on an mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes));
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar)));
}

// one MMA: D[tmem] (+)= A[desc a] B[desc b]^T
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar)));
}

// 16 consecutive FP32 columns of the warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&a)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
        "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15])
      : "r"(addr));
}

// 8 consecutive FP32 columns of the warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_ld8(uint32_t addr, uint32_t (&a)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7])
               : "r"(addr));
}

// x 2^sh for a double-float (exact power-of-two scaling; ldexpf only where 2^sh is not normal)
__device__ __forceinline__ float2 scale2(dfl::df x, int sh) {
  if (sh >= -126 && sh <= 127) {
    const float f = __int_as_float((127 + sh) << 23);
    return make_float2(x.hi * f, x.lo * f);
  }
  return make_float2(ldexpf(x.hi, sh), ldexpf(x.lo, sh));
}

}  // namespace tc
}  // namespace shbim
