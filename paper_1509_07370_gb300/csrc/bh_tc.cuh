// tcgen05 helpers shared by the tensor-core network evaluator (bh_mlp_tc.cu)
// and the tensor-core learned walk (bh_walk_learned_tc.cu): shared-memory
// matrix and instruction descriptors, MMA issue and commit, bounded mbarrier
// waits, tensor-memory loads, fences, and the bf16-pair GELU.
#pragma once
#include "bh_internal.cuh"

namespace bhg {
namespace {

// Bounded waits on the MMA barrier: at most kTcSpinLimit tries, each of which
// suspends the thread for at most kTcSuspendNs (it resumes as soon as the
// phase completes), so a wait that runs out takes about a second.
constexpr int kTcSpinLimit = 1 << 20;
constexpr uint32_t kTcSuspendNs = 1000;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(accumulate));
}
__device__ __forceinline__ void commit(unsigned long long *mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, uint32_t phase,
                                          int limit = kTcSpinLimit) {
  const uint32_t a = smem_u32(mbar);
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(phase), "r"(kTcSuspendNs)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes made visible to the tensor core.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 16 consecutive FP32 columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float v[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]),
        "=f"(v[14]), "=f"(v[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ float tmem_ld1(uint32_t addr) {
  float v;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=f"(v) : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  return v;
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// 2 GELU(a) in bf16 pairs, the same operations as the learned walk.
__device__ __forceinline__ uint32_t gelu2x(float lo, float hi) {
  const uint32_t a = bf16x2(lo, hi);
  uint32_t a2, p, z, t, r;
  asm("mul.rn.bf16x2 %0, %1, %1;" : "=r"(a2) : "r"(a));
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(p) : "r"(a2), "r"(0x3d123d12u), "r"(0x3f4c3f4cu));
  asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(z) : "r"(a), "r"(p));
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(z));
  asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(r) : "r"(a), "r"(t));
  return r;
}

// Row r (0..127) of a tile through the three layers of 64 columns: reads its
// accumulator columns (+ bias) from tensor memory, applies the GELU and
// writes the row of the next layer's K = 64 operand.
__device__ __forceinline__ void tc_epilogue(uint32_t col_addr, const float *bias, uint16_t *a2,
                                            int r) {
  unsigned char *base = reinterpret_cast<unsigned char *>(a2);
#pragma unroll
  for (int c0 = 0; c0 < 64; c0 += 16) {
    float v[16];
    tmem_ld16(col_addr + c0, v);
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float b0 = bias ? bias[c0 + 2 * i] : 0.0f, b1 = bias ? bias[c0 + 2 * i + 1] : 0.0f;
      w[i] = gelu2x(v[2 * i] + b0, v[2 * i + 1] + b1);
    }
    *reinterpret_cast<uint4 *>(base + tc_canon(r, c0, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(base + tc_canon(r, c0 + 8, 64)) =
        make_uint4(w[4], w[5], w[6], w[7]);
  }
}

}  // namespace
}  // namespace bhg
