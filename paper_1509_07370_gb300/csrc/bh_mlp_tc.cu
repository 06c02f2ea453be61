// bh_mlp_eval: the learned correction's network evaluated on a batch of pair
// feature rows with the fifth-generation tensor cores (tcgen05).
//
// One CTA is one warpgroup (4 warps) and works on tiles of 128 rows:
//   layer 1: D1[128 x 64]  = A1[128 x 16] B1^T   (1 MMA, K = 16)
//   layer 2: D2[128 x 64]  = A2[128 x 64] B2^T   (4 MMAs, K = 16 each)
//   layer 3: D3[128 x 16]  = A3[128 x 64] B3^T   (4 MMAs; column 0 is y)
// A and B are bf16 in shared memory in the canonical K-major layout without
// swizzle (core matrices of 8 rows x 16 bytes; the next core matrix along K
// is 128 bytes on, the next along M/N K/8 x 128 bytes on); the accumulators
// are FP32 in tensor memory (128 lanes = the tile's rows; D1 and D3 in
// columns 0.., D2 in columns 64..).  One thread issues the MMAs and commits
// them to an mbarrier; after each layer every warp reads its own 32 lanes
// (rows 32w .. 32w+31) back with tcgen05.ld, applies the bias and the GELU
// exactly as the learned walk does (2 GELU(a) in bf16 pairs; the next
// layer's weights are stored halved), and writes the next layer's A operand.
// b1 enters through a constant input 10, as in the walk.
//
// Waits on the mbarrier are bounded: on time-out the kernel raises a flag,
// stops, and the call returns BH_ERR_DEVICE_TIMEOUT.  probe_limit > 0 is the
// test of that path: the MMA-issuing thread issues and commits nothing, so
// the first wait (limited to probe_limit tries) runs out on a barrier no one
// arrives at, with no tensor-core work in flight; the kernel then takes the
// same failure path as a real time-out (flag, drain wait, tensor-memory
// release).
#include "bh_tc.cuh"

namespace bhg {
namespace {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr uint32_t kTmemCols = 128;

struct __align__(1024) TcSmem {
  uint16_t a1[kTcRows * 16];  // features, K = 16
  uint16_t a2[kTcRows * 64];  // hidden activations, K = 64 (layer-2 and layer-3 input)
  MlpTc w;                    // weights (canonical layout) and biases
  uint32_t tmem;              // tensor-memory base from tcgen05.alloc
  int unused;
  unsigned long long mbar;    // MMA completion
};

__global__ void __launch_bounds__(kTcThreads)
    k_mlp_tc(int64_t n, const float *__restrict__ x, const MlpTc *__restrict__ wts,
             float *__restrict__ y, unsigned *flags, int probe_limit) {
  extern __shared__ unsigned char smem_raw[];
  TcSmem &S = *reinterpret_cast<TcSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, warp = t >> 5;
  {  // weights (already in the canonical layout) and biases
    const uint4 *src = reinterpret_cast<const uint4 *>(wts);
    uint4 *dst = reinterpret_cast<uint4 *>(&S.w);
    for (int i = t; i < (int)(sizeof(MlpTc) / 16); i += kTcThreads) dst[i] = src[i];
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
    fence_async_smem();  // the initialised barrier, visible to the tensor core's arrivals
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
  const int r = t;  // this thread's row of the tile (its TMEM lane)
  uint32_t phase = 0;
  bool ok = true;
  const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    // features of row r, bf16, input 10 = 1 (bias), 11..15 = 0
    const int64_t row = tile * kTcRows + r;
    uint32_t w[8] = {0u, 0u, 0u, 0u, 0u, 0x3f80u, 0u, 0u};
    if (row < n) {
      const float *f = x + row * kMlpIn;
      w[0] = bf16x2(f[0], f[1]);
      w[1] = bf16x2(f[2], f[3]);
      w[2] = bf16x2(f[4], f[5]);
      w[3] = bf16x2(f[6], f[7]);
      w[4] = bf16x2(f[8], f[9]);
    }
    unsigned char *a1 = reinterpret_cast<unsigned char *>(S.a1);
    *reinterpret_cast<uint4 *>(a1 + tc_canon(r, 0, 16)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(a1 + tc_canon(r, 8, 16)) = make_uint4(w[4], w[5], w[6], w[7]);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0 && probe_limit == 0) {  // layer 1
      mma(tmem, sdesc(S.a1, 128, 256), sdesc(S.w.b1, 128, 256), idesc(128, 64), 0u);
      commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase, probe_limit ? probe_limit : kTcSpinLimit));
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    tc_epilogue(lane_base, nullptr, S.a2, r);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {  // layer 2
      for (int kk = 0; kk < 4; ++kk)  // K = 16 steps: two core matrices (256 bytes) each
        mma(tmem + 64, sdesc(S.a2 + 128 * kk, 128, 1024), sdesc(S.w.b2 + 128 * kk, 128, 1024),
            idesc(128, 64), kk > 0);
      commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase));
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    tc_epilogue(lane_base + 64, S.w.bias2, S.a2, r);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {  // layer 3 (N = 16; column 0 is the output)
      for (int kk = 0; kk < 4; ++kk)
        mma(tmem, sdesc(S.a2 + 128 * kk, 128, 1024), sdesc(S.w.b3 + 128 * kk, 128, 1024),
            idesc(128, 16), kk > 0);
      commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase));
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    const float v = tmem_ld1(lane_base);
    if (row < n) y[row] = v + S.w.bias3;
    fence_before();
    __syncthreads();
    fence_after();
  }
  if (!ok) {  // give the MMAs in flight (phase not reached) a last bounded wait, report
    if (t == 0) atomicOr(flags, 1u);
    mbar_wait(&S.mbar, phase);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
}

}  // namespace

// Dynamic shared memory per CTA: at least 56 KB, so that at most 4 CTAs share
// an SM and their tensor memory (4 x 128 of 512 columns) never runs out.
constexpr int kTcSmem = (int)sizeof(TcSmem) + 1024 > 56 * 1024 ? (int)sizeof(TcSmem) + 1024
                                                                 : 56 * 1024;

cudaError_t launch_mlp_tc(cudaStream_t s, int64_t n, const float *x, const MlpTc *w, float *y,
                          unsigned *flags, int probe_limit) {
  const int smem = kTcSmem;
  const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
  const int grid = (int)(ntiles < 4 * 152 ? ntiles : 4 * 152);
  if (grid <= 0) return cudaSuccess;
  k_mlp_tc<<<grid, kTcThreads, smem, s>>>(n, x, w, y, flags, probe_limit);
  return cudaGetLastError();
}

cudaError_t prepare_mlp_tc_kernel() {
  return cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
}

}  // namespace bhg
