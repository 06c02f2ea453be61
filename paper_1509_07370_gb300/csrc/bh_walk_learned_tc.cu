// The learned walk with the network on the fifth-generation tensor cores
// (tcgen05): the same walk, features, queue and arithmetic per row as
// k_walk_learned (bh_walk_learned.cu), with the rows of four warps evaluated
// together as one 128-row tile.
//
// A CTA is one warpgroup: four warps, each walking one 64-cell octant with
// its own row queue (a ring of 128 rows in shared memory).  A warp walks
// until it has 32 rows queued or its walk is over; then the four warps meet
// at a barrier and each puts its oldest (up to) 32 rows in rows 32w ..
// 32w+31 of the tile, which are the tensor-memory lanes warp w can read.
// One thread issues the three layers' MMAs (bf16 operands in shared memory
// in the canonical K-major layout, FP32 accumulators in tensor memory) and
// commits them to an mbarrier; every thread then runs its own row's
// epilogue (bias, GELU in bf16 pairs) into the next layer's operand, and at
// the end reads its row's y and adds c y to the row's target in row order.
// Which rows meet in a tile depends only on each warp's own walk, and each
// row's result only on that row, so results do not depend on timing.
//
// All decisions to meet, evaluate or stop are taken with CTA-wide reductions
// (__syncthreads_or / _and), so every thread passes the same barriers; waits
// for the MMAs are bounded: on time-out the kernel raises kErrTimeout and
// stops evaluating (bh_sync_status reports it).
#include "bh_walk_common.cuh"
#include "bh_tc.cuh"

namespace bhg {
namespace {

constexpr int kTWarps = 4;         // one warpgroup per CTA
constexpr int kTRing = 128;        // queue ring per warp (rows)
constexpr int kTTake = 32;         // rows per warp per tile
constexpr uint32_t kTCols = 128;   // tensor-memory columns per CTA (D1/D3: 0.., D2: 64..)

struct TcQueue {
  uint32_t x[kTRing * 8];  // 16 bf16 per row (32 bytes): 10 features, 1 (bias input), 0s
  float coef[kTRing];
  float corr[64];
  uint8_t owner[kTRing];
};
struct __align__(1024) TcWalkSmem {
  uint16_t a1[128 * 16];   // tile: features (canonical K-major, K = 16)
  uint16_t a2[128 * 64];   // tile: hidden activations (K = 64)
  MlpTc w;
  TcQueue q[kTWarps];
  uint32_t tmem;
  int unused;
  unsigned long long mbar;
};

// Appends one row to a warp's ring (same features as k_walk_learned).
__device__ __forceinline__ void tc_queue_row(TcQueue &Q, int slot, float dx, float dy, float dz,
                                             float r, float l, float dl, float inv_ml2,
                                             float qf, const WalkQuad &q, float coef,
                                             int target) {
  const float ux = dx * r, uy = dy * r, uz = dz * r;
  const float s = l * r;
  const float quu = 2.0f * (ux * (q.hxx * ux + q.qxy * uy + q.qxz * uz) +
                            uy * (q.hyy * uy + q.qyz * uz)) + 2.0f * q.hzz * uz * uz;
  const float f7 = quu * inv_ml2;
  uint4 *w = reinterpret_cast<uint4 *>(Q.x + slot * 8);
  w[0] = make_uint4(bf16x2(ux, uy), bf16x2(uz, s), bf16x2(s * s, s * s * s), bf16x2(dl, f7));
  w[1] = make_uint4(bf16x2(qf * inv_ml2, s * s * f7), 0x3f80u, 0u, 0u);  // input 10 = 1
  Q.coef[slot] = coef;
  Q.owner[slot] = (uint8_t)target;
}

template <bool KAHAN>
__global__ void __launch_bounds__(kTWarps * 32, 4)
    k_walk_learned_tc(unsigned nunits, const WalkRec *__restrict__ rec,
                      const WalkQuad *__restrict__ qrec, const float2 *__restrict__ aux,
                      const int4 *__restrict__ blk, const int *__restrict__ orig,
                      const int4 *__restrict__ fld, const double *__restrict__ invL,
                      const unsigned long long *__restrict__ mmax, double G,
                      const MlpTc *__restrict__ wts, float inv_smin, float *__restrict__ out,
                      unsigned *flags) {
  extern __shared__ unsigned char smem_raw[];
  TcWalkSmem &S = *reinterpret_cast<TcWalkSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(wts);
    uint4 *dst = reinterpret_cast<uint4 *>(&S.w);
    for (int i = t; i < (int)(sizeof(MlpTc) / 16); i += kTWarps * 32) dst[i] = src[i];
  }
  TcQueue &Q = S.q[wid];
  Q.corr[lane] = 0.0f;
  Q.corr[lane + 32] = 0.0f;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)));
    fence_async_smem();
  }
  if (wid == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem)),
                 "r"(kTCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = S.tmem;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * wid) << 16);

  // this warp's octant (a warp past the last unit walks nothing)
  const unsigned u = blockIdx.x * kTWarps + wid;
  const bool active = u < nunits;
  const unsigned p = active ? u >> 3 : 0u;
  const int4 F = fld[p];
  const unsigned n_nodes = (unsigned)F.y;
  const int ma = (int)((u & 7) << 6) | (lane << 1);
  const int4 B = blk[p];
  const int cx = (int)compact3(ma), cy = (int)compact3(ma >> 1), cz = (int)compact3(ma >> 2);
  const float hh = pow2f(-(B.x + 3 + 1));
  const float txa = __fmul_rn((float)(2 * (8 * B.y + cx) + 1), hh);
  const float txb = __fmul_rn((float)(2 * (8 * B.y + cx) + 3), hh);
  const float ty = __fmul_rn((float)(2 * (8 * B.z + cy) + 1), hh);
  const float tz = __fmul_rn((float)(2 * (8 * B.w + cz) + 1), hh);
  const u64 tx2 = pk(txa, txb);
  const unsigned lower = (1u << lane) - 1u;
  u64 sum = 0ull, comp = 0ull;
  unsigned next_a = (unsigned)F.x, next_b = (unsigned)F.x;
  unsigned node = active ? (unsigned)F.x : n_nodes;
  int head = 0, count = 0;  // ring state (warp-uniform)
  uint32_t phase = 0;
  bool ok = true;
  for (;;) {
    // walk until 32 rows are queued or the walk is over
    while (node < n_nodes && count < kTTake) {
      u64 q0, q1, q2, q3;
      load_rec(rec + node, q0, q1, q2, q3);
      float s2, skf;
      upk(q3, s2, skf);
      const unsigned skip = __float_as_uint(skf);
      float d2a, d2b, dy, dz;
      u64 dx2;
      dist2(tx2, ty, tz, q0, q1, d2a, d2b, dx2, dy, dz);
      const bool mine_a = next_a == node, mine_b = next_b == node;
      const bool take_a = mine_a && d2a > s2;
      const bool take_b = mine_b && d2b > s2;
      float ra = rsqrt_approx(d2a), rb = rsqrt_approx(d2b);
      ra = take_a ? ra : 0.0f;
      rb = take_b ? rb : 0.0f;
      accumulate2<KAHAN>(sum, comp, mul2(q2, pk(ra, rb)));
      if (s2 > 0.0f) {  // internal node: queue the accepted pairs the gate lets through
        const float2 lv = aux[node];
        const float g = __fmul_rn(lv.x, inv_smin);  // the gate, as in k_walk_learned
        const float g2 = __fmul_rn(g, g);
        const bool qa = take_a && d2a <= g2, qb = take_b && d2b <= g2;
        const unsigned ba = __ballot_sync(kFull, qa), bb = __ballot_sync(kFull, qb);
        if (ba | bb) {
          const WalkQuad q = qrec[node];
          float mf, mf2;
          upk(q2, mf, mf2);
          const float inv_ml2 = mf > 0.0f ? 1.0f / (mf * lv.x * lv.x) : 1.0f;
          const float qf = sqrtf(4.0f * (q.hxx * q.hxx + q.hyy * q.hyy + q.hzz * q.hzz) +
                                 2.0f * (q.qxy * q.qxy + q.qxz * q.qxz + q.qyz * q.qyz));
          const float dl = lv.y / lv.x;
          float dxa, dxb;
          upk(dx2, dxa, dxb);
          int k = count + __popc(ba & lower) + __popc(bb & lower);
          if (qa) {
            const float s = lv.x * ra;
            tc_queue_row(Q, (head + k++) & (kTRing - 1), dxa, dy, dz, ra, lv.x, dl, inv_ml2, qf,
                         q, mf * ra * s * s, 2 * lane);
          }
          if (qb) {
            const float s = lv.x * rb;
            tc_queue_row(Q, (head + k) & (kTRing - 1), dxb, dy, dz, rb, lv.x, dl, inv_ml2, qf, q,
                         mf * rb * s * s, 2 * lane + 1);
          }
          count += __popc(ba) + __popc(bb);
        }
      }
      if (skip == node + 9u) {  // bottom node: its 8 cells in one step
        const bool open_a = mine_a && !take_a, open_b = mine_b && !take_b;
        if (__any_sync(kFull, open_a || open_b)) {
#pragma unroll 2
          for (unsigned c = node + 1; c < node + 9u; ++c) {
            u64 c0, c1, c2, c3;
            load_rec(rec + c, c0, c1, c2, c3);
            float e2a, e2b, ey, ez;
            u64 ex2;
            dist2(tx2, ty, tz, c0, c1, e2a, e2b, ex2, ey, ez);
            float sa = rsqrt_approx(e2a), sb = rsqrt_approx(e2b);
            sa = (open_a && e2a > 0.0f) ? sa : 0.0f;
            sb = (open_b && e2b > 0.0f) ? sb : 0.0f;
            accumulate2<KAHAN>(sum, comp, mul2(c2, pk(sa, sb)));
          }
        }
        next_a = max(next_a, skip);
        next_b = max(next_b, skip);
      } else {
        const unsigned n1 = node + 1;
        next_a = max(next_a, take_a ? skip : n1);
        next_b = max(next_b, take_b ? skip : n1);
      }
      node = __reduce_min_sync(kFull, min(next_a, next_b));
    }
    // every warp has 32 rows or has finished: evaluate a tile, if any rows
    __syncwarp();
    if (!__syncthreads_or(count > 0) || !ok) break;
    const int take = count < kTTake ? count : kTTake;
    {  // this warp's rows into tile rows 32 wid + lane (zeros past `take`)
      const int r = 32 * wid + lane;
      uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
      if (lane < take) {
        const uint4 *src = reinterpret_cast<const uint4 *>(Q.x + ((head + lane) & (kTRing - 1)) * 8);
        lo = src[0];
        hi = src[1];
      }
      unsigned char *a1 = reinterpret_cast<unsigned char *>(S.a1);
      *reinterpret_cast<uint4 *>(a1 + tc_canon(r, 0, 16)) = lo;
      *reinterpret_cast<uint4 *>(a1 + tc_canon(r, 8, 16)) = hi;
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      mma(tmem, sdesc(S.a1, 128, 256), sdesc(S.w.b1, 128, 256), idesc(128, 64), 0u);
      commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase));
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    tc_epilogue(lane_base, nullptr, S.a2, t);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      for (int kk = 0; kk < 4; ++kk)
        mma(tmem + 64, sdesc(S.a2 + 128 * kk, 128, 1024), sdesc(S.w.b2 + 128 * kk, 128, 1024),
            idesc(128, 64), kk > 0);
      commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase));
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    tc_epilogue(lane_base + 64, S.w.bias2, S.a2, t);
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      for (int kk = 0; kk < 4; ++kk)
        mma(tmem, sdesc(S.a2 + 128 * kk, 128, 1024), sdesc(S.w.b3 + 128 * kk, 128, 1024),
            idesc(128, 16), kk > 0);
      commit(&S.mbar);
    }
    ok = __syncthreads_and(mbar_wait(&S.mbar, phase));
    if (!ok) break;
    phase ^= 1u;
    fence_after();
    {  // y of this lane's row; rows of one target added in row order
      const float y = tmem_ld1(lane_base) + S.w.bias3;
      const bool v = lane < take;
      const int slot = (head + lane) & (kTRing - 1);
      const int o = v ? (int)Q.owner[slot] : 64 + lane;
      const float cy = v ? Q.coef[slot] * y : 0.0f;
      const unsigned peers = __match_any_sync(kFull, o);
      const int rank = __popc(peers & lower);
      const int last = __reduce_max_sync(kFull, (unsigned)rank);
      for (int k = 0; k <= last; ++k) {
        if (v && rank == k) Q.corr[o] += cy;
        __syncwarp();
      }
    }
    head = (head + take) & (kTRing - 1);
    count -= take;
    fence_before();
    __syncthreads();
    fence_after();
  }
  if (!ok) {  // the MMA barrier did not complete in time
    if (t == 0) atomicOr(flags, kErrTimeout);
    mbar_wait(&S.mbar, phase);
  }
  __syncwarp();
  if (active) {
    accumulate2<KAHAN>(sum, comp, pk(Q.corr[2 * lane], Q.corr[2 * lane + 1]));
    const int64_t cell = (int64_t)orig[p] * kCellsPerBlock + cz * 64 + cy * 8 + cx;
    sum = finish2<KAHAN>(sum, comp);
    float sa, sb;
    upk(sum, sa, sb);
    const float scale = (float)(-G * invL[F.w] * pow2i(mass_exponent(mmax[F.w])));
    out[cell] = __fmul_rn(sa, scale);
    out[cell + 1] = __fmul_rn(sb, scale);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (wid == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTCols));
}

constexpr int kTcWalkSmem = (int)sizeof(TcWalkSmem) + 1024;

}  // namespace

cudaError_t prepare_learned_tc_kernel() {
  cudaError_t e = cudaFuncSetAttribute(k_walk_learned_tc<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kTcWalkSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_walk_learned_tc<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kTcWalkSmem);
  return e;
}

cudaError_t launch_walk_learned_tc(cudaStream_t s, bh_ctx *ctx, double G, void *out) {
  const Tree &t = ctx->tree;
  const unsigned nunits = (unsigned)t.nb * 8u;
  const unsigned grid = (nunits + kTWarps - 1) / kTWarps;
  const float inv_smin = learned_inv_smin(ctx);
  if (ctx->opt.kahan)
    k_walk_learned_tc<true><<<grid, kTWarps * 32, kTcWalkSmem, s>>>(
        nunits, t.d_rec, t.d_qrec, t.d_aux, t.d_blk, t.d_orig, t.d_fld, t.d_invL, t.d_mmax, G,
        ctx->d_mlp_tc, inv_smin, (float *)out, t.d_flags);
  else
    k_walk_learned_tc<false><<<grid, kTWarps * 32, kTcWalkSmem, s>>>(
        nunits, t.d_rec, t.d_qrec, t.d_aux, t.d_blk, t.d_orig, t.d_fld, t.d_invL, t.d_mmax, G,
        ctx->d_mlp_tc, inv_smin, (float *)out, t.d_flags);
  return cudaGetLastError();
}

}  // namespace bhg
