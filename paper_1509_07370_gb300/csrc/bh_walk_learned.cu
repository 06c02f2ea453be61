// The learned walk: the per-cell binary32 monopole walk of k_walk_pair with
// the learned residual correction added for every accepted internal node
// (features and network in bhgrav.h; the correction is not in the paper).
//
// Every (target, accepted internal node) pair is one row of the network (with
// the gate of bh_set_mlp_gate: only pairs with s = l/d >= s_min, decided in
// binary32 on the opening test's d^2: d2 <= fl(g * g), g = fl(l fl(1/s_min));
// inv_smin = +inf corrects every pair).  A
// warp queues its rows in shared memory as it walks: the pair's ten features
// as one bf16 row, the coefficient c = M s^2 / d and the target (0..63).  When
// 64 or more rows are queued, the warp evaluates the largest multiple of 16 of
// them on the tensor cores (mma.sync m16n8k16, bf16 in, FP32 accumulate) and
// moves the rest to the front; the last rows are evaluated when the walk
// ends.  Only accepted pairs are evaluated, never idle lanes.
//
// Inside one 16-row tile the activations stay in registers: the accumulator
// fragments of n-tiles 2j and 2j+1 of one layer, after the GELU and the bf16
// rounding, are exactly the A fragment of k-tile j of the next layer.  The
// kernel keeps 2 GELU(a) = a + a tanh(z) (one bf16 fma after the SFU tanh),
// and the next layer's weights are stored halved (exact in bf16) to absorb
// the factor 2.
//
// Each row adds c y to its target's correction sum, in row order (lanes that
// hold rows of the same target take turns), so results do not depend on
// timing; each target adds its correction sum to its potential at the end.
// The monopole part is the plain pair walk, term for term.
#include "bh_walk_common.cuh"

namespace bhg {
namespace {

constexpr int kLWarps = 8;      // warps per CTA (one block of 512 cells); 3 CTAs per SM
                                // (80 registers, 72 KB of shared memory each)
constexpr int kQRows = 128;     // queue capacity per warp (rows)
constexpr int kQFlush = 64;     // evaluate once this many rows are queued
constexpr int kXWords = 12;     // row stride of the queued features: 24 bf16 = 48 bytes
                                // (16 used; the stride keeps the A loads conflict-free)

struct WarpQueue {
  uint32_t x[kQRows * kXWords];
  float coef[kQRows];
  float y[kQRows];
  float corr[64];
  uint8_t owner[kQRows];
};
struct LearnSmem {
  MlpDev w;
  WarpQueue q[kLWarps];
};
static_assert(sizeof(MlpDev) % 16 == 0, "weights staged as 16-byte words");
static_assert(sizeof(WarpQueue) % 16 == 0, "queues start on 16-byte boundaries");

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// 2 GELU(a) for a pair of FP32 pre-activations, tanh form, in bf16 pairs:
// a rounded to bf16, z = a (c0 + c1 a^2) with c0 = sqrt(2/pi) and c1 =
// 0.044715 sqrt(2/pi) rounded to bf16 (0.796875, 0.0356445), t = tanh(z) on
// the SFU, result a + a t.  The activation is a bf16 value either way; this
// costs one conversion, four bf16 pair operations and one SFU operation.
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

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Appends one row: features of the pair (binary32, then bf16), c, target.
// Quadrupole and mass share the field's binary32 mass unit, so their ratio
// u^T Q u / (M l^2) is the physical one.
__device__ __forceinline__ void queue_row(WarpQueue &Q, int row, float dx, float dy, float dz,
                                          float r, float l, float dl, float inv_ml2, float qf,
                                          const WalkQuad &q, float coef, int target) {
  const float ux = dx * r, uy = dy * r, uz = dz * r;
  const float s = l * r;
  const float quu = 2.0f * (ux * (q.hxx * ux + q.qxy * uy + q.qxz * uz) +
                            uy * (q.hyy * uy + q.qyz * uz)) + 2.0f * q.hzz * uz * uz;
  const float f7 = quu * inv_ml2;
  uint4 *w = reinterpret_cast<uint4 *>(Q.x + row * kXWords);
  w[0] = make_uint4(bf16x2(ux, uy), bf16x2(uz, s), bf16x2(s * s, s * s * s), bf16x2(dl, f7));
  w[1] = make_uint4(bf16x2(qf * inv_ml2, s * s * f7), 0x3f80u, 0u, 0u);  // input 10 = 1
  Q.coef[row] = coef;
  Q.owner[row] = (uint8_t)target;
}

// Evaluates rows [0, n) of the queue (n rounded up to 16; rows beyond n are
// computed and ignored) and adds c y of each row to its target's sum.
__device__ __forceinline__ void evaluate(const MlpDev &W, WarpQueue &Q, int n, int lane) {
  const int gid = lane >> 2, tig = lane & 3;
  const uint2 *w1 = reinterpret_cast<const uint2 *>(&W.w1f[0][0][0]) + lane;
  const uint2 *w2 = reinterpret_cast<const uint2 *>(&W.w2f[0][0][0][0]) + lane;
  const uint2 *w3 = reinterpret_cast<const uint2 *>(&W.w3f[0][0][0]) + lane;
  const int mtiles = (n + 15) >> 4;
  for (int mt = 0; mt < mtiles; ++mt) {
    const uint32_t *xr = Q.x + (mt * 16 + gid) * kXWords + tig;
    const uint32_t a[4] = {xr[0], xr[8 * kXWords], xr[4], xr[8 * kXWords + 4]};
    uint32_t h[16];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // b1 comes in through input 10
      const uint2 b = w1[nt * 32];
      mma_bf16(c, a, b.x, b.y);
      const int j = nt >> 1, q = (nt & 1) * 2;
      h[4 * j + q] = gelu2x(c[0], c[1]);
      h[4 * j + q + 1] = gelu2x(c[2], c[3]);
    }
    uint32_t g[16];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float2 bb = *reinterpret_cast<const float2 *>(W.b2 + nt * 8 + 2 * tig);
      float c[4] = {bb.x, bb.y, bb.x, bb.y};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint2 b = w2[(nt * 4 + j) * 32];
        mma_bf16(c, &h[4 * j], b.x, b.y);
      }
      const int j = nt >> 1, q = (nt & 1) * 2;
      g[4 * j + q] = gelu2x(c[0], c[1]);
      g[4 * j + q + 1] = gelu2x(c[2], c[3]);
    }
    float c[4] = {W.b3, 0.0f, W.b3, 0.0f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint2 b = w3[j * 32];
      mma_bf16(c, &g[4 * j], b.x, b.y);
    }
    if (tig == 0) {  // output column 0
      Q.y[mt * 16 + gid] = c[0];
      Q.y[mt * 16 + gid + 8] = c[2];
    }
  }
  __syncwarp();
  for (int r0 = 0; r0 < n; r0 += 32) {
    const int r = r0 + lane;
    const bool v = r < n;
    const int o = v ? (int)Q.owner[r] : 64 + lane;  // idle lanes: keys of their own
    const float cy = v ? Q.coef[r] * Q.y[r] : 0.0f;
    const unsigned peers = __match_any_sync(kFull, o);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int last = __reduce_max_sync(kFull, (unsigned)rank);
    for (int k = 0; k <= last; ++k) {  // rows of one target in row order
      if (v && rank == k) Q.corr[o] += cy;
      __syncwarp();
    }
  }
}

template <bool KAHAN>
__global__ void __launch_bounds__(kLWarps * 32, 3)
    k_walk_learned(unsigned nunits, const WalkRec *__restrict__ rec,
                   const WalkQuad *__restrict__ qrec, const float2 *__restrict__ aux,
                   const int4 *__restrict__ blk, const int *__restrict__ orig,
                   const int4 *__restrict__ fld, const double *__restrict__ invL,
                   const unsigned long long *__restrict__ mmax, double G,
                   const MlpDev *__restrict__ mlp, float inv_smin, float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LearnSmem &S = *reinterpret_cast<LearnSmem *>(smem_raw);
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(mlp);
    uint4 *dst = reinterpret_cast<uint4 *>(&S.w);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 16); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned u = blockIdx.x * kLWarps + wid;
  if (u >= nunits) return;  // whole warps only, after the CTA-wide staging
  WarpQueue &Q = S.q[wid];
  Q.corr[lane] = 0.0f;
  Q.corr[lane + 32] = 0.0f;
  const unsigned p = u >> 3;
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
  unsigned node = (unsigned)F.x;
  int count = 0;  // queued rows (warp-uniform)
  for (;;) {
    const bool done = node >= n_nodes;
    if (!done) {
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
        const float2 lv = aux[node];  // node side, delta
        const float g = __fmul_rn(lv.x, inv_smin);
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
          int row = count + __popc(ba & lower) + __popc(bb & lower);
          if (qa) {
            const float s = lv.x * ra;
            queue_row(Q, row++, dxa, dy, dz, ra, lv.x, dl, inv_ml2, qf, q, mf * ra * s * s,
                      2 * lane);
          }
          if (qb) {
            const float s = lv.x * rb;
            queue_row(Q, row, dxb, dy, dz, rb, lv.x, dl, inv_ml2, qf, q, mf * rb * s * s,
                      2 * lane + 1);
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
    if (count >= kQFlush || (done && count > 0)) {
      __syncwarp();
      const int n = done ? count : (count & ~15);
      evaluate(S.w, Q, n, lane);
      const int tail = count - n;  // < 16 rows, moved to the front (rows >= 64 -> 0..15)
      for (int i = lane; i < tail * 8; i += 32)
        Q.x[(i >> 3) * kXWords + (i & 7)] = Q.x[(n + (i >> 3)) * kXWords + (i & 7)];
      if (lane < tail) {
        Q.coef[lane] = Q.coef[n + lane];
        Q.owner[lane] = Q.owner[n + lane];
      }
      __syncwarp();
      count = tail;
    }
    if (done) break;
  }
  __syncwarp();
  accumulate2<KAHAN>(sum, comp, pk(Q.corr[2 * lane], Q.corr[2 * lane + 1]));
  const int64_t cell = (int64_t)orig[p] * kCellsPerBlock + cz * 64 + cy * 8 + cx;
  sum = finish2<KAHAN>(sum, comp);
  float sa, sb;
  upk(sum, sa, sb);
  const float scale = (float)(-G * invL[F.w] * pow2i(mass_exponent(mmax[F.w])));
  out[cell] = __fmul_rn(sa, scale);
  out[cell + 1] = __fmul_rn(sb, scale);
}

}  // namespace

cudaError_t prepare_learned_kernels() {
  const int smem = (int)sizeof(LearnSmem);
  cudaError_t e = cudaFuncSetAttribute(k_walk_learned<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_walk_learned<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  return e;
}

cudaError_t launch_walk_learned(cudaStream_t s, bh_ctx *ctx, double G, void *out) {
  const Tree &t = ctx->tree;
  const unsigned nunits = (unsigned)t.nb * 8u;
  const int smem = (int)sizeof(LearnSmem);  // limit set by prepare_learned_kernels
  const bool kahan = ctx->opt.kahan != 0;
  const unsigned grid = (nunits + kLWarps - 1) / kLWarps;
  const float inv_smin = learned_inv_smin(ctx);
  if (kahan)
    k_walk_learned<true><<<grid, kLWarps * 32, smem, s>>>(
        nunits, t.d_rec, t.d_qrec, t.d_aux, t.d_blk, t.d_orig, t.d_fld, t.d_invL, t.d_mmax, G,
        ctx->d_mlp, inv_smin, (float *)out);
  else
    k_walk_learned<false><<<grid, kLWarps * 32, smem, s>>>(
        nunits, t.d_rec, t.d_qrec, t.d_aux, t.d_blk, t.d_orig, t.d_fld, t.d_invL, t.d_mmax, G,
        ctx->d_mlp, inv_smin, (float *)out);
  return cudaGetLastError();
}

}  // namespace bhg
