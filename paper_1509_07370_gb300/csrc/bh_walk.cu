// The Barnes-Hut walk: potential at every cell centre (Sec. 3.3).
//
// One warp owns one brick of 32 neighbouring cells of a block (a 4x4x2 set,
// local Morton indices 32q .. 32q+31), as the paper groups its cells
// (Sec. 3.1.1, Sec. 3.3).  The paper walks with a shared-memory stack pushed
// by lane 0 and an all() vote on the opening test.  This walk needs no stack:
// nodes are stored in pre-order, so a node's first child is the next node and
// its subtree ends at its skip index.  Each lane keeps `next`, the first node
// it still has to visit (0 = the root at the start).  At every step the warp
// takes the smallest `next` over its lanes (one __reduce_min_sync), all lanes
// load that node (one broadcast load), and the lanes whose `next` equals it
// apply the opening test of Eq. 4:
//   accepted -> add M / d, next = skip (the whole subtree is done)
//   opened   -> next = node + 1 (descend into the first child)
// Cells carry s2 = 0, so the test accepts every other cell (d2 > 0) and
// rejects only the lane's own cell (d2 = 0), which contributes nothing; for a
// cell node + 1 equals its skip, so no special case is needed.  Every lane
// thus visits exactly the nodes of its own recursive walk, in pre-order, and
// the result is the per-cell potential of the recursive definition; lanes
// whose `next` is further ahead simply wait (masked) for the warp to get
// there.  Each lane's `next` only grows, so the loop ends after at most
// n_nodes steps.  With the warp vote (paper mode) all lanes share `next`.
//
// The opening test is evaluated in binary32 with the exact operation order
// stated in the public header; interactions use the same d2 (F32 mode, Kahan
// sum) or recompute d in binary64 from the FP64 moments (F64 mode).
#include "bh_internal.cuh"

namespace bhg {
namespace {

constexpr int kWalkThreads = 256;
constexpr int kWarpsPerCta = kWalkThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

__global__ void k_prepare_s2(int64_t n, const float2 *__restrict__ aux, float2 *__restrict__ rec1,
                             float inv_theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 a = aux[i];
  float2 r = rec1[i];
  const float s = __fadd_rn(__fmul_rn(a.x, inv_theta), a.y);  // l/theta + delta
  r.x = __fmul_rn(s, s);
  rec1[i] = r;
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

template <bool F64, bool VOTE, bool KAHAN, bool COUNTS>
__global__ void __launch_bounds__(kWalkThreads)
    k_walk(int nbricks, unsigned n_nodes, const float4 *__restrict__ rec0,
           const float2 *__restrict__ rec1, const double4_32a *__restrict__ mom,
           const int4 *__restrict__ blk, const int *__restrict__ orig, float scale_f,
           double scale_d, void *__restrict__ out, int32_t *__restrict__ n_int,
           int32_t *__restrict__ n_test) {
  const int warp = blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= nbricks) return;  // whole warps only
  const int p = warp >> 4;      // sorted block
  const int m = ((warp & 15) << 5) | lane;  // local Morton index of this lane's cell
  const int4 B = blk[p];
  const int cx = (int)compact3(m), cy = (int)compact3(m >> 1), cz = (int)compact3(m >> 2);
  const int lc = B.x + 3;
  // cell centre in box units, exact in binary32: (2 i + 1) * 2^-(lc+1)
  const float hh = pow2f(-(lc + 1));
  const float tx = __fmul_rn((float)(2 * (8 * B.y + cx) + 1), hh);
  const float ty = __fmul_rn((float)(2 * (8 * B.z + cy) + 1), hh);
  const float tz = __fmul_rn((float)(2 * (8 * B.w + cz) + 1), hh);
  double txd = 0.0, tyd = 0.0, tzd = 0.0;
  if (F64) {
    txd = (double)tx;
    tyd = (double)ty;
    tzd = (double)tz;
  }

  float sum = 0.0f, comp = 0.0f;
  double sumd = 0.0;
  int ni = 0, nt = 0;
  unsigned next = 0;
  while (true) {
    const unsigned node = VOTE ? next : __reduce_min_sync(kFull, next);
    if (node >= n_nodes) break;
    const float4 a = __ldg(&rec0[node]);
    const float2 r = __ldg(&rec1[node]);
    const float dx = __fsub_rn(tx, a.x);
    const float dy = __fsub_rn(ty, a.y);
    const float dz = __fsub_rn(tz, a.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    const bool internal = r.x > 0.0f;
    bool take;
    bool mine = true;
    if (VOTE) {
      const bool acc = d2 > r.x;
      take = internal ? (__all_sync(kFull, acc) != 0) : acc;
      next = (internal && !take) ? node + 1 : __float_as_uint(r.y);
    } else {
      mine = (next == node);
      take = mine && (d2 > r.x);
      if (mine) next = take ? __float_as_uint(r.y) : node + 1;
    }
    if (COUNTS) {
      nt += (mine && internal) ? 1 : 0;
      ni += take ? 1 : 0;
    } else if (take) {
      if (F64) {
        const double4_32a md = mom[node];
        const double ex = txd - md.x, ey = tyd - md.y, ez = tzd - md.z;
        sumd += md.w / sqrt(ex * ex + ey * ey + ez * ez);
      } else {
        const float term = __fmul_rn(a.w, rsqrtf(d2));
        if (KAHAN) {
          const float y = __fsub_rn(term, comp);
          const float s = __fadd_rn(sum, y);
          comp = __fsub_rn(__fsub_rn(s, sum), y);
          sum = s;
        } else {
          sum = __fadd_rn(sum, term);
        }
      }
    }
  }
  const int64_t cell = (int64_t)orig[p] * kCellsPerBlock + cz * 64 + cy * 8 + cx;
  if (COUNTS) {
    n_int[cell] = ni;
    n_test[cell] = nt;
  } else if (F64) {
    reinterpret_cast<double *>(out)[cell] = sumd * scale_d;
  } else {
    const float total = KAHAN ? __fsub_rn(sum, comp) : sum;
    reinterpret_cast<float *>(out)[cell] = __fmul_rn(total, scale_f);
  }
}

template <bool F64, bool VOTE, bool KAHAN, bool COUNTS>
cudaError_t go(cudaStream_t s, int nbricks, unsigned n, const float4 *rec0, const float2 *rec1,
               const double4_32a *mom, const int4 *blk, const int *orig, double scale, void *out,
               int32_t *ni, int32_t *nt) {
  const int grid = (nbricks + kWarpsPerCta - 1) / kWarpsPerCta;
  k_walk<F64, VOTE, KAHAN, COUNTS><<<grid, kWalkThreads, 0, s>>>(
      nbricks, n, rec0, rec1, mom, blk, orig, (float)scale, scale, out, ni, nt);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_prepare_s2(cudaStream_t s, int64_t n_nodes, const float2 *aux, float2 *rec1,
                              float inv_theta) {
  const int threads = 256;
  const int64_t grid = (n_nodes + threads - 1) / threads;
  k_prepare_s2<<<(unsigned)grid, threads, 0, s>>>(n_nodes, aux, rec1, inv_theta);
  return cudaGetLastError();
}

cudaError_t launch_walk(cudaStream_t s, const bh_options &opt, int nb, int64_t n_nodes,
                        const float4 *rec0, const float2 *rec1, const double4_32a *mom,
                        const int4 *blk, const int *orig, double scale, void *out,
                        int32_t *n_int, int32_t *n_test) {
  const int nbricks = nb * 16;
  const unsigned n = (unsigned)n_nodes;
  const bool vote = opt.criterion == BH_CRIT_WARP_VOTE;
  if (n_int) {
    return vote ? go<false, true, false, true>(s, nbricks, n, rec0, rec1, mom, blk, orig, scale,
                                               out, n_int, n_test)
                : go<false, false, false, true>(s, nbricks, n, rec0, rec1, mom, blk, orig,
                                                scale, out, n_int, n_test);
  }
  if (opt.precision == BH_PREC_F64) {
    return vote ? go<true, true, false, false>(s, nbricks, n, rec0, rec1, mom, blk, orig, scale,
                                               out, nullptr, nullptr)
                : go<true, false, false, false>(s, nbricks, n, rec0, rec1, mom, blk, orig, scale,
                                                out, nullptr, nullptr);
  }
  if (opt.kahan) {
    return vote ? go<false, true, true, false>(s, nbricks, n, rec0, rec1, mom, blk, orig, scale,
                                               out, nullptr, nullptr)
                : go<false, false, true, false>(s, nbricks, n, rec0, rec1, mom, blk, orig, scale,
                                                out, nullptr, nullptr);
  }
  return vote ? go<false, true, false, false>(s, nbricks, n, rec0, rec1, mom, blk, orig, scale,
                                              out, nullptr, nullptr)
              : go<false, false, false, false>(s, nbricks, n, rec0, rec1, mom, blk, orig, scale,
                                               out, nullptr, nullptr);
}

}  // namespace bhg
