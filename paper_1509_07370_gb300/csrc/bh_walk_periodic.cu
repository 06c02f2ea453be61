// The Barnes-Hut walk with periodic boundaries (App. A).
//
// The traversal is the per-cell stackless walk of bh_walk.cu (pre-order
// nodes with skip indices, the warp steps to the smallest `next` of its
// targets, bottom nodes in one super-step, two x-neighbour targets per lane
// in packed binary32 pairs); what changes is the geometry and the term:
//  * every displacement is the minimum image: each box-unit component of
//    t - R is wrapped into [-1/2, 1/2] (dx > 0.5 -> dx - 1, dx < -0.5 ->
//    dx + 1, both exact in binary32), for the opening test of Eq. 4 and for
//    the term;
//  * an accepted node or another cell adds M psi(d) = M (1/d + chi(d)), chi
//    the smooth part of the Ewald field interpolated quadratically from the
//    table (bh_ewald.cuh): one 64-byte entry of interpolant coefficients
//    per target and 26 FMAs, the y and z indices shared by the x-neighbour
//    pair;
//  * the target's own cell adds its mass times chi(0): the field of its
//    periodic copies (the direct part 1/d is absent, as in the isolated walk).
// The table interpolation costs far more than 1/d, so a step evaluates it
// only when one of the warp's targets takes a node.
#include "bh_walk_common.cuh"
#include "bh_ewald.cuh"

namespace bhg {
namespace {

constexpr int kPWarpsPerCta = 8;
constexpr int kPMaxThreads = 512;

__device__ __forceinline__ float min_image(float d) {
  return d > 0.5f ? __fsub_rn(d, 1.0f) : (d < -0.5f ? __fadd_rn(d, 1.0f) : d);
}

// Minimum-image displacements of the pair of targets (tx2 = {txa, txb}, ty,
// tz) from a record's binary32 position, and the squared distances with the
// opening test's rounding: d2 = fma(dx, dx, fma(dz, dz, dy*dy)).
__device__ __forceinline__ void dist2_min_image(u64 tx2, float ty, float tz, u64 q0, u64 q1,
                                                float &d2a, float &d2b, u64 &dx2, float &dy,
                                                float &dz) {
  float py, pz, dxa, dxb;
  upk(q1, py, pz);
  upk(sub2(tx2, q0), dxa, dxb);
  dx2 = pk(min_image(dxa), min_image(dxb));
  dy = min_image(__fsub_rn(ty, py));
  dz = min_image(__fsub_rn(tz, pz));
  const float h = __fmaf_rn(dz, dz, __fmul_rn(dy, dy));
  upk(fma2(dx2, dx2, pk(h, h)), d2a, d2b);
}

// chi of the pair (the arithmetic of ewald_chi) for the targets whose flag
// is set (the others get 0).  The table is read through the L1 data stage
// one line per distinct entry and load, which bounds this walk, so a target
// that takes nothing loads nothing, and target b reuses a's entry when both
// fall on the same centre (the y and z parts of the index and fy, fz are
// shared by the x-neighbour pair).
__device__ __forceinline__ u64 chi_pair(const unsigned char *__restrict__ tab, int n, float s, u64 dx2,
                                        float dy, float dz, bool ua, bool ub) {
  float dxa, dxb, fxa, fxb, fy, fz;
  uint32_t C[16];
  upk(dx2, dxa, dxb);
  const int ca = ewald_axis(fabsf(dxa), s, n, fxa);
  const int cb = ewald_axis(fabsf(dxb), s, n, fxb);
  const int cy = ewald_axis(fabsf(dy), s, n, fy);
  const int cz = ewald_axis(fabsf(dz), s, n, fz);
  float chia = 0.0f, chib = 0.0f;
  if (ua) {
    ewald_load(tab, n, ca, cy, cz, C);
    chia = ewald_poly(C, fxa, fy, fz);
  }
  if (ub) {
    if (!ua || cb != ca) ewald_load(tab, n, cb, cy, cz, C);
    chib = ewald_poly(C, fxb, fy, fz);
  }
  return pk(chia, chib);
}

// M (1/d + chi) for the targets whose flag is set, 0 for the others; r = 1/d
// (0 for the target's own cell).
__device__ __forceinline__ u64 periodic_term2(u64 mm, float ra, float rb, u64 chi, bool ua,
                                              bool ub) {
  float ta, tb;
  upk(mul2(mm, add2(pk(ra, rb), chi)), ta, tb);
  return pk(ua ? ta : 0.0f, ub ? tb : 0.0f);
}

template <bool KAHAN, bool COUNTS>
__device__ __forceinline__ void walk_octant_periodic(
    unsigned u, int lane, const WalkRec *__restrict__ rec, const int4 *__restrict__ blk,
    const int *__restrict__ orig, const int4 *__restrict__ fld, const double *__restrict__ invL,
    const unsigned long long *__restrict__ mmax, const unsigned char *__restrict__ tab, int n, double G,
    float *__restrict__ out, int32_t *__restrict__ n_int, int32_t *__restrict__ n_test,
    int32_t *__restrict__ n_leaf) {
  const unsigned p = u >> 3;                          // sorted block
  const int4 F = fld[p];                              // this field's node range
  const unsigned n_nodes = (unsigned)F.y;
  const int ma = (int)((u & 7) << 6) | (lane << 1);   // local Morton index, even
  const int4 B = blk[p];
  const int cx = (int)compact3(ma), cy = (int)compact3(ma >> 1), cz = (int)compact3(ma >> 2);
  const int lc = B.x + 3;
  const float hh = pow2f(-(lc + 1));
  const float txa = __fmul_rn((float)(2 * (8 * B.y + cx) + 1), hh);
  const float txb = __fmul_rn((float)(2 * (8 * B.y + cx) + 3), hh);
  const float ty = __fmul_rn((float)(2 * (8 * B.z + cy) + 1), hh);
  const float tz = __fmul_rn((float)(2 * (8 * B.w + cz) + 1), hh);
  const u64 tx2 = pk(txa, txb);
  const float s = (float)(2 * n);

  u64 sum = 0ull, comp = 0ull;
  int nia = 0, nib = 0, nta = 0, ntb = 0, nla = 0, nlb = 0;
  unsigned next_a = (unsigned)F.x, next_b = (unsigned)F.x;
  unsigned node = (unsigned)F.x;
  while (node < n_nodes) {
    u64 q0, q1, q2, q3;
    load_rec(rec + node, q0, q1, q2, q3);
    float s2, skf;
    upk(q3, s2, skf);
    const unsigned skip = __float_as_uint(skf);
    float d2a, d2b, dy, dz;
    u64 dx2;
    dist2_min_image(tx2, ty, tz, q0, q1, d2a, d2b, dx2, dy, dz);
    const bool mine_a = next_a == node, mine_b = next_b == node;
    const bool take_a = mine_a && d2a > s2;
    const bool take_b = mine_b && d2b > s2;
    if (COUNTS) {
      const bool internal = s2 > 0.0f;
      nia += take_a;
      nib += take_b;
      nta += mine_a && internal;
      ntb += mine_b && internal;
      nla += take_a && !internal;
      nlb += take_b && !internal;
    } else if (__any_sync(kFull, take_a || take_b)) {
      const float ra = take_a ? rsqrt_approx(d2a) : 0.0f;
      const float rb = take_b ? rsqrt_approx(d2b) : 0.0f;
      accumulate2<KAHAN>(sum, comp,
                         periodic_term2(q2, ra, rb, chi_pair(tab, n, s, dx2, dy, dz, take_a, take_b),
                                        take_a, take_b));
    }
    if (skip == node + 9u) {  // bottom node: its 8 cells in one step
      const bool open_a = mine_a && !take_a, open_b = mine_b && !take_b;
      if (__any_sync(kFull, open_a || open_b)) {
#pragma unroll 1
        for (unsigned c = node + 1; c < node + 9u; ++c) {
          u64 c0, c1, c2, c3;
          load_rec(rec + c, c0, c1, c2, c3);
          float e2a, e2b, ey, ez;
          u64 ex2;
          dist2_min_image(tx2, ty, tz, c0, c1, e2a, e2b, ex2, ey, ez);
          if (COUNTS) {
            const bool la = open_a && e2a > 0.0f;  // the own cell is no interaction
            const bool lb = open_b && e2b > 0.0f;
            nia += la;
            nib += lb;
            nla += la;
            nlb += lb;
          } else {
            // every cell of the node, the own cell (e2 = 0) with chi(0) only
            const float ra = e2a > 0.0f ? rsqrt_approx(e2a) : 0.0f;
            const float rb = e2b > 0.0f ? rsqrt_approx(e2b) : 0.0f;
            accumulate2<KAHAN>(sum, comp,
                               periodic_term2(c2, ra, rb,
                                              chi_pair(tab, n, s, ex2, ey, ez, open_a, open_b),
                                              open_a, open_b));
          }
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
  const int64_t cell = (int64_t)orig[p] * kCellsPerBlock + cz * 64 + cy * 8 + cx;
  if (COUNTS) {
    n_int[cell] = nia;
    n_int[cell + 1] = nib;
    n_test[cell] = nta;
    n_test[cell + 1] = ntb;
    if (n_leaf) {
      n_leaf[cell] = nla;
      n_leaf[cell + 1] = nlb;
    }
  } else {
    sum = finish2<KAHAN>(sum, comp);
    float sa, sb;
    upk(sum, sa, sb);
    const float scale = (float)(-G * invL[F.w] * pow2i(mass_exponent(mmax[F.w])));
    out[cell] = __fmul_rn(sa, scale);
    out[cell + 1] = __fmul_rn(sb, scale);
  }
}

// One warp per octant: octant order[warp] when an order is given (the
// octants sorted by the time of their walks, longest first, so that the
// CTAs, issued in index order, start with the long walks and each holds
// octants of about equal length).  With `cycles`, lane 0 stores the SM clock
// cycles its octant's walk took.
template <bool KAHAN, bool COUNTS>
__global__ void __launch_bounds__(kPMaxThreads)
    k_walk_periodic(unsigned nunits, const unsigned *__restrict__ order,
                    unsigned long long *__restrict__ cycles, const WalkRec *__restrict__ rec,
                    const int4 *__restrict__ blk, const int *__restrict__ orig,
                    const int4 *__restrict__ fld, const double *__restrict__ invL,
                    const unsigned long long *__restrict__ mmax, const unsigned char *__restrict__ tab,
                    int n, double G, float *__restrict__ out, int32_t *__restrict__ n_int,
                    int32_t *__restrict__ n_test, int32_t *__restrict__ n_leaf) {
  const int lane = threadIdx.x & 31;
  const unsigned warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (warp >= nunits) return;  // whole warps only
  const unsigned u = order ? order[warp] : warp;
  const long long t0 = cycles ? clock64() : 0;
  walk_octant_periodic<KAHAN, COUNTS>(u, lane, rec, blk, orig, fld, invL, mmax, tab, n, G,
                                      out, n_int, n_test, n_leaf);
  if (cycles && lane == 0) cycles[u] = (unsigned long long)(clock64() - t0);
}

template <bool KAHAN, bool COUNTS>
cudaError_t go_periodic(cudaStream_t s, int nb, const WalkRec *rec, const int4 *blk,
                        const int *orig, const FieldArgs &fa, const unsigned char *tab, int n, double G,
                        void *out, int32_t *ni, int32_t *nt, int32_t *nl, int wpc,
                        const unsigned *order, unsigned long long *cycles) {
  const unsigned nunits = (unsigned)nb * 8u;
  const int w = wpc > 0 ? wpc : kPWarpsPerCta;
  const int grid = (int)((nunits + w - 1) / w);
  k_walk_periodic<KAHAN, COUNTS><<<grid, 32 * w, 0, s>>>(nunits, order, cycles, rec, blk, orig,
                                                         fa.fld, fa.invL, fa.mmax, tab, n, G,
                                                         (float *)out, ni, nt, nl);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_walk_periodic(cudaStream_t s, const bh_options &opt, int nb,
                                 const WalkRec *rec, const int4 *blk, const int *orig,
                                 const FieldArgs &fa, const unsigned char *tab, int n, double G,
                                 void *out, int32_t *n_int, int32_t *n_test, int32_t *n_leaf,
                                 int wpc, const unsigned *order, unsigned long long *cycles) {
  if (n_int)
    return go_periodic<false, true>(s, nb, rec, blk, orig, fa, tab, n, G, out, n_int, n_test,
                                    n_leaf, wpc, order, nullptr);
  return opt.kahan ? go_periodic<true, false>(s, nb, rec, blk, orig, fa, tab, n, G, out, nullptr,
                                              nullptr, nullptr, wpc, order, cycles)
                   : go_periodic<false, false>(s, nb, rec, blk, orig, fa, tab, n, G, out,
                                               nullptr, nullptr, nullptr, wpc, order, cycles);
}

}  // namespace bhg
