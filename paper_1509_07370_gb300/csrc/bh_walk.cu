// The Barnes-Hut walk: potential at every cell centre (Sec. 3.3).
//
// Traversal.  The paper walks with a shared-memory stack pushed by lane 0 and
// an all() vote on the opening test (Sec. 3.3).  This walk needs no stack:
// nodes are stored in pre-order, so a node's first child is the next node and
// its subtree ends at its skip index.  Every target cell keeps `next`, the
// first node it still has to visit (0 = the root at the start).  At each step
// the warp takes the smallest `next` over its lanes (one __reduce_min_sync),
// all lanes load that node (one broadcast 256-bit load), and the targets whose
// `next` equals it apply the opening test of Eq. 4:
//   accepted -> add M / d, next = skip (the whole subtree is done)
//   opened   -> next = node + 1 (descend into the first child)
// Cells carry s2 = 0: the test accepts every other cell (d2 > 0) and rejects
// only the target's own cell (d2 = 0), which then adds nothing; for a cell
// node + 1 is its skip, so no special case is needed.  Each target thus
// visits exactly the nodes of its own recursive walk, in pre-order, and gets
// the per-cell result of the recursive definition; targets whose `next` lies
// further ahead wait (masked) for the warp to get there.  `next` only grows,
// so a walk ends after at most n_nodes steps.  With the warp vote (paper mode)
// all lanes share `next`.
//
// Work layout.
//  * Per-cell binary32 walk (the default, k_walk_pair): one warp per 4x4x4
//    octant of a block (64 cells, local Morton indices 64o .. 64o+63); lane l
//    owns the two x-neighbours 64o+2l and 64o+2l+1.  They share ty, tz and
//    so dy, dz; their dx, d2, 1/d products and Kahan sums run as packed
//    f32x2 operations (two binary32 results per instruction, each rounded as
//    its scalar counterpart).  A CTA of 8 warps is one whole block.
//  * binary64 interactions and the paper's warp vote (k_walk_scalar): one
//    warp per 32-cell brick (4x4x2, local Morton 32q .. 32q+31), one target
//    per lane, as the paper groups its cells (Sec. 3.1.1, Sec. 3.3).
//
// The opening test is evaluated in binary32 with the operation order stated
// in the public header; the interaction uses the same d2 (binary32, Kahan
// sum) or recomputes d in binary64 from the FP64 moments.
#include "bh_walk_common.cuh"

namespace bhg {
namespace {

constexpr int kWalkThreads = 256;               // default CTA: 8 warps = one block
constexpr int kWarpsPerCta = kWalkThreads / 32;
constexpr int kMaxWalkThreads = 512;            // largest tunable CTA

__global__ void k_prepare_s2(int64_t n, const float2 *__restrict__ aux, WalkRec *__restrict__ rec,
                             float inv_theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 a = aux[i];
  const float s = __fadd_rn(__fmul_rn(a.x, inv_theta), a.y);  // l/theta + delta
  rec[i].s2 = __fmul_rn(s, s);
}

// ---- per-cell binary32 walk, two x-neighbour targets per lane ---------------
// Interaction pair of an accepted node with the quadrupole term:
// rinv (M + (d^T Q d / 2) rinv^4), i.e. M/d + (1/2) d^T Q d / d^5.
__device__ __forceinline__ u64 quad_term2(const WalkQuad *qr, u64 mm, u64 rr, u64 dx2, float dy,
                                          float dz) {
  u64 w0, w1, w2, w3;
  load_quad(qr, w0, w1, w2, w3);
  float hyy, hzz, qxy, qxz, qyz, unused;
  upk(w1, hyy, hzz);
  upk(w2, qxy, qxz);
  upk(w3, qyz, unused);
  const float u = __fmaf_rn(qxz, dz, __fmul_rn(qxy, dy));    // shared by the pair
  const float v = __fmaf_rn(hyy, dy, __fmul_rn(qyz, dz));
  const float c = __fmaf_rn(dy, v, __fmul_rn(__fmul_rn(hzz, dz), dz));
  const u64 hq = fma2(dx2, fma2(w0, dx2, pk(u, u)), pk(c, c));
  const u64 r2 = mul2(rr, rr);
  return mul2(rr, fma2(hq, mul2(r2, r2), mm));
}

// Walk of one 64-cell octant (unit u = 8 * sorted block + octant).
//
// Bottom nodes (whose 8 children are cells, stored right after them, so
// skip = node + 9) are taken in one step: the targets that open such a node
// interact with its 8 cells in an unrolled loop that needs no per-cell
// bookkeeping (cells are never opened), and every target then continues at
// node + 9.  Targets that do not open it have next >= node + 9 already: a
// target whose walk does not contain a node has accepted one of its
// ancestors and skipped past the ancestor's whole subtree.
template <bool KAHAN, bool COUNTS, bool QUAD>
__device__ __forceinline__ void walk_octant(unsigned u, int lane, const WalkRec *__restrict__ rec,
                                            const WalkQuad *__restrict__ qrec,
                                            const int4 *__restrict__ blk,
                                            const int *__restrict__ orig,
                                            const int4 *__restrict__ fld,
                                            const double *__restrict__ invL,
                                            const unsigned long long *__restrict__ mmax, double G,
                                            float *__restrict__ out, int32_t *__restrict__ n_int,
                                            int32_t *__restrict__ n_test,
                                            int32_t *__restrict__ n_leaf) {
  const unsigned p = u >> 3;                          // sorted block
  const int4 F = fld[p];                              // this field's node range
  const unsigned n_nodes = (unsigned)F.y;
  const int ma = (int)((u & 7) << 6) | (lane << 1);   // local Morton index, even: x bit 0
  const int4 B = blk[p];
  const int cx = (int)compact3(ma), cy = (int)compact3(ma >> 1), cz = (int)compact3(ma >> 2);
  const int lc = B.x + 3;
  // cell centres in box units, exact in binary32: (2 i + 1) * 2^-(lc+1)
  const float hh = pow2f(-(lc + 1));
  const float txa = __fmul_rn((float)(2 * (8 * B.y + cx) + 1), hh);
  const float txb = __fmul_rn((float)(2 * (8 * B.y + cx) + 3), hh);
  const float ty = __fmul_rn((float)(2 * (8 * B.z + cy) + 1), hh);
  const float tz = __fmul_rn((float)(2 * (8 * B.w + cz) + 1), hh);
  const u64 tx2 = pk(txa, txb);

  u64 sum = 0ull, comp = 0ull;  // (+0.0f, +0.0f) pairs
  int nia = 0, nib = 0, nta = 0, ntb = 0, nla = 0, nlb = 0;
  unsigned next_a = (unsigned)F.x, next_b = (unsigned)F.x;  // the field's root
  unsigned node = (unsigned)F.x;
  while (node < n_nodes) {
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
    if (COUNTS) {
      const bool internal = s2 > 0.0f;
      nia += take_a;
      nib += take_b;
      nta += mine_a && internal;
      ntb += mine_b && internal;
      nla += take_a && !internal;
      nlb += take_b && !internal;
    } else {
      float ra = rsqrt_approx(d2a), rb = rsqrt_approx(d2b);
      ra = take_a ? ra : 0.0f;
      rb = take_b ? rb : 0.0f;
      const u64 rr = pk(ra, rb);
      accumulate2<KAHAN>(sum, comp,
                         QUAD ? quad_term2(qrec + node, q2, rr, dx2, dy, dz) : mul2(q2, rr));
    }
    if (skip == node + 9u) {  // bottom node
      const bool open_a = mine_a && !take_a, open_b = mine_b && !take_b;
      if (__any_sync(kFull, open_a || open_b)) {
#pragma unroll 2
        for (unsigned c = node + 1; c < node + 9u; ++c) {
          u64 c0, c1, c2, c3;
          load_rec(rec + c, c0, c1, c2, c3);
          float e2a, e2b, ey, ez;
          u64 ex2;
          dist2(tx2, ty, tz, c0, c1, e2a, e2b, ex2, ey, ez);
          const bool la = open_a && e2a > 0.0f;  // every cell but the target's own
          const bool lb = open_b && e2b > 0.0f;
          if (COUNTS) {
            nia += la;
            nib += lb;
            nla += la;
            nlb += lb;
          } else {
            float ra = rsqrt_approx(e2a), rb = rsqrt_approx(e2b);
            ra = la ? ra : 0.0f;
            rb = lb ? rb : 0.0f;
            accumulate2<KAHAN>(sum, comp, mul2(c2, pk(ra, rb)));
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
    if (KAHAN) sum = sub2(sum, comp);
    float sa, sb;
    upk(sum, sa, sb);
    // -G/L times the field's binary32 mass unit 2^e (exact), rounded once
    const float scale = (float)(-G * invL[F.w] * pow2i(mass_exponent(mmax[F.w])));
    out[cell] = __fmul_rn(sa, scale);
    out[cell + 1] = __fmul_rn(sb, scale);
  }
}

// One warp per 64-cell octant; a CTA of 8 warps covers one block.  (A
// persistent SM-affine schedule with work stealing raised the L1 hit rate
// from 44 % to 57 % but ran 8 % slower on GB300, so the hardware schedule of a
// plain grid is kept.)
template <bool KAHAN, bool COUNTS, bool QUAD>
__global__ void __launch_bounds__(kMaxWalkThreads)
    k_walk_pair(unsigned nunits, const WalkRec *__restrict__ rec,
                const WalkQuad *__restrict__ qrec, const int4 *__restrict__ blk,
                const int *__restrict__ orig, const int4 *__restrict__ fld,
                const double *__restrict__ invL, const unsigned long long *__restrict__ mmax,
                double G, float *__restrict__ out, int32_t *__restrict__ n_int,
                int32_t *__restrict__ n_test, int32_t *__restrict__ n_leaf) {
  const int lane = threadIdx.x & 31;
  const unsigned warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (warp >= nunits) return;  // whole warps only
  walk_octant<KAHAN, COUNTS, QUAD>(warp, lane, rec, qrec, blk, orig, fld, invL, mmax, G, out,
                                   n_int, n_test, n_leaf);
}

// ---- one target per lane: binary64 interactions and/or the warp vote --------
template <bool F64, bool VOTE, bool KAHAN, bool COUNTS, bool QUAD>
__global__ void __launch_bounds__(kWalkThreads)
    k_walk_scalar(int nbricks, const WalkRec *__restrict__ rec,
                  const double4_32a *__restrict__ mom, const WalkQuad *__restrict__ qrec,
                  const double *__restrict__ q64, const int4 *__restrict__ blk,
                  const int *__restrict__ orig, const int4 *__restrict__ fld,
                  const double *__restrict__ invL, const unsigned long long *__restrict__ mmax,
                  double G, void *__restrict__ out,
                  int32_t *__restrict__ n_int, int32_t *__restrict__ n_test,
                  int32_t *__restrict__ n_leaf) {
  const int warp = blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= nbricks) return;  // whole warps only
  const int p = warp >> 4;      // sorted block
  const int m = ((warp & 15) << 5) | lane;  // local Morton index of this lane's cell
  const int4 B = blk[p];
  const int4 F = fld[p];        // this field's node range
  const unsigned n_nodes = (unsigned)F.y;
  const double scale_d = -G * invL[F.w];  // FP64 walk: physical FP64 moments
  // binary32 walk: the records' masses are in the field's unit 2^e
  const float scale_f = (float)(scale_d * pow2i(mass_exponent(mmax[F.w])));
  const int cx = (int)compact3(m), cy = (int)compact3(m >> 1), cz = (int)compact3(m >> 2);
  const int lc = B.x + 3;
  const float hh = pow2f(-(lc + 1));
  const float tx = __fmul_rn((float)(2 * (8 * B.y + cx) + 1), hh);
  const float ty = __fmul_rn((float)(2 * (8 * B.z + cy) + 1), hh);
  const float tz = __fmul_rn((float)(2 * (8 * B.w + cz) + 1), hh);

  float sum = 0.0f, comp = 0.0f;
  double sumd = 0.0;
  int ni = 0, nt = 0, nl = 0;
  unsigned next = (unsigned)F.x;  // the field's root
  unsigned node = (unsigned)F.x;
  while (node < n_nodes) {
    u64 q0, q1, q2, q3;
    load_rec(rec + node, q0, q1, q2, q3);
    float px, px2, py, pz, mf, mf2, s2, skf;
    upk(q0, px, px2);
    upk(q1, py, pz);
    upk(q2, mf, mf2);
    upk(q3, s2, skf);
    const unsigned skip = __float_as_uint(skf);
    const float dx = __fsub_rn(tx, px);
    const float dy = __fsub_rn(ty, py);
    const float dz = __fsub_rn(tz, pz);
    const float d2 = __fmaf_rn(dx, dx, __fmaf_rn(dz, dz, __fmul_rn(dy, dy)));
    const bool internal = s2 > 0.0f;
    bool mine = true, take;
    if (VOTE) {
      const bool acc = d2 > s2;
      take = internal ? (__all_sync(kFull, acc) != 0) : acc;
      next = (internal && !take) ? node + 1 : skip;
    } else {
      mine = next == node;
      take = mine && d2 > s2;
      next = max(next, take ? skip : node + 1);
    }
    if (COUNTS) {
      nt += (mine && internal) ? 1 : 0;
      ni += take ? 1 : 0;
      nl += (take && !internal) ? 1 : 0;
    } else if (F64) {
      if (take) {
        const double4_32a md = mom[node];
        const double ex = (double)tx - md.x, ey = (double)ty - md.y, ez = (double)tz - md.z;
        const double dd = ex * ex + ey * ey + ez * ez;
        const double rinv = 1.0 / sqrt(dd);
        double t = md.w * rinv;
        if (QUAD && internal) {
          const double *Q = q64 + 6 * (size_t)node;
          const double hq = 0.5 * (Q[0] * ex * ex + Q[1] * ey * ey + Q[2] * ez * ez) +
                            Q[3] * ex * ey + Q[4] * ex * ez + Q[5] * ey * ez;
          t += hq * rinv * rinv * rinv * rinv * rinv;
        }
        sumd += t;
      }
    } else {
      float r = rsqrt_approx(d2);
      r = take ? r : 0.0f;
      float term = __fmul_rn(mf, r);
      if (QUAD && internal) {  // cells carry no quadrupole (and have no record)
        const WalkQuad w = qrec[node];
        const float hq = dx * (w.hxx * dx + w.qxy * dy + w.qxz * dz) +
                         dy * (w.hyy * dy + w.qyz * dz) + w.hzz * dz * dz;
        const float r2 = r * r;
        term = r * (mf + hq * r2 * r2);
      }
      if (KAHAN) {
        const float y = __fsub_rn(term, comp);
        const float t = __fadd_rn(sum, y);
        comp = __fsub_rn(__fsub_rn(t, sum), y);
        sum = t;
      } else {
        sum = __fadd_rn(sum, term);
      }
    }
    node = VOTE ? next : __reduce_min_sync(kFull, next);
  }
  const int64_t cell = (int64_t)orig[p] * kCellsPerBlock + cz * 64 + cy * 8 + cx;
  if (COUNTS) {
    n_int[cell] = ni;
    n_test[cell] = nt;
    if (n_leaf) n_leaf[cell] = nl;
  } else if (F64) {
    reinterpret_cast<double *>(out)[cell] = sumd * scale_d;
  } else {
    const float total = KAHAN ? __fsub_rn(sum, comp) : sum;
    reinterpret_cast<float *>(out)[cell] = __fmul_rn(total, scale_f);
  }
}

template <bool KAHAN, bool COUNTS, bool QUAD>
cudaError_t go_pair(cudaStream_t s, int nb, const WalkRec *rec, const WalkQuad *qrec,
                    const int4 *blk, const int *orig, const FieldArgs &fa, double G, void *out,
                    int32_t *ni, int32_t *nt, int32_t *nl, int wpc) {
  const unsigned nunits = (unsigned)nb * 8u;
  const int w = wpc > 0 ? wpc : kWarpsPerCta;
  const int grid = (int)((nunits + w - 1) / w);
  k_walk_pair<KAHAN, COUNTS, QUAD><<<grid, 32 * w, 0, s>>>(
      nunits, rec, qrec, blk, orig, fa.fld, fa.invL, fa.mmax, G, (float *)out, ni, nt, nl);
  return cudaGetLastError();
}

template <bool F64, bool VOTE, bool KAHAN, bool COUNTS, bool QUAD>
cudaError_t go_scalar(cudaStream_t s, int nb, const WalkRec *rec, const double4_32a *mom,
                      const WalkQuad *qrec, const double *q64, const int4 *blk,
                      const int *orig, const FieldArgs &fa, double G, void *out, int32_t *ni,
                      int32_t *nt, int32_t *nl) {
  const int nbricks = nb * 16;
  const int grid = (nbricks + kWarpsPerCta - 1) / kWarpsPerCta;
  k_walk_scalar<F64, VOTE, KAHAN, COUNTS, QUAD><<<grid, kWalkThreads, 0, s>>>(
      nbricks, rec, mom, qrec, q64, blk, orig, fa.fld, fa.invL, fa.mmax, G, out, ni, nt, nl);
  return cudaGetLastError();
}

// Picks the kernel instance for the options.  The counting walk takes the
// same decisions as every walk of the same criterion (the opening test does
// not depend on precision, summation or the quadrupole term).
template <bool QUAD>
cudaError_t launch_walk_q(cudaStream_t s, const bh_options &opt, int nb, const WalkRec *rec,
                          const double4_32a *mom, const WalkQuad *qrec, const double *q64,
                          const int4 *blk, const int *orig, const FieldArgs &fa, double G,
                          void *out, int wpc) {
  const bool vote = opt.criterion == BH_CRIT_WARP_VOTE;
  if (opt.precision == BH_PREC_F64)
    return vote ? go_scalar<true, true, false, false, QUAD>(s, nb, rec, mom, qrec, q64, blk, orig,
                                                            fa, G, out, nullptr, nullptr, nullptr)
                : go_scalar<true, false, false, false, QUAD>(s, nb, rec, mom, qrec, q64, blk,
                                                             orig, fa, G, out, nullptr, nullptr,
                                                             nullptr);
  if (vote)
    return opt.kahan ? go_scalar<false, true, true, false, QUAD>(s, nb, rec, mom, qrec, q64, blk,
                                                                 orig, fa, G, out, nullptr,
                                                                 nullptr, nullptr)
                     : go_scalar<false, true, false, false, QUAD>(s, nb, rec, mom, qrec, q64,
                                                                  blk, orig, fa, G, out, nullptr,
                                                                  nullptr, nullptr);
  return opt.kahan ? go_pair<true, false, QUAD>(s, nb, rec, qrec, blk, orig, fa, G, out, nullptr,
                                                nullptr, nullptr, wpc)
                   : go_pair<false, false, QUAD>(s, nb, rec, qrec, blk, orig, fa, G, out,
                                                 nullptr, nullptr, nullptr, wpc);
}

}  // namespace

cudaError_t launch_prepare_s2(cudaStream_t s, int64_t n_nodes, const float2 *aux, WalkRec *rec,
                              float inv_theta) {
  const int threads = 256;
  const int64_t grid = (n_nodes + threads - 1) / threads;
  k_prepare_s2<<<(unsigned)grid, threads, 0, s>>>(n_nodes, aux, rec, inv_theta);
  return cudaGetLastError();
}

cudaError_t launch_walk(cudaStream_t s, const bh_options &opt, int nb, const WalkRec *rec,
                        const double4_32a *mom, const WalkQuad *qrec, const double *q64,
                        const int4 *blk, const int *orig, const FieldArgs &fa, double G,
                        void *out, int32_t *n_int, int32_t *n_test, int32_t *n_leaf, int wpc) {
  if (n_int)  // counting walk
    return opt.criterion == BH_CRIT_WARP_VOTE
               ? go_scalar<false, true, false, true, false>(s, nb, rec, mom, qrec, q64, blk, orig,
                                                           fa, G, out, n_int, n_test, n_leaf)
               : go_pair<false, true, false>(s, nb, rec, qrec, blk, orig, fa, G, out, n_int,
                                             n_test, n_leaf, wpc);
  if (opt.quadrupole)
    return launch_walk_q<true>(s, opt, nb, rec, mom, qrec, q64, blk, orig, fa, G, out, wpc);
  return launch_walk_q<false>(s, opt, nb, rec, mom, qrec, q64, blk, orig, fa, G, out, wpc);
}

}  // namespace bhg
