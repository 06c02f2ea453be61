// The Barnes-Hut walk: potential at every cell centre (Sec. 3.3).
//
// Traversal.  The paper walks with a shared-memory stack pushed by lane 0 and
// an all() vote on the opening test (Sec. 3.3).  This walk needs no stack:
// nodes are stored in pre-order, so a node's first child is the next node and
// its subtree ends at its skip index.  Every target cell keeps `next`, the
// first node it still has to visit (0 = the root at the start).  In the
// one-target-per-lane walk (k_walk_scalar) the warp takes the smallest `next`
// over its lanes at each step (one __reduce_min_sync), all lanes load that
// node (one broadcast load), and the targets whose `next` equals it apply the
// opening test of Eq. 4:
//   accepted -> add M / d, next = skip (the whole subtree is done)
//   opened   -> next = node + 1 (descend into the first child)
// Cells carry s2 = 0: the test accepts every other cell (d2 > 0) and rejects
// only the target's own cell (d2 = 0), which then adds nothing; for a cell
// node + 1 is its skip, so no special case is needed.  Each target thus
// visits exactly the nodes of its own recursive walk, in pre-order, and gets
// the per-cell result of the recursive definition; targets whose `next` lies
// further ahead wait (masked) for the warp to get there.  `next` only grows,
// so a walk ends after at most n_nodes steps.  With the warp vote (paper mode)
// all lanes share `next`.  The per-cell pair walk (walk_group) takes the same
// decisions in two modes that need no reduction: one vote per node while all
// targets sit at the same node, a lazy per-target `next` inside a subtree
// they disagree on.
//
// Work layout.
//  * Per-cell binary32 walk (the default, k_walk_pair / k_walk_queue): one
//    warp per 4x4x4 octant of a block (64 cells, local Morton indices 64o ..
//    64o+63), lane l owning the two x-neighbours 64o+2l and 64o+2l+1, or per
//    8x4x4 slab (128 cells, two such pairs per lane).  A lane's targets share
//    ty, tz and so dy, dz; their dx, d2, 1/d products and Kahan sums run as
//    packed f32x2 operations (two binary32 results per instruction, each
//    rounded as its scalar counterpart).  CTAs of 2 to 16 warps, on a plain
//    grid or a persistent one fed by a work counter (the launch shape).
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

constexpr int kWalkThreads = 256;               // CTA of the scalar walk: 8 bricks = half a block
constexpr int kWarpsPerCta = kWalkThreads / 32;
constexpr int kMaxWalkThreads = 512;            // largest tunable CTA
// Default launch shape of the per-cell walk (the fastest on GB300 for the
// spheroid and cloud-core workloads at theta 0.24 - 0.72): one target pair
// per lane (64-target octants), CTAs of 4 warps.
constexpr int kDefaultPairs = 1;
constexpr int kDefaultWarps = 4;

__global__ void k_prepare_s2(int64_t n, const float2 *__restrict__ aux, WalkRec *__restrict__ rec,
                             float inv_theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 a = aux[i];
  const float s = __fadd_rn(__fmul_rn(a.x, inv_theta), a.y);  // l/theta + delta
  rec[i].s2 = __fmul_rn(s, s);
}

// ---- per-cell binary32 walk, x-neighbour target pairs per lane -------------
//
// A warp walks for a group of targets that share every y and z coordinate
// pattern: lane l owns NP pairs of x-neighbours, pair k at x offset 4k, so
// all 2 NP targets of a lane have the same (y, z) and share dy, dz and
// dy^2 + dz^2.  NP = 1: the group is a 4x4x4 octant of a block (64 targets);
// NP = 2: two x-adjacent octants, a 8x4x4 slab (128 targets).  A larger group
// walks only a few percent more nodes than a smaller one (the union of its
// targets' walks), so every record loaded serves more targets: the record's
// broadcast to all 32 lanes (8 registers each) is what the L1 return path
// spends most of its time on.

// Per-target state of one lane: NP packed pairs.
template <int NP>
struct Lanes {
  u64 tx2[NP];              // {x_a, x_b} of pair k, box units
  u64 sum[NP], comp[NP];    // Kahan pair sums
  unsigned next_a[NP], next_b[NP];
  int ni[2 * NP], nt[2 * NP], nl[2 * NP];  // counting walk
};

// dy, dz and h = fma(dz, dz, dy * dy) of the lane's targets to a record, the
// shared part of the opening test's distance (fixed rounding: d2 = fma(dx,
// dx, h)).
__device__ __forceinline__ float dyz_part(float ty, float tz, u64 q1, float &dy, float &dz) {
  float py, pz;
  upk(q1, py, pz);
  dy = __fsub_rn(ty, py);
  dz = __fsub_rn(tz, pz);
  return __fmaf_rn(dz, dz, __fmul_rn(dy, dy));
}

// The terms of an accepted node for one pair: M/d, or with the quadrupole
// record w rinv (M + (d^T Q d / 2) rinv^4); qu = Qxy dy + Qxz dz and qc =
// dy (Qyy/2 dy + Qyz dz) + Qzz/2 dz^2 are shared by all pairs of the lane.
template <bool QUAD>
__device__ __forceinline__ u64 node_term2(u64 mm, u64 rr, u64 dx2, u64 w0, float qu, float qc) {
  if (!QUAD) return mul2(mm, rr);
  const u64 hq = fma2(dx2, fma2(w0, dx2, pk(qu, qu)), pk(qc, qc));
  const u64 r2 = mul2(rr, rr);
  return mul2(rr, fma2(hq, mul2(r2, r2), mm));
}

// The shared parts of a node's quadrupole term from its record (loaded with
// the node's walk record at the start of the step, so that its latency
// overlaps the opening test; w0 = {Qxx/2, Qxx/2}, w1 = {Qyy/2, Qzz/2},
// w2 = {Qxy, Qxz}, w3 = {Qyz, 0}).
__device__ __forceinline__ void quad_parts(u64 v0, u64 w1, u64 w2, u64 w3, float dy, float dz,
                                           u64 &w0, float &qu, float &qc) {
  w0 = v0;
  float hyy, hzz, qxy, qxz, qyz, unused;
  upk(w1, hyy, hzz);
  upk(w2, qxy, qxz);
  upk(w3, qyz, unused);
  qu = __fmaf_rn(qxz, dz, __fmul_rn(qxy, dy));
  const float v = __fmaf_rn(hyy, dy, __fmul_rn(qyz, dz));
  qc = __fmaf_rn(dy, v, __fmul_rn(__fmul_rn(hzz, dz), dz));
}

// The 8 cells of a bottom node (node + 1 .. node + 8) for the targets that
// opened it (oa[k] for target a of pair k, ob[k] for target b; kept as
// predicates, not packed into a bit mask, which took a few more instructions
// a step): every cell but the target's own (d2 > 0).
// Cells 2j and 2j + 1 are x-neighbours with the same y and z, so they share
// dy, dz and h too.  The 8 positive cell terms are summed plainly (a
// relative error of at most 7 units in the last place of their sum) and the
// sum joins the compensated total once.  (A second form of this loop for
// bottom nodes that hold none of the warp's targets, the openers' mask a
// factor on the mass instead of a compare and select per cell, took 8 more
// registers and made the walk slower.)
template <int NP, bool KAHAN, bool COUNTS>
__device__ __forceinline__ void bottom_cells(unsigned node, const bool (&oa)[NP],
                                             const bool (&ob)[NP],
                                             const WalkRec *__restrict__ rec, float ty,
                                             float tz, Lanes<NP> &L) {
  u64 part[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) part[k] = 0ull;
#pragma unroll 1
  for (unsigned c = node + 1; c < node + 9u; c += 2) {
    u64 c0, c1, c2, c3, e0, e1, e2, e3;
    load_rec(rec + c, c0, c1, c2, c3);
    load_rec(rec + c + 1, e0, e1, e2, e3);
    float dy, dz;
    const float h = dyz_part(ty, tz, c1, dy, dz);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const u64 px = j ? e0 : c0, mm = j ? e2 : c2;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const u64 dx2 = sub2(L.tx2[k], px);
        float e2a, e2b;
        upk(fma2(dx2, dx2, pk(h, h)), e2a, e2b);
        const bool la = oa[k] && e2a > 0.0f;
        const bool lb = ob[k] && e2b > 0.0f;
        if (COUNTS) {
          L.ni[2 * k] += la;
          L.ni[2 * k + 1] += lb;
          L.nl[2 * k] += la;
          L.nl[2 * k + 1] += lb;
        } else {
          float ra = rsqrt_approx(e2a), rb = rsqrt_approx(e2b);
          ra = la ? ra : 0.0f;
          rb = lb ? rb : 0.0f;
          part[k] = fma2(mm, pk(ra, rb), part[k]);
        }
      }
    }
  }
  if (!COUNTS) {
#pragma unroll
    for (int k = 0; k < NP; ++k) accumulate2<KAHAN>(L.sum[k], L.comp[k], part[k]);
  }
}

// Walk of one target group (unit u = (8 / NP) * sorted block + group; group
// g covers octants NP g .. NP g + NP - 1).
//
// Two modes.  While every target of the warp is at the same node (all `next`
// equal: "converged", as at the root), a step needs no per-target
// bookkeeping: each target still applies its own test, and one vote tells
// whether all accepted (add the terms, continue at skip), all opened
// (continue at node + 1) or they differ.  Where they differ, the targets
// part, and the subtree of that node is walked per target ("diverged").
// There a target takes part in the step at `node` when its `next` <= node
// (`next` is kept lazily: it only moves ahead of the warp when the target
// accepts a node that another target opens); the warp goes on at node + 1
// when some taking-part target opened the node, else at its skip index --
// which is the smallest next of all targets, as the recursive walk requires.
// Every target leaves a subtree at its skip index, so they all meet again at
// the end of the parted subtree, and the warp is converged once more.  Both
// modes take exactly the per-target decisions of the recursive definition;
// they differ only in the bookkeeping.
//
// Bottom nodes (whose 8 children are cells, stored right after them, so
// skip = node + 9) are taken in one step: the targets that open such a node
// interact with its 8 cells in an unrolled loop that needs no per-cell
// bookkeeping (cells are never opened), and every target then continues at
// node + 9.  Cells are only reached through their bottom node, so the walk
// never stops at a cell.
template <int NP, bool KAHAN, bool COUNTS, bool QUAD>
__device__ __forceinline__ void walk_group(unsigned u, int lane, const WalkRec *__restrict__ rec,
                                           const WalkQuad *__restrict__ qrec,
                                           const int4 *__restrict__ blk,
                                           const int *__restrict__ orig,
                                           const int4 *__restrict__ fld,
                                           const double *__restrict__ invL,
                                           const unsigned long long *__restrict__ mmax, double G,
                                           float *__restrict__ out, int32_t *__restrict__ n_int,
                                           int32_t *__restrict__ n_test,
                                           int32_t *__restrict__ n_leaf) {
  constexpr unsigned kGroups = 8 / NP;                // groups per block
  const unsigned p = u / kGroups;                     // sorted block
  const int4 F = fld[p];                              // this field's node range
  const unsigned n_nodes = (unsigned)F.y;
  const int o = (int)(u % kGroups) * NP;              // octant of pair 0
  const int ma = (o << 6) | (lane << 1);              // local Morton index, even: x bit 0
  const int4 B = blk[p];
  const int cx = (int)compact3(ma), cy = (int)compact3(ma >> 1), cz = (int)compact3(ma >> 2);
  const int lc = B.x + 3;
  // cell centres in box units, exact in binary32: (2 i + 1) * 2^-(lc+1)
  const float hh = pow2f(-(lc + 1));
  const float ty = __fmul_rn((float)(2 * (8 * B.z + cy) + 1), hh);
  const float tz = __fmul_rn((float)(2 * (8 * B.w + cz) + 1), hh);
  Lanes<NP> L;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int ix = 8 * B.y + cx + 4 * k;
    L.tx2[k] = pk(__fmul_rn((float)(2 * ix + 1), hh), __fmul_rn((float)(2 * ix + 3), hh));
    L.sum[k] = 0ull;  // (+0.0f, +0.0f)
    L.comp[k] = 0ull;
    L.ni[2 * k] = L.ni[2 * k + 1] = L.nt[2 * k] = L.nt[2 * k + 1] = 0;
    L.nl[2 * k] = L.nl[2 * k + 1] = 0;
  }

  unsigned node = (unsigned)F.x;  // the field's root
  while (node < n_nodes) {
    // ---- converged: every target is at `node`, an internal node ----
    u64 q0, q1, q2, q3;
    load_rec(rec + node, q0, q1, q2, q3);
    u64 p0 = 0ull, p1 = 0ull, p2 = 0ull, p3 = 0ull;
    if (QUAD && !COUNTS) load_quad(qrec + node, p0, p1, p2, p3);
    float s2, skf;
    upk(q3, s2, skf);
    const unsigned skip = __float_as_uint(skf);
    float dy, dz;
    const float h = dyz_part(ty, tz, q1, dy, dz);
    u64 dx2[NP];
    float d2a[NP], d2b[NP];
    bool ta[NP], tb[NP];
    bool all = true, any = false;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      dx2[k] = sub2(L.tx2[k], q0);
      upk(fma2(dx2[k], dx2[k], pk(h, h)), d2a[k], d2b[k]);
      ta[k] = d2a[k] > s2;
      tb[k] = d2b[k] > s2;
      all = all && ta[k] && tb[k];
      any = any || ta[k] || tb[k];
      if (COUNTS) {
        ++L.nt[2 * k];
        ++L.nt[2 * k + 1];
        L.ni[2 * k] += ta[k];
        L.ni[2 * k + 1] += tb[k];
      }
    }
    u64 w0 = 0ull;
    float qu = 0.0f, qc = 0.0f;
    if (__all_sync(kFull, all)) {  // every target accepts the node
      if (!COUNTS) {
        if (QUAD) quad_parts(p0, p1, p2, p3, dy, dz, w0, qu, qc);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const u64 rr = pk(rsqrt_approx(d2a[k]), rsqrt_approx(d2b[k]));
          accumulate2<KAHAN>(L.sum[k], L.comp[k], node_term2<QUAD>(q2, rr, dx2[k], w0, qu, qc));
        }
      }
      node = skip;
      continue;
    }
    const bool any_take = __any_sync(kFull, any);
    if (!COUNTS && any_take) {
      if (QUAD) quad_parts(p0, p1, p2, p3, dy, dz, w0, qu, qc);
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float ra = rsqrt_approx(d2a[k]), rb = rsqrt_approx(d2b[k]);
        ra = ta[k] ? ra : 0.0f;
        rb = tb[k] ? rb : 0.0f;
        accumulate2<KAHAN>(L.sum[k], L.comp[k],
                           node_term2<QUAD>(q2, pk(ra, rb), dx2[k], w0, qu, qc));
      }
    }
    if (skip == node + 9u) {  // bottom node: the openers meet its cells; all go on at skip
      bool oa[NP], ob[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        oa[k] = !ta[k];
        ob[k] = !tb[k];
      }
      bottom_cells<NP, KAHAN, COUNTS>(node, oa, ob, rec, ty, tz, L);
      node = skip;
      continue;
    }
    if (!any_take) {  // every target opens the node
      node = node + 1;
      continue;
    }
    // ---- diverged: the targets part inside the subtree [node + 1, end) ----
    const unsigned end = skip;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      L.next_a[k] = ta[k] ? skip : node + 1;
      L.next_b[k] = tb[k] ? skip : node + 1;
    }
    node = node + 1;  // some target opened the node
    while (node < end) {
      load_rec(rec + node, q0, q1, q2, q3);
      if (QUAD && !COUNTS) load_quad(qrec + node, p0, p1, p2, p3);
      upk(q3, s2, skf);
      const unsigned skp = __float_as_uint(skf);
      const float hd = dyz_part(ty, tz, q1, dy, dz);
      bool ma_[NP], mb_[NP];
      bool oa[NP], ob[NP];
      bool any_tk = false, any_op = false;
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        dx2[k] = sub2(L.tx2[k], q0);
        upk(fma2(dx2[k], dx2[k], pk(hd, hd)), d2a[k], d2b[k]);
        ma_[k] = L.next_a[k] <= node;
        mb_[k] = L.next_b[k] <= node;
        ta[k] = ma_[k] && d2a[k] > s2;
        tb[k] = mb_[k] && d2b[k] > s2;
        oa[k] = ma_[k] && !ta[k];
        ob[k] = mb_[k] && !tb[k];
        any_op = any_op || oa[k] || ob[k];
        any_tk = any_tk || ta[k] || tb[k];
        if (COUNTS) {  // internal: cells are only reached through bottom nodes
          L.ni[2 * k] += ta[k];
          L.ni[2 * k + 1] += tb[k];
          L.nt[2 * k] += ma_[k];
          L.nt[2 * k + 1] += mb_[k];
        }
      }
      if (!COUNTS && __any_sync(kFull, any_tk)) {
        if (QUAD) quad_parts(p0, p1, p2, p3, dy, dz, w0, qu, qc);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          float ra = rsqrt_approx(d2a[k]), rb = rsqrt_approx(d2b[k]);
          ra = ta[k] ? ra : 0.0f;
          rb = tb[k] ? rb : 0.0f;
          accumulate2<KAHAN>(L.sum[k], L.comp[k],
                             node_term2<QUAD>(q2, pk(ra, rb), dx2[k], w0, qu, qc));
        }
      }
      const bool opened = __any_sync(kFull, any_op);
      if (skp == node + 9u) {  // bottom node: all go on at skip
        if (opened) bottom_cells<NP, KAHAN, COUNTS>(node, oa, ob, rec, ty, tz, L);
        node = skp;
      } else if (opened) {  // takers of a node others open move ahead of the warp
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          L.next_a[k] = ta[k] ? skp : L.next_a[k];
          L.next_b[k] = tb[k] ? skp : L.next_b[k];
        }
        node = node + 1;
      } else {
        node = skp;
      }
    }
    node = end;  // every target leaves the subtree at its skip index
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int64_t cell = (int64_t)orig[p] * kCellsPerBlock + cz * 64 + cy * 8 + cx + 4 * k;
    if (COUNTS) {
      n_int[cell] = L.ni[2 * k];
      n_int[cell + 1] = L.ni[2 * k + 1];
      n_test[cell] = L.nt[2 * k];
      n_test[cell + 1] = L.nt[2 * k + 1];
      if (n_leaf) {
        n_leaf[cell] = L.nl[2 * k];
        n_leaf[cell + 1] = L.nl[2 * k + 1];
      }
    } else {
      u64 sm = L.sum[k];
      sm = finish2<KAHAN>(sm, L.comp[k]);
      float sa, sb;
      upk(sm, sa, sb);
      // -G/L times the field's binary32 mass unit 2^e (exact), rounded once
      const float scale = (float)(-G * invL[F.w] * pow2i(mass_exponent(mmax[F.w])));
      out[cell] = __fmul_rn(sa, scale);
      out[cell + 1] = __fmul_rn(sb, scale);
    }
  }
}

// One warp per target group (8 / NP groups per block), group order[warp] when
// an order is given.  (Schedules that keep an SM's warps on neighbouring
// octants -- SM- or CTA-affine ranges with stealing -- share more of the near
// field in L1 but ran 2-8 % slower on GB300.)
template <int NP, bool KAHAN, bool COUNTS, bool QUAD>
__global__ void __launch_bounds__(kMaxWalkThreads)
    k_walk_pair(unsigned nunits, const unsigned *__restrict__ order,
                const WalkRec *__restrict__ rec,
                const WalkQuad *__restrict__ qrec, const int4 *__restrict__ blk,
                const int *__restrict__ orig, const int4 *__restrict__ fld,
                const double *__restrict__ invL, const unsigned long long *__restrict__ mmax,
                double G, float *__restrict__ out, int32_t *__restrict__ n_int,
                int32_t *__restrict__ n_test, int32_t *__restrict__ n_leaf) {
  const int lane = threadIdx.x & 31;
  const unsigned warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (warp >= nunits) return;  // whole warps only
  const unsigned u = order ? order[warp] : warp;
  walk_group<NP, KAHAN, COUNTS, QUAD>(u, lane, rec, qrec, blk, orig, fld, invL, mmax, G, out,
                                      n_int, n_test, n_leaf);
}

// The same walk on a persistent grid: each warp takes `per_ticket`
// consecutive groups at a time from the work counter (one atomic add by lane
// 0; no waiting on other warps) until every group is taken.  In the groups'
// own order, consecutive groups are neighbouring octants; with `order` (the
// groups sorted by the time of their walks, longest first) the long walks
// start first and the short ones fill the end, so that fewer warps are left
// running alone at the end of the launch.  cycles (or null): the SM clock
// cycles of each group's walk, the measurement that order is made from.
template <int NP, bool KAHAN, bool COUNTS, bool QUAD>
__global__ void __launch_bounds__(kMaxWalkThreads)
    k_walk_queue(unsigned nunits, unsigned per_ticket, unsigned *__restrict__ counter,
                 const unsigned *__restrict__ order, unsigned long long *__restrict__ cycles,
                 const WalkRec *__restrict__ rec, const WalkQuad *__restrict__ qrec,
                 const int4 *__restrict__ blk, const int *__restrict__ orig,
                 const int4 *__restrict__ fld, const double *__restrict__ invL,
                 const unsigned long long *__restrict__ mmax, double G, float *__restrict__ out,
                 int32_t *__restrict__ n_int, int32_t *__restrict__ n_test,
                 int32_t *__restrict__ n_leaf) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned u0 = 0u;
    if (lane == 0) u0 = atomicAdd(counter, per_ticket);
    u0 = __shfl_sync(kFull, u0, 0);
    if (u0 >= nunits) return;
    const unsigned u1 = u0 + per_ticket < nunits ? u0 + per_ticket : nunits;
    for (unsigned i = u0; i < u1; ++i) {
      const unsigned u = order ? order[i] : i;
      const long long c0 = cycles ? clock64() : 0;
      walk_group<NP, KAHAN, COUNTS, QUAD>(u, lane, rec, qrec, blk, orig, fld, invL, mmax, G, out,
                                          n_int, n_test, n_leaf);
      if (cycles && lane == 0) cycles[u] = (unsigned long long)(clock64() - c0);
    }
  }
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
      if (KAHAN) {  // compensated as accumulate2 (bh_walk_common.cuh)
        const float t = __fadd_rn(sum, term);
        comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(sum, t), term));
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
    const float total = KAHAN ? __fadd_rn(sum, comp) : sum;
    reinterpret_cast<float *>(out)[cell] = __fmul_rn(total, scale_f);
  }
}

template <int NP, bool KAHAN, bool COUNTS, bool QUAD>
cudaError_t go_pair_np(cudaStream_t s, int nb, const WalkRec *rec, const WalkQuad *qrec,
                       const int4 *blk, const int *orig, const FieldArgs &fa, double G, void *out,
                       int32_t *ni, int32_t *nt, int32_t *nl, const WalkShape &shape) {
  const unsigned nunits = (unsigned)nb * (8u / NP);
  const int w = shape.warps > 0 ? shape.warps : kDefaultWarps;
  if (shape.ticket > 0 && shape.counter) {  // persistent: the CTAs that fit at once
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, k_walk_queue<NP, KAHAN, COUNTS, QUAD>, 32 * w, 0);
    if (e != cudaSuccess) return e;
    const unsigned warps_needed = (nunits + (unsigned)shape.ticket - 1) / (unsigned)shape.ticket;
    const unsigned ctas_needed = (warps_needed + (unsigned)w - 1) / (unsigned)w;
    const unsigned resident = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    const unsigned grid = ctas_needed < resident ? ctas_needed : resident;
    e = cudaMemsetAsync(shape.counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_walk_queue<NP, KAHAN, COUNTS, QUAD><<<grid, 32 * w, 0, s>>>(
        nunits, (unsigned)shape.ticket, shape.counter, shape.order, shape.cycles, rec, qrec, blk,
        orig, fa.fld, fa.invL, fa.mmax, G, (float *)out, ni, nt, nl);
    return cudaGetLastError();
  }
  const int grid = (int)((nunits + w - 1) / w);
  k_walk_pair<NP, KAHAN, COUNTS, QUAD><<<grid, 32 * w, 0, s>>>(
      nunits, shape.order, rec, qrec, blk, orig, fa.fld, fa.invL, fa.mmax, G, (float *)out, ni,
      nt, nl);
  return cudaGetLastError();
}

template <bool KAHAN, bool COUNTS, bool QUAD>
cudaError_t go_pair(cudaStream_t s, int nb, const WalkRec *rec, const WalkQuad *qrec,
                    const int4 *blk, const int *orig, const FieldArgs &fa, double G, void *out,
                    int32_t *ni, int32_t *nt, int32_t *nl, WalkShape shape) {
  const int np = shape.pairs > 0 ? shape.pairs : kDefaultPairs;
  if (np == 2)
    return go_pair_np<2, KAHAN, COUNTS, QUAD>(s, nb, rec, qrec, blk, orig, fa, G, out, ni, nt, nl,
                                              shape);
  return go_pair_np<1, KAHAN, COUNTS, QUAD>(s, nb, rec, qrec, blk, orig, fa, G, out, ni, nt, nl,
                                            shape);
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
                          void *out, WalkShape shape) {
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
                                                nullptr, nullptr, shape)
                   : go_pair<false, false, QUAD>(s, nb, rec, qrec, blk, orig, fa, G, out,
                                                 nullptr, nullptr, nullptr, shape);
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
                        void *out, int32_t *n_int, int32_t *n_test, int32_t *n_leaf,
                        WalkShape shape) {
  if (n_int)  // counting walk
    return opt.criterion == BH_CRIT_WARP_VOTE
               ? go_scalar<false, true, false, true, false>(s, nb, rec, mom, qrec, q64, blk, orig,
                                                           fa, G, out, n_int, n_test, n_leaf)
               : go_pair<false, true, false>(s, nb, rec, qrec, blk, orig, fa, G, out, n_int,
                                             n_test, n_leaf, shape);
  if (opt.quadrupole)
    return launch_walk_q<true>(s, opt, nb, rec, mom, qrec, q64, blk, orig, fa, G, out, shape);
  return launch_walk_q<false>(s, opt, nb, rec, mom, qrec, q64, blk, orig, fa, G, out, shape);
}

}  // namespace bhg
