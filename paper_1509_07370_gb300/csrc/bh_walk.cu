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
#include "bh_internal.cuh"

namespace bhg {
namespace {

constexpr int kWalkThreads = 256;               // default CTA: 8 warps = one block
constexpr int kWarpsPerCta = kWalkThreads / 32;
constexpr int kMaxWalkThreads = 512;            // largest tunable CTA
constexpr unsigned kFull = 0xffffffffu;
typedef unsigned long long u64;

__global__ void k_prepare_s2(int64_t n, const float2 *__restrict__ aux, WalkRec *__restrict__ rec,
                             float inv_theta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 a = aux[i];
  const float s = __fadd_rn(__fmul_rn(a.x, inv_theta), a.y);  // l/theta + delta
  rec[i].s2 = __fmul_rn(s, s);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// ---- packed binary32 pairs and raw loads (inline PTX) -----------------------
__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(u64 v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// 1/sqrt(x) on the special-function unit.  Only called where the value is
// used for x >= 2^-44 (an accepted node or another cell), so flushing
// subnormal inputs changes nothing.
__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// One 32-byte walk record as four 64-bit lanes:
//   q0 = {Px, Px}, q1 = {Py, Pz}, q2 = {M, M}, q3 = {s2, skip}
__device__ __forceinline__ void load_rec(const WalkRec *p, u64 &q0, u64 &q1, u64 &q2, u64 &q3) {
  asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
      : "=l"(q0), "=l"(q1), "=l"(q2), "=l"(q3)
      : "l"(p));
}

// One 32-byte quadrupole record: w0 = {Qxx/2, Qxx/2}, w1 = {Qyy/2, Qzz/2},
// w2 = {Qxy, Qxz}, w3 = {Qyz, 0}.
__device__ __forceinline__ void load_quad(const WalkQuad *p, u64 &w0, u64 &w1, u64 &w2, u64 &w3) {
  asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
      : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
      : "l"(p));
}

// ---- per-cell binary32 walk, two x-neighbour targets per lane ---------------
// Adds the pair `term` to the running (Kahan-compensated) pair sums.
template <bool KAHAN>
__device__ __forceinline__ void accumulate2(u64 &sum, u64 &comp, u64 term) {
  if (KAHAN) {
    const u64 y = sub2(term, comp);
    const u64 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
  } else {
    sum = add2(sum, term);
  }
}

// Squared distances of the two targets (tx2 = {txa, txb}, ty, tz) to the
// record's binary32 centre of mass, with the fixed rounding of the opening
// test: d2 = fma(dx, dx, fma(dz, dz, dy*dy)); the (dy, dz) part is shared.
__device__ __forceinline__ void dist2(u64 tx2, float ty, float tz, u64 q0, u64 q1, float &d2a,
                                      float &d2b, u64 &dx2, float &dy, float &dz) {
  float py, pz;
  upk(q1, py, pz);
  dx2 = sub2(tx2, q0);
  dy = __fsub_rn(ty, py);
  dz = __fsub_rn(tz, pz);
  const float h = __fmaf_rn(dz, dz, __fmul_rn(dy, dy));
  upk(fma2(dx2, dx2, pk(h, h)), d2a, d2b);
}

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
                                            const double *__restrict__ invL, double G,
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
    const float scale = (float)(-G * invL[F.w]);
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
                const double *__restrict__ invL, double G, float *__restrict__ out,
                int32_t *__restrict__ n_int, int32_t *__restrict__ n_test,
                int32_t *__restrict__ n_leaf) {
  const int lane = threadIdx.x & 31;
  const unsigned warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (warp >= nunits) return;  // whole warps only
  walk_octant<KAHAN, COUNTS, QUAD>(warp, lane, rec, qrec, blk, orig, fld, invL, G, out, n_int,
                                   n_test, n_leaf);
}

// ---- one target per lane: binary64 interactions and/or the warp vote --------
template <bool F64, bool VOTE, bool KAHAN, bool COUNTS, bool QUAD>
__global__ void __launch_bounds__(kWalkThreads)
    k_walk_scalar(int nbricks, const WalkRec *__restrict__ rec,
                  const double4_32a *__restrict__ mom, const WalkQuad *__restrict__ qrec,
                  const double *__restrict__ q64, const int4 *__restrict__ blk,
                  const int *__restrict__ orig, const int4 *__restrict__ fld,
                  const double *__restrict__ invL, double G, void *__restrict__ out,
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
  const double scale_d = -G * invL[F.w];
  const float scale_f = (float)scale_d;
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
      nunits, rec, qrec, blk, orig, fa.fld, fa.invL, G, (float *)out, ni, nt, nl);
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
      nbricks, rec, mom, qrec, q64, blk, orig, fa.fld, fa.invL, G, out, ni, nt, nl);
  return cudaGetLastError();
}

// ---- learned correction: the MLP on the tensor cores inside the walk --------
// At a step where any of the warp's 64 targets accepts an internal node, the
// warp evaluates y = MLP(x) for all 64 rows (row 2*lane+i = the lane's target
// i; rows of targets that do not accept are computed and ignored) with
// mma.sync m16n8k16 bf16 -> FP32: X[64x16] W1[16x64], H1[64x64] W2[64x64],
// H2[64x64] W3[64x8].  Activations pass through per-warp shared memory as
// bf16; weights are staged once per CTA.  The accepted term becomes
// (M/d)(1 + s^2 y).  (The warp-synchronous mma.sync form is used because the
// network runs per warp step inside the walk; a CTA-wide tcgen05 MMA would
// have to gather rows across warps that walk different nodes.)
constexpr int kLearnWarps = 8;
struct LearnSmem {
  MlpDev w;
  uint16_t x[kLearnWarps][64 * 16];
  uint16_t h[kLearnWarps][64 * 64];
  float y[kLearnWarps][64];
};

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ float tanh_approx(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float gelu_t(float a) {
  return 0.5f * a * (1.0f + tanh_approx(0.7978845608028654f * (a + 0.044715f * a * a * a)));
}
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// A fragment (16 rows from m0, 16 k from k0) of a row-major bf16 matrix with
// row stride ld (elements).
__device__ __forceinline__ void load_a(uint32_t a[4], const uint16_t *M, int ld, int m0, int k0,
                                       int gid, int tig) {
  const uint16_t *r0 = M + (m0 + gid) * ld + k0 + 2 * tig;
  const uint16_t *r1 = r0 + 8 * ld;
  a[0] = *reinterpret_cast<const uint32_t *>(r0);
  a[1] = *reinterpret_cast<const uint32_t *>(r1);
  a[2] = *reinterpret_cast<const uint32_t *>(r0 + 8);
  a[3] = *reinterpret_cast<const uint32_t *>(r1 + 8);
}

// y for the warp's 64 rows of X (written to y[64]).
__device__ void mlp_warp(const MlpDev &W, uint16_t *X, uint16_t *H, float *Y, int lane) {
  const int gid = lane >> 2, tig = lane & 3;
  // layer 1 (K = 16): H = gelu(X W1 + b1)
  for (int mt = 0; mt < 4; ++mt) {
    uint32_t a[4];
    load_a(a, X, 16, mt * 16, 0, gid, tig);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const uint16_t *b = W.w1t + (nt * 8 + gid) * 16 + 2 * tig;
      mma_bf16(c, a, *reinterpret_cast<const uint32_t *>(b),
               *reinterpret_cast<const uint32_t *>(b + 8));
      const int col = nt * 8 + 2 * tig;
      const float b0 = W.b1[col], b1 = W.b1[col + 1];
      *reinterpret_cast<uint32_t *>(H + (mt * 16 + gid) * 64 + col) =
          bf16x2(gelu_t(c[0] + b0), gelu_t(c[1] + b1));
      *reinterpret_cast<uint32_t *>(H + (mt * 16 + gid + 8) * 64 + col) =
          bf16x2(gelu_t(c[2] + b0), gelu_t(c[3] + b1));
    }
  }
  __syncwarp();
  // layer 2 (K = 64), rows of one m-tile at a time, in place
  for (int mt = 0; mt < 4; ++mt) {
    uint32_t a[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) load_a(a[kt], H, 64, mt * 16, kt * 16, gid, tig);
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      const uint16_t *b = W.w2t + (nt * 8 + gid) * 64 + 2 * tig;
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
        mma_bf16(c, a[kt], *reinterpret_cast<const uint32_t *>(b + kt * 16),
                 *reinterpret_cast<const uint32_t *>(b + kt * 16 + 8));
      const int col = nt * 8 + 2 * tig;
      const float b0 = W.b2[col], b1 = W.b2[col + 1];
      *reinterpret_cast<uint32_t *>(H + (mt * 16 + gid) * 64 + col) =
          bf16x2(gelu_t(c[0] + b0), gelu_t(c[1] + b1));
      *reinterpret_cast<uint32_t *>(H + (mt * 16 + gid + 8) * 64 + col) =
          bf16x2(gelu_t(c[2] + b0), gelu_t(c[3] + b1));
    }
    __syncwarp();
  }
  // layer 3 (N = 1, padded to 8): y = H2 W3 + b3
  for (int mt = 0; mt < 4; ++mt) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const uint16_t *b = W.w3t + gid * 64 + 2 * tig;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      uint32_t a[4];
      load_a(a, H, 64, mt * 16, kt * 16, gid, tig);
      mma_bf16(c, a, *reinterpret_cast<const uint32_t *>(b + kt * 16),
               *reinterpret_cast<const uint32_t *>(b + kt * 16 + 8));
    }
    if (tig == 0) {  // column 0 of the output tile
      Y[mt * 16 + gid] = c[0] + W.b3;
      Y[mt * 16 + gid + 8] = c[2] + W.b3;
    }
  }
  __syncwarp();
}

// Features of one (target, node) pair in binary32 (see bh_learn.cu), written
// as one bf16 row of 16 (10 used).
__device__ __forceinline__ void feature_row(uint16_t *row, float dx, float dy, float dz, float r,
                                            float l, float dl, float inv_ml2, float qf,
                                            const WalkQuad &q) {
  const float ux = dx * r, uy = dy * r, uz = dz * r;
  const float s = l * r;
  const float quu = 2.0f * (ux * (q.hxx * ux + q.qxy * uy + q.qxz * uz) +
                            uy * (q.hyy * uy + q.qyz * uz)) + 2.0f * q.hzz * uz * uz;
  const float f7 = quu * inv_ml2;
  uint32_t *w = reinterpret_cast<uint32_t *>(row);
  w[0] = bf16x2(ux, uy);
  w[1] = bf16x2(uz, s);
  w[2] = bf16x2(s * s, s * s * s);
  w[3] = bf16x2(dl, f7);
  w[4] = bf16x2(qf * inv_ml2, s * s * f7);
  w[5] = 0u;
  w[6] = 0u;
  w[7] = 0u;
}

template <bool KAHAN>
__global__ void __launch_bounds__(kLearnWarps * 32)
    k_walk_learned(unsigned nunits, const WalkRec *__restrict__ rec,
                   const WalkQuad *__restrict__ qrec, const float2 *__restrict__ aux,
                   const int4 *__restrict__ blk, const int *__restrict__ orig,
                   const int4 *__restrict__ fld, const double *__restrict__ invL, double G,
                   const MlpDev *__restrict__ mlp, float *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LearnSmem &S = *reinterpret_cast<LearnSmem *>(smem_raw);
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(mlp);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&S.w);
    for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned u = blockIdx.x * kLearnWarps + wid;
  if (u >= nunits) return;  // whole warps only, after the CTA-wide staging
  uint16_t *X = S.x[wid];
  uint16_t *H = S.h[wid];
  float *Y = S.y[wid];
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
  u64 sum = 0ull, comp = 0ull;
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
    dist2(tx2, ty, tz, q0, q1, d2a, d2b, dx2, dy, dz);
    const bool mine_a = next_a == node, mine_b = next_b == node;
    const bool take_a = mine_a && d2a > s2;
    const bool take_b = mine_b && d2b > s2;
    float ra = rsqrt_approx(d2a), rb = rsqrt_approx(d2b);
    ra = take_a ? ra : 0.0f;
    rb = take_b ? rb : 0.0f;
    u64 fac = pk(1.0f, 1.0f);  // 1 + s^2 y
    if (__any_sync(kFull, take_a || take_b) && s2 > 0.0f) {
      const float2 lv = aux[node];          // node side, delta
      const WalkQuad q = qrec[node];
      float mf, mf2;
      upk(q2, mf, mf2);
      const float inv_ml2 = mf > 0.0f ? 1.0f / (mf * lv.x * lv.x) : 1.0f;
      const float qf = sqrtf(4.0f * (q.hxx * q.hxx + q.hyy * q.hyy + q.hzz * q.hzz) +
                             2.0f * (q.qxy * q.qxy + q.qxz * q.qxz + q.qyz * q.qyz));
      float dxa, dxb;
      upk(dx2, dxa, dxb);
      feature_row(X + (2 * lane) * 16, dxa, dy, dz, ra, lv.x, lv.y / lv.x, inv_ml2, qf, q);
      feature_row(X + (2 * lane + 1) * 16, dxb, dy, dz, rb, lv.x, lv.y / lv.x, inv_ml2, qf, q);
      __syncwarp();
      mlp_warp(S.w, X, H, Y, lane);
      const float sa = lv.x * ra, sb = lv.x * rb;
      fac = pk(1.0f + sa * sa * Y[2 * lane], 1.0f + sb * sb * Y[2 * lane + 1]);
    }
    accumulate2<KAHAN>(sum, comp, mul2(mul2(q2, pk(ra, rb)), fac));
    if (skip == node + 9u) {  // bottom node: its 8 cells in one step (monopole)
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
  const int64_t cell = (int64_t)orig[p] * kCellsPerBlock + cz * 64 + cy * 8 + cx;
  if (KAHAN) sum = sub2(sum, comp);
  float sa, sb;
  upk(sum, sa, sb);
  const float scale = (float)(-G * invL[F.w]);
  out[cell] = __fmul_rn(sa, scale);
  out[cell + 1] = __fmul_rn(sb, scale);
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

cudaError_t launch_walk_learned(cudaStream_t s, bh_ctx *ctx, double G, void *out) {
  const Tree &t = ctx->tree;
  const unsigned nunits = (unsigned)t.nb * 8u;
  const int smem = (int)sizeof(LearnSmem);
  FieldArgs fa;
  fa.fld = t.d_fld;
  fa.invL = t.d_invL;
  cudaError_t e;
  const bool kahan = ctx->opt.kahan != 0;
  if (kahan)
    e = cudaFuncSetAttribute(k_walk_learned<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  else
    e = cudaFuncSetAttribute(k_walk_learned<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (nunits + kLearnWarps - 1) / kLearnWarps;
  if (kahan)
    k_walk_learned<true><<<grid, kLearnWarps * 32, smem, s>>>(
        nunits, t.d_rec, t.d_qrec, t.d_aux, t.d_blk, t.d_orig, t.d_fld, t.d_invL, G, ctx->d_mlp,
        (float *)out);
  else
    k_walk_learned<false><<<grid, kLearnWarps * 32, smem, s>>>(
        nunits, t.d_rec, t.d_qrec, t.d_aux, t.d_blk, t.d_orig, t.d_fld, t.d_invL, G, ctx->d_mlp,
        (float *)out);
  return cudaGetLastError();
}

}  // namespace bhg
