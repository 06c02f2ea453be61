// Tree construction and FP64 moments for the Barnes-Hut AMR solver.
//
// The paper builds its octree by inserting cells one at a time under locks
// (Sec. 3.2.2) and sums the node moments bottom-up with threads that wait on
// children still marked by a negative mass (Sec. 3.2.3).  Here neither locks
// nor spin waits are used.  Because the leaf blocks of an AMR mesh tile the
// box, the octree is fully determined by the block list: every cube that
// holds more than one block is split into 8, every block is an 8^3 subtree.
// So:
//   1. each block gets the Morton key of its lower corner on the level-21
//      lattice (k_block_keys) and blocks are put in key order (k_sort_blocks,
//      only if the caller's order is not already sorted);
//   2. consecutive keys must abut exactly (k_tile_and_count): this checks that
//      the blocks tile the box, and the trailing zero bits of a block's key
//      tell how many internal "top" nodes (cubes above the blocks) start at it
//      in pre-order;
//   3. an exclusive scan gives every block the pre-order index of its first
//      node (k_prestart_scan), from which top nodes get their skip pointers
//      (k_top_nodes) and their child lists (k_top_children: one binary
//      search per top node and octant, all in parallel);
//   4. one CTA per block reduces its 512 cells to 64, 8 and 1 nodes in shared
//      memory (k_blocks), and one short launch per level reduces the top
//      nodes, deepest level first (k_top_moments), reading each node's
//      children from its list.  (Measured: following skip pointers from the
//      first child instead took 13 us more per build -- a chain of 8
//      dependent loads per node and level; so did searching the children
//      one after another in one thread.  Not faster either: a single CTA
//      walking the levels with barriers, and a cluster of 8 CTAs doing so
//      with cluster barriers (0.330-0.345 ms per build instead of 0.310):
//      spread over the whole GPU a level's FP64 work finishes sooner than
//      the launches it saves.)
// Moments follow Eq. 5 with the children summed in octant order, in FP64 with
// explicitly rounded operations (no contraction), so results are
// reproducible bit for bit.
//
// Several independent fields (meshes, each in its own box) can be built at
// once: their block lists are concatenated (fstart[f] = first block of field
// f), blocks are sorted within their field, every field gets its own tree,
// and the trees' pre-order node ranges follow each other in one node array.
// The formulas above hold unchanged over the concatenation: the pre-order
// index of the first node of block p is still 585 p + (top nodes before p),
// and a field's range ends where the next field's first node starts.
#include "bh_internal.cuh"

namespace bhg {
namespace {

__device__ __forceinline__ unsigned long long key_span(int level) {
  return 1ull << (3 * (kKeyLevels - level));  // volume of a level cube in level-21 cells
}

__device__ __forceinline__ unsigned long long block_key(int lb, int i, int j, int k) {
  const int sh = kKeyLevels - lb;
  return spread3((unsigned long long)i << sh) | (spread3((unsigned long long)j << sh) << 1) |
         (spread3((unsigned long long)k << sh) << 2);
}

// Returns true when (lb, ijk) is a valid block; raises error bits otherwise.
__device__ __forceinline__ bool valid_block(int lb, int i, int j, int k, unsigned *flags) {
  if (lb < 0 || lb > kMaxBlockLevel) {
    atomicOr(flags, kErrLevel);
    return false;
  }
  const int n = 1 << lb;
  if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) {
    atomicOr(flags, kErrCoord);
    return false;
  }
  return true;
}

// Field of caller block b: the last f with fstart[f] <= b.
__device__ __forceinline__ int field_of(int b, int nfields, const int *fstart) {
  int a = 0, e = nfields;  // invariant: fstart[a] <= b < fstart[e]
  while (e - a > 1) {
    const int m = (a + e) >> 1;
    if (fstart[m] <= b) a = m; else e = m;
  }
  return a;
}

__global__ void k_block_keys(int nb, const int *__restrict__ level, const int *__restrict__ ijk,
                             unsigned long long *__restrict__ key, int *__restrict__ idx,
                             unsigned *flags, int nfields, const int *__restrict__ fstart,
                             int *__restrict__ fid) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int f = field_of(b, nfields, fstart);
  fid[b] = f;
  const int lb = level[b];
  const int i = ijk[3 * b], j = ijk[3 * b + 1], k = ijk[3 * b + 2];
  unsigned long long kb = ~0ull;
  if (valid_block(lb, i, j, k, flags)) kb = block_key(lb, i, j, k);
  key[b] = kb;
  idx[b] = b;
  // is the caller's order already the key order?  (compare with block b+1
  // of the same field)
  if (b + 1 < fstart[f + 1]) {
    const int l2 = level[b + 1];
    unsigned long long k2 = ~0ull;
    if (l2 >= 0 && l2 <= kMaxBlockLevel) k2 = block_key(l2, ijk[3 * b + 3], ijk[3 * b + 4], ijk[3 * b + 5]);
    if (!(kb < k2)) atomicOr(flags + 1, 1u);
  }
}

// Stable LSD radix sort of (key, idx), one CTA per field (its segment of the
// block list), 4 bits per pass, 16 passes, result back in buffer 0.  Block
// lists are small (a 16M-cell mesh has ~32k blocks), and the sort only runs
// when the caller's block order is not already the Morton order.
constexpr int kSortThreads = 512;
__global__ void __launch_bounds__(kSortThreads)
    k_sort_blocks(const int *__restrict__ fstart, unsigned long long *k0, int *v0,
                  unsigned long long *k1, int *v1, const unsigned *flags) {
  if (flags[1] == 0u) return;  // already sorted
  const int off = fstart[blockIdx.x];
  const int n = fstart[blockIdx.x + 1] - off;
  k0 += off;
  v0 += off;
  k1 += off;
  v1 += off;
  __shared__ int hist[16 * kSortThreads];
  __shared__ int part[kSortThreads];
  const int t = threadIdx.x;
  const int per = (n + kSortThreads - 1) / kSortThreads;
  const int beg = min(t * per, n), end = min(beg + per, n);
  unsigned long long *kin = k0, *kout = k1;
  int *vin = v0, *vout = v1;
  for (int pass = 0; pass < 16; ++pass) {
    const int sh = 4 * pass;
    int cnt[16];
#pragma unroll
    for (int d = 0; d < 16; ++d) cnt[d] = 0;
    for (int i = beg; i < end; ++i) cnt[(kin[i] >> sh) & 15]++;
#pragma unroll
    for (int d = 0; d < 16; ++d) hist[d * kSortThreads + t] = cnt[d];
    __syncthreads();
    int s = 0;
    for (int j = 0; j < 16; ++j) s += hist[16 * t + j];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < kSortThreads; off <<= 1) {
      const int v = t >= off ? part[t - off] : 0;
      __syncthreads();
      part[t] += v;
      __syncthreads();
    }
    int run = part[t] - s;
    for (int j = 0; j < 16; ++j) {
      const int c = hist[16 * t + j];
      hist[16 * t + j] = run;
      run += c;
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < 16; ++d) cnt[d] = hist[d * kSortThreads + t];
    for (int i = beg; i < end; ++i) {
      const unsigned long long kk = kin[i];
      const int pos = cnt[(kk >> sh) & 15]++;
      kout[pos] = kk;
      vout[pos] = vin[i];
    }
    __syncthreads();
    unsigned long long *tk = kin; kin = kout; kout = tk;
    int *tv = vin; vin = vout; vout = tv;
  }
}

__device__ __forceinline__ int top_start_level(unsigned long long key) {
  // smallest level j such that the key is aligned to a level-j cube
  const int tz = key ? __ffsll((long long)key) - 1 : 64;
  return max(0, kKeyLevels - tz / 3);
}

__global__ void k_tile_and_count(int nb, const unsigned long long *__restrict__ key,
                                 const int *__restrict__ idx, const int *__restrict__ level,
                                 const int *__restrict__ ijk, int *__restrict__ count,
                                 int4 *__restrict__ blk, int *__restrict__ orig,
                                 unsigned *flags, const int *__restrict__ fstart,
                                 const int *__restrict__ fid, int *__restrict__ pos) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  const int b = idx[p];
  if (pos) pos[b] = p;  // sorted position of caller block b
  const int lb = level[b];
  const unsigned long long kp = key[p];
  const int f = fid[b];
  int cnt = 0;
  if (kp != ~0ull && lb >= 0 && lb <= kMaxBlockLevel) {
    bool ok = true;
    if (p == fstart[f]) {
      ok = ok && kp == 0ull;
    } else {
      const int lprev = level[idx[p - 1]];
      const unsigned long long kprev = key[p - 1];
      ok = ok && kprev != ~0ull && lprev >= 0 && lprev <= kMaxBlockLevel &&
           kprev + key_span(lprev) == kp;
    }
    if (p == fstart[f + 1] - 1) ok = ok && kp + key_span(lb) == (1ull << 63);
    if (!ok) atomicOr(flags, kErrTiling);
    cnt = max(0, lb - top_start_level(kp));
  }
  count[p] = cnt;
  blk[p] = make_int4(lb, ijk[3 * b], ijk[3 * b + 1], ijk[3 * b + 2]);
  orig[p] = b;
}

// prestart[p] = 585 p + sum_{q<p} count[q]: pre-order index of the first node
// that belongs to block p (its first top node, else its root).  One CTA.
constexpr int kScanThreads = 1024;
__global__ void __launch_bounds__(kScanThreads)
    k_prestart_scan(int nb, const int *__restrict__ count, int *__restrict__ prestart,
                    unsigned *flags) {
  __shared__ int part[kScanThreads];
  const int t = threadIdx.x;
  const int per = (nb + kScanThreads - 1) / kScanThreads;
  const int beg = min(t * per, nb), end = min(beg + per, nb);
  int s = 0;
  for (int i = beg; i < end; ++i) s += count[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {
    const int v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int i = beg; i < end; ++i) {
    prestart[i] = kNodesPerBlock * i + run;
    run += count[i];
  }
  if (t == kScanThreads - 1) flags[2] = (unsigned)part[t];
}

__device__ __forceinline__ float pow2f(int e) {  // 2^e for -126 <= e <= 127, exact
  return __int_as_float((127 + e) << 23);
}
__device__ __forceinline__ double pow2d(int e) {  // 2^e for -1022 <= e <= 1023, exact
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// Also records, per block, its field's node range: fld[p] = {first node of
// the field (its root), one past its last node, first block of the next
// field, field index}.
__global__ void k_top_nodes(int nb, const unsigned long long *__restrict__ key,
                            const int4 *__restrict__ blk, const int *__restrict__ count,
                            const int *__restrict__ prestart, int64_t n_nodes,
                            WalkRec *__restrict__ rec, float2 *__restrict__ aux,
                            uint8_t *__restrict__ lvl, unsigned *flags, int nfields,
                            const int *__restrict__ fstart, const int *__restrict__ fid,
                            const int *__restrict__ orig, int4 *__restrict__ fld) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  const int f = fid[orig[p]];
  const int fend = fstart[f + 1];
  const int64_t node_end = fend < nb ? (int64_t)prestart[fend] : n_nodes;
  fld[p] = make_int4(prestart[fstart[f]], (int)node_end, fend, f);
  const int cnt = count[p];
  if (cnt == 0) return;
  const int lb = blk[p].x;
  const int j0 = lb - cnt;
  const unsigned long long kp = key[p];
  for (int k = j0; k < lb; ++k) {
    const int64_t id = (int64_t)prestart[p] + (k - j0);
    // first block whose key lies beyond this cube: its first node follows the subtree
    const unsigned long long lim = kp + (1ull << (3 * (kKeyLevels - k)));
    int a = p + 1, e = fend;
    while (a < e) {
      const int m = (a + e) >> 1;
      if (key[m] < lim) a = m + 1; else e = m;
    }
    const int64_t skip = a < fend ? (int64_t)prestart[a] : node_end;
    if (id < 0 || id >= n_nodes || skip > n_nodes) {
      atomicOr(flags, kErrIndex);
      continue;
    }
    rec[id].skip = (unsigned)skip;
    aux[id] = make_float2(pow2f(-k), 0.0f);
    lvl[id] = (uint8_t)k;
  }
}

// Child lists of the top nodes, for the moment pass: entry 8 slot + o holds
// the pre-order index of child o of the top node with compact index
// slot = prestart[p] - 585 p + r (the r-th top node that starts at block p,
// level k = j0 + r; prestart[p] - 585 p counts the top nodes before p).
// Child o's cube starts at key kp + o 8^(21-k-1), so its first block q is
// found by one binary search, and the child is q's top node of level k + 1
// or, if q is a block of level k + 1, q's root.  One thread per (top node,
// octant), all independent: the moment pass then reads its children
// directly instead of chasing skip pointers one after another.
__global__ void k_top_children(int nb, const unsigned long long *__restrict__ key,
                               const int4 *__restrict__ blk, const int *__restrict__ count,
                               const int *__restrict__ prestart, int64_t n_nodes,
                               const int *__restrict__ fstart, const int *__restrict__ fid,
                               const int *__restrict__ orig, int *__restrict__ child,
                               int64_t child_slots, unsigned *flags) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nb * 8) return;
  const int p = (int)(tid >> 3), o = (int)(tid & 7);
  const int r = blockIdx.y;
  const int cnt = count[p];
  if (r >= cnt) return;
  const int lb = blk[p].x, k = lb - cnt + r;
  const int fend = fstart[fid[orig[p]] + 1];
  const int64_t slot = (int64_t)prestart[p] - (int64_t)kNodesPerBlock * p + r;
  if (k < 0 || k >= kKeyLevels || slot < 0 || slot >= child_slots) {
    atomicOr(flags, kErrIndex);
    return;
  }
  const unsigned long long start = key[p] + (unsigned long long)o * key_span(k + 1);
  int q = p;
  if (o > 0) {
    int a = p + 1, e = fend;
    while (a < e) {
      const int m = (a + e) >> 1;
      if (key[m] < start) a = m + 1; else e = m;
    }
    q = a;
  }
  if (q >= fend || key[q] != start) {  // a complete tiling starts every cube with a block
    atomicOr(flags, kErrIndex);
    return;
  }
  const int lq = blk[q].x, cq = count[q];
  int64_t idx = -1;
  if (k + 1 < lq && k + 1 >= lq - cq) idx = (int64_t)prestart[q] + (k + 1 - (lq - cq));
  else if (k + 1 == lq) idx = (int64_t)prestart[q] + cq;
  if (idx <= 0 || idx >= n_nodes) {
    atomicOr(flags, kErrIndex);
    return;
  }
  child[8 * slot + o] = (int)idx;
}

// Moments of one internal node from its 8 children (Eq. 5), children in
// octant order, every operation rounded once.  c = geometric centre.
struct Moment {
  double x, y, z, m, delta;
  double ox, oy, oz;  // R - geometric centre
};
__device__ __forceinline__ void accumulate(double &M, double &Sx, double &Sy, double &Sz,
                                           double m, double x, double y, double z) {
  M = __dadd_rn(M, m);
  Sx = __dadd_rn(Sx, __dmul_rn(m, x));
  Sy = __dadd_rn(Sy, __dmul_rn(m, y));
  Sz = __dadd_rn(Sz, __dmul_rn(m, z));
}
__device__ __forceinline__ Moment finish(double M, double Sx, double Sy, double Sz, double cx,
                                         double cy, double cz) {
  Moment r;
  r.m = M;
  if (M > 0.0) {
    r.x = __ddiv_rn(Sx, M);
    r.y = __ddiv_rn(Sy, M);
    r.z = __ddiv_rn(Sz, M);
  } else {  // a massless node sits at its geometric centre
    r.x = cx;
    r.y = cy;
    r.z = cz;
  }
  const double ox = __dsub_rn(r.x, cx), oy = __dsub_rn(r.y, cy), oz = __dsub_rn(r.z, cz);
  r.delta = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ox, ox), __dmul_rn(oy, oy)), __dmul_rn(oz, oz)));
  r.ox = ox;
  r.oy = oy;
  r.oz = oz;
  return r;
}

// (i + 1/2) 2^-level, the centre coordinate of cube i at `level` in box units:
// 2i + 1 < 2^22 and level <= 21, so it is formed exactly in binary32 and
// widened (the same value as the FP64 expression, without FP64 operations).
__device__ __forceinline__ float centre_coord_f(int i, int level) {
  return __fmul_rn((float)(2 * i + 1), pow2f(-(level + 1)));
}
__device__ __forceinline__ double centre_coord(int i, int level) {
  return (double)centre_coord_f(i, level);
}

__device__ __forceinline__ WalkRec make_rec(double x, double y, double z, double m,
                                            int64_t skip) {
  WalkRec w;
  w.px = __double2float_rn(x);
  w.py = __double2float_rn(y);
  w.pz = __double2float_rn(z);
  w.m = __double2float_rn(m);
  w.s2 = 0.0f;
  w.skip = (unsigned)skip;
  w.pad[0] = w.pad[1] = 0.0f;
  return w;
}

// inv_unit = 2^-e of the field's binary32 mass unit (the record's mass).
// inv_theta > 0: also the squared opening radius s2 = fl(fl(l fl(1/theta)) +
// delta)^2 from the same binary32 l and delta as k_prepare_s2 (identical).
// Returns the record's binary32 mass (in the field's unit).
__device__ __forceinline__ float store_internal(int64_t id, int64_t skip, int level,
                                                const Moment &r, double4_32a *mom, WalkRec *rec,
                                                float2 *aux, uint8_t *lvl, double inv_unit,
                                                float inv_theta) {
  mom[id] = make_double4_32a(r.x, r.y, r.z, r.m);
  WalkRec w = make_rec(r.x, r.y, r.z, r.m * inv_unit, skip);
  const float l = pow2f(-level), delta = __double2float_rn(r.delta);
  if (inv_theta > 0.0f) {
    const float s = __fadd_rn(__fmul_rn(l, inv_theta), delta);
    w.s2 = __fmul_rn(s, s);
  }
  rec[id] = w;
  aux[id] = make_float2(l, delta);
  if (lvl) lvl[id] = (uint8_t)level;
  return w.m;
}

// Quadrupole about the parent's centre of mass (parallel-axis rule): the
// child's own quadrupole plus m (3 s s^T - |s|^2 I), s = child COM - parent
// COM.  Order: xx, yy, zz, xy, xz, yz.  Cells have none.
__device__ __forceinline__ void add_shifted(double Q[6], const double *Qc, double m, double sx,
                                            double sy, double sz) {
  const double s2 = sx * sx + sy * sy + sz * sz;
  Q[0] += m * (3.0 * sx * sx - s2);
  Q[1] += m * (3.0 * sy * sy - s2);
  Q[2] += m * (3.0 * sz * sz - s2);
  Q[3] += m * (3.0 * sx * sy);
  Q[4] += m * (3.0 * sx * sz);
  Q[5] += m * (3.0 * sy * sz);
  if (Qc)
    for (int a = 0; a < 6; ++a) Q[a] += Qc[a];
}

// Binary32 version, used when the walk is binary32: the quadrupole term is a
// small correction rounded to binary32 anyway, and GB300 runs FP64 far slower
// than FP32.  fm is the child's mass in the field's binary32 mass unit; the
// shift s is formed in FP64 (a difference of nearby centres of mass) and
// then rounded (top nodes), or inside a block from binary32 offsets (below).
__device__ __forceinline__ void add_shifted_f(float Q[6], const float *Qc, float fm, double sx,
                                              double sy, double sz) {
  const float x = __double2float_rn(sx), y = __double2float_rn(sy), z = __double2float_rn(sz);
  const float s2 = x * x + y * y + z * z;
  Q[0] += fm * (3.0f * x * x - s2);
  Q[1] += fm * (3.0f * y * y - s2);
  Q[2] += fm * (3.0f * z * z - s2);
  Q[3] += fm * (3.0f * x * y);
  Q[4] += fm * (3.0f * x * z);
  Q[5] += fm * (3.0f * y * z);
  if (Qc)
    for (int a = 0; a < 6; ++a) Q[a] += Qc[a];
}

// The same with the shift given in binary32.  Inside a block it is formed as
// s = (c_child - c_parent) + (o_child - o_parent), o = R - c the binary32
// offsets of the centres of mass from the geometric centres c: c_child -
// c_parent is +-l/4 (exact) and every term is of the node's size, so s
// carries an absolute error of a few 2^-24 l -- the quadrupole, a sum of
// m s s^T terms against M l^2, keeps about 2^-22 relative accuracy -- and
// needs no FP64 operation (GB300 issues FP64 at a small fraction of FP32).
__device__ __forceinline__ void add_shifted_ff(float Q[6], const float *Qc, float fm, float x,
                                               float y, float z) {
  const float s2 = x * x + y * y + z * z;
  Q[0] += fm * (3.0f * x * x - s2);
  Q[1] += fm * (3.0f * y * y - s2);
  Q[2] += fm * (3.0f * z * z - s2);
  Q[3] += fm * (3.0f * x * y);
  Q[4] += fm * (3.0f * x * z);
  Q[5] += fm * (3.0f * y * z);
  if (Qc)
    for (int a = 0; a < 6; ++a) Q[a] += Qc[a];
}

__device__ __forceinline__ void store_quad_f(int64_t id, const float Q[6], WalkQuad *qrec) {
  WalkQuad w;
  w.hxx = 0.5f * Q[0];
  w.hyy = 0.5f * Q[1];
  w.hzz = 0.5f * Q[2];
  w.qxy = Q[3];
  w.qxz = Q[4];
  w.qyz = Q[5];
  w.pad[0] = w.pad[1] = 0.0f;
  qrec[id] = w;
}

// The quadrupole of a node back from its binary32 walk record.
__device__ __forceinline__ void load_quad_f(const WalkQuad &w, float Q[6]) {
  Q[0] = 2.0f * w.hxx;
  Q[1] = 2.0f * w.hyy;
  Q[2] = 2.0f * w.hzz;
  Q[3] = w.qxy;
  Q[4] = w.qxz;
  Q[5] = w.qyz;
}

// FP64 quadrupole (physical) and its binary32 walk record {Qxx/2, Qyy/2,
// Qzz/2, Qxy, Qxz, Qyz} in the field's mass unit (inv_unit = 2^-e):
// the halves fold the 1/2 of the quadrupole term.
__device__ __forceinline__ void store_quad(int64_t id, const double Q[6], double *q64,
                                           WalkQuad *qrec, double inv_unit) {
  for (int a = 0; a < 6; ++a) q64[6 * id + a] = Q[a];
  const double u = inv_unit;
  WalkQuad w;
  w.hxx = __double2float_rn(0.5 * Q[0] * u);
  w.hyy = __double2float_rn(0.5 * Q[1] * u);
  w.hzz = __double2float_rn(0.5 * Q[2] * u);
  w.qxy = __double2float_rn(Q[3] * u);
  w.qxz = __double2float_rn(Q[4] * u);
  w.qyz = __double2float_rn(Q[5] * u);
  w.pad[0] = w.pad[1] = 0.0f;
  qrec[id] = w;
}

constexpr int kBlockThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kBlockThreads)
    k_blocks(int nb, const int4 *__restrict__ blk, const int *__restrict__ orig,
             const int *__restrict__ count, const int *__restrict__ prestart,
             const T *__restrict__ density, const double *__restrict__ Lf,
             const int *__restrict__ fid, const unsigned long long *__restrict__ mmax,
             float inv_theta, int64_t n_nodes,
             double4_32a *__restrict__ mom, WalkRec *__restrict__ rec, float2 *__restrict__ aux,
             uint8_t *__restrict__ lvl, double *__restrict__ q64, WalkQuad *__restrict__ qrec,
             unsigned *flags) {
  __shared__ double cm[512], cxs[512], cys[512], czs[512];  // cells, local Morton order
  __shared__ float cmu[512];                                // cell mass, binary32 unit
  const bool quad64 = q64 != nullptr;                       // FP64 quadrupoles
  const bool quad32 = !quad64 && qrec != nullptr;           // binary32 quadrupoles
  const int p = blockIdx.x;
  const int t = threadIdx.x;
  const int4 B = blk[p];
  const int lb = B.x;
  if (lb < 0 || lb > kMaxBlockLevel) return;  // flagged earlier
  const int64_t root = (int64_t)prestart[p] + count[p];
  if (root < 0 || root + kNodesPerBlock > n_nodes) {
    if (t == 0) atomicOr(flags, kErrIndex);
    return;
  }
  const int lc = lb + 3;
  const int field = fid[orig[p]];
  const double L = Lf[field];                  // box side of this block's field
  const double inv_unit = pow2i(-mass_exponent(mmax[field]));  // binary32 mass unit
  const double hs = pow2d(-lc);               // cell side, box units
  const double h = __dmul_rn(L, hs);          // cell side, physical
  const double vol = __dmul_rn(__dmul_rn(h, h), h);
  const T *rho = density + (int64_t)orig[p] * kCellsPerBlock;
  bool bad = false;
  for (int i = t; i < kCellsPerBlock; i += kBlockThreads) {
    const T rv = rho[i];
    if (!(rv >= T(0)) || isinf(rv)) bad = true;  // checked in the input's precision
    const double r = (double)rv;
    const int cx = i & 7, cy = (i >> 3) & 7, cz = i >> 6;
    const int m = (int)(spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2));
    const float fx = centre_coord_f(8 * B.y + cx, lc);
    const float fy = centre_coord_f(8 * B.z + cy, lc);
    const float fz = centre_coord_f(8 * B.w + cz, lc);
    const double ux = fx, uy = fy, uz = fz;
    const double mass = __dmul_rn(r, vol);
    const float mu = __double2float_rn(mass * inv_unit);
    cm[m] = mass;
    cmu[m] = mu;
    cxs[m] = ux;
    cys[m] = uy;
    czs[m] = uz;
    const int64_t id = root + cell_offset(m);
    mom[id] = make_double4_32a(ux, uy, uz, mass);
    WalkRec w;  // make_rec without the conversions: the centre is a binary32 value
    w.px = fx;
    w.py = fy;
    w.pz = fz;
    w.m = mu;
    w.s2 = 0.0f;
    w.skip = (unsigned)(id + 1);
    w.pad[0] = w.pad[1] = 0.0f;
    rec[id] = w;
    aux[id] = make_float2(0.0f, 0.0f);
    lvl[id] = (uint8_t)lc;
  }
  if (bad) atomicOr(flags, kErrDensity);
  __syncthreads();
  if (t < 64) {  // nodes at level lb+2: q = 8p + r, children = cells 8q..8q+7
    const int q = t;
    const int qx = (int)compact3(q), qy = (int)compact3(q >> 1), qz = (int)compact3(q >> 2);
    const double cx = centre_coord(4 * B.y + qx, lb + 2);
    const double cy = centre_coord(4 * B.z + qy, lb + 2);
    const double cz = centre_coord(4 * B.w + qz, lb + 2);
    double M = 0.0, Sx = 0.0, Sy = 0.0, Sz = 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o)
      accumulate(M, Sx, Sy, Sz, cm[8 * q + o], cxs[8 * q + o], cys[8 * q + o], czs[8 * q + o]);
    const Moment r = finish(M, Sx, Sy, Sz, cx, cy, cz);
    const int64_t id = root + 2 + 73 * (q >> 3) + 9 * (q & 7);
    store_internal(id, id + 9, lb + 2, r, mom, rec, aux, lvl, inv_unit, inv_theta);
    if (quad64) {
      double Q[6] = {0, 0, 0, 0, 0, 0};
      for (int o = 0; o < 8; ++o) {
        const int k = 8 * q + o;
        add_shifted(Q, nullptr, cm[k], cxs[k] - r.x, cys[k] - r.y, czs[k] - r.z);
      }
      store_quad(id, Q, q64, qrec, inv_unit);
    } else if (quad32) {
      // children: cells at c +- h/2 (h = 2^-(lb+3)) with o = 0
      const float ox = __double2float_rn(r.ox), oy = __double2float_rn(r.oy),
                  oz = __double2float_rn(r.oz);
      const float hc = pow2f(-(lb + 4));
      float Q[6] = {0, 0, 0, 0, 0, 0};
      for (int o = 0; o < 8; ++o) {
        const float dx = (o & 1) ? hc : -hc, dy = (o & 2) ? hc : -hc, dz = (o & 4) ? hc : -hc;
        add_shifted_ff(Q, nullptr, cmu[8 * q + o], __fsub_rn(dx, ox), __fsub_rn(dy, oy),
                       __fsub_rn(dz, oz));
      }
      store_quad_f(id, Q, qrec);
    }
  }
}

// The 8 nodes at level lb+1 of every block (STAGE 1) or every block's root
// (STAGE 0), one node per thread over all blocks, so that the FP64 work runs
// in full warps (in one CTA per block these levels kept 8 and 1 lanes of a
// warp busy at the cost of a whole warp).  Their children -- written by
// k_blocks (stage 1) or by stage 1 (stage 0) -- are read back from the node
// arrays; the arithmetic is that of k_blocks (Eq. 5 in octant order; the
// binary32 quadrupole shift from the children's binary32 centre-of-mass
// offsets), so the results are the same bit for bit.
template <int STAGE>
__global__ void __launch_bounds__(256)
    k_block_upper(int nb, const int4 *__restrict__ blk, const int *__restrict__ orig,
                  const int *__restrict__ count, const int *__restrict__ prestart,
                  const int *__restrict__ fid, const unsigned long long *__restrict__ mmax,
                  float inv_theta, int64_t n_nodes, double4_32a *__restrict__ mom,
                  WalkRec *__restrict__ rec, float2 *__restrict__ aux, uint8_t *__restrict__ lvl,
                  double *__restrict__ q64, WalkQuad *__restrict__ qrec) {
  constexpr int kPer = STAGE ? 8 : 1;  // nodes of this level per block
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nb * kPer) return;
  const int p = (int)(i / kPer), c = (int)(i % kPer);
  const int4 B = blk[p];
  const int lb = B.x;
  if (lb < 0 || lb > kMaxBlockLevel) return;  // flagged by k_block_keys
  const int64_t root = (int64_t)prestart[p] + count[p];
  if (root < 0 || root + kNodesPerBlock > n_nodes) return;  // flagged by k_blocks
  const double inv_unit = pow2i(-mass_exponent(mmax[fid[orig[p]]]));
  const int lev = STAGE ? lb + 1 : lb;
  const int ix = STAGE ? 2 * B.y + (c & 1) : B.y;
  const int iy = STAGE ? 2 * B.z + ((c >> 1) & 1) : B.z;
  const int iz = STAGE ? 2 * B.w + ((c >> 2) & 1) : B.w;
  const int64_t id = STAGE ? root + 1 + 73 * c : root;
  const int64_t skip = STAGE ? id + 73 : root + kNodesPerBlock;
  const int64_t first = id + 1, stride = STAGE ? 9 : 73;  // child o at first + stride o
  const double cx = centre_coord(ix, lev), cy = centre_coord(iy, lev), cz = centre_coord(iz, lev);
  double M = 0.0, Sx = 0.0, Sy = 0.0, Sz = 0.0;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const double4_32a ch = mom[first + stride * o];
    accumulate(M, Sx, Sy, Sz, ch.w, ch.x, ch.y, ch.z);
  }
  const Moment r = finish(M, Sx, Sy, Sz, cx, cy, cz);
  store_internal(id, skip, lev, r, mom, rec, aux, lvl, inv_unit, inv_theta);
  if (q64) {
    double Q[6] = {0, 0, 0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
      const int64_t k = first + stride * o;
      const double4_32a ch = mom[k];
      add_shifted(Q, q64 + 6 * k, ch.w, ch.x - r.x, ch.y - r.y, ch.z - r.z);
    }
    store_quad(id, Q, q64, qrec, inv_unit);
  } else if (qrec) {
    const float ox = __double2float_rn(r.ox), oy = __double2float_rn(r.oy),
                oz = __double2float_rn(r.oz);
    const float hc = pow2f(-(lev + 2));  // child centre - centre: +-2^-(lev+2)
    float Q[6] = {0, 0, 0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
      const int64_t k = first + stride * o;
      const double4_32a ch = mom[k];
      // the child's binary32 offset R - c from its own centre, as k_blocks formed it
      const float gx = __double2float_rn(__dsub_rn(ch.x, centre_coord(2 * ix + (o & 1), lev + 1)));
      const float gy =
          __double2float_rn(__dsub_rn(ch.y, centre_coord(2 * iy + ((o >> 1) & 1), lev + 1)));
      const float gz =
          __double2float_rn(__dsub_rn(ch.z, centre_coord(2 * iz + ((o >> 2) & 1), lev + 1)));
      float Qc[6];
      load_quad_f(qrec[k], Qc);
      const float dx = (o & 1) ? hc : -hc, dy = (o & 2) ? hc : -hc, dz = (o & 4) ? hc : -hc;
      add_shifted_ff(Q, Qc, rec[k].m, __fsub_rn(__fadd_rn(dx, gx), ox),
                     __fsub_rn(__fadd_rn(dy, gy), oy), __fsub_rn(__fadd_rn(dz, gz), oz));
    }
    store_quad_f(id, Q, qrec);
  }
}

// The top node of sorted block p at `level` (the block starts cnt = count[p]
// top nodes, levels lb - cnt .. lb - 1): its children are top nodes one level
// down or block roots, read from its child list (k_top_children).
__device__ __forceinline__ void top_moment(int p, int level, const unsigned long long *key,
                                           const int4 *blk, const int *count,
                                           const int *prestart, int64_t n_nodes,
                                           double4_32a *mom, WalkRec *rec, float2 *aux,
                                           double *q64, WalkQuad *qrec, unsigned *flags,
                                           const int4 *fld, const unsigned long long *mmax,
                                           float inv_theta, const int *__restrict__ child_list,
                                           int64_t child_slots) {
  const int cnt = count[p];
  const int lb = blk[p].x;
  const int j0 = lb - cnt;
  const int64_t id = (int64_t)prestart[p] + (level - j0);
  const unsigned long long kp = key[p];
  const int sh = kKeyLevels - level;
  const double cx = centre_coord((int)(compact3(kp) >> sh), level);
  const double cy = centre_coord((int)(compact3(kp >> 1) >> sh), level);
  const double cz = centre_coord((int)(compact3(kp >> 2) >> sh), level);
  double M = 0.0, Sx = 0.0, Sy = 0.0, Sz = 0.0;
  const int64_t slot = id - (int64_t)kNodesPerBlock * p;
  if (slot < 0 || slot >= child_slots) {
    atomicOr(flags, kErrIndex);
    return;
  }
  int64_t child[8];  // from the child list, kept for the quadrupoles
  for (int o = 0; o < 8; ++o) {
    const int64_t c = child_list[8 * slot + o];
    if (c <= 0 || c >= n_nodes) {
      atomicOr(flags, kErrIndex);
      return;
    }
    child[o] = c;
  }
  for (int o = 0; o < 8; ++o) {
    const double4_32a ch = mom[child[o]];
    accumulate(M, Sx, Sy, Sz, ch.w, ch.x, ch.y, ch.z);
  }
  const Moment r = finish(M, Sx, Sy, Sz, cx, cy, cz);
  const int64_t skip = rec[id].skip;
  const double inv_unit = pow2i(-mass_exponent(mmax[fld[p].w]));
  store_internal(id, skip, level, r, mom, rec, aux, nullptr, inv_unit, inv_theta);
  if (q64) {
    double Q[6] = {0, 0, 0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
      const double4_32a ch = mom[child[o]];
      add_shifted(Q, q64 + 6 * child[o], ch.w, ch.x - r.x, ch.y - r.y, ch.z - r.z);
    }
    store_quad(id, Q, q64, qrec, inv_unit);
  } else if (qrec) {
    float Q[6] = {0, 0, 0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
      const double4_32a ch = mom[child[o]];
      float Qc[6];
      load_quad_f(qrec[child[o]], Qc);
      add_shifted_f(Q, Qc, __double2float_rn(ch.w * inv_unit), ch.x - r.x, ch.y - r.y,
                    ch.z - r.z);
    }
    store_quad_f(id, Q, qrec);
  }
}

// One launch per level (any number of top nodes).
__global__ void k_top_moments(int nb, int level, const unsigned long long *__restrict__ key,
                              const int4 *__restrict__ blk, const int *__restrict__ count,
                              const int *__restrict__ prestart, int64_t n_nodes,
                              double4_32a *__restrict__ mom, WalkRec *__restrict__ rec,
                              float2 *__restrict__ aux, double *__restrict__ q64,
                              WalkQuad *__restrict__ qrec, unsigned *flags,
                              const int4 *__restrict__ fld,
                              const unsigned long long *__restrict__ mmax, float inv_theta,
                              const int *__restrict__ child_list, int64_t child_slots) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  const int cnt = count[p];
  const int lb = blk[p].x;
  if (cnt == 0 || level < lb - cnt || level >= lb) return;
  top_moment(p, level, key, blk, count, prestart, n_nodes, mom, rec, aux, q64, qrec, flags, fld,
             mmax, inv_theta, child_list, child_slots);
}

// Largest cell mass m = rho h^3 of each field (FP64, rounded as in k_blocks),
// as an atomic max on its bits (a non-negative double orders like its bits).
// One CTA per caller block; invalid levels and densities are skipped here
// and reported by the other kernels.
template <typename T>
__global__ void __launch_bounds__(kBlockThreads)
    k_mass_max(int nb, const int *__restrict__ level, const T *__restrict__ density,
               const double *__restrict__ Lf, const int *__restrict__ fid,
               unsigned long long *__restrict__ mmax) {
  const int b = blockIdx.x;
  const int lb = level[b];
  if (lb < 0 || lb > kMaxBlockLevel) return;
  const int field = fid[b];
  const double h = __dmul_rn(Lf[field], pow2d(-(lb + 3)));
  const double vol = __dmul_rn(__dmul_rn(h, h), h);
  const T *rho = density + (int64_t)b * kCellsPerBlock;
  T mx = 0;  // the largest density, in its own precision (max is exact)
  for (int i = threadIdx.x; i < kCellsPerBlock; i += kBlockThreads) {
    const T r = rho[i];
    if (r >= T(0) && !isinf(r)) mx = r > mx ? r : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const T v = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = v > mx ? v : mx;
  }
  __shared__ T warp_max[kBlockThreads / 32];
  if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {  // one atomic per block, and only when it can raise the max
    for (int w = 1; w < kBlockThreads / 32; ++w) mx = warp_max[w] > mx ? warp_max[w] : mx;
    if (mx > T(0)) {
      const unsigned long long bits =
          (unsigned long long)__double_as_longlong(__dmul_rn((double)mx, vol));
      if (bits > *(volatile unsigned long long *)(mmax + field)) atomicMax(mmax + field, bits);
    }
  }
}

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_block_keys(cudaStream_t s, int nb, const int *level, const int *ijk,
                              unsigned long long *key, int *idx, unsigned *flags,
                              const FieldArgs &fa) {
  k_block_keys<<<grid_for(nb, 256), 256, 0, s>>>(nb, level, ijk, key, idx, flags, fa.nfields,
                                                  fa.fstart, fa.fid);
  return cudaGetLastError();
}

cudaError_t launch_sort_blocks(cudaStream_t s, unsigned long long *key[2], int *idx[2],
                               unsigned *flags, const FieldArgs &fa) {
  k_sort_blocks<<<fa.nfields, kSortThreads, 0, s>>>(fa.fstart, key[0], idx[0], key[1], idx[1],
                                                     flags);
  return cudaGetLastError();
}

cudaError_t launch_tile_and_count(cudaStream_t s, int nb, const unsigned long long *key,
                                  const int *idx, const int *level, const int *ijk, int *count,
                                  int4 *blk, int *orig, unsigned *flags, const FieldArgs &fa,
                                  int *pos) {
  k_tile_and_count<<<grid_for(nb, 256), 256, 0, s>>>(nb, key, idx, level, ijk, count, blk, orig,
                                                      flags, fa.fstart, fa.fid, pos);
  return cudaGetLastError();
}

cudaError_t launch_prestart_scan(cudaStream_t s, int nb, const int *count, int *prestart,
                                 unsigned *flags) {
  k_prestart_scan<<<1, kScanThreads, 0, s>>>(nb, count, prestart, flags);
  return cudaGetLastError();
}

cudaError_t launch_top_nodes(cudaStream_t s, int nb, const unsigned long long *key,
                             const int4 *blk, const int *count, const int *prestart,
                             int64_t n_nodes, WalkRec *rec, float2 *aux, uint8_t *lvl,
                             unsigned *flags, const FieldArgs &fa, const int *orig,
                             int max_level, int *child, int64_t child_slots) {
  k_top_nodes<<<grid_for(nb, 256), 256, 0, s>>>(nb, key, blk, count, prestart, n_nodes, rec,
                                                 aux, lvl, flags, fa.nfields, fa.fstart, fa.fid,
                                                 orig, fa.fld);
  if (max_level > 0) {  // a block starts at most max_level top nodes
    const dim3 grid((unsigned)grid_for((int64_t)nb * 8, 256), (unsigned)max_level);
    k_top_children<<<grid, 256, 0, s>>>(nb, key, blk, count, prestart, n_nodes, fa.fstart,
                                         fa.fid, orig, child, child_slots, flags);
  }
  return cudaGetLastError();
}

cudaError_t launch_blocks(cudaStream_t s, int nb, const int4 *blk, const int *orig,
                          const int *count, const int *prestart, const void *density,
                          int density_is_fp64, const FieldArgs &fa, int64_t n_nodes,
                          double4_32a *mom, WalkRec *rec, float2 *aux, uint8_t *lvl, double *q64,
                          WalkQuad *qrec, unsigned *flags) {
  if (density_is_fp64)
    k_blocks<double><<<nb, kBlockThreads, 0, s>>>(nb, blk, orig, count, prestart,
                                                   (const double *)density, fa.L, fa.fid,
                                                   fa.mmax, fa.inv_theta, n_nodes, mom, rec, aux,
                                                   lvl, q64, qrec, flags);
  else
    k_blocks<float><<<nb, kBlockThreads, 0, s>>>(nb, blk, orig, count, prestart,
                                                  (const float *)density, fa.L, fa.fid, fa.mmax,
                                                  fa.inv_theta, n_nodes, mom, rec, aux, lvl, q64,
                                                  qrec, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_block_upper<1><<<grid_for((int64_t)nb * 8, 256), 256, 0, s>>>(
      nb, blk, orig, count, prestart, fa.fid, fa.mmax, fa.inv_theta, n_nodes, mom, rec, aux, lvl,
      q64, qrec);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_block_upper<0><<<grid_for(nb, 256), 256, 0, s>>>(
      nb, blk, orig, count, prestart, fa.fid, fa.mmax, fa.inv_theta, n_nodes, mom, rec, aux, lvl,
      q64, qrec);
  return cudaGetLastError();
}

cudaError_t launch_mass_max(cudaStream_t s, int nb, const int *level, const void *density,
                            int density_is_fp64, const FieldArgs &fa) {
  if (density_is_fp64)
    k_mass_max<double><<<nb, kBlockThreads, 0, s>>>(nb, level, (const double *)density, fa.L,
                                                     fa.fid, fa.mmax);
  else
    k_mass_max<float><<<nb, kBlockThreads, 0, s>>>(nb, level, (const float *)density, fa.L,
                                                    fa.fid, fa.mmax);
  return cudaGetLastError();
}

cudaError_t launch_top_tree(cudaStream_t s, int nb, int max_level, int64_t n_top,
                            const unsigned long long *key, const int4 *blk, const int *count,
                            const int *prestart, int64_t n_nodes, double4_32a *mom, WalkRec *rec,
                            float2 *aux, double *q64, WalkQuad *qrec, unsigned *flags,
                            const FieldArgs &fa, const int *child, int64_t child_slots) {
  if (n_top <= 0) return cudaSuccess;
  for (int lev = max_level - 1; lev >= 0; --lev) {
    const cudaError_t e = launch_top_moments(s, nb, lev, key, blk, count, prestart, n_nodes, mom,
                                             rec, aux, q64, qrec, flags, fa, child, child_slots);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_top_moments(cudaStream_t s, int nb, int level, const unsigned long long *key,
                               const int4 *blk, const int *count, const int *prestart,
                               int64_t n_nodes, double4_32a *mom, WalkRec *rec, float2 *aux,
                               double *q64, WalkQuad *qrec, unsigned *flags, const FieldArgs &fa,
                               const int *child, int64_t child_slots) {
  k_top_moments<<<grid_for(nb, 256), 256, 0, s>>>(nb, level, key, blk, count, prestart,
                                                   n_nodes, mom, rec, aux, q64, qrec, flags,
                                                   fa.fld, fa.mmax, fa.inv_theta, child,
                                                   child_slots);
  return cudaGetLastError();
}

}  // namespace bhg
