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
//      lattice (k_keys_mass, which also finds each field's largest cell
//      mass, the binary32 mass unit) and blocks are put in key order
//      (k_sort_blocks, only if the caller's order is not already sorted);
//   2. consecutive keys must abut exactly (k_tile_and_count): this checks that
//      the blocks tile the box, and the trailing zero bits of a block's key
//      tell how many internal "top" nodes (cubes above the blocks) start at it
//      in pre-order;
//   3. an exclusive scan gives every block the pre-order index of its first
//      node (k_prestart_scan), from which top nodes get their skip pointers
//      (k_top_nodes) and their child lists (k_top_children: one binary
//      search per top node and octant, all in parallel);
//   4. one CTA per block reduces its 512 cells to its 64 bottom nodes in
//      shared memory (k_blocks); one more launch (k_upper_tree) does the
//      rest: the 8 level-one nodes and the root of every block, in full
//      warps, then the top tree, which it climbs by arrival counts -- the
//      thread that finishes the last of a node's 8 children computes the
//      node and climbs on, so no thread waits and no launch per level is
//      needed.  (Measured before: one launch per top level, each reading its
//      nodes from child lists, cost 12-18 us a level, mostly launch and
//      latency for a few hundred nodes; the paper's version has threads
//      wait on children still marked by a negative mass.)
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

// Morton key of caller block b (field f) and its field index; notes in
// flags[1] whether the caller's order differs from the key order (compared
// with block b+1 of the same field).
__device__ __forceinline__ void key_of_block(int b, int f, const int *__restrict__ level,
                                             const int *__restrict__ ijk,
                                             unsigned long long *__restrict__ key,
                                             int *__restrict__ idx, unsigned *flags,
                                             const int *__restrict__ fstart,
                                             int *__restrict__ fid) {
  fid[b] = f;
  const int lb = level[b];
  const int i = ijk[3 * b], j = ijk[3 * b + 1], k = ijk[3 * b + 2];
  unsigned long long kb = ~0ull;
  if (valid_block(lb, i, j, k, flags)) kb = block_key(lb, i, j, k);
  key[b] = kb;
  idx[b] = b;
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
                                 const int *__restrict__ fid, int *__restrict__ pos,
                                 int *__restrict__ bparent) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nb) return;
  const int b = idx[p];
  if (pos) pos[b] = p;  // sorted position of caller block b
  bparent[p] = -1;      // a field's only block has no parent; k_top_children sets the rest
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

// binary64 <-> binary32 conversions of the moment kernels.  (Measured: a
// general bit-level version on the integer pipes -- 64-bit integer
// arithmetic is several instructions a step -- made k_blocks 7 % and the
// level-one nodes 75 % slower than the conversion instructions.)
__device__ __forceinline__ double widen(float f) { return (double)f; }
// A positive normal binary32 value as binary64 (exact): the exponent rebased
// from 127 to 1023 and the 23 fraction bits moved up by 29, three 32-bit
// integer operations instead of a conversion on GB300's narrow FP64 pipe.
// Used for cube centres, (2i + 1) 2^-(level + 1) > 0.
__device__ __forceinline__ double widen_pos(float f) {
  const unsigned b = __float_as_uint(f);
  return __hiloint2double((int)((b >> 3) + ((1023u - 127u) << 20)), (int)(b << 29));
}
// fl32(x 2^k), 2^k a power of two that scales x exactly.  For a normal x
// whose scaled value stays normal the product is x with k added to its
// exponent (an integer add on the high word); zeros and the rest take the
// FP64 multiplication.
__device__ __forceinline__ float narrow_scaled(double x, int k) {
  const int hi = __double2hiint(x);
  const int E = (hi >> 20) & 0x7ff;
  if (E > 0 && E + k > 0 && E + k < 0x7ff)
    return __double2float_rn(__hiloint2double(hi + (k << 20), __double2loint(x)));
  return __double2float_rn(x * pow2d(k));
}
__device__ __forceinline__ float narrow(double x) { return __double2float_rn(x); }
__device__ __forceinline__ double as_f64(float v) { return widen(v); }
__device__ __forceinline__ double as_f64(double v) { return v; }

// Also records, per block, its field's node range: fld[p] = {first node of
// the field (its root), one past its last node, first block of the next
// field, field index}.
__global__ void k_top_nodes(int nb, const unsigned long long *__restrict__ key,
                            const int4 *__restrict__ blk, const int *__restrict__ count,
                            const int *__restrict__ prestart, int64_t n_nodes,
                            WalkRec *__restrict__ rec, float2 *__restrict__ aux,
                            uint8_t *__restrict__ lvl, unsigned *flags, int nfields,
                            const int *__restrict__ fstart, const int *__restrict__ fid,
                            const int *__restrict__ orig, int4 *__restrict__ fld,
                            TopArgs top) {
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
    const int64_t slot = id - (int64_t)kNodesPerBlock * p;
    if (id < 0 || id >= n_nodes || skip > n_nodes || slot < 0 || slot >= top.slots) {
      atomicOr(flags, kErrIndex);
      continue;
    }
    rec[id].skip = (unsigned)skip;
    aux[id] = make_float2(pow2f(-k), 0.0f);
    lvl[id] = (uint8_t)k;
    const int sh = kKeyLevels - k;
    top.slot[2 * slot] = make_int4((int)id, (int)skip, (int)(compact3(kp) >> sh),
                                   (int)(compact3(kp >> 1) >> sh));
    top.slot[2 * slot + 1] = make_int4((int)(compact3(kp >> 2) >> sh), k, f, p);
    top.parent[slot] = -1;  // a field's root; k_top_children sets the others
    top.arrive[slot] = 0u;
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
// directly instead of chasing skip pointers one after another.  Also records
// each child's parent slot (TopArgs::parent, TopArgs::bparent), by which the
// moment pass climbs the top tree.
__global__ void k_top_children(int nb, const unsigned long long *__restrict__ key,
                               const int4 *__restrict__ blk, const int *__restrict__ count,
                               const int *__restrict__ prestart, int64_t n_nodes,
                               const int *__restrict__ fstart, const int *__restrict__ fid,
                               const int *__restrict__ orig, TopArgs top, unsigned *flags) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nb * 8) return;
  const int p = (int)(tid >> 3), o = (int)(tid & 7);
  const int r = blockIdx.y;
  const int cnt = count[p];
  if (r >= cnt) return;
  const int lb = blk[p].x, k = lb - cnt + r;
  const int fend = fstart[fid[orig[p]] + 1];
  const int64_t slot = (int64_t)prestart[p] - (int64_t)kNodesPerBlock * p + r;
  if (k < 0 || k >= kKeyLevels || slot < 0 || slot >= top.slots) {
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
  top.child[8 * slot + o] = (int)idx;
  if (k + 1 < lq) {  // a top node: its slot
    const int64_t cs = idx - (int64_t)kNodesPerBlock * q;
    if (cs < 0 || cs >= top.slots) {
      atomicOr(flags, kErrIndex);
      return;
    }
    top.parent[cs] = (int)slot;
  } else {  // block q's root
    top.bparent[q] = (int)slot;
  }
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
// The first term of the sums: 0 + m = m and 0 + fl(m x) = fl(m x) (masses and
// box coordinates are >= 0), so the sums start from it.
__device__ __forceinline__ void accumulate_first(double &M, double &Sx, double &Sy, double &Sz,
                                                 double m, double x, double y, double z) {
  M = m;
  Sx = __dmul_rn(m, x);
  Sy = __dmul_rn(m, y);
  Sz = __dmul_rn(m, z);
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
  return widen_pos(centre_coord_f(i, level));
}

// ku: the exponent of the field's inverse binary32 mass unit (the record's
// mass is fl(m 2^ku)).
__device__ __forceinline__ WalkRec make_rec(double x, double y, double z, double m, int ku,
                                            int64_t skip) {
  WalkRec w;
  w.px = narrow(x);
  w.py = narrow(y);
  w.pz = narrow(z);
  w.m = narrow_scaled(m, ku);
  w.s2 = 0.0f;
  w.skip = (unsigned)skip;
  w.pad[0] = w.pad[1] = 0.0f;
  return w;
}

// ku = -e for the field's binary32 mass unit 2^e (the record's mass).
// inv_theta > 0: also the squared opening radius s2 = fl(fl(l fl(1/theta)) +
// delta)^2 from the same binary32 l and delta as k_prepare_s2 (identical).
// Returns the record's binary32 mass (in the field's unit).
// keep_off: also keep the binary32 offset R - c of the centre of mass from
// the geometric centre, x and y in the record's two spare words (z goes
// into the quadrupole record's, store_quad_f), for the parent's quadrupole
// shift.
__device__ __forceinline__ float store_internal(int64_t id, int64_t skip, int level,
                                                const Moment &r, double4_32a *mom, WalkRec *rec,
                                                float2 *aux, uint8_t *lvl, int ku,
                                                float inv_theta, bool keep_off = false) {
  mom[id] = make_double4_32a(r.x, r.y, r.z, r.m);
  WalkRec w = make_rec(r.x, r.y, r.z, r.m, ku, skip);
  if (keep_off) {
    w.pad[0] = narrow(r.ox);
    w.pad[1] = narrow(r.oy);
  }
  const float l = pow2f(-level), delta = narrow(r.delta);
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
  const float x = narrow(sx), y = narrow(sy), z = narrow(sz);
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

// oz: the node's binary32 offset R_z - c_z (see store_internal), or 0.
__device__ __forceinline__ void store_quad_f(int64_t id, const float Q[6], WalkQuad *qrec,
                                             float oz = 0.0f) {
  WalkQuad w;
  w.hxx = 0.5f * Q[0];
  w.hyy = 0.5f * Q[1];
  w.hzz = 0.5f * Q[2];
  w.qxy = Q[3];
  w.qxz = Q[4];
  w.qyz = Q[5];
  w.pad[0] = oz;
  w.pad[1] = 0.0f;
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
  const int ku = -mass_exponent(mmax[field]);  // binary32 mass unit 2^-ku
  const double inv_unit = pow2i(ku);
  const double hs = pow2d(-lc);               // cell side, box units
  const double h = __dmul_rn(L, hs);          // cell side, physical
  const double vol = __dmul_rn(__dmul_rn(h, h), h);
  const T *rho = density + (int64_t)orig[p] * kCellsPerBlock;
  bool bad = false;
  for (int i = t; i < kCellsPerBlock; i += kBlockThreads) {
    const T rv = rho[i];
    if (!(rv >= T(0)) || isinf(rv)) bad = true;  // checked in the input's precision
    const double r = as_f64(rv);
    const int cx = i & 7, cy = (i >> 3) & 7, cz = i >> 6;
    const int m = (int)(spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2));
    const float fx = centre_coord_f(8 * B.y + cx, lc);
    const float fy = centre_coord_f(8 * B.z + cy, lc);
    const float fz = centre_coord_f(8 * B.w + cz, lc);
    const double ux = widen_pos(fx), uy = widen_pos(fy), uz = widen_pos(fz);
    const double mass = __dmul_rn(r, vol);
    const float mu = narrow_scaled(mass, ku);
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
  // nodes at level lb+2: q = 8p + r, children = cells 8q..8q+7; warps 0-1
  // on even CTAs, 2-3 on odd ones, so that this FP64 work of the CTAs on an
  // SM is spread over its four schedulers
  if ((t >> 6) == (p & 1)) {
    const int q = t & 63;
    const int qx = (int)compact3(q), qy = (int)compact3(q >> 1), qz = (int)compact3(q >> 2);
    const double cx = centre_coord(4 * B.y + qx, lb + 2);
    const double cy = centre_coord(4 * B.z + qy, lb + 2);
    const double cz = centre_coord(4 * B.w + qz, lb + 2);
    double M, Sx, Sy, Sz;
    accumulate_first(M, Sx, Sy, Sz, cm[8 * q], cxs[8 * q], cys[8 * q], czs[8 * q]);
#pragma unroll
    for (int o = 1; o < 8; ++o)
      accumulate(M, Sx, Sy, Sz, cm[8 * q + o], cxs[8 * q + o], cys[8 * q + o], czs[8 * q + o]);
    const Moment r = finish(M, Sx, Sy, Sz, cx, cy, cz);
    const int64_t id = root + 2 + 73 * (q >> 3) + 9 * (q & 7);
    store_internal(id, id + 9, lb + 2, r, mom, rec, aux, lvl, ku, inv_theta, quad32);
    if (quad64) {
      double Q[6] = {0, 0, 0, 0, 0, 0};
      for (int o = 0; o < 8; ++o) {
        const int k = 8 * q + o;
        add_shifted(Q, nullptr, cm[k], cxs[k] - r.x, cys[k] - r.y, czs[k] - r.z);
      }
      store_quad(id, Q, q64, qrec, inv_unit);
    } else if (quad32) {
      // children: cells at c +- h/2 (h = 2^-(lb+3)) with o = 0
      const float ox = narrow(r.ox), oy = narrow(r.oy), oz = narrow(r.oz);
      const float hc = pow2f(-(lb + 4));
      float Q[6] = {0, 0, 0, 0, 0, 0};
      for (int o = 0; o < 8; ++o) {
        const float dx = (o & 1) ? hc : -hc, dy = (o & 2) ? hc : -hc, dz = (o & 4) ? hc : -hc;
        add_shifted_ff(Q, nullptr, cmu[8 * q + o], __fsub_rn(dx, ox), __fsub_rn(dy, oy),
                       __fsub_rn(dz, oz));
      }
      store_quad_f(id, Q, qrec, oz);
    }
  }
}

// Loads of node data written by other CTAs of the same launch: through L2
// (ld.global.cg), after the arrival count has said that the writers are done.
__device__ __forceinline__ double4_32a ld_mom_cg(const double4_32a *p) {
  const double2 a = __ldcg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldcg(reinterpret_cast<const double2 *>(p) + 1);
  return make_double4_32a(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ WalkQuad ld_quad_cg(const WalkQuad *p) {
  const float4 a = __ldcg(reinterpret_cast<const float4 *>(p));
  const float2 b = __ldcg(reinterpret_cast<const float2 *>(p) + 2);
  WalkQuad w;
  w.hxx = a.x;
  w.hyy = a.y;
  w.hzz = a.z;
  w.qxy = a.w;
  w.qxz = b.x;
  w.qyz = b.y;
  w.pad[0] = w.pad[1] = 0.0f;
  return w;
}

// A level-one node of a block (level lev = lb + 1) from its 8 children, the
// bottom nodes at first + 9 o, one thread per node.  Eq. 5 in octant order;
// the binary32 quadrupole shift from the children's binary32 centre-of-mass
// offsets, as k_blocks forms it.
__device__ __forceinline__ void level_one_node(int lev, int ix, int iy, int iz, int64_t id,
                                               int64_t skip, int64_t first, int ku,
                                               double inv_unit, float inv_theta,
                                               double4_32a *mom, WalkRec *rec, float2 *aux,
                                               uint8_t *lvl, double *q64, WalkQuad *qrec) {
  constexpr int64_t stride = 9;
  const double cx = centre_coord(ix, lev), cy = centre_coord(iy, lev), cz = centre_coord(iz, lev);
  double4_32a ch[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) ch[o] = mom[first + stride * o];
  double M, Sx, Sy, Sz;
  accumulate_first(M, Sx, Sy, Sz, ch[0].w, ch[0].x, ch[0].y, ch[0].z);
#pragma unroll
  for (int o = 1; o < 8; ++o) accumulate(M, Sx, Sy, Sz, ch[o].w, ch[o].x, ch[o].y, ch[o].z);
  const Moment r = finish(M, Sx, Sy, Sz, cx, cy, cz);
  const bool quad32 = qrec && !q64;
  store_internal(id, skip, lev, r, mom, rec, aux, lvl, ku, inv_theta, quad32);
  if (q64) {
    double Q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int64_t k = first + stride * o;
      add_shifted(Q, q64 + 6 * k, ch[o].w, ch[o].x - r.x, ch[o].y - r.y, ch[o].z - r.z);
    }
    store_quad(id, Q, q64, qrec, inv_unit);
  } else if (qrec) {
    const float ox = narrow(r.ox), oy = narrow(r.oy), oz = narrow(r.oz);
    const float hc = pow2f(-(lev + 2));  // child centre - centre: +-2^-(lev+2)
    float Q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int64_t k = first + stride * o;
      // the child's binary32 offset R - c from its own centre, as k_blocks
      // formed it (narrow(R - c) in FP64) and kept in its spare words
      const WalkRec cr = rec[k];
      const WalkQuad cq = qrec[k];
      float Qc[6];
      load_quad_f(cq, Qc);
      const float dx = (o & 1) ? hc : -hc, dy = (o & 2) ? hc : -hc, dz = (o & 4) ? hc : -hc;
      add_shifted_ff(Q, Qc, cr.m, __fsub_rn(__fadd_rn(dx, cr.pad[0]), ox),
                     __fsub_rn(__fadd_rn(dy, cr.pad[1]), oy),
                     __fsub_rn(__fadd_rn(dz, cq.pad[0]), oz));
    }
    store_quad_f(id, Q, qrec, oz);
  }
}

// One node computed by a group of 8 lanes of a warp (lanes gbase..gbase+7,
// mask gmask); lane o of the group brings child o (node index `child`).  A
// lone thread spends about 90 clocks on each dependent FP64 instruction here,
// so the node's FP64 work is spread over the group: the four sums of Eq. 5
// on lanes k = o & 3 (k = 0: M, as fl(m 1) = m; 1-3: the x, y, z moments),
// each in octant order; the divisions by M on lanes 1-3; the FP64
// differences of the quadrupole shifts on all eight.  The binary32
// quadrupole sum then runs on every lane from the shuffled terms in octant
// order.  Every value is the one the one-thread form computes, bit for bit.
// ROOT: a block's root (children: its level-one nodes; shift from their
// binary32 offsets, as inside a block; ix, iy, iz its cube); else a top
// node (children from its list; shift = the FP64 difference of the centres
// of mass, rounded).  CG: read the children through L2.
template <bool ROOT, bool CG>
__device__ __forceinline__ void group_node(unsigned gmask, int gbase, int o, int lev, int ix,
                                           int iy, int iz, double cx, double cy, double cz,
                                           int64_t id, int64_t skip, int64_t child, int ku,
                                           double inv_unit, float inv_theta, double4_32a *mom,
                                           WalkRec *rec, float2 *aux, uint8_t *lvl, double *q64,
                                           WalkQuad *qrec) {
  const double4_32a c = CG ? ld_mom_cg(mom + child) : mom[child];
  WalkQuad qc = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, {0.0f, 0.0f}};
  float fm = 0.0f, gx = 0.0f, gy = 0.0f;
  if (qrec && !q64) {  // issued with the moments, used after the FP64 part
    qc = CG ? ld_quad_cg(qrec + child) : qrec[child];
    fm = CG ? __ldcg(&rec[child].m) : rec[child].m;
    if (ROOT) {  // a level-one child's binary32 offset R - c (level_one_node kept it)
      gx = rec[child].pad[0];
      gy = rec[child].pad[1];
    }
  }
  const int k = o & 3;
  double S = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const double mj = __shfl_sync(gmask, c.w, gbase + j);
    const double xj = __shfl_sync(gmask, c.x, gbase + j);
    const double yj = __shfl_sync(gmask, c.y, gbase + j);
    const double zj = __shfl_sync(gmask, c.z, gbase + j);
    const double t = __dmul_rn(mj, k == 0 ? 1.0 : (k == 1 ? xj : (k == 2 ? yj : zj)));
    S = j == 0 ? t : __dadd_rn(S, t);
  }
  const double M = __shfl_sync(gmask, S, gbase);
  const double cc = k == 1 ? cx : (k == 2 ? cy : cz);
  const double R = M > 0.0 ? __ddiv_rn(S, M) : cc;  // a massless node sits at its centre
  const double off = __dsub_rn(R, cc);
  const double sq = __dmul_rn(off, off);
  Moment r;
  r.m = M;
  r.x = __shfl_sync(gmask, R, gbase + 1);
  r.y = __shfl_sync(gmask, R, gbase + 2);
  r.z = __shfl_sync(gmask, R, gbase + 3);
  r.ox = __shfl_sync(gmask, off, gbase + 1);
  r.oy = __shfl_sync(gmask, off, gbase + 2);
  r.oz = __shfl_sync(gmask, off, gbase + 3);
  r.delta = __dsqrt_rn(__dadd_rn(__dadd_rn(__shfl_sync(gmask, sq, gbase + 1),
                                           __shfl_sync(gmask, sq, gbase + 2)),
                                 __shfl_sync(gmask, sq, gbase + 3)));
  if (o == 0) store_internal(id, skip, lev, r, mom, rec, aux, lvl, ku, inv_theta);
  if (q64) {  // FP64 quadrupoles (the FP64 walk): on lane 0, as the one-thread form
    int64_t kids[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) kids[j] = __shfl_sync(gmask, child, gbase + j);
    if (o == 0) {
      double Q[6] = {0, 0, 0, 0, 0, 0};
      for (int j = 0; j < 8; ++j) {
        const int64_t kj = kids[j];
        const double4_32a cj = CG ? ld_mom_cg(mom + kj) : mom[kj];
        double Qc[6];
        for (int a = 0; a < 6; ++a) Qc[a] = CG ? __ldcg(q64 + 6 * kj + a) : q64[6 * kj + a];
        add_shifted(Q, Qc, cj.w, cj.x - r.x, cj.y - r.y, cj.z - r.z);
      }
      store_quad(id, Q, q64, qrec, inv_unit);
    }
    return;
  }
  if (!qrec) return;
  float sx, sy, sz;  // this lane's child: its shift from the node's centre of mass
  if (ROOT) {
    const float hc = pow2f(-(lev + 2));
    const float gz = qc.pad[0];
    const float dx = (o & 1) ? hc : -hc, dy = (o & 2) ? hc : -hc, dz = (o & 4) ? hc : -hc;
    sx = __fsub_rn(__fadd_rn(dx, gx), narrow(r.ox));
    sy = __fsub_rn(__fadd_rn(dy, gy), narrow(r.oy));
    sz = __fsub_rn(__fadd_rn(dz, gz), narrow(r.oz));
  } else {
    sx = narrow(c.x - r.x);
    sy = narrow(c.y - r.y);
    sz = narrow(c.z - r.z);
  }
  float Q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const WalkQuad qj = {__shfl_sync(gmask, qc.hxx, gbase + j), __shfl_sync(gmask, qc.hyy, gbase + j),
                         __shfl_sync(gmask, qc.hzz, gbase + j), __shfl_sync(gmask, qc.qxy, gbase + j),
                         __shfl_sync(gmask, qc.qxz, gbase + j), __shfl_sync(gmask, qc.qyz, gbase + j),
                         {0.0f, 0.0f}};
    float Qc[6];
    load_quad_f(qj, Qc);
    add_shifted_ff(Q, Qc, __shfl_sync(gmask, fm, gbase + j), __shfl_sync(gmask, sx, gbase + j),
                   __shfl_sync(gmask, sy, gbase + j), __shfl_sync(gmask, sz, gbase + j));
  }
  if (o == 0) store_quad_f(id, Q, qrec);
}

// The top node whose slot holds {a, b} (made by k_top_nodes: node, skip, cube,
// level, field) and whose child o is c, by a group of 8 lanes; its
// children -- top nodes one level down or block roots -- were written by
// other CTAs and are read through L2.  ku: the field's mass-unit exponent.
// False when the slot is inconsistent (a failed geometry).
__device__ __forceinline__ bool top_node(unsigned gmask, int gbase, int o, int4 a, int4 b,
                                         int64_t c, int ku, int nb, int nfields,
                                         int64_t n_nodes, double4_32a *mom, WalkRec *rec,
                                         float2 *aux, double *q64, WalkQuad *qrec,
                                         float inv_theta) {
  const int level = b.y;
  if (a.x < 0 || a.x >= n_nodes || level < 0 || level >= kKeyLevels || b.z < 0 ||
      b.z >= nfields || b.w < 0 || b.w >= nb)
    return false;
  if (__any_sync(gmask, c <= 0 || c >= n_nodes)) return false;
  group_node<false, true>(gmask, gbase, o, level, 0, 0, 0, centre_coord(a.z, level),
                          centre_coord(a.w, level), centre_coord(b.x, level), a.x, a.y, c, ku,
                          pow2i(ku), inv_theta, mom, rec, aux, nullptr, q64, qrec);
  return true;
}

// Everything above the 64 bottom nodes of the blocks, in one launch.  A CTA
// takes kUpperBlocks sorted blocks: (1) their 8 level-one nodes, one per
// thread, so that the FP64 work runs in full warps; (2) after a CTA barrier,
// their roots, one per group of 8 lanes; (3) the top tree, climbed without
// waiting: a group that has finished a node adds one to its parent's
// arrival count, and the group that brings it to 8 computes the parent (the
// other seven are done) and climbs on; the rest stop.  No thread ever waits
// for another, the count is put back to 0 by the group that used it, and
// the results do not depend on which group computes a node: every node is
// the same function of its children in octant order, as in the paper's
// bottom-up pass (Sec. 3.2.3, there with threads that wait on their
// children).
constexpr int kUpperBlocks = 16;
__global__ void __launch_bounds__(8 * kUpperBlocks)
    k_upper_tree(int nb, int nfields, const int4 *__restrict__ blk, const int *__restrict__ orig,
                 const int *__restrict__ count, const int *__restrict__ prestart,
                 const int *__restrict__ fid, const unsigned long long *__restrict__ mmax,
                 float inv_theta, int64_t n_nodes, double4_32a *mom, WalkRec *rec, float2 *aux,
                 uint8_t *lvl, double *q64, WalkQuad *qrec, unsigned *flags, TopArgs top) {
  const int p0 = blockIdx.x * kUpperBlocks;
  const int t = threadIdx.x;
  {  // (1) level-one nodes: block p0 + t/8, octant t%8
    const int p = p0 + t / 8, c = t % 8;
    if (p < nb) {
      const int4 B = blk[p];
      const int lb = B.x;
      const int64_t root = (int64_t)prestart[p] + count[p];
      if (lb >= 0 && lb <= kMaxBlockLevel && root >= 0 && root + kNodesPerBlock <= n_nodes) {
        const int ku = -mass_exponent(mmax[fid[orig[p]]]);
        const int64_t id = root + 1 + 73 * c;
        level_one_node(lb + 1, 2 * B.y + (c & 1), 2 * B.z + ((c >> 1) & 1),
                       2 * B.w + ((c >> 2) & 1), id, id + 73, id + 1, ku, pow2i(ku), inv_theta,
                       mom, rec, aux, lvl, q64, qrec);
      }
    }
  }
  __syncthreads();
  // (2) roots: block p0 + t/8 by the group of lanes t & ~7
  const int o = t & 7, gbase = t & 24;
  const unsigned gmask = 0xFFu << gbase;
  const int p = p0 + t / 8;
  if (p >= nb) return;
  const int4 B = blk[p];
  const int lb = B.x;
  const int64_t root = (int64_t)prestart[p] + count[p];
  if (lb < 0 || lb > kMaxBlockLevel || root < 0 || root + kNodesPerBlock > n_nodes) return;
  const int ku = -mass_exponent(mmax[fid[orig[p]]]);
  group_node<true, false>(gmask, gbase, o, lb, B.y, B.z, B.w, centre_coord(B.y, lb),
                          centre_coord(B.z, lb), centre_coord(B.w, lb), root,
                          root + kNodesPerBlock, root + 1 + 73 * o, ku, pow2i(ku), inv_theta, mom,
                          rec, aux, lvl, q64, qrec);
  // (3) climb: the parent top node of this root, then its parents
  int s = top.bparent[p];
  while (s >= 0) {
    if (s >= top.slots) {  // a failed geometry
      if (o == 0) atomicOr(flags, kErrIndex);
      return;
    }
    // what the parent's computation needs from earlier launches, read before
    // the arrival so that only its children's moments remain after it
    const int4 a = top.slot[2 * (int64_t)s], b = top.slot[2 * (int64_t)s + 1];
    const int64_t c = top.child[8 * (int64_t)s + o];
    const int up = top.parent[s];
    const int kuf = b.z >= 0 && b.z < nfields ? -mass_exponent(mmax[b.z]) : 0;
    unsigned before = 0u;
    if (o == 0) {
      __threadfence();  // this node's moments (lane 0 wrote them) before the arrival
      before = atomicAdd(top.arrive + s, 1u);
    }
    before = __shfl_sync(gmask, before, gbase);
    if (before != 7u) {
      if (before > 7u && o == 0) atomicOr(flags, kErrIndex);
      return;
    }
    __threadfence();  // the other children's moments after their arrivals
    if (o == 0) top.arrive[s] = 0u;
    if (!top_node(gmask, gbase, o, a, b, c, kuf, nb, nfields, n_nodes, mom, rec, aux, q64, qrec,
                  inv_theta)) {
      if (o == 0) atomicOr(flags, kErrIndex);
      return;
    }
    s = up;
  }
}

// Largest cell mass m = rho h^3 of each field (FP64, rounded as in k_blocks),
// as an atomic max on its bits (a non-negative double orders like its bits):
// the part of caller block b (level lb, field f), by all threads of a CTA.
// Invalid densities (negative, NaN, infinite) are skipped and flagged here,
// in the build's first kernel, so that the host can report them before the
// moments are done (k_blocks flags them too).
template <typename T>
__device__ __forceinline__ void block_mass_max(int b, int field, int lb,
                                               const T *__restrict__ density,
                                               const double *__restrict__ Lf,
                                               unsigned long long *__restrict__ mmax,
                                               unsigned *flags) {
  const T *rho = density + (int64_t)b * kCellsPerBlock;
  T mx = 0;  // the largest density, in its own precision (max is exact)
  bool bad = false;
  for (int i = threadIdx.x; i < kCellsPerBlock; i += kBlockThreads) {
    const T r = rho[i];
    if (r >= T(0) && !isinf(r)) mx = r > mx ? r : mx;
    else bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kErrDensity);
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
      const double h = __dmul_rn(Lf[field], pow2d(-(lb + 3)));
      const double vol = __dmul_rn(__dmul_rn(h, h), h);
      const unsigned long long bits =
          (unsigned long long)__double_as_longlong(__dmul_rn(as_f64(mx), vol));
      if (bits > *(volatile unsigned long long *)(mmax + field)) atomicMax(mmax + field, bits);
    }
  }
}

// The largest cell mass alone (a new density on the same tree).  One CTA per
// caller block.
template <typename T>
__global__ void __launch_bounds__(kBlockThreads)
    k_mass_max(int nb, const int *__restrict__ level, const T *__restrict__ density,
               const double *__restrict__ Lf, const int *__restrict__ fid,
               unsigned long long *__restrict__ mmax, unsigned *flags) {
  const int b = blockIdx.x;
  const int lb = level[b];
  if (lb < 0 || lb > kMaxBlockLevel) return;
  block_mass_max(b, fid[b], lb, density, Lf, mmax, flags);
}

// The build's first kernel: block keys and the largest cell mass together,
// one CTA per caller block (thread 0 forms the key).
template <typename T>
__global__ void __launch_bounds__(kBlockThreads)
    k_keys_mass(int nb, const int *__restrict__ level, const int *__restrict__ ijk,
                unsigned long long *__restrict__ key, int *__restrict__ idx, unsigned *flags,
                int nfields, const int *__restrict__ fstart, int *__restrict__ fid,
                const T *__restrict__ density, const double *__restrict__ Lf,
                unsigned long long *__restrict__ mmax) {
  const int b = blockIdx.x;
  const int f = field_of(b, nfields, fstart);
  if (threadIdx.x == 0) key_of_block(b, f, level, ijk, key, idx, flags, fstart, fid);
  const int lb = level[b];
  if (lb < 0 || lb > kMaxBlockLevel) return;
  block_mass_max(b, f, lb, density, Lf, mmax, flags);
}

inline int grid_for(int64_t n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_keys_mass(cudaStream_t s, int nb, const int *level, const int *ijk,
                             unsigned long long *key, int *idx, unsigned *flags,
                             const FieldArgs &fa, const void *density, int density_is_fp64) {
  if (density_is_fp64)
    k_keys_mass<double><<<nb, kBlockThreads, 0, s>>>(nb, level, ijk, key, idx, flags, fa.nfields,
                                                      fa.fstart, fa.fid, (const double *)density,
                                                      fa.L, fa.mmax);
  else
    k_keys_mass<float><<<nb, kBlockThreads, 0, s>>>(nb, level, ijk, key, idx, flags, fa.nfields,
                                                     fa.fstart, fa.fid, (const float *)density,
                                                     fa.L, fa.mmax);
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
                                  const TopArgs &top, int *pos) {
  k_tile_and_count<<<grid_for(nb, 256), 256, 0, s>>>(nb, key, idx, level, ijk, count, blk, orig,
                                                      flags, fa.fstart, fa.fid, pos, top.bparent);
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
                             int max_level, const TopArgs &top) {
  k_top_nodes<<<grid_for(nb, 256), 256, 0, s>>>(nb, key, blk, count, prestart, n_nodes, rec,
                                                 aux, lvl, flags, fa.nfields, fa.fstart, fa.fid,
                                                 orig, fa.fld, top);
  if (max_level > 0) {  // a block starts at most max_level top nodes
    const dim3 grid((unsigned)grid_for((int64_t)nb * 8, 256), (unsigned)max_level);
    k_top_children<<<grid, 256, 0, s>>>(nb, key, blk, count, prestart, n_nodes, fa.fstart,
                                         fa.fid, orig, top, flags);
  }
  return cudaGetLastError();
}

cudaError_t launch_mass_max(cudaStream_t s, int nb, const int *level, const void *density,
                            int density_is_fp64, const FieldArgs &fa, unsigned *flags) {
  if (density_is_fp64)
    k_mass_max<double><<<nb, kBlockThreads, 0, s>>>(nb, level, (const double *)density, fa.L,
                                                     fa.fid, fa.mmax, flags);
  else
    k_mass_max<float><<<nb, kBlockThreads, 0, s>>>(nb, level, (const float *)density, fa.L,
                                                    fa.fid, fa.mmax, flags);
  return cudaGetLastError();
}

cudaError_t launch_moments(cudaStream_t s, int nb, const int4 *blk, const int *orig,
                           const int *count, const int *prestart, const void *density, int density_is_fp64, const FieldArgs &fa,
                           int64_t n_nodes, double4_32a *mom, WalkRec *rec, float2 *aux,
                           uint8_t *lvl, double *q64, WalkQuad *qrec, unsigned *flags,
                           const TopArgs &top, cudaEvent_t before_upper) {
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
  if (before_upper && (e = cudaStreamWaitEvent(s, before_upper, 0)) != cudaSuccess) return e;
  k_upper_tree<<<grid_for(nb, kUpperBlocks), 8 * kUpperBlocks, 0, s>>>(
      nb, fa.nfields, blk, orig, count, prestart, fa.fid, fa.mmax, fa.inv_theta, n_nodes, mom,
      rec, aux, lvl, q64, qrec, flags, top);
  return cudaGetLastError();
}

}  // namespace bhg
