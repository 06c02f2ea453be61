// Internal declarations shared by the translation units of libbhgrav.
//
// Node storage (all arrays indexed by the node's pre-order position: a
// depth-first visit of the octree in octant order o = ox + 2 oy + 4 oz, so a
// node's first child sits right after it and its subtree is contiguous):
//   mom  double4 {Rx, Ry, Rz, M}  FP64 centre of mass (box units) and mass
//   rec  WalkRec (32 bytes)       what the walk reads, 24 bytes in a 128-bit
//                                 and a 64-bit load: the centre of mass and
//                                 mass rounded to binary32, the mass in its
//                                 field's binary32 mass unit (below), the
//                                 squared opening radius s2 for the current
//                                 theta (0 for cells), and the index of the
//                                 first node after the subtree; 8 bytes of
//                                 padding keep records 32-byte aligned
//   aux  float2  {l, delta}       node side and |R - centre| in binary32
//                                 (both 0 for cells)
//   lvl  uint8                    node level
// Leaf blocks are renumbered in Morton order of their lower corner ("sorted
// position" p); blk[p] = {level, bi, bj, bk}, orig[p] = caller block index.
//
// Binary32 mass unit.  Binary32 records (walk and quadrupole records) hold
// masses divided by 2^e_f, with e_f = (binary exponent of the largest cell
// mass of field f) - 40, so that the largest cell mass lies in [2^40, 2^41)
// whatever the physical units (cgs included).  Then, with at most 2^24 cells
// per field and distances down to 2^-21 of the box, no binary32 sum exceeds
// ~2^86, and the quadrupole term of the deepest nodes (cells of 2^-21 of the
// box, d^T Q d / 2 ~ m l^2 d^2 ~ 2^-88 for a cell 1e-12 as heavy as the
// heaviest one) stays far above the binary32 underflow (2^-126).  Scaling by
// a power of two is exact, so the binary32 walk computes the same numbers as
// with unscaled masses wherever those were in range; it multiplies its sum
// back by 2^e_f.  FP64 moments (mom, q64) stay physical.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <limits>
#include <vector>

#include "bhgrav.h"  // -I include

namespace bhg {

constexpr int kCellsPerBlock = 512;
constexpr int kNodesPerBlock = 585;  // 1 + 8 + 64 + 512
constexpr int kMaxBlockLevel = 18;   // cells at level <= 21: 63-bit Morton keys
constexpr int kKeyLevels = 21;

// Error bits raised by device-side validation.
enum : unsigned {
  kErrLevel = 1u,        // level outside [0, 18]
  kErrCoord = 2u,        // coordinate outside [0, 2^level)
  kErrTiling = 4u,       // sorted blocks leave a gap or overlap
  kErrDensity = 8u,      // negative or non-finite density
  kErrIndex = 16u,       // a node index fell outside the allocation
  kErrTimeout = 32u,     // a bounded wait for the tensor core gave up
};

// Every warp lane needs every field of the record it walks through, so each
// load is delivered to all 32 lanes: only the six fields the walk uses are
// read (24 bytes; the L1 returns a warp's data 128 bytes per cycle).
struct __align__(32) WalkRec {
  float px, py, pz;  // centre of mass, box units
  float m;           // mass in the field's binary32 unit
  float s2;          // (l/theta + delta)^2 in binary32; 0 for cells
  unsigned skip;     // first node after this node's subtree
  float pad[2];
};
static_assert(sizeof(WalkRec) == 32, "walk record must be 32 bytes");

// Quadrupole walk record (quadrupole or learned option), box units and the
// field's binary32 mass unit: half the diagonal of Q and the off-diagonal
// terms (read as 24 bytes, like WalkRec), so that
//   d^T Q d / 2 = dx (Qxx/2 dx + Qxy dy + Qxz dz) + dy (Qyy/2 dy + Qyz dz)
//                 + Qzz/2 dz^2.
struct __align__(32) WalkQuad {
  float hxx, hyy, hzz, qxy;
  float qxz, qyz;
  float pad[2];
};
static_assert(sizeof(WalkQuad) == 32, "quadrupole record must be 32 bytes");

// Launch shape of the per-cell binary32 walk: warps per CTA, x-neighbour
// target pairs per lane (a warp's group of targets: 1 pair = a 4x4x4 octant,
// 2 pairs = a 8x4x4 slab), and the schedule: ticket = 0 a plain grid of one
// warp per group; ticket = k > 0 a persistent grid (as many CTAs as fit on
// the GPU at once) whose warps take k groups at a time from `counter` (a
// device word that the launch resets) until all are taken.  0 = defaults.
// longest = 1: the groups are walked in the tree's walk order (longest walk
// first, made by bh_autotune); order: that permutation of the groups (group
// order[i] is the i-th to be walked: taken i-th from the counter, or walked
// by warp i of a plain grid), or null for the groups' own order.  cycles
// (persistent grid only, else null): receives the SM clock cycles each
// group's walk took, per group.
struct WalkShape {
  int warps = 0;
  int pairs = 0;
  int ticket = 0;
  int longest = 0;
  unsigned *counter = nullptr;
  const unsigned *order = nullptr;
  unsigned long long *cycles = nullptr;
};

// Top nodes (the cubes above the blocks), by slot = their rank among the
// top nodes in pre-order, made once per geometry by k_top_nodes and
// k_top_children for the moment pass, which climbs the top tree by arrival
// counts.  All in one allocation of top_ints(nb_cap) ints.
struct TopArgs {
  int *child = nullptr;         // 8 per slot: pre-order index of child o
  int4 *slot = nullptr;         // 2 per slot: {node, skip, cube x, cube y},
                                //             {cube z, level, field, sorted block}
  int *parent = nullptr;        // per slot: parent slot, -1 for a field's root
  unsigned *arrive = nullptr;   // per slot: children done in this pass (0 between passes)
  int *bparent = nullptr;       // per sorted block: the slot of its root's parent, or -1
  int64_t slots = 0;            // capacity in slots
};
// Top nodes number (nb_f - 1)/7 per field, so fewer than nb/4 in all.
constexpr int64_t top_slots(int64_t nb_cap) { return nb_cap / 4; }
constexpr int64_t top_ints(int64_t nb_cap) { return 18 * top_slots(nb_cap) + nb_cap; }
inline TopArgs top_args(int *base, int64_t nb_cap) {
  TopArgs a;
  const int64_t S = top_slots(nb_cap);
  a.child = base;
  a.slot = reinterpret_cast<int4 *>(base + 8 * S);
  a.parent = base + 16 * S;
  a.arrive = reinterpret_cast<unsigned *>(base + 17 * S);
  a.bparent = base + 18 * S;
  a.slots = S;
  return a;
}

struct Tree {
  // block arrays (capacity nb_cap)
  int *d_level = nullptr, *d_ijk = nullptr;
  unsigned long long *d_key[2] = {nullptr, nullptr};
  int *d_idx[2] = {nullptr, nullptr};
  int *d_count = nullptr, *d_prestart = nullptr;
  int4 *d_blk = nullptr;
  int *d_orig = nullptr;
  int *d_pos = nullptr;         // sorted position of each caller block
  int *d_top = nullptr;         // top-node lists (TopArgs, top_ints(nb_cap) ints)
  unsigned *d_flags = nullptr;  // [0] error bits, [1] unsorted flag, [2] top-node total,
                                // [4] work counter of the persistent walk (8 entries)
  unsigned *h_flags = nullptr;  // pinned mirror of d_flags
  // fields
  int nfields = 0;
  int *d_fstart = nullptr;      // nfields + 1
  int *d_fid = nullptr;         // per caller block
  int4 *d_fld = nullptr;        // per sorted block
  double *d_invL = nullptr;     // per field
  double *d_L = nullptr;        // per field
  unsigned long long *d_mmax = nullptr;  // per field, largest cell mass (bits)
  int nf_cap = 0;
  // d_mmax, d_L, d_invL, d_fstart, d_level and d_ijk live in d_geo, which a
  // build fills from its pinned mirror h_geo in one copy (geo_done: that copy)
  unsigned char *d_geo = nullptr, *h_geo = nullptr;
  int64_t geo_nb_cap = 0;
  cudaEvent_t geo_done = nullptr;
  std::vector<double> h_L;      // per field, host copy
  std::vector<int64_t> h_fnode; // first node of each field, then the total
  // batched solve: CUDA graph of (moments for new densities + walk)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  const void *graph_density = nullptr;
  void *graph_out = nullptr;
  int graph_fp64 = -1;
  double graph_theta = 0.0, graph_G = 0.0;
  WalkShape shape;              // tuned launch shape of the walk (0 = defaults)
  // walk order of the groups made by bh_autotune, longest walk first, for one
  // (np = 1) or two (np = 2) target pairs per lane: d_order[np - 1] holds
  // order_n[np - 1] group indices (0 = none); used while the tree has that
  // many groups
  unsigned *d_order[2] = {nullptr, nullptr};
  int64_t order_n[2] = {0, 0}, order_cap[2] = {0, 0};
  int64_t nb_cap = 0;
  // node arrays (capacity node_cap)
  double4_32a *d_mom = nullptr;
  WalkRec *d_rec = nullptr;
  float2 *d_aux = nullptr;
  uint8_t *d_lvl = nullptr;
  int64_t node_cap = 0;
  double *d_q64 = nullptr;      // 6 per node, FP64 quadrupoles (quadrupole option)
  WalkQuad *d_qrec = nullptr;   // binary32 quadrupole walk records
  int64_t quad_cap = 0;
  // host staging for the density of bh_solve_host
  void *d_stage_in = nullptr, *d_stage_out = nullptr;
  int64_t stage_in_bytes = 0, stage_out_bytes = 0;
  // current tree
  int nb = 0;
  int max_block_level = 0;
  int64_t n_nodes = 0;
  double lo[3] = {0, 0, 0};
  double L = 1.0;
  bool built = false;
  float s2_inv_theta = -1.0f;  // inverse theta the s2 field was prepared for
  float last_inv_theta = 0.0f; // of the last walk: builds prepare s2 for it
};

// Several fields (independent meshes) built and walked together: their
// blocks are concatenated; fstart[f] .. fstart[f+1]-1 are field f's blocks
// (nfields + 1 entries), fid[b] the field of caller block b, fld[p] = {first
// node, end node, first block of the next field, field} per sorted block, and
// invL[f] = 1 / box side of field f.  One field is the ordinary case.
struct FieldArgs {
  int nfields;
  const int *fstart;
  int *fid;
  int4 *fld;
  const double *invL;
  const double *L;   // box side per field
  unsigned long long *mmax;  // per field: bits of the largest FP64 cell mass
  // > 0: the moment kernels also write the squared opening radius of every
  // internal node for this 1/theta (as k_prepare_s2 would); 0: they write 0
  float inv_theta;
};

// The binary32 mass unit 2^e of a field from the bits of its largest cell
// mass (a non-negative double): e = its binary exponent - 40; 0 for zero.
__host__ __device__ inline int mass_exponent(unsigned long long bits) {
  const int E = (int)((bits >> 52) & 0x7ff);
  if (E == 0) return 0;                   // zero (or subnormal) masses
  const int e = E - 1023 - 40;
  return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}
// 2^e as a double, |e| <= 1022.
__host__ __device__ inline double pow2i(int e) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)(1023 + e) << 52);
#else
  const unsigned long long u = (unsigned long long)(1023 + e) << 52;
  double d;
  memcpy(&d, &u, sizeof d);
  return d;
#endif
}

// ---- build kernels (bh_build.cu) -------------------------------------------
// Every launcher returns the cudaError_t of its launch.
// Block keys (caller order, fid too) and the largest cell mass of every field
// (atomic max on fa.mmax, which the caller zeroes first): one launch.
cudaError_t launch_keys_mass(cudaStream_t s, int nb, const int *level, const int *ijk,
                             unsigned long long *key, int *idx, unsigned *flags,
                             const FieldArgs &fa, const void *density, int density_is_fp64);
cudaError_t launch_sort_blocks(cudaStream_t s, unsigned long long *key[2], int *idx[2],
                               unsigned *flags, const FieldArgs &fa);
cudaError_t launch_tile_and_count(cudaStream_t s, int nb, const unsigned long long *key,
                                  const int *idx, const int *level, const int *ijk,
                                  int *count, int4 *blk, int *orig, unsigned *flags,
                                  const FieldArgs &fa, const TopArgs &top, int *pos = nullptr);
cudaError_t launch_prestart_scan(cudaStream_t s, int nb, const int *count, int *prestart,
                                 unsigned *flags);
// Skip pointers of the top nodes and their lists (TopArgs); max_level = the
// largest block level.
cudaError_t launch_top_nodes(cudaStream_t s, int nb, const unsigned long long *key,
                             const int4 *blk, const int *count, const int *prestart,
                             int64_t n_nodes, WalkRec *rec, float2 *aux, uint8_t *lvl,
                             unsigned *flags, const FieldArgs &fa, const int *orig,
                             int max_level, const TopArgs &top);
// Largest cell mass of every field alone (a new density on the same tree).
// Negative or non-finite densities set kErrDensity in flags.
cudaError_t launch_mass_max(cudaStream_t s, int nb, const int *level, const void *density,
                            int density_is_fp64, const FieldArgs &fa, unsigned *flags);
// Every node's moments: cells and bottom nodes (k_blocks), then the rest of
// the blocks and the top tree (k_upper_tree), two launches.  before_upper:
// an event the second launch waits for (the top-node lists made on another
// stream), or null.
cudaError_t launch_moments(cudaStream_t s, int nb, const int4 *blk, const int *orig,
                           const int *count, const int *prestart, const void *density, int density_is_fp64, const FieldArgs &fa,
                           int64_t n_nodes, double4_32a *mom, WalkRec *rec, float2 *aux,
                           uint8_t *lvl, double *q64, WalkQuad *qrec, unsigned *flags,
                           const TopArgs &top, cudaEvent_t before_upper = nullptr);
// Raises the dynamic shared-memory limit of the learned walk (more than 48 KB)
// on the current device; called once per context, outside any graph capture.
cudaError_t prepare_learned_kernels();

// ---- walk kernels (bh_walk.cu) ---------------------------------------------
cudaError_t launch_prepare_s2(cudaStream_t s, int64_t n_nodes, const float2 *aux, WalkRec *rec,
                              float inv_theta);
// out: float* (F32) or double* (F64); counts: optional per-cell n_int/n_test.
// Potential scale of field f: -G * invL[f] (times the field's mass unit for
// the binary32 walk).  shape = the launch shape of the per-cell binary32
// walk (warps per CTA, target pairs per lane; 0 = defaults), tunable.
cudaError_t launch_walk(cudaStream_t s, const bh_options &opt, int nb, const WalkRec *rec,
                        const double4_32a *mom, const WalkQuad *qrec, const double *q64,
                        const int4 *blk, const int *orig, const FieldArgs &fa, double G,
                        void *out, int32_t *n_int, int32_t *n_test, int32_t *n_leaf = nullptr,
                        WalkShape shape = WalkShape());

// ---- small device helpers ---------------------------------------------------
// Spread the low 21 bits of v so bit b lands at bit 3b.
__host__ __device__ inline unsigned long long spread3(unsigned long long v) {
  v &= 0x1FFFFFull;
  v = (v | (v << 32)) & 0x1F00000000FFFFull;
  v = (v | (v << 16)) & 0x1F0000FF0000FFull;
  v = (v | (v << 8)) & 0x100F00F00F00F00Full;
  v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}
// Inverse of spread3.
__host__ __device__ inline unsigned long long compact3(unsigned long long v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10C30C30C30C30C3ull;
  v = (v ^ (v >> 4)) & 0x100F00F00F00F00Full;
  v = (v ^ (v >> 8)) & 0x1F0000FF0000FFull;
  v = (v ^ (v >> 16)) & 0x1F00000000FFFFull;
  v = (v ^ (v >> 32)) & 0x1FFFFFull;
  return v;
}

// Position of a node inside its block's 585-node pre-order subtree.
//   block root 0; child p (0..7) at 1 + 73p; grandchild (p, r) at 2 + 73p + 9r;
//   cell with local Morton index m = 64p + 8r + s at 3 + 73p + 9r + s.
__host__ __device__ inline int cell_offset(int m) {
  return 3 + 73 * (m >> 6) + 9 * ((m >> 3) & 7) + (m & 7);
}

// ---- learned correction (bh_learn.cu, bh_walk.cu) ---------------------------
constexpr int kMlpIn = 10, kMlpH = 64;
// FP32 master weights, flat: W1[10][64], b1[64], W2[64][64], b2[64], W3[64], b3
constexpr int kMlpNW = kMlpIn * kMlpH + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;
// Inference copy for the tensor-core walk, in the B-fragment order of
// mma.sync m16n8k16 (bf16): for each (n-tile, k-tile), 32 lanes x {b0, b1};
// lane (g = lane / 4, t = lane % 4) holds W[k0 + 2t .. k0 + 2t + 1][n0 + g] in
// b0 and W[k0 + 2t + 8 .. k0 + 2t + 9][n0 + g] in b1, the lower k in the low
// half.  Layer 1: K = 16: inputs 0..9 the features, input 10 a constant 1
// whose weights are b1 (so b1 is rounded to bf16 and added by the tensor
// core), inputs 11..15 zero; 8 n-tiles.  Layer 2: 8 n-tiles x 4 k-tiles;
// layer 3: 4 k-tiles of one n-tile whose column 0 is the output.  The walk
// carries activations as 2 GELU(a), so layer-2 and layer-3 weights are
// stored halved (exact in bf16).  b2, b3 FP32.
struct MlpDev {
  uint32_t w1f[8][32][2];
  uint32_t w2f[8][4][32][2];
  uint32_t w3f[4][32][2];
  float b2[kMlpH];
  float b3;
  float pad[3];
};

// Weights of the tcgen05 evaluator (bh_mlp_eval), bf16 operands in the
// canonical K-major layout without swizzle: element (r, k) of an operand with
// K columns at byte tc_canon(r, k, K) (core matrices of 8 rows x 16 bytes).
// b1: W1^T with b1 at input 10 (N = 64, K = 16); b2: W2^T halved (64 x 64);
// b3: W3^T halved in row 0 of 16 (N = 16, K = 64).  The same bf16 values as
// the walk's MlpDev.
struct MlpTc {
  uint16_t b1[64 * 16];
  uint16_t b2[64 * 64];
  uint16_t b3[16 * 64];
  float bias2[kMlpH];
  float bias3;
  float pad[3];
};
__host__ __device__ constexpr int tc_canon(int r, int k, int K) {
  return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// n rows of features x[n][10] -> y[n] on the tensor cores; flags[0] |= 1 if a
// bounded wait gave up.  probe_limit > 0 (tests of the time-out path only):
// no MMA is issued and the first wait gives up after probe_limit tries.
cudaError_t launch_mlp_tc(cudaStream_t s, int64_t n, const float *x, const MlpTc *w, float *y,
                          unsigned *flags, int probe_limit = 0);
cudaError_t prepare_mlp_tc_kernel();
// The learned walk with the network on tcgen05 (bh_walk_learned_tc.cu).
cudaError_t prepare_learned_tc_kernel();
cudaError_t launch_walk_learned_tc(cudaStream_t s, bh_ctx *ctx, double G, void *out);

// ---- device allocations (bh_abi.cu) ------------------------------------------
// Every device buffer the library owns is allocated through here.  Fault
// injection for tests of the out-of-memory paths: with the environment
// variable BHGRAV_FAIL_ALLOC_AFTER=n, the allocations after the first n made
// since the variable took that value fail with cudaErrorMemoryAllocation --
// nothing is allocated and no device fault is involved.
cudaError_t dev_malloc_bytes(void **p, size_t bytes);
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
  return dev_malloc_bytes(reinterpret_cast<void **>(p), bytes);
}

// ---- periodic boundaries (bh_ewald.cu, bh_walk_periodic.cu) ----------------
// The Ewald table of grid n and series range N (layout in bh_ewald.cuh):
// FP64 values at the (n+2)^3 points into scratch, then n^3 entries of 64
// bytes (the interpolants' coefficients) into tab.
cudaError_t launch_ewald_table(cudaStream_t s, int n, int N, double *scratch,
                               unsigned char *tab);
// chi at npts displacements r[npts][3] by the walk's interpolation.
cudaError_t launch_ewald_eval(cudaStream_t s, int64_t npts, const float *r,
                              const unsigned char *tab, int n, float *out);
// The binary32 per-cell walk with periodic boundaries; counts as launch_walk.
// wpc: warps per CTA (0 = default); order: the octants' walk order or null;
// cycles (potential only, else null): each octant's walk time in SM cycles.
cudaError_t launch_walk_periodic(cudaStream_t s, const bh_options &opt, int nb,
                                 const WalkRec *rec, const int4 *blk, const int *orig,
                                 const FieldArgs &fa, const unsigned char *tab, int n,
                                 double G,
                                 void *out, int32_t *n_int, int32_t *n_test, int32_t *n_leaf,
                                 int wpc, const unsigned *order = nullptr,
                                 unsigned long long *cycles = nullptr);

}  // namespace bhg

// The context (shared by the C-ABI translation units).
struct bh_ctx {
  bh_options opt;
  int device = 0;
  cudaStream_t stream = nullptr;
  // a second stream of the build: the top nodes' records and child lists are
  // made on it while k_blocks runs on `stream` (fork / join events)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bhg::Tree tree;
  bhg::MlpDev *d_mlp = nullptr;  // learned correction, set by bh_set_mlp
  double mlp_s_min = 0.0;        // its gate (bh_set_mlp_gate): no network below s = l/d
  bhg::MlpTc *d_mlp_tc = nullptr;   // the same network for bh_mlp_eval
  unsigned *d_tc_flag = nullptr;    // time-out flag of bh_mlp_eval
  unsigned char *d_ewald = nullptr; // periodic boundaries: the Ewald table
  int ewald_n = 0, ewald_series = 0;
  // statistics (bh_stats): events of the timing option (build start/end,
  // potential start/end), theta of the last potential, device totals of the
  // last bh_walk_counts
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool build_timed = false, potential_timed = false;
  double last_theta = 0.0;
  unsigned long long *d_counts = nullptr;
  bool counts_valid = false, counts_have_cells = false;
  char err[512] = {0};
};

namespace bhg {
// The gate of the learned walks as the kernels take it: fl32(1/s_min), or
// +inf (every accepted internal node corrected) for s_min = 0.
inline float learned_inv_smin(const bh_ctx *ctx) {
  return ctx->mlp_s_min > 0.0 ? (float)(1.0 / ctx->mlp_s_min)
                              : std::numeric_limits<float>::infinity();
}
// Records a one-line reason on the context and returns st.
bh_status ctx_fail(bh_ctx *c, bh_status st, const char *fmt, ...);
// Checks theta and the tree, and prepares the opening radii for theta.
bh_status ctx_prepare(bh_ctx *ctx, double theta);
cudaError_t launch_walk_learned(cudaStream_t s, bh_ctx *ctx, double G, void *out);
}  // namespace bhg
