/*
 * bhgrav -- Barnes-Hut gravitational potential at every cell centre of an
 * octree AMR mesh, on one NVIDIA GB300 (sm_103a).
 *
 * The method is the GPU Barnes-Hut tree solver of Lukat & Banerjee,
 * "A GPU accelerated Barnes-Hut tree code for FLASH4":
 *   - the octree is the AMR block tree extended down to single cells
 *     (Sec. 1; Sec. 2; Sec. 3.2.2);
 *   - every node carries its mass M, centre of mass R (Eq. 5) and the offset
 *     delta = |R - geometric centre| (Sec. 3.2.3, Fig. opening_angles);
 *   - the potential of a cell is the sum of -G M / d over the nodes accepted
 *     by the opening test d > l/theta + delta (Eq. 4) and -G m / d over the
 *     other cells reached (Sec. 3.3); theta is the runtime parameter
 *     grv_bh_gpuLimAngle, 0 < theta <= 1 (App. B).
 *
 * Calling convention (all entry points):
 *   - Block geometry (level, ijk) is passed in HOST memory.  Densities, the
 *     potential and every other array argument are DEVICE pointers on the
 *     context's device, owned by the caller.  The library owns its tree
 *     buffers from bh_build until the next bh_build or bh_destroy.
 *   - Work is issued on the context's CUDA stream.  bh_build returns once
 *     the geometry and the density are validated (it waits once, for the
 *     build's first kernels, to report their errors); the moments are then
 *     still being computed on the stream.  bh_potential only enqueues: the
 *     output is ready once the stream reaches that point.  Device inputs are
 *     read in stream order: keep them unchanged until the stream has passed
 *     the call that reads them.
 *   - No exceptions cross this boundary.  Every call returns a bh_status;
 *     bh_last_error() gives a one-line reason for the last failure on that
 *     context.  A context must not be used from two threads at once;
 *     separate contexts are independent.
 *
 * Mesh layout:
 *   - The box is the cube [box_lo, box_lo + box_len)^3.
 *   - Block b has level[b] in [0, 18] and integer coordinates ijk[3b..3b+2]
 *     in [0, 2^level[b]); it covers a cube of side box_len / 2^level[b] and
 *     holds 8^3 cells of side box_len / 2^(level[b]+3).  The leaf blocks must
 *     tile the box exactly (no gaps, no overlaps); they may come in any order.
 *     A 2:1 level balance is not required.
 *   - Cell arrays (density, potential) are [nblocks][8][8][8] in the caller's
 *     block order, indexed [b][cz][cy][cx], x fastest.
 */
#ifndef BHGRAV_H
#define BHGRAV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bh_ctx bh_ctx;

typedef enum {
  BH_OK = 0,
  BH_ERR_ARG = 1,             /* bad argument: null pointer, theta, G, negative/NaN density */
  BH_ERR_GEOMETRY = 2,        /* blocks do not tile the box, or a level/coordinate is out of range */
  BH_ERR_OOM = 3,             /* device allocation failed */
  BH_ERR_CUDA = 4,            /* a CUDA runtime call failed */
  BH_ERR_DEVICE_TIMEOUT = 5,  /* reserved: a bounded device wait gave up */
  BH_ERR_STATE = 6            /* call out of order (e.g. bh_potential before bh_build) */
} bh_status;

/* Arithmetic of the walk.  Node moments are always FP64 (Sec. 3.2.3). */
enum { BH_PREC_F32 = 0, BH_PREC_F64 = 1 };
/* Opening test scope: per target cell (the recursive definition of Sec. 2),
 * or the paper's warp vote (Sec. 3.3): 32 neighbouring cells (a 4x4x2 brick
 * of a block) accept a node only if all 32 accept it. */
enum { BH_CRIT_PER_CELL = 0, BH_CRIT_WARP_VOTE = 1 };

typedef struct {
  int precision;  /* BH_PREC_F32 (default): binary32 interaction arithmetic;
                     BH_PREC_F64: binary64 interaction arithmetic */
  int criterion;  /* BH_CRIT_PER_CELL (default) or BH_CRIT_WARP_VOTE */
  int kahan;      /* F32 only: 1 (default) compensated (Kahan) summation, 0 plain */
  int quadrupole; /* 0 (default): monopole nodes, as in the paper.  1: every
                     accepted node also adds its quadrupole term,
                     -G (1/2) d^T Q d / |d|^5 with Q = sum m (3 x x^T - |x|^2 I)
                     about the node's centre of mass (not in the paper: the
                     next term of the multipole expansion; the opening test is
                     unchanged).  Quadrupoles are reduced in binary32 for the
                     binary32 walk and in FP64 for the FP64 walk; they cost 32
                     (binary32) or 80 (FP64) more bytes per internal node. */
  int learned;    /* 0 (default).  1: every accepted node's term M/d is
                     multiplied by (1 + s^2 y), y = MLP(pair features), with the
                     network set by bh_set_mlp and evaluated on the tensor
                     cores by each warp as it walks (mma.sync, bf16 in, FP32
                     accumulate).  2: the same walk and arithmetic with the
                     rows of four warps evaluated together as 128-row tiles by
                     tcgen05 (FP32 accumulators in tensor memory); the same
                     results, slower on GB300 (the warps wait for each other).
                     Not in the paper; see bh_learn_pairs.  Needs the binary32
                     per-cell walk; excludes the quadrupole term. */
  int timing;     /* 0 (default).  1: bh_build, bh_build_batch, bh_update_density
                     and bh_potential bracket their device work with CUDA events
                     on the context's stream, for bh_stats (not while the
                     stream is being captured into a graph). */
  int periodic;   /* 0 (default): isolated boundaries (Eq. 2).  1: periodic
                     boundaries (App. A): every node's or cell's term M/d
                     becomes M psi(d), psi the Ewald field of a unit mass and
                     all its periodic copies with the mean density
                     subtracted, psi = 1/d + chi(d), chi interpolated from a
                     table (see bh_set_ewald); the opening test and the terms
                     use the minimum-image displacement (each box-unit
                     component wrapped into [-1/2, 1/2]:
                     dx > 0.5 -> fl(dx - 1), dx < -0.5 -> fl(dx + 1)), and
                     every cell also gets its own mass times chi(0), the
                     field of its periodic copies.  Needs the binary32
                     per-cell walk without the quadrupole or learned options. */
  int reserved[1];
} bh_options;

/* Fills *opt with the defaults: F32 walk, per-cell test, Kahan summation,
 * monopole nodes. */
void bh_default_options(bh_options *opt);

/* Creates a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * opt may be NULL for the defaults.  On success *out owns the context. */
bh_status bh_create(bh_ctx **out, const bh_options *opt, int device, void *cuda_stream);

/* Builds the octree of the mesh and its FP64 moments (Sec. 3.1.1 "collect
 * cell data", Sec. 3.2.2 tree build, Sec. 3.2.3 centres of gravity, Eq. 5).
 *   nblocks          number of leaf blocks (>= 1)
 *   level, ijk       HOST arrays [nblocks] and [nblocks][3], see "Mesh layout"
 *   box_lo, box_len  HOST double[3] lower corner and the side (> 0) of the box
 *   density          DEVICE array of nblocks*512 values, float (density_is_fp64
 *                    = 0) or double (1); every value finite and >= 0.  Cell
 *                    mass is density * cell volume.  Read on the stream until
 *                    the build's last kernel, which may run after the return.
 * Errors: BH_ERR_ARG, BH_ERR_GEOMETRY (nothing usable is kept: a later
 * bh_potential returns BH_ERR_STATE), BH_ERR_OOM, BH_ERR_CUDA. */
bh_status bh_build(bh_ctx *ctx, int nblocks, const int32_t *level, const int32_t *ijk,
                   const double *box_lo, double box_len, const void *density,
                   int density_is_fp64);

/* Potential at every cell centre (Sec. 3.3; Eq. 4 opening test, Eq. 2 terms
 * without the printed 1/2 of the energy sum):
 *   Phi_t = -G * ( sum over accepted nodes n of M_n / |r_t - R_n|
 *                + sum over the other cells c reached of m_c / |r_t - r_c| ).
 *   theta   opening parameter, 0 < theta <= 1
 *   G       gravitational constant (finite)
 *   out     DEVICE array of nblocks*512 values in the density layout: float
 *           for BH_PREC_F32, double for BH_PREC_F64.
 * The opening test is evaluated in binary32 (round to nearest) in box units
 * with this fixed order, so that any binary32 implementation of it reaches
 * the same decisions:
 *   s  = fl(fl(l * fl(1/theta)) + fl(delta)),  s2 = fl(s * s)
 *   dx = fl(t.x - fl(R.x)), dy, dz likewise
 *   d2 = fma(dx, dx, fma(dz, dz, fl(dy * dy)));  accept iff d2 > s2.
 * The interaction sum is binary32 with Kahan compensation or binary64 per
 * the context options.
 * Errors: BH_ERR_STATE (no tree), BH_ERR_ARG, BH_ERR_CUDA. */
bh_status bh_potential(bh_ctx *ctx, double theta, double G, void *out);

/* Several independent meshes ("fields") at once: one tree per field, all
 * built by the same kernel launches and walked by one launch of bh_potential
 * (each cell only sees its own field).  Not in the paper: batching for many
 * small solves, whose single launches would each fill only part of the GPU.
 *   nfields          number of fields (>= 1)
 *   nblocks          HOST int32[nfields], blocks per field
 *   level, ijk       HOST arrays of all fields' blocks, field after field
 *   box_lo, box_len  HOST double[nfields][3] and double[nfields]: each field's box
 *   density          DEVICE array, field after field, 512 values per block
 * Cell arrays (density, potential) follow the concatenated block order.
 * bh_potential, bh_walk_counts, bh_export_* then cover all fields.  Same
 * errors as bh_build. */
bh_status bh_build_batch(bh_ctx *ctx, int nfields, const int32_t *nblocks, const int32_t *level,
                         const int32_t *ijk, const double *box_lo, const double *box_len,
                         const void *density, int density_is_fp64);

/* New densities on the current geometry: recomputes the moments (and
 * quadrupoles) only, without the geometry work and without synchronising
 * the stream.  Densities are checked on the device; bh_sync_status reports a
 * negative or non-finite value (BH_ERR_ARG).  BH_ERR_STATE if no tree. */
bh_status bh_update_density(bh_ctx *ctx, const void *density, int density_is_fp64);

/* Synchronises the context's stream and reports errors the device raised
 * since the last build or density update (BH_OK if none). */
bh_status bh_sync_status(bh_ctx *ctx);

/* Times the binary32 per-cell walk of the current tree at this theta for
 * every launch shape it offers -- CTAs of 2, 4, 8 and 16 warps; warps that
 * walk for 64 targets (a 4x4x4 octant of a block, one pair of x-neighbours
 * per lane) or 128 targets (a 8x4x4 slab, two pairs per lane); either a
 * plain grid of one warp per group or a persistent grid (as many CTAs as the
 * GPU holds at once) whose warps take 1, 2 or 4 groups at a time from a work
 * counter; and the groups in their own (Morton) order or longest walk first
 * (the periodic walk: CTA width and order, one pair per lane, plain grid) --
 * each twice, then the four fastest five times more -- and keeps the fastest
 * for later walks.  For the longest-first order it first walks the tree once
 * at this theta (the persistent grid; the periodic walk on its plain grid),
 * recording the SM clock cycles of every group's walk, and
 * sorts the groups by them (on the host); that order is kept with the
 * context, like the shape, and used while the tree has the same number of
 * groups (a permutation of the groups: it can only change the speed).  All shapes
 * give bit-identical potentials.  shape (may be NULL) receives four ints:
 * {warps per CTA, target pairs per lane, groups per take (0 = plain grid),
 * longest first (0/1)}; all 0 for walk modes with a fixed launch shape.
 * Allocates a scratch output once and the order (4 bytes per group). */
bh_status bh_autotune(bh_ctx *ctx, double theta, int *shape);

/* Sets the launch shape of the binary32 per-cell walk (the four values
 * bh_autotune chooses among), e.g. one found by an earlier bh_autotune on
 * the same kind of mesh: warps per CTA (1..16), target pairs per lane (1 or
 * 2), groups per take of the persistent grid (0 = plain grid, 1..64) and
 * longest_first (1: the walk order made by the last bh_autotune, 0: the
 * groups' own order); 0 for the first two means the default.  Potentials do
 * not depend on the shape (bit for bit).  Drops a captured bh_solve_graph
 * graph.  BH_ERR_ARG for values out of range (the periodic walk: one pair,
 * plain grid); BH_ERR_STATE for longest_first = 1 without an order. */
bh_status bh_set_walk_shape(bh_ctx *ctx, int warps_per_cta, int pairs_per_lane,
                            int groups_per_take, int longest_first);

/* bh_update_density + bh_potential as ONE CUDA graph launch: the first call
 * (or a call with a different density/out pointer, density type, theta or G)
 * tunes the walk if it was not tuned yet, captures the sequence on the
 * context's stream and instantiates it; later calls replay it.  The context
 * must run on a created (non-default) stream.  Nothing is synchronised:
 * out is ready when the stream reaches the end of the graph; density errors
 * are reported by bh_sync_status.  Errors: BH_ERR_STATE, BH_ERR_ARG,
 * BH_ERR_CUDA. */
bh_status bh_solve_graph(bh_ctx *ctx, const void *density, int density_is_fp64, double theta,
                         double G, void *out);

/* Same walk as bh_potential, but instead of the potential it writes, per
 * cell in the density layout, the number of interactions n_int (accepted
 * nodes plus other cells reached), of opening tests n_test (internal nodes
 * examined) and, if n_cell is not NULL, of the interactions that are with
 * single cells (a subset of n_int).  DEVICE int32 arrays of nblocks*512
 * entries.  Used to count the algorithmic work of a walk. */
bh_status bh_walk_counts(bh_ctx *ctx, double theta, int32_t *n_int, int32_t *n_test,
                         int32_t *n_cell);

/* Sizes of the current tree: leaf cells, all nodes (cells + internal), and
 * the deepest cell level.  Any pointer may be NULL.  BH_ERR_STATE if no tree. */
bh_status bh_tree_size(const bh_ctx *ctx, int64_t *n_cells, int64_t *n_nodes, int *max_level);

/* Copies the node table (pre-order of a depth-first visit in octant order
 * o = ox + 2 oy + 4 oz, children after their parent) to DEVICE arrays of
 * n_nodes entries (any pointer may be NULL):
 *   M      double   node mass
 *   R      double*3 centre of mass in box units u = (x - box_lo)/box_len
 *   delta  float    |R - geometric centre| in box units, rounded to binary32
 *   skip   int32    index of the first node after this node's subtree
 *   level  int32    node level (0 = the box)
 * For inspection and tests; not needed to compute the potential. */
bh_status bh_export_nodes(const bh_ctx *ctx, double *M, double *R, float *delta, int32_t *skip,
                          int32_t *level);

/* Copies the quadrupole of every node (pre-order, 6 values per node:
 * xx, yy, zz, xy, xz, yz, box units, about the node's centre of mass; zero
 * for cells; FP64 values for an FP64 context, binary32 ones widened to double
 * otherwise) to the DEVICE array Q of 6*n_nodes doubles.  BH_ERR_STATE if no
 * tree or if the context was created without the quadrupole option. */
bh_status bh_export_quadrupoles(const bh_ctx *ctx, double *Q);

/* One-call form for callers whose data live in HOST memory: copies the
 * density (float or double per density_is_fp64) to the device, builds the
 * tree, walks it and writes the potential to out_host (float or double per
 * the context precision), then synchronises the stream.  A pinned out_host
 * (cudaMallocHost / cudaHostAlloc / cudaHostRegister) is written by the walk
 * directly through its device address; a pageable one receives a copy from a
 * device staging buffer (allocated once, kept by the context).  The density
 * goes through a device staging buffer; pinned, it copies at full bandwidth.
 * Same errors as the calls it makes. */
bh_status bh_solve_host(bh_ctx *ctx, int nblocks, const int32_t *level, const int32_t *ijk,
                        const double *box_lo, double box_len, const void *density_host,
                        int density_is_fp64, double theta, double G, void *out_host);

/* Allocation-free solve of one small mesh.  (The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * e.g. a host code whose GPU memory is entirely reserved by its own pool
 * allocator, or one that must not let a library enter cudaMalloc/cudaFree,
 * which may synchronise the device.)
 * Computes what bh_create (default options: binary32 per-cell walk with
 * Kahan sum) + bh_build + bh_potential compute, on the CURRENT device and on
 * `cuda_stream` (a cudaStream_t, NULL = legacy default stream), without any
 * context and without allocating: the tree lives in one fixed array in device
 * global memory (about 2.7 MB, held by every GPU that loads this library until
 * the process exits).
 *   nblocks        1 .. 64 blocks (at most 32,768 cells); more -> BH_ERR_ARG
 *   level, ijk, box_lo, box_len, density, density_is_fp64: as bh_build
 *   theta, G       as bh_potential
 *   out            DEVICE float array of nblocks*512 values (density layout)
 * The call synchronises the stream once, after the tree build, to check the
 * geometry and the density; it returns with the walk enqueued on the stream.
 * All calls share the fixed array and leave the last call's tree in it:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  The first call on a device looks up the
 * array's device address (with that device current); make that first call
 * before any stream capture on the device.
 * Errors: BH_ERR_ARG, BH_ERR_GEOMETRY, BH_ERR_CUDA (no message string: there
 * is no context). */
bh_status bh_solve_noalloc(int nblocks, const int32_t *level, const int32_t *ijk,
                           const double *box_lo, double box_len, const void *density,
                           int density_is_fp64, double theta, double G, float *out,
                           void *cuda_stream);

/* ---- learned residual correction (not in the paper) -------------------------
 * Features x of an accepted (target, node) pair, s = l/|d|, u = d/|d|:
 *   x = [u_x, u_y, u_z, s, s^2, s^3, delta/l, u^T Q u/(M l^2), |Q|_F/(M l^2),
 *        s^2 u^T Q u/(M l^2)]
 * Network: 10 -> 64 -> 64 -> 1, tanh-form GELU, weights flat in FP32 as
 * W1[10][64], b1[64], W2[64][64], b2[64], W3[64], b3 (4865 floats). */

/* Training pairs generated by the method itself: for each DEVICE target cell
 * index (caller layout, int64), every internal node its per-cell walk at theta
 * accepts, with the pair's features feat[10] and eps = (the node's exact
 * contribution, summed over its cells in FP64)/(M/|d|) - 1.  feat (cap*10)
 * and eps (cap) are DEVICE float arrays; node (DEVICE int64, cap, may be NULL)
 * receives the node index of each pair (pairs come in no particular order);
 * *count (HOST) receives the number of pairs found (only the first cap are
 * written).  Needs a tree with quadrupole records (quadrupole or learned
 * option).  Synchronises the stream. */
bh_status bh_learn_pairs(bh_ctx *ctx, double theta, int64_t ntargets, const int64_t *targets,
                         int64_t cap, float *feat, float *eps, int64_t *node, int64_t *count);

/* Training targets of n pairs: z = eps / s^2 with s = feat[3] (DEVICE float
 * arrays feat[n][10], eps[n] from bh_learn_pairs; z[n] written), the network
 * output for which the learned walk's term (M/d)(1 + s^2 z) equals the
 * node's exact contribution.  Not in the paper.  Enqueued on cuda_stream. */
bh_status bh_learn_targets(int64_t n, const float *feat, const float *eps, float *z,
                           void *cuda_stream);

/* Gradient of the mean squared error of MLP(x) against z over n samples
 * (DEVICE x[n][10], z[n], weights w), written to DEVICE grad[4865]; the loss
 * to DEVICE *loss.  FP32.  Enqueued on cuda_stream. */
bh_status bh_mlp_grad(int64_t n, const float *x, const float *z, const float *w, float *grad,
                      float *loss, void *cuda_stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) of the DEVICE weights w with
 * DEVICE moments m, v (4865 each, zero before step 1); step counts from 1. */
bh_status bh_mlp_adam(const float *grad, float *w, float *m, float *v, int step, float lr,
                      void *cuda_stream);

/* Sets the network of the learned walk from HOST FP32 weights; the weights
 * are rounded to bf16 (round to nearest even) for the tensor cores, biases
 * stay FP32.  bh_get_mlp returns the weights in use (bf16 values widened). */
bh_status bh_set_mlp(bh_ctx *ctx, const float *w_host);
bh_status bh_get_mlp(const bh_ctx *ctx, float *w_host);

/* Gate of the learned walk (not in the paper): the network corrects an
 * accepted internal node only while s = l/|d| >= s_min, since its correction
 * (M/|d|) s^2 y shrinks with s^2.  Decided in binary32 on the opening test's
 * d2 (see bh_options.criterion) with a fixed rounding: corrected iff
 * d2 <= fl(g * g), g = fl(l * fl(1/s_min)); the other accepted nodes keep
 * their plain term M/|d|.  s_min = 0 (the default) corrects every accepted
 * internal node.  BH_ERR_ARG unless 0 <= s_min < 1. */
bh_status bh_set_mlp_gate(bh_ctx *ctx, double s_min);

/* ---- statistics (not in the paper) ---------------------------------------- */
typedef struct {
  int64_t n_cells;           /* leaf cells of the current tree, all fields (0: no tree) */
  int64_t n_nodes;           /* nodes: cells + internal nodes, (N - 1)/7 of them per field */
  int32_t n_blocks;          /* leaf blocks */
  int32_t n_fields;          /* fields of the last bh_build (1) or bh_build_batch */
  int32_t max_level;         /* deepest cell level (block level + 3) */
  int32_t built;             /* 1 once a tree is built and validated */
  double last_theta;         /* theta of the last bh_potential (0: none yet) */
  double build_ms;           /* device time of the last bh_build / bh_build_batch /
                                bh_update_density; -1 unless the timing option is on */
  double potential_ms;       /* device time of the last bh_potential (opening radii +
                                walk); -1 unless the timing option is on */
  int64_t interactions;      /* totals over all cells of the last bh_walk_counts call: */
  int64_t tests;             /*   interactions, opening tests of internal nodes and */
  int64_t cell_interactions; /*   interactions with single cells; -1 if none yet */
  int64_t device_bytes;      /* device memory held by the context's tree buffers */
} bh_stats_t;

/* Sizes of the current tree, the device times of the last build and
 * potential (timing option) and the work totals of the last bh_walk_counts.
 * Waits for the recorded events and copies 24 bytes from the device, so it
 * synchronises with the work it reports on.  BH_ERR_ARG on null pointers. */
bh_status bh_stats(const bh_ctx *ctx, bh_stats_t *out);

/* Evaluates the network set by bh_set_mlp on n rows of pair features
 * (DEVICE FP32 x[n][10], the layout of bh_learn_pairs) into DEVICE FP32 y[n],
 * on the tensor cores (tcgen05: bf16 operands in shared memory, FP32
 * accumulators in tensor memory), with the same rounding as the learned walk:
 * features, b1 and hidden activations in bf16, the GELU in bf16 pairs.  Not in
 * the paper.  Synchronises the stream.  BH_ERR_STATE without a network;
 * BH_ERR_DEVICE_TIMEOUT if a bounded wait for the tensor core gave up. */
bh_status bh_mlp_eval(bh_ctx *ctx, int64_t n, const float *x, float *y);

/* ---- periodic boundaries (App. A) ----------------------------------------
 * The Ewald field of a unit mass in the box (box units, period 1), mean
 * density subtracted, split as 1/r = erf(a r)/r + erfc(a r)/r with a = 2:
 *   psi(r) = sum_n erfc(a|r+n|)/|r+n|
 *          + (1/pi) sum_{k!=0} exp(-pi^2 |k|^2/a^2)/|k|^2 cos(2 pi k.r) - pi/a^2
 * (n, k integer triples with components in [-n_series, n_series], the
 * paper's gpuEwaldSeriesN), and chi(r) = psi(r) - 1/|r|, smooth around the
 * origin.  The table holds chi at the points (i, j, k) h, h = 1/(2 n_grid),
 * i, j, k = 0 .. n_grid + 1 (the octant [0, 1/2 + h]^3; chi is even in each
 * coordinate).  At u = |minimum-image displacement| the walk interpolates
 * quadratically: per axis c = floor(u/h + 1/2) clamped to [1, n_grid],
 * f = u/h - c, weights f(f-1)/2, 1 - f^2, f(f+1)/2 for the points c-1, c,
 * c+1; chi(u) = sum of the 27 weight products times the table values. */

/* Computes the table on the device (FP64 sums) for the periodic walk of
 * this context and keeps it as n_grid^3 entries of 64 bytes: per grid
 * centre the 27 coefficients of its quadratic interpolant, the value and
 * first-order ones in binary32, the 23 smaller ones in binary16 (they change
 * chi by less than 3e-7).  A context created with the periodic option starts
 * with n_grid = 64, n_series = 3 (16 MB; interpolation error about 3e-6,
 * series converged to 1e-13).  n_grid in [2, 256], n_series in [1, 8], else
 * BH_ERR_ARG; BH_ERR_OOM if the table does not fit.  Synchronises the
 * context's stream. */
bh_status bh_set_ewald(bh_ctx *ctx, int n_grid, int n_series);

/* chi at n box-unit displacements (DEVICE FP32 r[n][3], each component in
 * [-1/2, 1/2]) into DEVICE FP32 chi[n], by the walk's interpolation of the
 * table.  BH_ERR_STATE without a table (context not periodic and no
 * bh_set_ewald call); enqueued on the context's stream. */
bh_status bh_ewald_eval(bh_ctx *ctx, int64_t n, const float *r, float *chi);

/* Reason for the last failure on ctx ("" if none).  Valid until the next call. */
const char *bh_last_error(const bh_ctx *ctx);

/* Releases the context and every buffer the library allocated.  NULL is a no-op. */
void bh_destroy(bh_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BHGRAV_H */
