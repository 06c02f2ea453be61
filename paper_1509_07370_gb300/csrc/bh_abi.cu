// C-ABI of libbhgrav: argument checking, buffer ownership, the order of the
// build and walk launches, the choice of walk for the context's options, the
// Ewald table's lifetime and the batched (CUDA graph) solve.  The method's
// arithmetic lives in the other translation units (bh_build.cu, bh_walk.cu,
// bh_walk_periodic.cu with bh_ewald.cu, bh_walk_learned*.cu with bh_learn.cu
// and bh_mlp_tc.cu); this file only holds the small export kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "bh_internal.cuh"

namespace bhg {
cudaError_t dev_malloc_bytes(void **p, size_t bytes) {
  static std::mutex mu;
  static std::string armed;  // the variable's value the count belongs to
  static long long made = 0;
  const char *env = std::getenv("BHGRAV_FAIL_ALLOC_AFTER");
  if (env && *env) {
    std::lock_guard<std::mutex> lock(mu);
    if (armed != env) {
      armed = env;
      made = 0;
    }
    if (made >= std::atoll(env)) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    ++made;
  }
  return cudaMalloc(p, bytes);
}
}  // namespace bhg

namespace {

// A named NVTX range around each entry point's host work (header-only NVTX:
// a no-op unless a profiler is attached), so that timelines show the calls.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

bh_status fail(bh_ctx *c, bh_status st, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define BH_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? BH_ERR_OOM : BH_ERR_CUDA,   \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

template <typename T>
void release(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

void free_blocks(bhg::Tree &t) {
  release(t.d_key[0]);
  release(t.d_key[1]);
  release(t.d_idx[0]);
  release(t.d_idx[1]);
  release(t.d_count);
  release(t.d_prestart);
  release(t.d_blk);
  release(t.d_orig);
  release(t.d_fid);
  release(t.d_fld);
  release(t.d_pos);
  release(t.d_top);
  t.nb_cap = 0;
}

void free_nodes(bhg::Tree &t) {
  release(t.d_mom);
  release(t.d_rec);
  release(t.d_aux);
  release(t.d_lvl);
  t.node_cap = 0;
  release(t.d_q64);
  release(t.d_qrec);
  t.quad_cap = 0;
}

bh_status ensure_blocks(bh_ctx *ctx, int nb) {
  bhg::Tree &t = ctx->tree;
  if (t.nb_cap >= nb) return BH_OK;
  free_blocks(t);
  const size_t n = (size_t)nb;
  BH_CUDA(bhg::dev_malloc(&t.d_key[0], n * sizeof(unsigned long long)));
  BH_CUDA(bhg::dev_malloc(&t.d_key[1], n * sizeof(unsigned long long)));
  BH_CUDA(bhg::dev_malloc(&t.d_idx[0], n * sizeof(int)));
  BH_CUDA(bhg::dev_malloc(&t.d_idx[1], n * sizeof(int)));
  BH_CUDA(bhg::dev_malloc(&t.d_count, n * sizeof(int)));
  BH_CUDA(bhg::dev_malloc(&t.d_prestart, n * sizeof(int)));
  BH_CUDA(bhg::dev_malloc(&t.d_blk, n * sizeof(int4)));
  BH_CUDA(bhg::dev_malloc(&t.d_orig, n * sizeof(int)));
  BH_CUDA(bhg::dev_malloc(&t.d_fid, n * sizeof(int)));
  BH_CUDA(bhg::dev_malloc(&t.d_pos, n * sizeof(int)));
  BH_CUDA(bhg::dev_malloc(&t.d_fld, n * sizeof(int4)));
  BH_CUDA(bhg::dev_malloc(&t.d_top, (size_t)bhg::top_ints(nb) * sizeof(int)));
  t.nb_cap = nb;
  return BH_OK;
}

bh_status ensure_nodes(bh_ctx *ctx, int64_t n_nodes) {
  bhg::Tree &t = ctx->tree;
  const bool quad = ctx->opt.quadrupole != 0 || ctx->opt.learned != 0;
  const bool quad64 = ctx->opt.quadrupole && ctx->opt.precision == BH_PREC_F64;
  if (t.node_cap >= n_nodes && (!quad || t.quad_cap >= n_nodes)) return BH_OK;
  free_nodes(t);
  if (quad) {
    if (quad64) BH_CUDA(bhg::dev_malloc(&t.d_q64, (size_t)n_nodes * 6 * sizeof(double)));
    BH_CUDA(bhg::dev_malloc(&t.d_qrec, (size_t)n_nodes * sizeof(bhg::WalkQuad)));
    t.quad_cap = n_nodes;
  }
  const size_t n = (size_t)n_nodes;
  BH_CUDA(bhg::dev_malloc(&t.d_mom, n * sizeof(double4_32a)));
  BH_CUDA(bhg::dev_malloc(&t.d_rec, n * sizeof(bhg::WalkRec)));
  BH_CUDA(bhg::dev_malloc(&t.d_aux, n * sizeof(float2)));
  BH_CUDA(bhg::dev_malloc(&t.d_lvl, n * sizeof(uint8_t)));
  t.node_cap = n_nodes;
  return BH_OK;
}

bh_status use_device(bh_ctx *ctx) {
  BH_CUDA(cudaSetDevice(ctx->device));
  return BH_OK;
}

// The geometry a build takes from the host lives in one device region with a
// pinned host mirror, so that a build uploads it in one copy:
// [mmax (nf u64, zeroed) | L, 1/L (nf f64 each) | fstart (nf + 1 int) |
//  level (nb int) | ijk (3 nb int)], nf = nf_cap, nb = geo_nb_cap.
struct GeoLayout {
  size_t L, invL, fstart, level, ijk, end;
};
GeoLayout geo_layout(int64_t nf, int64_t nb) {
  GeoLayout g;
  g.L = 8 * nf;
  g.invL = 16 * nf;
  g.fstart = 24 * nf;
  g.level = (g.fstart + 4 * (nf + 1) + 15) & ~(size_t)15;
  g.ijk = g.level + 4 * nb;
  g.end = g.ijk + 12 * nb;
  return g;
}

void free_fields(bhg::Tree &t) {
  release(t.d_geo);
  if (t.h_geo) cudaFreeHost(t.h_geo);
  t.h_geo = nullptr;
  t.d_mmax = nullptr;
  t.d_L = t.d_invL = nullptr;
  t.d_fstart = t.d_level = t.d_ijk = nullptr;
  t.nf_cap = 0;
  t.geo_nb_cap = 0;
}

void drop_graph(bhg::Tree &t) {
  if (t.graph_exec) cudaGraphExecDestroy(t.graph_exec);
  if (t.graph) cudaGraphDestroy(t.graph);
  t.graph_exec = nullptr;
  t.graph = nullptr;
  t.graph_density = nullptr;
  t.graph_out = nullptr;
}

bh_status ensure_fields(bh_ctx *ctx, int nfields, int nb) {
  bhg::Tree &t = ctx->tree;
  if (t.nf_cap >= nfields && t.geo_nb_cap >= nb) return BH_OK;
  const int64_t nf = std::max<int64_t>(nfields, t.nf_cap);
  const int64_t nbc = std::max<int64_t>(nb, t.geo_nb_cap);
  free_fields(t);
  const GeoLayout g = geo_layout(nf, nbc);
  BH_CUDA(bhg::dev_malloc(&t.d_geo, g.end));
  BH_CUDA(cudaHostAlloc((void **)&t.h_geo, g.end, cudaHostAllocDefault));
  t.d_mmax = reinterpret_cast<unsigned long long *>(t.d_geo);
  t.d_L = reinterpret_cast<double *>(t.d_geo + g.L);
  t.d_invL = reinterpret_cast<double *>(t.d_geo + g.invL);
  t.d_fstart = reinterpret_cast<int *>(t.d_geo + g.fstart);
  t.d_level = reinterpret_cast<int *>(t.d_geo + g.level);
  t.d_ijk = reinterpret_cast<int *>(t.d_geo + g.ijk);
  t.nf_cap = (int)nf;
  t.geo_nb_cap = nbc;
  return BH_OK;
}

bhg::FieldArgs field_args(bhg::Tree &t) {
  bhg::FieldArgs fa;
  fa.nfields = t.nfields;
  fa.fstart = t.d_fstart;
  fa.fid = t.d_fid;
  fa.fld = t.d_fld;
  fa.invL = t.d_invL;
  fa.L = t.d_L;
  fa.mmax = t.d_mmax;
  fa.inv_theta = t.last_inv_theta;
  return fa;
}

// Moments of the current geometry from a density (k_blocks, then
// k_upper_tree); stream-ordered, no host synchronisation.
bh_status enqueue_moments(bh_ctx *ctx, const void *density, int density_is_fp64,
                          bool mmax_ready = false, cudaEvent_t before_upper = nullptr) {
  bhg::Tree &t = ctx->tree;
  cudaStream_t s = ctx->stream;
  // FP64 quadrupoles for the FP64 walk, binary32 ones for the binary32 walk
  double *q64 = ctx->opt.quadrupole && ctx->opt.precision == BH_PREC_F64 ? t.d_q64 : nullptr;
  bhg::WalkQuad *qrec = (ctx->opt.quadrupole || ctx->opt.learned) ? t.d_qrec : nullptr;
  const bhg::FieldArgs fa = field_args(t);
  // binary32 mass unit of every field (largest cell mass), unless the build's
  // first kernel found it, then the moments
  if (!mmax_ready) {
    BH_CUDA(cudaMemsetAsync(t.d_mmax, 0, (size_t)t.nfields * sizeof(unsigned long long), s));
    BH_CUDA(bhg::launch_mass_max(s, t.nb, t.d_level, density, density_is_fp64, fa, t.d_flags));
  }
  BH_CUDA(bhg::launch_moments(s, t.nb, t.d_blk, t.d_orig, t.d_count, t.d_prestart, density, density_is_fp64, fa, t.n_nodes, t.d_mom, t.d_rec, t.d_aux,
                              t.d_lvl, q64, qrec, t.d_flags, bhg::top_args(t.d_top, t.nb_cap),
                              before_upper));
  return BH_OK;
}

// Records event i of the timing option on the context's stream; not while
// the stream is being captured into a graph (replays are not timed).
bool timing_mark(bh_ctx *ctx, int i) {
  if (!ctx->opt.timing) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;
  }
  if (!ctx->ev[i] && cudaEventCreate(&ctx->ev[i]) != cudaSuccess) {
    cudaGetLastError();
    ctx->ev[i] = nullptr;
    return false;
  }
  if (cudaEventRecord(ctx->ev[i], ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Totals of the per-cell counts of a counting walk: out[0] += sum n_int,
// out[1] += sum n_test, out[2] += sum n_cell (if given).
__global__ void k_sum_counts(int64_t n, const int32_t *__restrict__ a,
                             const int32_t *__restrict__ b, const int32_t *__restrict__ c,
                             unsigned long long *out) {
  unsigned long long sa = 0, sb = 0, sc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    sa += (unsigned)a[i];
    sb += (unsigned)b[i];
    if (c) sc += (unsigned)c[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_down_sync(0xffffffffu, sa, o);
    sb += __shfl_down_sync(0xffffffffu, sb, o);
    sc += __shfl_down_sync(0xffffffffu, sc, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, sa);
    atomicAdd(out + 1, sb);
    if (c) atomicAdd(out + 2, sc);
  }
}

// Tree and moments of nfields meshes (one field = bh_build).  Waits once,
// for the input checks of the first kernels, to report geometry and density
// errors; the moments are still running on the stream when it returns.
bh_status build_fields(bh_ctx *ctx, int nfields, const int32_t *nblocks, const int32_t *level,
                       const int32_t *ijk, const double *box_lo, const double *box_len,
                       const void *density, int density_is_fp64, const char *who) {
  bhg::Tree &t = ctx->tree;
  t.built = false;
  drop_graph(t);
  if (nfields <= 0 || !nblocks || !level || !ijk || !box_lo || !box_len || !density)
    return fail(ctx, BH_ERR_ARG, "%s: nblocks must be >= 1 and pointers non-null", who);
  if (density_is_fp64 != 0 && density_is_fp64 != 1)
    return fail(ctx, BH_ERR_ARG, "%s: density_is_fp64 must be 0 or 1", who);
  std::vector<int> fstart(nfields + 1, 0);
  std::vector<int64_t> fnode(nfields + 1, 0);
  std::vector<double> invL(nfields), L(nfields);
  int64_t nb64 = 0, n_nodes = 0, tops = 0;
  for (int f = 0; f < nfields; ++f) {
    const int nbf = nblocks[f];
    if (nbf <= 0) return fail(ctx, BH_ERR_ARG, "%s: field %d has no blocks", who, f);
    if (!(box_len[f] > 0.0) || !std::isfinite(box_len[f]) || !std::isfinite(box_lo[3 * f]) ||
        !std::isfinite(box_lo[3 * f + 1]) || !std::isfinite(box_lo[3 * f + 2]))
      return fail(ctx, BH_ERR_ARG, "%s: box_len must be finite and > 0, box_lo finite", who);
    // a tiling has nb = 1 + 7k blocks
    if ((nbf - 1) % 7 != 0)
      return fail(ctx, BH_ERR_GEOMETRY, "%s: %d blocks cannot tile a cube (need 1 + 7k)", who,
                  nbf);
    fstart[f] = (int)nb64;
    fnode[f] = n_nodes;
    nb64 += nbf;
    tops += (nbf - 1) / 7;
    n_nodes += (int64_t)bhg::kNodesPerBlock * nbf + (nbf - 1) / 7;
    L[f] = box_len[f];
    invL[f] = 1.0 / box_len[f];
  }
  // node indices must fit 31 bits
  if (n_nodes >= (int64_t)0x7fffffff || nb64 >= (int64_t)0x7fffffff)
    return fail(ctx, BH_ERR_ARG, "%s: %lld blocks exceed the 2^31 node limit", who,
                (long long)nb64);
  const int nb = (int)nb64;
  fstart[nfields] = nb;
  fnode[nfields] = n_nodes;
  int max_level = 0;
  for (int b = 0; b < nb; ++b) {
    if (level[b] < 0 || level[b] > bhg::kMaxBlockLevel)
      return fail(ctx, BH_ERR_GEOMETRY, "%s: block %d has level %d outside [0, 18]", who, b,
                  level[b]);
    max_level = level[b] > max_level ? level[b] : max_level;
  }
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  if ((st = ensure_blocks(ctx, nb)) != BH_OK) return st;
  if ((st = ensure_fields(ctx, nfields, nb)) != BH_OK) return st;
  if ((st = ensure_nodes(ctx, n_nodes)) != BH_OK) return st;
  t.nfields = nfields;
  t.nb = nb;
  t.n_nodes = n_nodes;
  t.max_block_level = max_level;
  t.h_L = L;
  t.h_fnode = fnode;
  cudaStream_t s = ctx->stream;
  const bhg::FieldArgs fa = field_args(t);
  const bhg::TopArgs top = bhg::top_args(t.d_top, t.nb_cap);
  // the host geometry, with zeroed largest masses, into the pinned mirror and
  // up in one copy (the last build's copy ended before its wait on the
  // flags returned)
  const GeoLayout g = geo_layout(t.nf_cap, t.geo_nb_cap);
  if (t.geo_done) BH_CUDA(cudaEventSynchronize(t.geo_done));  // a copy left by a failed build
  else BH_CUDA(cudaEventCreateWithFlags(&t.geo_done, cudaEventDisableTiming));
  memset(t.h_geo, 0, (size_t)nfields * sizeof(unsigned long long));
  memcpy(t.h_geo + g.L, L.data(), (size_t)nfields * sizeof(double));
  memcpy(t.h_geo + g.invL, invL.data(), (size_t)nfields * sizeof(double));
  memcpy(t.h_geo + g.fstart, fstart.data(), (size_t)(nfields + 1) * sizeof(int));
  memcpy(t.h_geo + g.level, level, (size_t)nb * sizeof(int));
  memcpy(t.h_geo + g.ijk, ijk, 3 * (size_t)nb * sizeof(int));
  ctx->build_timed = false;
  const bool timed = timing_mark(ctx, 0);
  BH_CUDA(cudaMemsetAsync(t.d_flags, 0, 4 * sizeof(unsigned), s));
  BH_CUDA(cudaMemcpyAsync(t.d_geo, t.h_geo, g.ijk + 12 * (size_t)nb, cudaMemcpyHostToDevice, s));
  BH_CUDA(cudaEventRecord(t.geo_done, s));
  BH_CUDA(bhg::launch_keys_mass(s, nb, t.d_level, t.d_ijk, t.d_key[0], t.d_idx[0], t.d_flags, fa,
                                density, density_is_fp64));
  BH_CUDA(bhg::launch_sort_blocks(s, t.d_key, t.d_idx, t.d_flags, fa));
  BH_CUDA(bhg::launch_tile_and_count(s, nb, t.d_key[0], t.d_idx[0], t.d_level, t.d_ijk,
                                     t.d_count, t.d_blk, t.d_orig, t.d_flags, fa, top, t.d_pos));
  BH_CUDA(bhg::launch_prestart_scan(s, nb, t.d_count, t.d_prestart, t.d_flags));
  // the top nodes' records and child lists (needed from k_upper_tree on) on
  // the side stream, beside k_blocks, which writes only the blocks' nodes
  if (!ctx->side || !ctx->fork || !ctx->join) {  // made once, all three or none
    int lo_prio = 0, hi_prio = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, hi_prio);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      if (join) cudaEventDestroy(join);
      if (fork) cudaEventDestroy(fork);
      if (side) cudaStreamDestroy(side);
    }
    BH_CUDA(e);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->join) cudaEventDestroy(ctx->join);
    ctx->side = side;
    ctx->fork = fork;
    ctx->join = join;
  }
  BH_CUDA(cudaEventRecord(ctx->fork, s));
  BH_CUDA(cudaStreamWaitEvent(ctx->side, ctx->fork, 0));
  BH_CUDA(bhg::launch_top_nodes(ctx->side, nb, t.d_key[0], t.d_blk, t.d_count, t.d_prestart,
                                n_nodes, t.d_rec, t.d_aux, t.d_lvl, t.d_flags, fa, t.d_orig,
                                max_level, top));
  // Every check of the input is done by now (levels, coordinates and density
  // in k_keys_mass, the tiling in k_tile_and_count, the top-node count in
  // k_prestart_scan, top indexes in k_top_nodes/k_top_children): the flags go
  // to the host from the side stream while k_blocks runs, and the host waits
  // for them alone, so that the walk the caller enqueues next follows the
  // moments with no gap.  (k_blocks may set bits of its own meanwhile; the
  // copy then sees them or not, and they are set only on a failed geometry or
  // density, which the copied bits already report.)
  BH_CUDA(cudaMemcpyAsync(t.h_flags, t.d_flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          ctx->side));
  BH_CUDA(cudaEventRecord(ctx->join, ctx->side));
  if ((st = enqueue_moments(ctx, density, density_is_fp64, true, ctx->join)) != BH_OK) return st;
  ctx->build_timed = timed && timing_mark(ctx, 1);
  BH_CUDA(cudaEventSynchronize(ctx->join));
  const unsigned e = t.h_flags[0];
  if (e & (bhg::kErrLevel | bhg::kErrCoord))
    return fail(ctx, BH_ERR_GEOMETRY, "%s: a block coordinate lies outside its level", who);
  if (e & bhg::kErrTiling)
    return fail(ctx, BH_ERR_GEOMETRY, "%s: the blocks do not tile the box (gap or overlap)", who);
  if ((int64_t)t.h_flags[2] != tops || (e & bhg::kErrIndex))
    return fail(ctx, BH_ERR_GEOMETRY, "%s: inconsistent block tree (%u internal nodes)", who,
                t.h_flags[2]);
  if (e & bhg::kErrDensity)
    return fail(ctx, BH_ERR_ARG, "%s: density has a negative or non-finite value", who);
  for (int a = 0; a < 3; ++a) t.lo[a] = box_lo[a];
  t.L = box_len[0];
  // the moment kernels prepared s2 for the last walk's theta, if any
  t.s2_inv_theta = fa.inv_theta > 0.0f ? fa.inv_theta : -1.0f;
  t.built = true;
  return BH_OK;
}

}  // namespace

extern "C" {

void bh_default_options(bh_options *opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = BH_PREC_F32;
  opt->criterion = BH_CRIT_PER_CELL;
  opt->kahan = 1;
}

// Default Ewald table of a periodic context: interpolation error about 3e-6
// of chi(0), series converged to 1e-13.
constexpr int kEwaldGrid = 64, kEwaldSeries = 3;

// Computes the Ewald table (n, N) on the context's stream and makes it the
// context's table; synchronises once (to free the FP64 scratch).
static bh_status set_ewald(bh_ctx *ctx, int n, int N) {
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const int64_t m = n + 2;
  double *scratch = nullptr;
  unsigned char *tab = nullptr;
  if (bhg::dev_malloc(&scratch, m * m * m * sizeof(double)) != cudaSuccess ||
      bhg::dev_malloc(&tab, (int64_t)n * n * n * 64) != cudaSuccess) {
    cudaGetLastError();
    release(scratch);
    release(tab);
    return fail(ctx, BH_ERR_OOM, "Ewald table: device allocation failed");
  }
  cudaError_t e = bhg::launch_ewald_table(ctx->stream, n, N, scratch, tab);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  release(scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(tab);
    return fail(ctx, BH_ERR_CUDA, "Ewald table: %s", cudaGetErrorString(e));
  }
  drop_graph(ctx->tree);  // a captured walk holds the old table
  release(ctx->d_ewald);
  ctx->d_ewald = tab;
  ctx->ewald_n = n;
  ctx->ewald_series = N;
  return BH_OK;
}

// The walk of the context's options on stream s: the potential into out, or
// with n_int / n_test (and optional n_leaf) the per-cell counts.
static cudaError_t enqueue_walk(bh_ctx *ctx, cudaStream_t s, double G, void *out,
                                int32_t *n_int, int32_t *n_test, int32_t *n_leaf,
                                bhg::WalkShape shape) {
  bhg::Tree &t = ctx->tree;
  if (ctx->opt.periodic) {  // one pair per lane, a plain grid, optionally longest first
    const int64_t groups = (int64_t)t.nb * 8;
    const unsigned *order = shape.longest && t.order_n[0] == groups ? t.d_order[0] : nullptr;
    return bhg::launch_walk_periodic(s, ctx->opt, t.nb, t.d_rec, t.d_blk, t.d_orig,
                                     field_args(t), ctx->d_ewald, ctx->ewald_n, G, out, n_int,
                                     n_test, n_leaf, shape.warps, order, shape.cycles);
  }
  if (!n_int && ctx->opt.learned == 2) return bhg::launch_walk_learned_tc(s, ctx, G, out);
  if (!n_int && ctx->opt.learned) return bhg::launch_walk_learned(s, ctx, G, out);
  shape.counter = t.d_flags + 4;  // the work counter of the persistent walk
  {  // the groups' walk order made by bh_autotune, while it fits the tree
    const int np = shape.pairs > 0 ? shape.pairs : 1;
    const int64_t groups = (int64_t)t.nb * (8 / np);
    shape.order = (shape.longest && np <= 2 && t.order_n[np - 1] == groups) ? t.d_order[np - 1]
                                                                             : nullptr;
  }
  return bhg::launch_walk(s, ctx->opt, t.nb, t.d_rec, t.d_mom, t.d_qrec, t.d_q64, t.d_blk,
                          t.d_orig, field_args(t), G, out, n_int, n_test, n_leaf, shape);
}

bh_status bh_create(bh_ctx **out, const bh_options *opt, int device, void *cuda_stream) {
  if (!out) return BH_ERR_ARG;
  *out = nullptr;
  bh_options o;
  bh_default_options(&o);
  if (opt) o = *opt;
  if ((o.precision != BH_PREC_F32 && o.precision != BH_PREC_F64) ||
      (o.criterion != BH_CRIT_PER_CELL && o.criterion != BH_CRIT_WARP_VOTE) ||
      (o.kahan != 0 && o.kahan != 1) || (o.quadrupole != 0 && o.quadrupole != 1) ||
      (o.learned < 0 || o.learned > 2) || (o.timing != 0 && o.timing != 1) ||
      (o.periodic != 0 && o.periodic != 1))
    return BH_ERR_ARG;
  // periodic boundaries: the binary32 per-cell walk with monopole terms
  if (o.periodic && (o.precision != BH_PREC_F32 || o.criterion != BH_CRIT_PER_CELL ||
                     o.quadrupole || o.learned))
    return BH_ERR_ARG;
  // the learned walk is the binary32 per-cell walk, with the network in place
  // of the quadrupole term
  if (o.learned && (o.precision != BH_PREC_F32 || o.criterion != BH_CRIT_PER_CELL ||
                    o.quadrupole))
    return BH_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return device < 0 ? BH_ERR_ARG : BH_ERR_CUDA;
  }
  bh_ctx *ctx = new (std::nothrow) bh_ctx();
  if (!ctx) return BH_ERR_OOM;
  ctx->opt = o;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaSetDevice(device) != cudaSuccess || bhg::prepare_learned_kernels() != cudaSuccess ||
      bhg::prepare_mlp_tc_kernel() != cudaSuccess ||
      bhg::prepare_learned_tc_kernel() != cudaSuccess ||
      bhg::dev_malloc(&ctx->tree.d_flags, 8 * sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&ctx->tree.h_flags, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->tree.d_flags) cudaFree(ctx->tree.d_flags);
    if (ctx->tree.h_flags) cudaFreeHost(ctx->tree.h_flags);
    delete ctx;
    return BH_ERR_CUDA;
  }
  if (o.periodic) {
    const bh_status st = set_ewald(ctx, kEwaldGrid, kEwaldSeries);
    if (st != BH_OK) {
      bh_destroy(ctx);
      return st;
    }
  }
  *out = ctx;
  return BH_OK;
}

bh_status bh_build(bh_ctx *ctx, int nblocks, const int32_t *level, const int32_t *ijk,
                   const double *box_lo, double box_len, const void *density,
                   int density_is_fp64) {
  const Range range_("bh_build");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (nblocks <= 0) {
    ctx->tree.built = false;
    return fail(ctx, BH_ERR_ARG, "bh_build: nblocks must be >= 1 and pointers non-null");
  }
  const int32_t nb = nblocks;
  return build_fields(ctx, 1, &nb, level, ijk, box_lo, &box_len, density, density_is_fp64,
                      "bh_build");
}

bh_status bh_build_batch(bh_ctx *ctx, int nfields, const int32_t *nblocks, const int32_t *level,
                         const int32_t *ijk, const double *box_lo, const double *box_len,
                         const void *density, int density_is_fp64) {
  const Range range_("bh_build_batch");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  return build_fields(ctx, nfields, nblocks, level, ijk, box_lo, box_len, density,
                      density_is_fp64, "bh_build_batch");
}

bh_status bh_update_density(bh_ctx *ctx, const void *density, int density_is_fp64) {
  const Range range_("bh_update_density");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (!ctx->tree.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!density || (density_is_fp64 != 0 && density_is_fp64 != 1))
    return fail(ctx, BH_ERR_ARG, "bh_update_density: bad density");
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  ctx->build_timed = false;
  const bool timed = timing_mark(ctx, 0);
  BH_CUDA(cudaMemsetAsync(ctx->tree.d_flags, 0, sizeof(unsigned), ctx->stream));
  // the records are rewritten (s2 included, and delta changes with the
  // density), with s2 for the last walk's theta if there was one
  const float inv_theta = ctx->tree.last_inv_theta;
  ctx->tree.s2_inv_theta = inv_theta > 0.0f ? inv_theta : -1.0f;
  st = enqueue_moments(ctx, density, density_is_fp64);
  ctx->build_timed = st == BH_OK && timed && timing_mark(ctx, 1);
  return st;
}

bh_status bh_sync_status(bh_ctx *ctx) {
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  bhg::Tree &t = ctx->tree;
  BH_CUDA(cudaMemcpyAsync(t.h_flags, t.d_flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost,
                          ctx->stream));
  BH_CUDA(cudaStreamSynchronize(ctx->stream));
  if (t.h_flags[0] & bhg::kErrDensity)
    return fail(ctx, BH_ERR_ARG, "density has a negative or non-finite value");
  if (t.h_flags[0] & bhg::kErrTimeout)
    return fail(ctx, BH_ERR_DEVICE_TIMEOUT, "a bounded wait for the tensor core gave up");
  if (t.h_flags[0] & ~bhg::kErrDensity)
    return fail(ctx, BH_ERR_GEOMETRY, "device error flags 0x%x", t.h_flags[0]);
  return BH_OK;
}

static bh_status prepare(bh_ctx *ctx, double theta);

}  // extern "C"

namespace bhg {
bh_status ctx_fail(bh_ctx *c, bh_status st, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return st;
}
bh_status ctx_prepare(bh_ctx *ctx, double theta) { return prepare(ctx, theta); }
}  // namespace bhg

extern "C" {

static bh_status prepare(bh_ctx *ctx, double theta) {
  bhg::Tree &t = ctx->tree;
  if (!t.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!(theta > 0.0) || !(theta <= 1.0))
    return fail(ctx, BH_ERR_ARG, "theta must lie in (0, 1], got %g", theta);
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const float inv_theta = (float)(1.0 / theta);
  t.last_inv_theta = inv_theta;
  if (inv_theta != t.s2_inv_theta) {
    BH_CUDA(bhg::launch_prepare_s2(ctx->stream, t.n_nodes, t.d_aux, t.d_rec, inv_theta));
    t.s2_inv_theta = inv_theta;
  }
  return BH_OK;
}

bh_status bh_potential(bh_ctx *ctx, double theta, double G, void *out) {
  const Range range_("bh_potential");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (!ctx->tree.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!out) return fail(ctx, BH_ERR_ARG, "bh_potential: out is null");
  if (!std::isfinite(G)) return fail(ctx, BH_ERR_ARG, "bh_potential: G must be finite");
  if (ctx->opt.learned && !ctx->d_mlp)
    return fail(ctx, BH_ERR_STATE, "learned walk: call bh_set_mlp first");
  ctx->potential_timed = false;
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const bool timed = timing_mark(ctx, 2);
  if ((st = prepare(ctx, theta)) != BH_OK) return st;
  BH_CUDA(enqueue_walk(ctx, ctx->stream, G, out, nullptr, nullptr, nullptr, ctx->tree.shape));
  ctx->potential_timed = timed && timing_mark(ctx, 3);
  ctx->last_theta = theta;
  return BH_OK;
}

bh_status bh_walk_counts(bh_ctx *ctx, double theta, int32_t *n_int, int32_t *n_test,
                         int32_t *n_cell) {
  const Range range_("bh_walk_counts");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (!ctx->tree.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!n_int || !n_test) return fail(ctx, BH_ERR_ARG, "bh_walk_counts: null output");
  bh_status st = prepare(ctx, theta);
  if (st != BH_OK) return st;
  bhg::Tree &t = ctx->tree;
  BH_CUDA(enqueue_walk(ctx, ctx->stream, 0.0, nullptr, n_int, n_test, n_cell, t.shape));
  // totals for bh_stats
  ctx->counts_valid = false;
  if (!ctx->d_counts) BH_CUDA(bhg::dev_malloc(&ctx->d_counts, 3 * sizeof(unsigned long long)));
  BH_CUDA(cudaMemsetAsync(ctx->d_counts, 0, 3 * sizeof(unsigned long long), ctx->stream));
  const int64_t ncell = (int64_t)t.nb * bhg::kCellsPerBlock;
  k_sum_counts<<<4 * 152, 256, 0, ctx->stream>>>(ncell, n_int, n_test, n_cell, ctx->d_counts);
  BH_CUDA(cudaGetLastError());
  ctx->counts_valid = true;
  ctx->counts_have_cells = n_cell != nullptr;
  return BH_OK;
}

bh_status bh_tree_size(const bh_ctx *ctx, int64_t *n_cells, int64_t *n_nodes, int *max_level) {
  if (!ctx) return BH_ERR_ARG;
  if (!ctx->tree.built) return BH_ERR_STATE;
  if (n_cells) *n_cells = (int64_t)ctx->tree.nb * bhg::kCellsPerBlock;
  if (n_nodes) *n_nodes = ctx->tree.n_nodes;
  if (max_level) *max_level = ctx->tree.max_block_level + 3;
  return BH_OK;
}

namespace {
__global__ void k_export(int64_t n, const double4_32a *mom, const bhg::WalkRec *rec, const float2 *aux,
                         const uint8_t *lvl, double *M, double *R, float *delta, int32_t *skip,
                         int32_t *level) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a m = mom[i];
  if (M) M[i] = m.w;
  if (R) {
    R[3 * i] = m.x;
    R[3 * i + 1] = m.y;
    R[3 * i + 2] = m.z;
  }
  if (delta) delta[i] = aux[i].y;
  if (skip) skip[i] = (int32_t)rec[i].skip;
  if (level) level[i] = lvl[i];
}
}  // namespace

namespace {
// Quadrupoles are stored for internal nodes only; cells (node side 0) get
// zeros.  FP64 values if they were built (FP64 walk), else the binary32 ones.
// Nodes [i0, i1) of one field, whose binary32 mass unit is 2^e.
__global__ void k_export_quad(int64_t i0, int64_t i1, const double *q64,
                              const bhg::WalkQuad *qrec, const float2 *aux,
                              const unsigned long long *mmax, int field, double *Q) {
  const int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= i1) return;
  const bool cell = aux[i].x == 0.0f;
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (!cell && q64) {
    for (int a = 0; a < 6; ++a) v[a] = q64[6 * i + a];
  } else if (!cell) {  // binary32 record in the field's mass unit 2^e
    const bhg::WalkQuad w = qrec[i];
    const double u = bhg::pow2i(bhg::mass_exponent(mmax[field]));
    v[0] = 2.0 * w.hxx * u;
    v[1] = 2.0 * w.hyy * u;
    v[2] = 2.0 * w.hzz * u;
    v[3] = w.qxy * u;
    v[4] = w.qxz * u;
    v[5] = w.qyz * u;
  }
  for (int a = 0; a < 6; ++a) Q[6 * i + a] = v[a];
}
}  // namespace

bh_status bh_export_nodes(const bh_ctx *cctx, double *M, double *R, float *delta, int32_t *skip,
                          int32_t *level) {
  bh_ctx *ctx = const_cast<bh_ctx *>(cctx);
  if (!ctx) return BH_ERR_ARG;
  if (!ctx->tree.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const bhg::Tree &t = ctx->tree;
  const int threads = 256;
  k_export<<<(unsigned)((t.n_nodes + threads - 1) / threads), threads, 0, ctx->stream>>>(
      t.n_nodes, t.d_mom, t.d_rec, t.d_aux, t.d_lvl, M, R, delta, skip, level);
  BH_CUDA(cudaGetLastError());
  return BH_OK;
}

bh_status bh_export_quadrupoles(const bh_ctx *cctx, double *Q) {
  bh_ctx *ctx = const_cast<bh_ctx *>(cctx);
  if (!ctx) return BH_ERR_ARG;
  if (!ctx->tree.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!ctx->opt.quadrupole && !ctx->opt.learned)
    return fail(ctx, BH_ERR_STATE, "the context was created without the quadrupole option");
  if (!Q) return fail(ctx, BH_ERR_ARG, "bh_export_quadrupoles: Q is null");
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const int threads = 256;
  const bhg::Tree &t = ctx->tree;
  for (int f = 0; f < t.nfields; ++f) {
    const int64_t i0 = t.h_fnode[f], i1 = t.h_fnode[f + 1];
    k_export_quad<<<(unsigned)((i1 - i0 + threads - 1) / threads), threads, 0, ctx->stream>>>(
        i0, i1, t.d_q64, t.d_qrec, t.d_aux, t.d_mmax, f, Q);
    BH_CUDA(cudaGetLastError());
  }
  return BH_OK;
}

// The walk order of the groups for one and for two target pairs per lane,
// longest walk first: one walk of the tree at the prepared theta on the
// persistent grid (4-warp CTAs, one group per take; the periodic walk: its
// plain grid of 4-warp CTAs, one pair per lane) records the SM clock
// cycles of each group's walk, under the load of a whole launch; the groups
// are sorted by them on the host (stable, so equal times keep their Morton
// order) and the order goes up.  The persistent walk then starts the long
// walks first and ends with the short ones, and the plain grid's CTAs
// (issued in index order) do the same.  Only bh_autotune does this; the
// potentials it writes to the scratch output are not used.
static bh_status make_walk_order(bh_ctx *ctx, int npairs) {
  bhg::Tree &t = ctx->tree;
  for (int np = 1; np <= npairs; ++np) {
    const int64_t groups = (int64_t)t.nb * (8 / np);
    std::vector<unsigned long long> cyc;
    try {
      cyc.resize(groups);
    } catch (const std::bad_alloc &) {
      return fail(ctx, BH_ERR_OOM, "bh_autotune: no host memory for the group times");
    }
    unsigned long long *d_cyc = nullptr;
    BH_CUDA(bhg::dev_malloc(&d_cyc, (size_t)groups * sizeof(unsigned long long)));
    bhg::WalkShape sh;
    sh.warps = 4;
    sh.pairs = np;
    sh.ticket = 1;
    sh.cycles = d_cyc;
    cudaError_t e = enqueue_walk(ctx, ctx->stream, 1.0, t.d_stage_out, nullptr, nullptr, nullptr,
                                 sh);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cyc.data(), d_cyc, (size_t)groups * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    release(d_cyc);
    BH_CUDA(e);
    std::vector<unsigned> order(groups);
    for (int64_t g = 0; g < groups; ++g) order[g] = (unsigned)g;
    std::stable_sort(order.begin(), order.end(),
                     [&](unsigned a, unsigned b) { return cyc[a] > cyc[b]; });
    unsigned *&d = t.d_order[np - 1];
    if (t.order_cap[np - 1] < groups) {
      release(d);
      t.order_cap[np - 1] = 0;
      t.order_n[np - 1] = 0;
      BH_CUDA(bhg::dev_malloc(&d, (size_t)groups * sizeof(unsigned)));
      t.order_cap[np - 1] = groups;
    }
    BH_CUDA(cudaMemcpyAsync(d, order.data(), (size_t)groups * sizeof(unsigned),
                            cudaMemcpyHostToDevice, ctx->stream));
    BH_CUDA(cudaStreamSynchronize(ctx->stream));  // the host vector goes out of scope
    t.order_n[np - 1] = groups;
  }
  return BH_OK;
}

bh_status bh_autotune(bh_ctx *ctx, double theta, int *shape) {
  const Range range_("bh_autotune");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  bh_status st = prepare(ctx, theta);
  if (st != BH_OK) return st;
  bhg::Tree &t = ctx->tree;
  const bool tunable = ctx->opt.precision == BH_PREC_F32 &&
                       ctx->opt.criterion == BH_CRIT_PER_CELL && !ctx->opt.learned;
  // the periodic walk has one target pair per lane and a plain grid: its CTA
  // width and the octants' order are tuned
  const int npairs = ctx->opt.periodic ? 1 : 2;
  if (tunable) {
    const int64_t out_bytes = (int64_t)t.nb * bhg::kCellsPerBlock * sizeof(float);
    if (t.stage_out_bytes < out_bytes) {
      release(t.d_stage_out);
      t.stage_out_bytes = 0;
      BH_CUDA(bhg::dev_malloc(&t.d_stage_out, out_bytes));
      t.stage_out_bytes = out_bytes;
    }
    if ((st = make_walk_order(ctx, npairs)) != BH_OK) return st;
    struct Events {  // released on every return
      cudaEvent_t e[2] = {nullptr, nullptr};
      ~Events() {
        for (cudaEvent_t x : e)
          if (x) cudaEventDestroy(x);
      }
    } ev;
    BH_CUDA(cudaEventCreate(&ev.e[0]));
    BH_CUDA(cudaEventCreate(&ev.e[1]));
    const int cand[4] = {2, 4, 8, 16};
    const int tickets[4] = {0, 1, 2, 4};  // plain grid, or persistent with 1/2/4 groups a grab
    const int nticket = ctx->opt.periodic ? 1 : 4;
    std::vector<bhg::WalkShape> shapes;
    for (int np = 1; np <= npairs; ++np)
      for (int ti = 0; ti < nticket * 4 * 2; ++ti) {  // CTA width x schedule x order
        bhg::WalkShape sh;
        sh.warps = cand[ti % 4];
        sh.pairs = np;
        sh.ticket = tickets[(ti / 4) % nticket];
        sh.longest = ti / (4 * nticket);
        shapes.push_back(sh);
      }
    // the shortest of `reps` more walks in shape k, into tmin[k]
    std::vector<float> tmin(shapes.size(), 1e30f);
    auto time_shape = [&](size_t k, int reps) -> cudaError_t {
      for (int rep = 0; rep < reps; ++rep) {
        cudaError_t e = cudaEventRecord(ev.e[0], ctx->stream);
        if (e == cudaSuccess)
          e = enqueue_walk(ctx, ctx->stream, 1.0, t.d_stage_out, nullptr, nullptr, nullptr,
                           shapes[k]);
        if (e == cudaSuccess) e = cudaEventRecord(ev.e[1], ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev.e[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]);
        if (e != cudaSuccess) return e;
        tmin[k] = ms < tmin[k] ? ms : tmin[k];
      }
      return cudaSuccess;
    };
    // every shape twice, then the four fastest five times more: the pick
    // is the shortest walk seen, of shapes that were all timed seven times
    for (size_t k = 0; k < shapes.size(); ++k) BH_CUDA(time_shape(k, 2));
    std::vector<size_t> rank(shapes.size());
    for (size_t k = 0; k < rank.size(); ++k) rank[k] = k;
    std::stable_sort(rank.begin(), rank.end(), [&](size_t a, size_t b) { return tmin[a] < tmin[b]; });
    const size_t finalists = rank.size() < 4 ? rank.size() : 4;
    for (size_t i = 0; i < finalists; ++i) BH_CUDA(time_shape(rank[i], 5));
    size_t pick = rank[0];
    for (size_t i = 1; i < finalists; ++i)
      if (tmin[rank[i]] < tmin[pick]) pick = rank[i];
    const bhg::WalkShape best_s = shapes[pick];
    t.shape = best_s;
    drop_graph(t);
  }
  if (shape) {
    shape[0] = tunable ? t.shape.warps : 0;
    shape[1] = tunable ? t.shape.pairs : 0;
    shape[2] = tunable ? t.shape.ticket : 0;
    shape[3] = tunable ? t.shape.longest : 0;
  }
  return BH_OK;
}

bh_status bh_set_walk_shape(bh_ctx *ctx, int warps_per_cta, int pairs_per_lane,
                            int groups_per_take, int longest_first) {
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (!(warps_per_cta == 0 || (warps_per_cta >= 1 && warps_per_cta <= 16)) ||
      !(pairs_per_lane >= 0 && pairs_per_lane <= 2) ||
      !(groups_per_take >= 0 && groups_per_take <= 64) ||
      (longest_first != 0 && longest_first != 1))
    return fail(ctx, BH_ERR_ARG,
                "bh_set_walk_shape: warps 0..16, pairs 0..2, groups 0..64, longest_first 0/1");
  if (ctx->opt.periodic && (pairs_per_lane > 1 || groups_per_take > 0))
    return fail(ctx, BH_ERR_ARG, "bh_set_walk_shape: the periodic walk has one pair per lane "
                                 "and a plain grid");
  const int np = pairs_per_lane > 0 ? pairs_per_lane : 1;
  if (longest_first && ctx->tree.order_n[np - 1] == 0)
    return fail(ctx, BH_ERR_STATE, "bh_set_walk_shape: no walk order (run bh_autotune first)");
  ctx->tree.shape.warps = warps_per_cta;
  ctx->tree.shape.pairs = pairs_per_lane;
  ctx->tree.shape.ticket = groups_per_take;
  ctx->tree.shape.longest = longest_first;
  drop_graph(ctx->tree);  // a captured walk holds the old shape
  return BH_OK;
}

bh_status bh_solve_graph(bh_ctx *ctx, const void *density, int density_is_fp64, double theta,
                         double G, void *out) {
  const Range range_("bh_solve_graph");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  bhg::Tree &t = ctx->tree;
  if (!t.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build or bh_build_batch first");
  if (!density || !out || (density_is_fp64 != 0 && density_is_fp64 != 1))
    return fail(ctx, BH_ERR_ARG, "bh_solve_graph: null buffer or bad density type");
  if (!(theta > 0.0) || !(theta <= 1.0) || !std::isfinite(G))
    return fail(ctx, BH_ERR_ARG, "bh_solve_graph: theta must lie in (0, 1] and G be finite");
  if (!ctx->stream)
    return fail(ctx, BH_ERR_ARG, "bh_solve_graph: needs a context on a created (non-default) "
                                 "CUDA stream");
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const bool same = t.graph_exec && t.graph_density == density && t.graph_out == out &&
                    t.graph_fp64 == density_is_fp64 && t.graph_theta == theta && t.graph_G == G;
  if (!same) {
    drop_graph(t);
    if (t.shape.warps == 0 && (st = bh_autotune(ctx, theta, nullptr)) != BH_OK) return st;
    cudaStream_t s = ctx->stream;
    BH_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    bh_status cap = BH_OK;
    cudaError_t e = cudaMemsetAsync(t.d_flags, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
      cap = enqueue_moments(ctx, density, density_is_fp64);
      if (cap == BH_OK)
        e = bhg::launch_prepare_s2(s, t.n_nodes, t.d_aux, t.d_rec, (float)(1.0 / theta));
      if (cap == BH_OK && e == cudaSuccess && ctx->opt.learned && !ctx->d_mlp)
        cap = fail(ctx, BH_ERR_STATE, "learned walk: call bh_set_mlp first");
      if (cap == BH_OK && e == cudaSuccess)
        e = enqueue_walk(ctx, s, G, out, nullptr, nullptr, nullptr, t.shape);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &g);
    if (cap != BH_OK || e != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return cap != BH_OK ? cap
                          : fail(ctx, BH_ERR_CUDA, "bh_solve_graph: capture failed: %s",
                                 cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    t.graph = g;
    BH_CUDA(cudaGraphInstantiate(&t.graph_exec, t.graph, 0));
    t.graph_density = density;
    t.graph_out = out;
    t.graph_fp64 = density_is_fp64;
    t.graph_theta = theta;
    t.graph_G = G;
  }
  BH_CUDA(cudaGraphLaunch(t.graph_exec, ctx->stream));
  t.s2_inv_theta = t.last_inv_theta = (float)(1.0 / theta);
  return BH_OK;
}

bh_status bh_solve_host(bh_ctx *ctx, int nblocks, const int32_t *level, const int32_t *ijk,
                        const double *box_lo, double box_len, const void *density_host,
                        int density_is_fp64, double theta, double G, void *out_host) {
  const Range range_("bh_solve_host");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (nblocks <= 0 || !density_host || !out_host)
    return fail(ctx, BH_ERR_ARG, "bh_solve_host: nblocks >= 1 and non-null buffers required");
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  bhg::Tree &t = ctx->tree;
  const int64_t ncell = (int64_t)nblocks * bhg::kCellsPerBlock;
  const int64_t in_bytes = ncell * (density_is_fp64 ? 8 : 4);
  const int64_t out_bytes = ncell * (ctx->opt.precision == BH_PREC_F64 ? 8 : 4);
  if (t.stage_in_bytes < in_bytes) {
    release(t.d_stage_in);
    t.stage_in_bytes = 0;
    BH_CUDA(bhg::dev_malloc(&t.d_stage_in, in_bytes));
    t.stage_in_bytes = in_bytes;
  }
  // A pinned (page-locked, mapped) output buffer is written by the walk
  // itself, through its device address: on GB300 the stores cross the
  // NVLink chip-to-chip link to the Grace host memory while the walk runs,
  // instead of a copy after it.  Other output buffers get the staged copy.
  // (The density is copied in either way: read twice by the build's kernels
  // across the link, it made the call slower than one copy to HBM.)
  void *direct = nullptr;
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, out_host) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer) direct = pa.devicePointer;
  } else {
    cudaGetLastError();  // not a pointer CUDA knows: pageable memory
  }
  if (!direct && t.stage_out_bytes < out_bytes) {
    release(t.d_stage_out);
    t.stage_out_bytes = 0;
    BH_CUDA(bhg::dev_malloc(&t.d_stage_out, out_bytes));
    t.stage_out_bytes = out_bytes;
  }
  BH_CUDA(cudaMemcpyAsync(t.d_stage_in, density_host, in_bytes, cudaMemcpyHostToDevice,
                          ctx->stream));
  st = bh_build(ctx, nblocks, level, ijk, box_lo, box_len, t.d_stage_in, density_is_fp64);
  if (st != BH_OK) return st;
  st = bh_potential(ctx, theta, G, direct ? direct : t.d_stage_out);
  if (st != BH_OK) return st;
  if (!direct)
    BH_CUDA(cudaMemcpyAsync(out_host, t.d_stage_out, out_bytes, cudaMemcpyDeviceToHost,
                            ctx->stream));
  BH_CUDA(cudaStreamSynchronize(ctx->stream));
  return BH_OK;
}

bh_status bh_stats(const bh_ctx *ctx, bh_stats_t *out) {
  if (!ctx || !out) return BH_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  const bhg::Tree &t = ctx->tree;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return BH_ERR_CUDA;
  }
  out->built = t.built ? 1 : 0;
  if (t.built) {
    out->n_cells = (int64_t)t.nb * bhg::kCellsPerBlock;
    out->n_nodes = t.n_nodes;
    out->n_blocks = t.nb;
    out->n_fields = t.nfields;
    out->max_level = t.max_block_level + 3;
  }
  out->last_theta = ctx->last_theta;
  out->build_ms = out->potential_ms = -1.0;
  float ms = 0.0f;
  if (ctx->build_timed && cudaEventSynchronize(ctx->ev[1]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]) == cudaSuccess)
    out->build_ms = ms;
  if (ctx->potential_timed && cudaEventSynchronize(ctx->ev[3]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]) == cudaSuccess)
    out->potential_ms = ms;
  cudaGetLastError();
  out->interactions = out->tests = out->cell_interactions = -1;
  if (ctx->counts_valid) {
    unsigned long long c[3];
    if (cudaMemcpyAsync(c, ctx->d_counts, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
      cudaGetLastError();
      return BH_ERR_CUDA;
    }
    out->interactions = (int64_t)c[0];
    out->tests = (int64_t)c[1];
    out->cell_interactions = ctx->counts_have_cells ? (int64_t)c[2] : -1;
  }
  // per block: level, ijk, 2 keys, 2 indices, count, prestart, blk, orig, fid,
  // pos, fld, and 8 bytes of top-node child lists
  int64_t b = t.nb_cap * (int64_t)(4 + 12 + 8 + 8 + 4 + 4 + 4 + 4 + 16 + 4 + 4 + 4 + 16 + 8);
  b += t.node_cap * (int64_t)(sizeof(double4_32a) + sizeof(bhg::WalkRec) + sizeof(float2) + 1);
  b += t.quad_cap * (int64_t)sizeof(bhg::WalkQuad) + (t.d_q64 ? t.quad_cap * 48 : 0);
  b += t.nf_cap * (int64_t)(sizeof(int) + 2 * sizeof(double)) + (t.nf_cap ? 4 : 0);
  b += t.stage_in_bytes + t.stage_out_bytes + 4 * sizeof(unsigned);
  if (ctx->d_mlp) b += sizeof(bhg::MlpDev) + sizeof(bhg::MlpTc) + sizeof(unsigned);
  if (ctx->d_counts) b += 3 * sizeof(unsigned long long);
  if (ctx->d_ewald) b += (int64_t)ctx->ewald_n * ctx->ewald_n * ctx->ewald_n * 64;
  out->device_bytes = b;
  return BH_OK;
}

bh_status bh_set_ewald(bh_ctx *ctx, int n_grid, int n_series) {
  const Range range_("bh_set_ewald");
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (n_grid < 2 || n_grid > 256 || n_series < 1 || n_series > 8)
    return fail(ctx, BH_ERR_ARG, "bh_set_ewald: n_grid in [2, 256], n_series in [1, 8]");
  return set_ewald(ctx, n_grid, n_series);
}

bh_status bh_ewald_eval(bh_ctx *ctx, int64_t n, const float *r, float *chi) {
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (!ctx->d_ewald) return fail(ctx, BH_ERR_STATE, "bh_ewald_eval: no Ewald table");
  if (n < 0 || (n > 0 && (!r || !chi)))
    return fail(ctx, BH_ERR_ARG, "bh_ewald_eval: bad size or null buffer");
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  BH_CUDA(bhg::launch_ewald_eval(ctx->stream, n, r, ctx->d_ewald, ctx->ewald_n, chi));
  return BH_OK;
}

const char *bh_last_error(const bh_ctx *ctx) { return ctx ? ctx->err : "null context"; }

void bh_destroy(bh_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  drop_graph(ctx->tree);
  free_blocks(ctx->tree);
  free_nodes(ctx->tree);
  free_fields(ctx->tree);
  release(ctx->tree.d_stage_in);
  release(ctx->tree.d_stage_out);
  release(ctx->tree.d_flags);
  release(ctx->tree.d_order[0]);
  release(ctx->tree.d_order[1]);
  release(ctx->d_mlp);
  release(ctx->d_mlp_tc);
  release(ctx->d_tc_flag);
  release(ctx->d_counts);
  release(ctx->d_ewald);
  for (cudaEvent_t &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->tree.h_flags) cudaFreeHost(ctx->tree.h_flags);
  if (ctx->tree.geo_done) cudaEventDestroy(ctx->tree.geo_done);
  delete ctx;
}

}  // extern "C"
