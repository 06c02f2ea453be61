// C-ABI of libbhgrav: argument checking, buffer ownership and the order of
// the build and walk launches.  The arithmetic lives in bh_build.cu and
// bh_walk.cu; this file holds no kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "bh_internal.cuh"

struct bh_ctx {
  bh_options opt;
  int device = 0;
  cudaStream_t stream = nullptr;
  bhg::Tree tree;
  char err[512] = {0};
};

namespace {

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
  release(t.d_level);
  release(t.d_ijk);
  release(t.d_key[0]);
  release(t.d_key[1]);
  release(t.d_idx[0]);
  release(t.d_idx[1]);
  release(t.d_count);
  release(t.d_prestart);
  release(t.d_blk);
  release(t.d_orig);
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
  BH_CUDA(cudaMalloc(&t.d_level, n * sizeof(int)));
  BH_CUDA(cudaMalloc(&t.d_ijk, 3 * n * sizeof(int)));
  BH_CUDA(cudaMalloc(&t.d_key[0], n * sizeof(unsigned long long)));
  BH_CUDA(cudaMalloc(&t.d_key[1], n * sizeof(unsigned long long)));
  BH_CUDA(cudaMalloc(&t.d_idx[0], n * sizeof(int)));
  BH_CUDA(cudaMalloc(&t.d_idx[1], n * sizeof(int)));
  BH_CUDA(cudaMalloc(&t.d_count, n * sizeof(int)));
  BH_CUDA(cudaMalloc(&t.d_prestart, n * sizeof(int)));
  BH_CUDA(cudaMalloc(&t.d_blk, n * sizeof(int4)));
  BH_CUDA(cudaMalloc(&t.d_orig, n * sizeof(int)));
  t.nb_cap = nb;
  return BH_OK;
}

bh_status ensure_nodes(bh_ctx *ctx, int64_t n_nodes) {
  bhg::Tree &t = ctx->tree;
  const bool quad = ctx->opt.quadrupole != 0;
  const bool quad64 = quad && ctx->opt.precision == BH_PREC_F64;
  if (t.node_cap >= n_nodes && (!quad || t.quad_cap >= n_nodes)) return BH_OK;
  free_nodes(t);
  if (quad) {
    if (quad64) BH_CUDA(cudaMalloc(&t.d_q64, (size_t)n_nodes * 6 * sizeof(double)));
    BH_CUDA(cudaMalloc(&t.d_qrec, (size_t)n_nodes * sizeof(bhg::WalkQuad)));
    t.quad_cap = n_nodes;
  }
  const size_t n = (size_t)n_nodes;
  BH_CUDA(cudaMalloc(&t.d_mom, n * sizeof(double4_32a)));
  BH_CUDA(cudaMalloc(&t.d_rec, n * sizeof(bhg::WalkRec)));
  BH_CUDA(cudaMalloc(&t.d_aux, n * sizeof(float2)));
  BH_CUDA(cudaMalloc(&t.d_lvl, n * sizeof(uint8_t)));
  t.node_cap = n_nodes;
  return BH_OK;
}

bh_status use_device(bh_ctx *ctx) {
  BH_CUDA(cudaSetDevice(ctx->device));
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

bh_status bh_create(bh_ctx **out, const bh_options *opt, int device, void *cuda_stream) {
  if (!out) return BH_ERR_ARG;
  *out = nullptr;
  bh_options o;
  bh_default_options(&o);
  if (opt) o = *opt;
  if ((o.precision != BH_PREC_F32 && o.precision != BH_PREC_F64) ||
      (o.criterion != BH_CRIT_PER_CELL && o.criterion != BH_CRIT_WARP_VOTE) ||
      (o.kahan != 0 && o.kahan != 1) || (o.quadrupole != 0 && o.quadrupole != 1))
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
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaMalloc(&ctx->tree.d_flags, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&ctx->tree.h_flags, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->tree.d_flags) cudaFree(ctx->tree.d_flags);
    if (ctx->tree.h_flags) cudaFreeHost(ctx->tree.h_flags);
    delete ctx;
    return BH_ERR_CUDA;
  }
  *out = ctx;
  return BH_OK;
}

bh_status bh_build(bh_ctx *ctx, int nblocks, const int32_t *level, const int32_t *ijk,
                   const double *box_lo, double box_len, const void *density,
                   int density_is_fp64) {
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  bhg::Tree &t = ctx->tree;
  t.built = false;
  if (nblocks <= 0 || !level || !ijk || !box_lo || !density)
    return fail(ctx, BH_ERR_ARG, "bh_build: nblocks must be >= 1 and pointers non-null");
  if (!(box_len > 0.0) || !std::isfinite(box_len) || !std::isfinite(box_lo[0]) ||
      !std::isfinite(box_lo[1]) || !std::isfinite(box_lo[2]))
    return fail(ctx, BH_ERR_ARG, "bh_build: box_len must be finite and > 0, box_lo finite");
  if (density_is_fp64 != 0 && density_is_fp64 != 1)
    return fail(ctx, BH_ERR_ARG, "bh_build: density_is_fp64 must be 0 or 1");
  // a tiling has nb = 1 + 7k blocks; node count must fit a 32-bit index
  if ((nblocks - 1) % 7 != 0)
    return fail(ctx, BH_ERR_GEOMETRY, "bh_build: %d blocks cannot tile a cube (need 1 + 7k)",
                nblocks);
  const int64_t n_nodes = (int64_t)bhg::kNodesPerBlock * nblocks + (nblocks - 1) / 7;
  if (n_nodes >= (int64_t)0x7fffffff)
    return fail(ctx, BH_ERR_ARG, "bh_build: %d blocks exceed the 2^31 node limit", nblocks);
  int max_level = 0;
  for (int b = 0; b < nblocks; ++b) {
    if (level[b] < 0 || level[b] > bhg::kMaxBlockLevel)
      return fail(ctx, BH_ERR_GEOMETRY, "bh_build: block %d has level %d outside [0, 18]", b,
                  level[b]);
    max_level = level[b] > max_level ? level[b] : max_level;
  }
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  if ((st = ensure_blocks(ctx, nblocks)) != BH_OK) return st;
  if ((st = ensure_nodes(ctx, n_nodes)) != BH_OK) return st;
  cudaStream_t s = ctx->stream;
  const int nb = nblocks;
  // FP64 quadrupoles for the FP64 walk, binary32 ones for the binary32 walk
  double *q64 = ctx->opt.quadrupole && ctx->opt.precision == BH_PREC_F64 ? t.d_q64 : nullptr;
  bhg::WalkQuad *qrec = ctx->opt.quadrupole ? t.d_qrec : nullptr;
  BH_CUDA(cudaMemsetAsync(t.d_flags, 0, 4 * sizeof(unsigned), s));
  BH_CUDA(cudaMemcpyAsync(t.d_level, level, nb * sizeof(int), cudaMemcpyHostToDevice, s));
  BH_CUDA(cudaMemcpyAsync(t.d_ijk, ijk, 3 * (size_t)nb * sizeof(int), cudaMemcpyHostToDevice, s));
  BH_CUDA(bhg::launch_block_keys(s, nb, t.d_level, t.d_ijk, t.d_key[0], t.d_idx[0], t.d_flags));
  BH_CUDA(bhg::launch_sort_blocks(s, nb, t.d_key, t.d_idx, t.d_flags, nullptr));
  BH_CUDA(bhg::launch_tile_and_count(s, nb, t.d_key[0], t.d_idx[0], t.d_level, t.d_ijk,
                                     t.d_count, t.d_blk, t.d_orig, t.d_flags));
  BH_CUDA(bhg::launch_prestart_scan(s, nb, t.d_count, t.d_prestart, t.d_flags));
  BH_CUDA(bhg::launch_top_nodes(s, nb, t.d_key[0], t.d_blk, t.d_count, t.d_prestart, n_nodes,
                                t.d_rec, t.d_aux, t.d_lvl, t.d_flags));
  BH_CUDA(bhg::launch_blocks(s, nb, t.d_blk, t.d_orig, t.d_count, t.d_prestart, density,
                             density_is_fp64, box_len, n_nodes, t.d_mom, t.d_rec, t.d_aux,
                             t.d_lvl, q64, qrec, t.d_flags));
  for (int lev = max_level - 1; lev >= 0; --lev)
    BH_CUDA(bhg::launch_top_moments(s, nb, lev, t.d_key[0], t.d_blk, t.d_count, t.d_prestart,
                                    n_nodes, t.d_mom, t.d_rec, t.d_aux, q64, qrec, t.d_flags));
  BH_CUDA(cudaMemcpyAsync(t.h_flags, t.d_flags, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  BH_CUDA(cudaStreamSynchronize(s));
  const unsigned e = t.h_flags[0];
  if (e & (bhg::kErrLevel | bhg::kErrCoord))
    return fail(ctx, BH_ERR_GEOMETRY, "bh_build: a block coordinate lies outside its level");
  if (e & bhg::kErrTiling)
    return fail(ctx, BH_ERR_GEOMETRY, "bh_build: the blocks do not tile the box (gap or overlap)");
  if ((int64_t)t.h_flags[2] != (nb - 1) / 7 || (e & bhg::kErrIndex))
    return fail(ctx, BH_ERR_GEOMETRY, "bh_build: inconsistent block tree (%u internal nodes)",
                t.h_flags[2]);
  if (e & bhg::kErrDensity)
    return fail(ctx, BH_ERR_ARG, "bh_build: density has a negative or non-finite value");
  t.nb = nb;
  t.max_block_level = max_level;
  t.n_nodes = n_nodes;
  for (int a = 0; a < 3; ++a) t.lo[a] = box_lo[a];
  t.L = box_len;
  t.s2_inv_theta = -1.0f;
  t.built = true;
  return BH_OK;
}

static bh_status prepare(bh_ctx *ctx, double theta) {
  bhg::Tree &t = ctx->tree;
  if (!t.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!(theta > 0.0) || !(theta <= 1.0))
    return fail(ctx, BH_ERR_ARG, "theta must lie in (0, 1], got %g", theta);
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const float inv_theta = (float)(1.0 / theta);
  if (inv_theta != t.s2_inv_theta) {
    BH_CUDA(bhg::launch_prepare_s2(ctx->stream, t.n_nodes, t.d_aux, t.d_rec, inv_theta));
    t.s2_inv_theta = inv_theta;
  }
  return BH_OK;
}

bh_status bh_potential(bh_ctx *ctx, double theta, double G, void *out) {
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (!ctx->tree.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!out) return fail(ctx, BH_ERR_ARG, "bh_potential: out is null");
  if (!std::isfinite(G)) return fail(ctx, BH_ERR_ARG, "bh_potential: G must be finite");
  bh_status st = prepare(ctx, theta);
  if (st != BH_OK) return st;
  bhg::Tree &t = ctx->tree;
  const double scale = -G / t.L;
  BH_CUDA(bhg::launch_walk(ctx->stream, ctx->opt, t.nb, t.n_nodes, t.d_rec, t.d_mom, t.d_qrec,
                           t.d_q64, t.d_blk, t.d_orig, scale, out, nullptr, nullptr));
  return BH_OK;
}

bh_status bh_walk_counts(bh_ctx *ctx, double theta, int32_t *n_int, int32_t *n_test,
                         int32_t *n_cell) {
  if (!ctx) return BH_ERR_ARG;
  ctx->err[0] = 0;
  if (!ctx->tree.built) return fail(ctx, BH_ERR_STATE, "no tree: call bh_build first");
  if (!n_int || !n_test) return fail(ctx, BH_ERR_ARG, "bh_walk_counts: null output");
  bh_status st = prepare(ctx, theta);
  if (st != BH_OK) return st;
  bhg::Tree &t = ctx->tree;
  BH_CUDA(bhg::launch_walk(ctx->stream, ctx->opt, t.nb, t.n_nodes, t.d_rec, t.d_mom, t.d_qrec,
                           t.d_q64, t.d_blk, t.d_orig, 0.0, nullptr, n_int, n_test,
                           n_cell));
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
__global__ void k_export_quad(int64_t n, const double *q64, const bhg::WalkQuad *qrec,
                              const float2 *aux, double *Q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool cell = aux[i].x == 0.0f;
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (!cell && q64) {
    for (int a = 0; a < 6; ++a) v[a] = q64[6 * i + a];
  } else if (!cell) {
    const bhg::WalkQuad w = qrec[i];
    v[0] = 2.0 * w.hxx;
    v[1] = 2.0 * w.hyy;
    v[2] = 2.0 * w.hzz;
    v[3] = w.qxy;
    v[4] = w.qxz;
    v[5] = w.qyz;
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
  if (!ctx->opt.quadrupole)
    return fail(ctx, BH_ERR_STATE, "the context was created without the quadrupole option");
  if (!Q) return fail(ctx, BH_ERR_ARG, "bh_export_quadrupoles: Q is null");
  bh_status st = use_device(ctx);
  if (st != BH_OK) return st;
  const int threads = 256;
  k_export_quad<<<(unsigned)((ctx->tree.n_nodes + threads - 1) / threads), threads, 0,
                  ctx->stream>>>(ctx->tree.n_nodes, ctx->tree.d_q64, ctx->tree.d_qrec,
                                 ctx->tree.d_aux, Q);
  BH_CUDA(cudaGetLastError());
  return BH_OK;
}

bh_status bh_solve_host(bh_ctx *ctx, int nblocks, const int32_t *level, const int32_t *ijk,
                        const double *box_lo, double box_len, const void *density_host,
                        int density_is_fp64, double theta, double G, void *out_host) {
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
    BH_CUDA(cudaMalloc(&t.d_stage_in, in_bytes));
    t.stage_in_bytes = in_bytes;
  }
  if (t.stage_out_bytes < out_bytes) {
    release(t.d_stage_out);
    t.stage_out_bytes = 0;
    BH_CUDA(cudaMalloc(&t.d_stage_out, out_bytes));
    t.stage_out_bytes = out_bytes;
  }
  BH_CUDA(cudaMemcpyAsync(t.d_stage_in, density_host, in_bytes, cudaMemcpyHostToDevice,
                          ctx->stream));
  st = bh_build(ctx, nblocks, level, ijk, box_lo, box_len, t.d_stage_in, density_is_fp64);
  if (st != BH_OK) return st;
  st = bh_potential(ctx, theta, G, t.d_stage_out);
  if (st != BH_OK) return st;
  BH_CUDA(cudaMemcpyAsync(out_host, t.d_stage_out, out_bytes, cudaMemcpyDeviceToHost,
                          ctx->stream));
  BH_CUDA(cudaStreamSynchronize(ctx->stream));
  return BH_OK;
}

const char *bh_last_error(const bh_ctx *ctx) { return ctx ? ctx->err : "null context"; }

void bh_destroy(bh_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_blocks(ctx->tree);
  free_nodes(ctx->tree);
  release(ctx->tree.d_stage_in);
  release(ctx->tree.d_stage_out);
  release(ctx->tree.d_flags);
  if (ctx->tree.h_flags) cudaFreeHost(ctx->tree.h_flags);
  delete ctx;
}

}  // extern "C"
