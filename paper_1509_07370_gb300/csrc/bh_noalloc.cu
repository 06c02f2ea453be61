// bh_solve_noalloc: the whole solve (tree, FP64 moments, binary32 walk) for a
// small mesh without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a host code whose GPU memory is fully
// reserved up front by its own pool allocator (so a library allocation would
// fail or fragment that pool), or a caller that must not let the library
// enter the CUDA allocator at all, since cudaMalloc/cudaFree may synchronise
// the device and stall the caller's other streams.  For them the tree of one
// mesh of at most kNoAllocMaxBlocks blocks is kept in a fixed array in device
// global memory, declared below, which every GPU that loads this library
// holds until the process exits.
//
// Sharing rules: every call, from any thread and on any stream, uses the same
// array and leaves the last call's tree in it.  Calls whose work overlaps on
// the GPU race on it and corrupt each other's results, so callers must
// serialise them (one stream, or stream order between calls).  Everything a
// call reads is written by that same call first; the error flags are cleared
// at the start of each call.
//
// Set-up: the first call on a device, with that device current, looks up the
// device address of the array (cudaGetSymbolAddress) and caches it; this
// first call should come before any stream capture on that device.
//
// The kernels are the ones of bh_build / bh_potential, given pointers into
// the fixed array instead of allocated buffers.
#include <cmath>
#include <mutex>

#include "bh_internal.cuh"

namespace bhg {
namespace {

constexpr int kNoAllocMaxBlocks = 64;  // 32,768 cells
constexpr int64_t kNoAllocMaxNodes =
    (int64_t)kNodesPerBlock * kNoAllocMaxBlocks + (kNoAllocMaxBlocks - 1) / 7;
constexpr int kMaxDevices = 64;

constexpr size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffLevel = 0;
constexpr size_t kOffIjk = up256(kOffLevel + sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffKey0 = up256(kOffIjk + 3 * sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffKey1 = up256(kOffKey0 + sizeof(unsigned long long) * kNoAllocMaxBlocks);
constexpr size_t kOffIdx0 = up256(kOffKey1 + sizeof(unsigned long long) * kNoAllocMaxBlocks);
constexpr size_t kOffIdx1 = up256(kOffIdx0 + sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffCount = up256(kOffIdx1 + sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffPrestart = up256(kOffCount + sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffBlk = up256(kOffPrestart + sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffOrig = up256(kOffBlk + sizeof(int4) * kNoAllocMaxBlocks);
constexpr size_t kOffFlags = up256(kOffOrig + sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffFstart = up256(kOffFlags + 4 * sizeof(unsigned));   // one field
constexpr size_t kOffFid = up256(kOffFstart + 2 * sizeof(int));
constexpr size_t kOffFld = up256(kOffFid + sizeof(int) * kNoAllocMaxBlocks);
constexpr size_t kOffBox = up256(kOffFld + sizeof(int4) * kNoAllocMaxBlocks);  // L, 1/L
constexpr size_t kOffMmax = up256(kOffBox + 2 * sizeof(double));  // largest cell mass
constexpr size_t kOffMom = up256(kOffMmax + sizeof(unsigned long long));
constexpr size_t kOffRec = up256(kOffMom + sizeof(double4_32a) * kNoAllocMaxNodes);
constexpr size_t kOffAux = up256(kOffRec + sizeof(WalkRec) * kNoAllocMaxNodes);
constexpr size_t kOffLvl = up256(kOffAux + sizeof(float2) * kNoAllocMaxNodes);
constexpr size_t kOffTop = up256(kOffLvl + sizeof(uint8_t) * kNoAllocMaxNodes);  // TopArgs
constexpr size_t kScratchBytes = up256(kOffTop + sizeof(int) * top_ints(kNoAllocMaxBlocks));  // ~2.7 MB

// The fixed scratch.  In host code this name is only a stand-in for the
// symbol: host code must use the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Geometry {  // passed by value as a kernel parameter (1 KB)
  int level[kNoAllocMaxBlocks];
  int ijk[3 * kNoAllocMaxBlocks];
};

// Copies the block geometry from the kernel parameter into the scratch,
// describes the single field, and clears the error flags of this call.
__global__ void k_stage_geometry(Geometry g, int nb, int *level, int *ijk, unsigned *flags,
                                 int *fstart, double *box, double L, unsigned long long *mmax) {
  const int t = threadIdx.x;
  if (t < 4) flags[t] = 0u;
  if (t == 0) {
    fstart[0] = 0;
    fstart[1] = nb;
    box[0] = L;
    box[1] = 1.0 / L;
    *mmax = 0ull;
  }
  for (int i = t; i < nb; i += blockDim.x) level[i] = g.level[i];
  for (int i = t; i < 3 * nb; i += blockDim.x) ijk[i] = g.ijk[i];
}

std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once).
bh_status scratch_on_current_device(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return BH_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BH_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return BH_OK;
}

#define NA_CUDA(call)                         \
  do {                                        \
    if ((call) != cudaSuccess) {              \
      cudaGetLastError();                     \
      return BH_ERR_CUDA;                     \
    }                                         \
  } while (0)

}  // namespace
}  // namespace bhg

extern "C" bh_status bh_solve_noalloc(int nblocks, const int32_t *level, const int32_t *ijk,
                                      const double *box_lo, double box_len, const void *density,
                                      int density_is_fp64, double theta, double G, float *out,
                                      void *cuda_stream) {
  using namespace bhg;
  if (nblocks <= 0 || !level || !ijk || !box_lo || !density || !out) return BH_ERR_ARG;
  if (nblocks > kNoAllocMaxBlocks) return BH_ERR_ARG;  // beyond the fixed scratch
  if (!(box_len > 0.0) || !std::isfinite(box_len) || !(theta > 0.0) || !(theta <= 1.0) ||
      !std::isfinite(G) || (density_is_fp64 != 0 && density_is_fp64 != 1))
    return BH_ERR_ARG;
  for (int a = 0; a < 3; ++a)  // the box origin, as bh_build checks it
    if (!std::isfinite(box_lo[a])) return BH_ERR_ARG;
  if ((nblocks - 1) % 7 != 0) return BH_ERR_GEOMETRY;
  Geometry g;
  int max_level = 0;
  for (int b = 0; b < nblocks; ++b) {
    if (level[b] < 0 || level[b] > kMaxBlockLevel) return BH_ERR_GEOMETRY;
    g.level[b] = level[b];
    for (int a = 0; a < 3; ++a) g.ijk[3 * b + a] = ijk[3 * b + a];
    max_level = level[b] > max_level ? level[b] : max_level;
  }
  unsigned char *base = nullptr;
  bh_status st = scratch_on_current_device(&base);
  if (st != BH_OK) return st;
  const int nb = nblocks;
  const int64_t n_nodes = (int64_t)kNodesPerBlock * nb + (nb - 1) / 7;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int *d_level = (int *)(base + kOffLevel);
  int *d_ijk = (int *)(base + kOffIjk);
  unsigned long long *d_key[2] = {(unsigned long long *)(base + kOffKey0),
                                  (unsigned long long *)(base + kOffKey1)};
  int *d_idx[2] = {(int *)(base + kOffIdx0), (int *)(base + kOffIdx1)};
  int *d_count = (int *)(base + kOffCount);
  int *d_prestart = (int *)(base + kOffPrestart);
  int4 *d_blk = (int4 *)(base + kOffBlk);
  int *d_orig = (int *)(base + kOffOrig);
  unsigned *d_flags = (unsigned *)(base + kOffFlags);
  double4_32a *d_mom = (double4_32a *)(base + kOffMom);
  WalkRec *d_rec = (WalkRec *)(base + kOffRec);
  float2 *d_aux = (float2 *)(base + kOffAux);
  uint8_t *d_lvl = (uint8_t *)(base + kOffLvl);
  const TopArgs top = top_args((int *)(base + kOffTop), kNoAllocMaxBlocks);
  int *d_fstart = (int *)(base + kOffFstart);
  double *d_box = (double *)(base + kOffBox);
  FieldArgs fa;
  fa.nfields = 1;
  fa.fstart = d_fstart;
  fa.fid = (int *)(base + kOffFid);
  fa.fld = (int4 *)(base + kOffFld);
  fa.L = d_box;
  fa.invL = d_box + 1;
  fa.mmax = (unsigned long long *)(base + kOffMmax);
  fa.inv_theta = 0.0f;  // s2 is prepared below

  k_stage_geometry<<<1, 256, 0, s>>>(g, nb, d_level, d_ijk, d_flags, d_fstart, d_box, box_len,
                                     fa.mmax);
  NA_CUDA(cudaGetLastError());
  NA_CUDA(launch_keys_mass(s, nb, d_level, d_ijk, d_key[0], d_idx[0], d_flags, fa, density,
                           density_is_fp64));
  NA_CUDA(launch_sort_blocks(s, d_key, d_idx, d_flags, fa));
  NA_CUDA(launch_tile_and_count(s, nb, d_key[0], d_idx[0], d_level, d_ijk, d_count, d_blk,
                                d_orig, d_flags, fa, top));
  NA_CUDA(launch_prestart_scan(s, nb, d_count, d_prestart, d_flags));
  NA_CUDA(launch_top_nodes(s, nb, d_key[0], d_blk, d_count, d_prestart, n_nodes, d_rec, d_aux,
                           d_lvl, d_flags, fa, d_orig, max_level, top));
  NA_CUDA(launch_moments(s, nb, d_blk, d_orig, d_count, d_prestart, density,
                         density_is_fp64, fa, n_nodes, d_mom, d_rec, d_aux, d_lvl, nullptr, nullptr,
                         d_flags, top));
  // the walk must only run on a valid tree: check the flags first
  unsigned h_flags[4] = {0, 0, 0, 0};
  NA_CUDA(cudaMemcpyAsync(h_flags, d_flags, sizeof(h_flags), cudaMemcpyDeviceToHost, s));
  NA_CUDA(cudaStreamSynchronize(s));
  if (h_flags[0] & (kErrLevel | kErrCoord | kErrTiling | kErrIndex)) return BH_ERR_GEOMETRY;
  if ((int64_t)h_flags[2] != (nb - 1) / 7) return BH_ERR_GEOMETRY;
  if (h_flags[0] & kErrDensity) return BH_ERR_ARG;
  NA_CUDA(launch_prepare_s2(s, n_nodes, d_aux, d_rec, (float)(1.0 / theta)));
  bh_options opt;
  bh_default_options(&opt);
  NA_CUDA(launch_walk(s, opt, nb, d_rec, d_mom, nullptr, nullptr, d_blk, d_orig, fa, G, out,
                      nullptr, nullptr, nullptr, WalkShape()));
  return BH_OK;
}
