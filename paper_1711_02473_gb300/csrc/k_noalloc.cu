// k_noalloc.cu -- the p-adaptive DQ batched action for callers that cannot
// allocate device memory.
//
// sfx_plan_* allocates its tile list and tile counter with cudaMalloc when the
// plan is created.  Some callers may not allocate at the point where they
// need the action: code that runs while a memory pool owns the whole device,
// code whose allocations must all happen at start-up, or code inside a
// library that forbids allocating in its solve phase.  This entry point
// builds the same tile list on the device, into one fixed scratch array that
// lives in this file, and runs the same persistent kernel; it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The scratch array is a file-scope __device__ array: every GPU that loads the
// library holds it (about 5 MB) until the process exits.  Host code may not
// use its name as a device address (the host symbol is only a stand-in), so
// the first call on each device, with that device current, looks the device
// address up with cudaGetSymbolAddress and caches it.  Every call checks that
// the context's device is current, since the cached address and the mesh
// belong to that device.
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "kern_common.cuh"

namespace sfx {

// Largest mesh the scratch array can describe.
constexpr int64_t kNoAllocMaxCells = 262144;

namespace {

// word offsets of the scratch layout (int32 words)
constexpr int64_t kMetaWords = 64;
constexpr int64_t kSortedOff = kMetaWords;                      // kNoAllocMaxCells cell ids
constexpr int64_t kTilesOff = kSortedOff + kNoAllocMaxCells;    // kNoAllocMaxCells tiles of 4 words
constexpr int64_t kScratchWords = kTilesOff + 4 * kNoAllocMaxCells;
// meta words
constexpr int kCount = 0;    // [1..8] cells per degree
constexpr int kBegin = 9;    // [9+p] first position of degree p in the sorted list
constexpr int kTileOff = 18; // [18+p] first tile of degree p
constexpr int kCursor = 27;  // [27+p] scatter cursor
constexpr int kNTiles = 40;
constexpr int kCounter = 41;

struct TileSizes {
  int cb[kMaxDeg + 1];
};

}  // namespace

static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchWords];

namespace {

// A cell takes part only if its degree is in 1..kMaxDeg and its block of the
// vectors is [off[c], off[c+1]) with off[c+1] - off[c] = (degree + 1)^3 and
// off[0] = 0.  Cells that pass therefore have disjoint blocks inside
// [0, off[ncell]); a cell that fails is flagged and skipped by every stage,
// so the kernels never index x or y through it.
__device__ __forceinline__ bool na_cell_ok(const int32_t* degree, const int64_t* off, int64_t c, int* d_out) {
  const int d = degree[c];
  if (d < 1 || d > kMaxDeg) return false;
  const int64_t o0 = off[c], o1 = off[c + 1];
  const int64_t n = (int64_t)(d + 1) * (d + 1) * (d + 1);
  if (o0 < 0 || o1 - o0 != n || (c == 0 && o0 != 0)) return false;
  *d_out = d;
  return true;
}

__global__ void k_na_histogram(const int32_t* degree, const int64_t* off, int64_t ncell, int32_t* sc,
                               uint32_t* status) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    int d;
    if (!na_cell_ok(degree, off, c, &d)) { atomicOr(status, SFX_DEV_BADCELL); continue; }
    atomicAdd(&sc[kCount + d], 1);
  }
}

__global__ void k_na_layout(int32_t* sc, TileSizes ts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int begin = 0;
  for (int p = 1; p <= kMaxDeg; ++p) {
    sc[kBegin + p] = begin;
    sc[kCursor + p] = begin;
    begin += sc[kCount + p];
  }
  int run = 0;
  for (int p = kMaxDeg; p >= 1; --p) {  // largest degree first
    sc[kTileOff + p] = run;
    run += (sc[kCount + p] + ts.cb[p] - 1) / ts.cb[p];
  }
  sc[kNTiles] = run;
  sc[kCounter] = 0;
}

__global__ void k_na_scatter(const int32_t* degree, const int64_t* off, int64_t ncell, int32_t* sc) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    int d;
    if (!na_cell_ok(degree, off, c, &d)) continue;
    const int pos = atomicAdd(&sc[kCursor + d], 1);
    sc[kSortedOff + pos] = (int32_t)c;
  }
}

__global__ void k_na_tiles(int32_t* sc, TileSizes ts, int64_t max_tiles) {
  const int nt = sc[kNTiles];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt && t < max_tiles;
       t += (int64_t)gridDim.x * blockDim.x) {
    int p = kMaxDeg;
    while (p > 1 && t >= sc[kTileOff + p - 1]) --p;  // tile offsets grow as p falls
    const int k = (int)(t - sc[kTileOff + p]);
    const int first = sc[kBegin + p] + k * ts.cb[p];
    const int end = sc[kBegin + p] + sc[kCount + p];
    BatchTile* tiles = reinterpret_cast<BatchTile*>(sc + kTilesOff);
    BatchTile b;
    b.p = p;
    b.form = 0;
    b.first = first;
    b.count = end - first < ts.cb[p] ? end - first : ts.cb[p];
    tiles[t] = b;
  }
}

// Zero the blocks of the cells that pass the check, one warp per cell (the
// blocks are contiguous: off[c] * nrhs .. off[c+1] * nrhs).
__global__ void k_na_zero(const int32_t* degree, const int64_t* off, int64_t ncell, int nrhs, double* y) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < ncell; c += warps) {
    int d;
    if (!na_cell_ok(degree, off, c, &d)) continue;
    const int64_t i0 = off[c] * nrhs, i1 = off[c + 1] * nrhs;
    for (int64_t i = i0 + lane; i < i1; i += 32) y[i] = 0.0;
  }
}

// device address of the scratch array, looked up once per device
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {nullptr};

}  // namespace

int upload_all_tables();

namespace {
sfx_status noalloc_body(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree, const int64_t* cell_offset,
                        sfx_form form, const sfx_form_params* params, const double* x, double* y, int nrhs,
                        void* stream);
}  // namespace

}  // namespace sfx

using namespace sfx;

extern "C" sfx_status sfx_padaptive_action_noalloc(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree,
                                                   const int64_t* cell_offset, sfx_form form,
                                                   const sfx_form_params* params, const double* x, double* y,
                                                   int nrhs, void* stream) {
  if (!ctx || !mesh || !degree || !cell_offset || !x || !y || x == y || nrhs < 1 || nrhs > 64) return SFX_ERR_ARG;
  if (ctx->device < 0 || ctx->device >= kMaxDevices || mesh->ctx != ctx || !mesh->d_vmap) return SFX_ERR_ARG;
  if (form != SFX_MASS && form != SFX_LAPLACE && form != SFX_HELMHOLTZ) return SFX_ERR_UNSUPPORTED;
  if (mesh->ncell > kNoAllocMaxCells) return SFX_ERR_RANGE;
  nvtxRangePushA("sfx_padaptive_action_noalloc");
  const sfx_status st = noalloc_body(ctx, mesh, degree, cell_offset, form, params, x, y, nrhs, stream);
  nvtxRangePop();
  return st;
}

namespace sfx {
namespace {

sfx_status noalloc_body(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree, const int64_t* cell_offset,
                        sfx_form form, const sfx_form_params* params, const double* x, double* y, int nrhs,
                        void* stream) {
  // the cached scratch address, the mesh and the status word belong to
  // ctx->device: it must be the current device on every call
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != ctx->device) return SFX_ERR_ARG;
  int32_t* sc = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[ctx->device]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SFX_ERR_CUDA;
      if (upload_all_tables() != 0) return SFX_ERR_CUDA;
      g_addr[ctx->device] = ptr;
    }
    sc = static_cast<int32_t*>(g_addr[ctx->device]);
  }
  TileSizes ts;
  int cb[kMaxDeg + 1];
  size_t smem = 0;
  int grid = 0;
  if (batched_config(cb, &smem, &grid) != 0) return SFX_ERR_CUDA;
  for (int p = 0; p <= kMaxDeg; ++p) ts.cb[p] = p ? cb[p] : 1;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t ncell = mesh->ncell;
  const int nb = (int)((ncell + 255) / 256 < 1024 ? (ncell + 255) / 256 : 1024);
  // the scratch keeps the previous call's contents: clear the counters first
  if (cudaMemsetAsync(sc, 0, kMetaWords * sizeof(int32_t), s) != cudaSuccess) return SFX_ERR_CUDA;
  k_na_histogram<<<nb, 256, 0, s>>>(degree, cell_offset, ncell, sc, ctx->d_status);
  k_na_layout<<<1, 1, 0, s>>>(sc, ts);
  k_na_scatter<<<nb, 256, 0, s>>>(degree, cell_offset, ncell, sc);
  k_na_tiles<<<nb, 256, 0, s>>>(sc, ts, ncell);
  k_na_zero<<<nb * 8 < 4096 ? nb * 8 : 4096, 256, 0, s>>>(degree, cell_offset, ncell, nrhs, y);
  if (cudaGetLastError() != cudaSuccess) return SFX_ERR_CUDA;
  const sfx_form_params pr = params ? *params : sfx_form_params{1.0, -1.0, 0.0, 0.0};
  BatchArgs b{};
  b.base.map = nullptr;
  b.base.dq_off = cell_offset;
  b.base.vmap = mesh->d_vmap;
  b.base.xyz = mesh->d_xyz;
  b.base.x = x;
  b.base.nrhs = nrhs;
  b.base.r0 = 0;
  b.base.r1 = nrhs;
  b.base.status = ctx->d_status;
  b.sorted_cells = sc + kSortedOff;
  b.tiles = reinterpret_cast<const BatchTile*>(sc + kTilesOff);
  b.ntiles = 0;
  b.ntiles_dev = sc + kNTiles;
  b.counter = sc + kCounter;
  b.ncell_total = ncell;
  b.y[0] = y;
  b.alpha[0] = form == SFX_HELMHOLTZ ? pr.alpha : 1.0;
  b.beta[0] = form == SFX_HELMHOLTZ ? pr.beta : 1.0;
  b.form_id[0] = form;
  return batched_launch(b, grid, smem, stream) == 0 ? SFX_OK : SFX_ERR_CUDA;
}

}  // namespace
}  // namespace sfx
