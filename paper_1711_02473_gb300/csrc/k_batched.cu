// k_batched.cu -- one persistent launch for a p-adaptive DQ mesh, several
// forms and several right-hand sides.
//
// The host sorts the cells by degree and cuts each degree's list into tiles of
// cb(p) cells (one CTA's worth), one tile list per form, largest degree first.
// A fixed grid of CTAs (one per SM, or as many as fit) takes tiles from a
// global counter with atomicAdd until the list is exhausted; each tile runs the
// same device body as the per-colour kernel (scalar_body.cuh) for all
// right-hand sides, so the FP64 geometry of a cell is computed once per form
// for all RHS.  The loop ends after at most ntiles + grid counter increments;
// no CTA waits on another.
#include "scalar_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_batched)

namespace {

// threads per CTA and dynamic shared memory of the persistent kernel: the
// kernel's registers (the bodies of every degree and form in one kernel) allow
// one CTA per SM, so it takes nearly all the shared memory a CTA can have
// (227 KB less 1 KB for the kernel's static variables; a tile of the Helmholtz
// form then holds three DQ_8 cells instead of two; the other forms and
// degrees already had their team limit)
#ifndef SFX_BATCH_THREADS
#define SFX_BATCH_THREADS 256
#endif
#ifndef SFX_BATCH_SMEM_KB
#define SFX_BATCH_SMEM_KB 226
#endif
constexpr int kBT = SFX_BATCH_THREADS;
constexpr size_t kBudget = (size_t)SFX_BATCH_SMEM_KB * 1024;

template <int N, int FORM>
constexpr int cb_of() {
  using Sh = ScalarShape<N, FORM>;
  int cb = kBT / Sh::N2 > 0 ? kBT / Sh::N2 : 1;  // one team of N^2 threads per cell
  while (cb > 1 && (Sh::N3 + 16) * 8 + (size_t)cb * Sh::TEAM * 8 > kBudget) --cb;
  return cb;
}

template <int N>
__device__ __forceinline__ void run_tile(int form, const ActArgs& a, int64_t nc, double* sm) {
  switch (form) {
    // tiles serve every RHS: the factors are staged once per cell (geo_once)
    case SFX_MASS: scalar_tile_fp64<N, true, SFX_MASS>(a, nc, 0, cb_of<N, SFX_MASS>(), sm, true); break;
    case SFX_LAPLACE: scalar_tile_fp64<N, true, SFX_LAPLACE>(a, nc, 0, cb_of<N, SFX_LAPLACE>(), sm, true); break;
    default: scalar_tile_fp64<N, true, SFX_HELMHOLTZ>(a, nc, 0, cb_of<N, SFX_HELMHOLTZ>(), sm, true); break;
  }
}

__global__ void __launch_bounds__(kBT) k_batched_dq_fp64(const BatchArgs b) {
  extern __shared__ double sm[];
  __shared__ int s_tile;
#pragma unroll 1
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(b.counter, 1);
    __syncthreads();
    const int tix = s_tile;
    __syncthreads();
    if (tix >= (b.ntiles_dev ? *b.ntiles_dev : b.ntiles)) break;
    const BatchTile tl = b.tiles[tix];
    ActArgs a = b.base;
    a.cells = b.sorted_cells + tl.first;
    a.ncells = tl.count;
    a.y = b.y[tl.form];
    a.alpha = b.alpha[tl.form];
    a.beta = b.beta[tl.form];
    const int form = b.form_id[tl.form];
    switch (tl.p) {
      case 1: run_tile<2>(form, a, b.ncell_total, sm); break;
      case 2: run_tile<3>(form, a, b.ncell_total, sm); break;
      case 3: run_tile<4>(form, a, b.ncell_total, sm); break;
      case 4: run_tile<5>(form, a, b.ncell_total, sm); break;
      case 5: run_tile<6>(form, a, b.ncell_total, sm); break;
      case 6: run_tile<7>(form, a, b.ncell_total, sm); break;
      case 7: run_tile<8>(form, a, b.ncell_total, sm); break;
      default: run_tile<9>(form, a, b.ncell_total, sm); break;
    }
    __syncthreads();
  }
}

template <int N>
int cb_min(int form_mask) {
  // the tile size for a degree is the team count every form of the plan can host
  int cb = 1 << 30;
  if (form_mask & 1) cb = cb_of<N, SFX_MASS>() < cb ? cb_of<N, SFX_MASS>() : cb;
  if (form_mask & 2) cb = cb_of<N, SFX_LAPLACE>() < cb ? cb_of<N, SFX_LAPLACE>() : cb;
  if (form_mask & 4) cb = cb_of<N, SFX_HELMHOLTZ>() < cb ? cb_of<N, SFX_HELMHOLTZ>() : cb;
  return cb;
}

}  // namespace

// Team counts per degree (a tile must fit every form's shared-memory layout:
// the minimum over the three forms), the dynamic shared memory of the
// persistent kernel and its grid (CTAs resident on all SMs).
// Cells per tile: the tuned value (sfx_tune_set_cells_per_cta, kind 5) where
// one is set, at most the layout's count; smaller tiles give the tile counter
// finer pieces to balance across the SMs.  Only launch geometry changes: each
// cell's arithmetic is the same.
int batched_config(int* cb, size_t* smem, int* grid) {
  batched_tile_sizes(cb);
  for (int p = 1; p <= kMaxDeg; ++p) {
    const int t = tuned_cells_per_cta(SFX_TUNE_BATCHED, p, cb[p]);
    cb[p] = t >= 1 && t < cb[p] ? t : cb[p];
  }
  *smem = kBudget;
  cudaError_t e = cudaFuncSetAttribute(k_batched_dq_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBudget);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batched_dq_fp64, kBT, kBudget)) != cudaSuccess)
    return (int)e;
  *grid = sms * (per > 0 ? per : 1);
  return 0;
}

int batched_tile_sizes(int* cb) {
  cb[0] = 0;
  cb[1] = cb_min<2>(7); cb[2] = cb_min<3>(7); cb[3] = cb_min<4>(7); cb[4] = cb_min<5>(7);
  cb[5] = cb_min<6>(7); cb[6] = cb_min<7>(7); cb[7] = cb_min<8>(7); cb[8] = cb_min<9>(7);
  return 0;
}

int batched_launch(const BatchArgs& b, int grid, size_t smem, void* stream) {
  k_batched_dq_fp64<<<grid, kBT, smem, (cudaStream_t)stream>>>(b);
  return (int)cudaGetLastError();
}

}  // namespace sfx
