#pragma once
// batched_mixed_body.cuh -- the persistent p-adaptive batch (several forms,
// several right-hand sides, cells of every degree in one launch) with the
// split-precision tile body: each tile is cb cells of one degree and one form,
// run by scalar_tile_mixed (the contractions on the tensor cores, the
// geometry, weight scaling and scatter in FP64; Sec. 3.3, Eqs. coeff_eval and
// form_eval, with B = I for DQ_p).  Instantiated once per input format in
// k_batched_mixed_tf32.cu and k_batched_mixed_bf16.cu.
//
// Same schedule as k_batched_dq_fp64: the host sorts the cells by degree and
// cuts each degree's list into tiles, largest degree first; a grid of CTAs
// resident on every SM takes tiles from a global counter until the list is
// exhausted, so no CTA waits on another.
#include "scalar_mixed_body.cuh"

namespace sfx {
namespace {

// Four CTAs per SM (64 registers a thread, a few spilled; each CTA 55 KB of
// shared memory, which still holds one DQ_8 cell of any form with its staged
// factors), measured on the 200k-cell, 16-RHS, two-form batch against one,
// two and three CTAs per SM (191, 128 and 80 registers): 19.8 ms against
// 41.5, 25.1 and 20.8 -- the tile body is latency-bound and wants resident
// warps.
#ifndef SFX_BATCHM_CTAS
#define SFX_BATCHM_CTAS 4
#endif
constexpr int kBTM = 256;  // threads per CTA, every degree
constexpr int kCtasM = SFX_BATCHM_CTAS;
constexpr size_t kBudgetM = (size_t)(227 / kCtasM - 1) * 1024;

// Cells per tile for degree p = N - 1: the most (up to 32 for n <= 3, else 16)
// whose shared-memory layout fits, for every form of the mask; 0 if not even
// one cell fits.
template <int N>
int cb_mixed(int form_mask, bool geo_once) {
  int cb = N <= 3 ? 32 : 16;
  bool ok = true;
  auto fit = [&](size_t (*bytes)(int, bool, bool)) {
    while (cb > 1 && bytes(cb, geo_once, false) > kBudgetM) --cb;
    if (bytes(cb, geo_once, false) > kBudgetM) ok = false;
  };
  if (form_mask & 1) fit(&MixedShape<N, SFX_MASS>::bytes);
  if (form_mask & 2) fit(&MixedShape<N, SFX_LAPLACE>::bytes);
  if (form_mask & 4) fit(&MixedShape<N, SFX_HELMHOLTZ>::bytes);
  return ok ? cb : 0;
}

template <int N, int PREC>
__device__ __forceinline__ void run_tile_mixed(int form, const ActArgs& a, int64_t nc, int cb, bool geo_once,
                                               double* smd) {
  switch (form) {
    case SFX_MASS:
      scalar_tile_mixed<N, true, SFX_MASS, PREC, false, false, kBTM>(a, nc, 0, cb, geo_once, smd);
      break;
    case SFX_LAPLACE:
      scalar_tile_mixed<N, true, SFX_LAPLACE, PREC, false, false, kBTM>(a, nc, 0, cb, geo_once, smd);
      break;
    default:
      scalar_tile_mixed<N, true, SFX_HELMHOLTZ, PREC, false, false, kBTM>(a, nc, 0, cb, geo_once, smd);
      break;
  }
}

template <int PREC>
__global__ void __launch_bounds__(kBTM, kCtasM) k_batched_dq_mixed(const BatchArgs b, const bool geo_once) {
  extern __shared__ double smd[];
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
    // the tile's own cell count sets its shared-memory layout (at most the
    // degree's tile size, which the host sized to fit)
    switch (tl.p) {
      case 1: run_tile_mixed<2, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
      case 2: run_tile_mixed<3, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
      case 3: run_tile_mixed<4, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
      case 4: run_tile_mixed<5, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
      case 5: run_tile_mixed<6, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
      case 6: run_tile_mixed<7, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
      case 7: run_tile_mixed<8, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
      default: run_tile_mixed<9, PREC>(form, a, b.ncell_total, tl.count, geo_once, smd); break;
    }
    __syncthreads();
  }
}

// Host side: tile sizes per degree for the plan's forms, the dynamic shared
// memory and the persistent grid (the CTAs resident on every SM).
template <int PREC>
int batched_mixed_config_prec(int form_mask, int nrhs, int* cb, size_t* smem, int* grid) {
  const bool geo_once = nrhs > 1;
  cb[0] = 0;
  cb[1] = cb_mixed<2>(form_mask, geo_once); cb[2] = cb_mixed<3>(form_mask, geo_once);
  cb[3] = cb_mixed<4>(form_mask, geo_once); cb[4] = cb_mixed<5>(form_mask, geo_once);
  cb[5] = cb_mixed<6>(form_mask, geo_once); cb[6] = cb_mixed<7>(form_mask, geo_once);
  cb[7] = cb_mixed<8>(form_mask, geo_once); cb[8] = cb_mixed<9>(form_mask, geo_once);
  for (int p = 1; p <= kMaxDeg; ++p) {
    if (cb[p] < 1) return (int)cudaErrorInvalidValue;  // a layout that does not fit: no plan
    const int t = tuned_cells_per_cta(SFX_TUNE_BATCHED_MIXED, p, cb[p]);
    cb[p] = t >= 1 && t < cb[p] ? t : cb[p];
  }
  *smem = kBudgetM;
  auto kern = k_batched_dq_mixed<PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBudgetM);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBTM, kBudgetM)) != cudaSuccess) return (int)e;
  *grid = sms * (per > 0 ? per : 1);
  return 0;
}

template <int PREC>
int batched_mixed_launch_prec(const BatchArgs& b, int nrhs, int grid, size_t smem, void* stream) {
  k_batched_dq_mixed<PREC><<<grid, kBTM, smem, (cudaStream_t)stream>>>(b, nrhs > 1);
  return (int)cudaGetLastError();
}

}  // namespace
}  // namespace sfx
