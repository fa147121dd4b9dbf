// k_scalar.cu -- per-colour launches of the FP64 scalar-form action (the
// device body is in scalar_body.cuh).
#include "scalar_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_scalar)

namespace {

template <int N, bool DQ, int FORM, bool STORED>
__global__ void __launch_bounds__(256, 2) k_action_scalar_fp64(const ActArgs a, const int64_t ncell_total,
                                                           const bool geo_once) {
  extern __shared__ double sm[];
  const int cb = blockDim.x / (N * N);
  scalar_tile_fp64<N, DQ, FORM, STORED>(a, ncell_total, (int64_t)blockIdx.x * cb, cb, sm, geo_once);
}

template <int N, bool DQ, int FORM>
int launch_fp64(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = ScalarShape<N, FORM>;
  // several RHS: stage the factors once per cell; one RHS: form them at the point
  const bool geo_once = a.r1 - a.r0 > 1 || a.stage_factors;
  const size_t per_team = (size_t)Sh::team_doubles(geo_once) * sizeof(double);
  const size_t fixed = (Sh::N3 + 16) * sizeof(double);
  const size_t budget = 200 * 1024;
  int cb = tuned_cells_per_cta(SFX_TUNE_SCALAR_FP64, N - 1, Sh::MAXCB);
  if (cb > Sh::MAXCB) cb = Sh::MAXCB;  // one team of N^2 threads per cell, <= 256 threads
  while (cb > 1 && fixed + cb * per_team > budget) --cb;
  const size_t smem = fixed + cb * per_team;
  auto kern = a.qd64 ? k_action_scalar_fp64<N, DQ, FORM, true> : k_action_scalar_fp64<N, DQ, FORM, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  e = launch_kernel(kern, (unsigned)grid, cb * Sh::N2, smem, s, a.overlap_prev != 0, a, ncell_total, geo_once);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

template <int N, bool DQ>
int dispatch_form(sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (form) {
    case SFX_MASS: return launch_fp64<N, DQ, SFX_MASS>(a, nc, s);
    case SFX_LAPLACE: return launch_fp64<N, DQ, SFX_LAPLACE>(a, nc, s);
    case SFX_HELMHOLTZ: return launch_fp64<N, DQ, SFX_HELMHOLTZ>(a, nc, s);
    default: return -1;
  }
}

template <int N>
int dispatch_family(bool dq, sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  return dq ? dispatch_form<N, true>(form, a, nc, s) : dispatch_form<N, false>(form, a, nc, s);
}

}  // namespace

int launch_action_scalar_mixed_tf32(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);
int launch_action_scalar_mixed_bf16(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);

int launch_action_scalar_mixed_ws_tf32(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);
int launch_action_scalar_mixed_ws_bf16(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);

int launch_action_scalar_mixed(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                               void* stream) {
  // the warp-specialised kernel where it applies (Laplace part, p >= 3,
  // geometry in the kernel), else the one-role kernel
  int e = -1;
  if (prec == SFX_PREC_TF32X3) e = launch_action_scalar_mixed_ws_tf32(sp, form, a, stream);
  if (prec == SFX_PREC_BF16X3) e = launch_action_scalar_mixed_ws_bf16(sp, form, a, stream);
  if (e != -1) return e;
  if (prec == SFX_PREC_TF32X3) return launch_action_scalar_mixed_tf32(sp, form, a, stream);
  if (prec == SFX_PREC_BF16X3) return launch_action_scalar_mixed_bf16(sp, form, a, stream);
  return -1;
}

int launch_scalar_fp64_degree(int p, bool dq, sfx_form form, const ActArgs& a, int64_t nc, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (p) {
    case 1: return dispatch_family<2>(dq, form, a, nc, s);
    case 2: return dispatch_family<3>(dq, form, a, nc, s);
    case 3: return dispatch_family<4>(dq, form, a, nc, s);
    case 4: return dispatch_family<5>(dq, form, a, nc, s);
    case 5: return dispatch_family<6>(dq, form, a, nc, s);
    case 6: return dispatch_family<7>(dq, form, a, nc, s);
    case 7: return dispatch_family<8>(dq, form, a, nc, s);
    case 8: return dispatch_family<9>(dq, form, a, nc, s);
  }
  return -1;
}

int launch_action_scalar(const sfx_space* sp, sfx_form form, sfx_precision prec, sfx_algo algo,
                         const ActArgs& a, void* stream) {
  if (algo == SFX_ALGO_NAIVE) {
    if (prec != SFX_PREC_FP64) return -1;
    return launch_action_scalar_naive(sp, form, a, stream);
  }
  if (prec != SFX_PREC_FP64) return launch_action_scalar_mixed(sp, form, prec, a, stream);
  const bool dq = sp->family == SFX_DQ;
  const int64_t nc = sp->mesh->ncell;
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 1: return dispatch_family<2>(dq, form, a, nc, s);
    case 2: return dispatch_family<3>(dq, form, a, nc, s);
    case 3: return dispatch_family<4>(dq, form, a, nc, s);
    case 4: return dispatch_family<5>(dq, form, a, nc, s);
    case 5: return dispatch_family<6>(dq, form, a, nc, s);
    case 6: return dispatch_family<7>(dq, form, a, nc, s);
    case 7: return dispatch_family<8>(dq, form, a, nc, s);
    case 8: return dispatch_family<9>(dq, form, a, nc, s);
  }
  return -1;
}

}  // namespace sfx
