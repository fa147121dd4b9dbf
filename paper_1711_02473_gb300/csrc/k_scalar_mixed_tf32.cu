// k_scalar_mixed_tf32.cu -- TF32x3 instantiation of the split-precision scalar
// actions (body in scalar_mixed_body.cuh).  The two formats are separate
// translation units so that the build compiles them in parallel.
#include "scalar_mixed_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_scalar_mixed_tf32)

namespace {

template <int N, bool DQ, int FORM, int PREC>
int launch_mixed(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = MixedShape<N, FORM>;
  const bool stored = a.qd32 != nullptr;
  const bool geo_once = a.nrhs > 1;
  const size_t budget = 200 * 1024;
  // cells per CTA: the autotuned value, else enough fibers for dense tiles
  int cb = tuned_cells_per_cta(stored ? SFX_TUNE_SCALAR_MIXED_STORED : SFX_TUNE_SCALAR_MIXED, N - 1,
                               (N <= 3) ? 32 : 16);
  if (cb < 1) cb = 1;
  while (cb > 1 && Sh::bytes(cb, geo_once, stored) > budget) --cb;
  const size_t smem = Sh::bytes(cb, geo_once, stored);
  auto kern = stored ? k_action_scalar_mixed<N, DQ, FORM, PREC, true> : k_action_scalar_mixed<N, DQ, FORM, PREC, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  e = launch_kernel(kern, (unsigned)grid, Sh::NT, smem, s, a.overlap_prev != 0, a, ncell_total, cb, geo_once);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

template <int N, bool DQ>
int dispatch_form(sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (form) {
    case SFX_MASS: return launch_mixed<N, DQ, SFX_MASS, SFX_PREC_TF32X3>(a, nc, s);
    case SFX_LAPLACE: return launch_mixed<N, DQ, SFX_LAPLACE, SFX_PREC_TF32X3>(a, nc, s);
    case SFX_HELMHOLTZ: return launch_mixed<N, DQ, SFX_HELMHOLTZ, SFX_PREC_TF32X3>(a, nc, s);
    default: return -1;
  }
}

template <int N>
int dispatch(bool dq, sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  return dq ? dispatch_form<N, true>(form, a, nc, s) : dispatch_form<N, false>(form, a, nc, s);
}

}  // namespace

int launch_action_scalar_mixed_tf32(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  const bool dq = sp->family == SFX_DQ;
  const int64_t nc = sp->mesh->ncell;
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 1: return dispatch<2>(dq, form, a, nc, s);
    case 2: return dispatch<3>(dq, form, a, nc, s);
    case 3: return dispatch<4>(dq, form, a, nc, s);
    case 4: return dispatch<5>(dq, form, a, nc, s);
    case 5: return dispatch<6>(dq, form, a, nc, s);
    case 6: return dispatch<7>(dq, form, a, nc, s);
    case 7: return dispatch<8>(dq, form, a, nc, s);
    case 8: return dispatch<9>(dq, form, a, nc, s);
  }
  return -1;
}

}  // namespace sfx
