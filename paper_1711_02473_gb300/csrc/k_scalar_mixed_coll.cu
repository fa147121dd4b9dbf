// k_scalar_mixed_coll.cu -- TF32x3 split-precision Q_p actions with the
// collocated Gauss-Lobatto rule (B = I; only the derivative contractions run
// on the tensor cores; Sec. 2.5 and the "underintegration" case of Sec. 4.1).
// Body in scalar_mixed_body.cuh with COLL = true.
#include "scalar_mixed_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_scalar_mixed_coll)

namespace {

template <int N, int FORM>
int launch(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = MixedShape<N, FORM>;
  const bool geo_once = a.nrhs > 1;
  const size_t budget = 200 * 1024;
  int cb = tuned_cells_per_cta(SFX_TUNE_SCALAR_MIXED, N - 1, (N <= 3) ? 32 : 16);
  if (cb < 1) cb = 1;
  while (cb > 1 && Sh::bytes(cb, geo_once, false) > budget) --cb;
  const size_t smem = Sh::bytes(cb, geo_once, false);
  auto kern = k_action_scalar_mixed<N, true, FORM, SFX_PREC_TF32X3, false, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  kern<<<(unsigned)grid, Sh::NT, smem, s>>>(a, ncell_total, cb, geo_once);
  return (int)cudaGetLastError();
}

template <int N>
int dispatch_form(sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (form) {
    case SFX_MASS: return launch<N, SFX_MASS>(a, nc, s);
    case SFX_LAPLACE: return launch<N, SFX_LAPLACE>(a, nc, s);
    case SFX_HELMHOLTZ: return launch<N, SFX_HELMHOLTZ>(a, nc, s);
    default: return -1;
  }
}

}  // namespace

int launch_action_scalar_mixed_coll(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  if (sp->family != SFX_Q || a.qd32) return -1;
  const int64_t nc = sp->mesh->ncell;
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 1: return dispatch_form<2>(form, a, nc, s);
    case 2: return dispatch_form<3>(form, a, nc, s);
    case 3: return dispatch_form<4>(form, a, nc, s);
    case 4: return dispatch_form<5>(form, a, nc, s);
    case 5: return dispatch_form<6>(form, a, nc, s);
    case 6: return dispatch_form<7>(form, a, nc, s);
    case 7: return dispatch_form<8>(form, a, nc, s);
    case 8: return dispatch_form<9>(form, a, nc, s);
  }
  return -1;
}

}  // namespace sfx
