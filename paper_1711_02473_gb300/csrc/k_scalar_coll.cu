// k_scalar_coll.cu -- FP64 Q_p actions (mass, Laplace, Helmholtz) with the
// collocated Gauss-Lobatto rule: the p+1 GLL points per direction are the
// Q_p nodes, so the value tabulation is the identity and only the derivative
// contractions remain (Sec. 2.5, Eq. colocated; the "underintegration" case of
// Sec. 4.1, whose substitution makes each reference derivative a single 1D
// derivative table times two deltas).  Same device body as k_scalar.cu
// (scalar_body.cuh) with COLL = true; per-colour launches, deterministic.
#include "scalar_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_scalar_coll)

namespace {

template <int N, int FORM>
__global__ void __launch_bounds__(256, 2) k_action_scalar_coll_fp64(const ActArgs a, const int64_t ncell_total,
                                                                    const bool geo_once) {
  extern __shared__ double sm[];
  const int cb = blockDim.x / (N * N);
  scalar_tile_fp64<N, true, FORM, false, true>(a, ncell_total, (int64_t)blockIdx.x * cb, cb, sm, geo_once);
}

template <int N, int FORM>
int launch(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = ScalarShape<N, FORM>;
  const bool geo_once = a.r1 - a.r0 > 1;
  const size_t per_team = (size_t)Sh::team_doubles(geo_once) * sizeof(double);
  const size_t fixed = (Sh::N3 + 16) * sizeof(double);
  const size_t budget = 200 * 1024;
  int cb = tuned_cells_per_cta(SFX_TUNE_SCALAR_FP64, N - 1, Sh::MAXCB);
  if (cb > Sh::MAXCB) cb = Sh::MAXCB;  // one team of N^2 threads per cell, <= 256 threads
  while (cb > 1 && fixed + cb * per_team > budget) --cb;
  const size_t smem = fixed + cb * per_team;
  auto kern = k_action_scalar_coll_fp64<N, FORM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  kern<<<(unsigned)grid, cb * Sh::N2, smem, s>>>(a, ncell_total, geo_once);
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

int launch_action_scalar_coll(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  if (sp->family != SFX_Q) return -1;
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
