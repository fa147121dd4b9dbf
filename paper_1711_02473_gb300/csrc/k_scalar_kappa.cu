// k_scalar_kappa.cu -- FP64 action of the weighted Laplace form
// a(u, v) = int kappa grad u . grad v (Sec. 1.1, Eq. weighted_laplace) on Q_p
// and DQ_p: the coefficient kappa, given by its dofs in the same space, is
// interpolated to the Gauss points with the value contractions B (sum
// factorisation, Sec. 3.3, Eq. coeff_eval) and scales the geometric factor
// P = w S G G^T at each point.  Device body: scalar_body.cuh with KAP = true.
#include "scalar_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_scalar_kappa)

namespace {

template <int N, bool DQ>
__global__ void __launch_bounds__(256, 2) k_action_weighted_fp64(const ActArgs a, const int64_t ncell_total,
                                                                 const bool geo_once) {
  extern __shared__ double sm[];
  const int cb = blockDim.x / (N * N);
  scalar_tile_fp64<N, DQ, SFX_LAPLACE, false, false, true>(a, ncell_total, (int64_t)blockIdx.x * cb, cb, sm,
                                                           geo_once);
}

template <int N, bool DQ>
int launch(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = ScalarShape<N, SFX_LAPLACE, true>;
  const bool geo_once = a.r1 - a.r0 > 1;
  const size_t per_team = (size_t)Sh::team_doubles(geo_once) * sizeof(double);
  const size_t fixed = (Sh::N3 + 16) * sizeof(double);
  const size_t budget = 200 * 1024;
  int cb = tuned_cells_per_cta(SFX_TUNE_SCALAR_FP64, N - 1, Sh::MAXCB);
  if (cb > Sh::MAXCB) cb = Sh::MAXCB;
  while (cb > 1 && fixed + cb * per_team > budget) --cb;
  const size_t smem = fixed + cb * per_team;
  auto kern = k_action_weighted_fp64<N, DQ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  kern<<<(unsigned)grid, cb * Sh::N2, smem, s>>>(a, ncell_total, geo_once);
  return (int)cudaGetLastError();
}

template <int N>
int dispatch(bool dq, const ActArgs& a, int64_t nc, cudaStream_t s) {
  return dq ? launch<N, true>(a, nc, s) : launch<N, false>(a, nc, s);
}

}  // namespace

int launch_action_weighted(const sfx_space* sp, const ActArgs& a, void* stream) {
  if (sp->family != SFX_Q && sp->family != SFX_DQ) return -1;
  const bool dq = sp->family == SFX_DQ;
  const int64_t nc = sp->mesh->ncell;
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 1: return dispatch<2>(dq, a, nc, s);
    case 2: return dispatch<3>(dq, a, nc, s);
    case 3: return dispatch<4>(dq, a, nc, s);
    case 4: return dispatch<5>(dq, a, nc, s);
    case 5: return dispatch<6>(dq, a, nc, s);
    case 6: return dispatch<7>(dq, a, nc, s);
    case 7: return dispatch<8>(dq, a, nc, s);
    case 8: return dispatch<9>(dq, a, nc, s);
  }
  return -1;
}

}  // namespace sfx
