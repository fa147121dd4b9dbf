// k_qdata.cu -- geometric factors at the quadrature points, computed once per
// space in FP64 and stored (the "P^(k,l)" of Sec. 3.2, with the weight and
// |J| folded in, for every point of every cell).
//
// Per point: J from the trilinear coordinate field (column tables, as in the
// action kernels), S = det J, adj J rows r_k, and
//   P_kl = (w/S) r_k . r_l   (= w S (G G^T)_kl)   and   W = w S.
// The actions that use them (SFX_ALGO_STORED) skip the per-point geometry:
// a memory-for-arithmetic trade that suits GB300's narrow FP64 pipe when the
// same operator is applied many times.
#include "kern_common.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_qdata)

namespace {

template <int N>
__global__ void __launch_bounds__(128) k_qdata(const int32_t* vmap, const double* xyz, int64_t ncell, double* d64,
                                               float* d32, uint32_t* status) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const Tab1D& T = c_tab[N - 1];
  __shared__ double X[8][3], Jc[3][N2][3], xq[N];
  __shared__ int bad;
  const int64_t cell = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid < 24) X[tid / 3][tid % 3] = xyz[(int64_t)vmap[cell * 8 + tid / 3] * 3 + tid % 3];
  if (tid < N) xq[tid] = T.x[tid];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int i = tid; i < N2; i += blockDim.x) jacobian_columns<N>(X, xq, Jc, i);
  __syncthreads();
  for (int qp = tid; qp < N3; qp += blockDim.x) {
    const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
    const double* c0 = Jc[0][q2 * N + q3];
    const double* c1 = Jc[1][q1 * N + q3];
    const double* c2 = Jc[2][q1 * N + q2];
    double r0[3], r1[3], r2[3];
    cross3(c1, c2, r0);
    cross3(c2, c0, r1);
    cross3(c0, c1, r2);
    const double S = dot3(c0, r0);
    if (!(S > 0.0)) bad = 1;
    const double w = T.w[q1] * T.w[q2] * T.w[q3];
    const double ws = w / S;
    const double v[7] = {ws * dot3(r0, r0), ws * dot3(r1, r1), ws * dot3(r2, r2), ws * dot3(r0, r1),
                         ws * dot3(r0, r2), ws * dot3(r1, r2), w * S};
    for (int j = 0; j < 7; ++j) {
      const int64_t at = (cell * 7 + j) * N3 + qp;
      if (d64) d64[at] = v[j];
      if (d32) d32[at] = (float)v[j];
    }
  }
  __syncthreads();
  if (bad && tid == 0) atomicOr(status, SFX_DEV_INVERTED);
}

template <int N>
int go(const sfx_space* sp, sfx_qdata* q, uint32_t* st, cudaStream_t s) {
  k_qdata<N><<<(unsigned)sp->mesh->ncell, 128, 0, s>>>(sp->mesh->d_vmap, sp->mesh->d_xyz, sp->mesh->ncell, q->d64,
                                                         q->d32, st);
  return (int)cudaGetLastError();
}

}  // namespace

int launch_qdata(const sfx_space* sp, sfx_qdata* q, uint32_t* st, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 1: return go<2>(sp, q, st, s);
    case 2: return go<3>(sp, q, st, s);
    case 3: return go<4>(sp, q, st, s);
    case 4: return go<5>(sp, q, st, s);
    case 5: return go<6>(sp, q, st, s);
    case 6: return go<7>(sp, q, st, s);
    case 7: return go<8>(sp, q, st, s);
    case 8: return go<9>(sp, q, st, s);
  }
  return -1;
}

}  // namespace sfx
