// k_naive.cu -- scalar-form actions without sum factorisation (FP64).
//
// The coefficient is evaluated at every 3D point as a sum over all local basis
// functions, u(xi_q) = sum_i U_i Psi_i(xi_q) with Psi_i(xi_q) formed as the
// product of its three 1D factors (the dense tabulation of Sec. 1.1 Eq.
// fiat_table, built on the fly), and the test integral sums over all points
// again: O(n^6) per cell, the cost class of the un-factorised kernels the
// paper compares against (Sec. 3.3, Table form_ordo).  Geometry and pointwise
// physics are identical to the sum-factorised kernel.
#include "kern_common.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_naive)

namespace {

constexpr int kNT = 128;

template <int N>
struct NaiveSm {
  static constexpr int N2 = N * N, N3 = N2 * N;
  double B[N][N], D[N][N], W3[N3], xq[N];
  double U[N3], F0[N3], F1[N3], F2[N3], FV[N3], K[6][N3], WS[N3];
  double X[8][3], Jc[3][N2][3];
  int bad;
};

template <int N, bool DQ, int FORM>
__global__ void __launch_bounds__(kNT) k_action_scalar_naive(const ActArgs a, const int64_t ncell_total) {
  constexpr int N2 = N * N, N3 = N2 * N;
  constexpr bool LAP = FORM != SFX_MASS, MAS = FORM != SFX_LAPLACE;
  const Tab1D& T = c_tab[N - 1];
  extern __shared__ double raw[];
  NaiveSm<N>& S_ = *reinterpret_cast<NaiveSm<N>*>(raw);
  auto& B = S_.B;
  auto& D = S_.D;
  auto& W3 = S_.W3;
  auto& xq = S_.xq;
  auto& U = S_.U;
  auto& F0 = S_.F0;
  auto& F1 = S_.F1;
  auto& F2 = S_.F2;
  auto& FV = S_.FV;
  auto& K = S_.K;
  auto& WS = S_.WS;
  auto& X = S_.X;
  auto& Jc = S_.Jc;
  int& bad = S_.bad;
  const int tid = threadIdx.x;
  int cell = 0;
  if (!slot_cell(a, blockIdx.x, ncell_total, &cell)) return;  // uniform over the CTA
  for (int i = tid; i < N2; i += kNT) {
    const int q = i / N, j = i % N;
    B[q][j] = DQ ? (q == j ? 1.0 : 0.0) : T.Bc[q][j];
    D[q][j] = DQ ? T.Dq[q][j] : T.Dc[q][j];
  }
  for (int i = tid; i < N3; i += kNT) W3[i] = T.w[i / N2] * T.w[(i / N) % N] * T.w[i % N];
  if (tid < N) xq[tid] = T.x[tid];
  if (tid < 24) X[tid / 3][tid % 3] = a.xyz[(int64_t)a.vmap[(int64_t)cell * 8 + tid / 3] * 3 + tid % 3];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int i = tid; i < N2; i += kNT) jacobian_columns<N>(X, xq, Jc, i);
  __syncthreads();
  const double alpha = FORM == SFX_HELMHOLTZ ? a.alpha : 1.0;
  const double beta = FORM == SFX_HELMHOLTZ ? a.beta : 1.0;
  for (int qp = tid; qp < N3; qp += kNT) {
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
    const double ws = alpha * W3[qp] / S;
    K[0][qp] = ws * dot3(r0, r0); K[1][qp] = ws * dot3(r1, r1); K[2][qp] = ws * dot3(r2, r2);
    K[3][qp] = ws * dot3(r0, r1); K[4][qp] = ws * dot3(r0, r2); K[5][qp] = ws * dot3(r1, r2);
    WS[qp] = beta * W3[qp] * S;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) set_flag(a.status, SFX_DEV_INVERTED);
    if (a.cell_vectors)
      for (int i = tid; i < N3 * a.nrhs; i += kNT) a.y[(int64_t)blockIdx.x * N3 * a.nrhs + i] = 0.0;
    return;
  }
  const int32_t* mrow = a.map + (int64_t)cell * N3;
  for (int r = 0; r < a.nrhs; ++r) {
    for (int l = tid; l < N3; l += kNT) U[l] = a.x[(int64_t)mrow[l] * a.nrhs + r];
    __syncthreads();
    for (int qp = tid; qp < N3; qp += kNT) {
      const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
      double u = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
      for (int l = 0; l < N3; ++l) {
        const int i1 = l / N2, i2 = (l / N) % N, i3 = l % N;
        const double b1 = B[q1][i1], b2 = B[q2][i2], b3 = B[q3][i3];
        const double c = U[l];
        if (MAS) u += c * (b1 * b2 * b3);
        if (LAP) {
          g0 += c * (D[q1][i1] * b2 * b3);
          g1 += c * (b1 * D[q2][i2] * b3);
          g2 += c * (b1 * b2 * D[q3][i3]);
        }
      }
      if (LAP) {
        F0[qp] = K[0][qp] * g0 + K[3][qp] * g1 + K[4][qp] * g2;
        F1[qp] = K[3][qp] * g0 + K[1][qp] * g1 + K[5][qp] * g2;
        F2[qp] = K[4][qp] * g0 + K[5][qp] * g1 + K[2][qp] * g2;
      }
      if (MAS) FV[qp] = WS[qp] * u;
    }
    __syncthreads();
    for (int l = tid; l < N3; l += kNT) {
      const int i1 = l / N2, i2 = (l / N) % N, i3 = l % N;
      double b = 0.0;
      for (int qp = 0; qp < N3; ++qp) {
        const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
        const double b1 = B[q1][i1], b2 = B[q2][i2], b3 = B[q3][i3];
        if (MAS) b += FV[qp] * (b1 * b2 * b3);
        if (LAP) b += F0[qp] * (D[q1][i1] * b2 * b3) + F1[qp] * (b1 * D[q2][i2] * b3) + F2[qp] * (b1 * b2 * D[q3][i3]);
      }
      if (a.cell_vectors) a.y[((int64_t)blockIdx.x * N3 + l) * a.nrhs + r] = b;
      else a.y[(int64_t)mrow[l] * a.nrhs + r] += b;
    }
    __syncthreads();
  }
}

template <int N, bool DQ, int FORM>
int launch_k(const ActArgs& a, int64_t nc, cudaStream_t s) {
  const size_t smem = sizeof(NaiveSm<N>);
  auto kern = k_action_scalar_naive<N, DQ, FORM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<(unsigned)a.ncells, kNT, smem, s>>>(a, nc);
  return (int)cudaGetLastError();
}

template <int N, bool DQ>
int launch_n(sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (form) {
    case SFX_MASS: return launch_k<N, DQ, SFX_MASS>(a, nc, s);
    case SFX_LAPLACE: return launch_k<N, DQ, SFX_LAPLACE>(a, nc, s);
    case SFX_HELMHOLTZ: return launch_k<N, DQ, SFX_HELMHOLTZ>(a, nc, s);
    default: return -1;
  }
}

template <int N>
int launch_f(bool dq, sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  return dq ? launch_n<N, true>(form, a, nc, s) : launch_n<N, false>(form, a, nc, s);
}

}  // namespace

int launch_action_scalar_naive(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  const bool dq = sp->family == SFX_DQ;
  const int64_t nc = sp->mesh->ncell;
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 1: return launch_f<2>(dq, form, a, nc, s);
    case 2: return launch_f<3>(dq, form, a, nc, s);
    case 3: return launch_f<4>(dq, form, a, nc, s);
    case 4: return launch_f<5>(dq, form, a, nc, s);
    case 5: return launch_f<6>(dq, form, a, nc, s);
    case 6: return launch_f<7>(dq, form, a, nc, s);
    case 7: return launch_f<8>(dq, form, a, nc, s);
    case 8: return launch_f<9>(dq, form, a, nc, s);
  }
  return -1;
}

}  // namespace sfx
