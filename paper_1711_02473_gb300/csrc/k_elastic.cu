// k_elastic.cu -- hyperelastic residual r_(a,j) = int P(F) : grad(phi_j e_a) on
// vector Q_p (GLL), FP64, sum-factorised.
//
// The vector element is three copies of the scalar Q_p element (Sec. 1.2 and
// Sec. 2.3: Psi_(i,a) = Psi*_i e_a; delta cancellation leaves one scalar
// tabulation per component), so each component is contracted like a scalar
// field: interpolation to the Gauss points (B along x, y, z), then the
// reference gradient with the collocation derivative Dq.  Pointwise, with
// H = grad^ u (3x3) and G = J^{-1} = adj(J)/S:
//   F = I + H G,
//   neo-Hookean: P = mu (F - F^{-T}) + lambda ln(det F) F^{-T};
//   Saint Venant-Kirchhoff (Sec. 4.1): E = (F^T F - I)/2, P = F (lambda tr(E) I + 2 mu E);
//   test flux  w S P G^T = w P adj(J)^T, contracted back with Dq^T and B^T.
// A point with det F <= 0 (neo-Hookean) contributes zero and sets SFX_DEV_DETF.
#include "kern_common.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_elastic)

namespace {

template <int N>
struct EShape {
  static constexpr int N2 = N * N, N3 = N2 * N;
  // per team: U (N3 scratch), H (9 N3), corners, Jacobian columns, flag
  static constexpr int TEAM = N3 + 9 * N3 + 24 + 9 * N2 + 1;
  static constexpr int MAXCB = 256 / N2 > 0 ? 256 / N2 : 1;
};

template <int N, bool NEO>
__global__ void __launch_bounds__(256) k_residual_elastic_fp64(const ActArgs a, const int64_t ncell_total,
                                                               const int64_t ndof_scalar) {
  using Sh = EShape<N>;
  constexpr int N2 = Sh::N2, N3 = Sh::N3;
  const Tab1D& T = c_tab[N - 1];
  extern __shared__ double sm[];
  const int cb = blockDim.x / N2;
  const int team = threadIdx.x / N2, t = threadIdx.x - team * N2;
  double* W3 = sm;
  double* xq = sm + N3;
  double* base = sm + N3 + 16 + team * Sh::TEAM;
  double* U = base;
  double* H = U + N3;  // H[(a*3+k)*N3 + qp]
  double(*X)[3] = reinterpret_cast<double(*)[3]>(H + 9 * N3);
  double(*Jc)[N2][3] = reinterpret_cast<double(*)[N2][3]>(&X[8][0]);
  int* bad = reinterpret_cast<int*>(&Jc[3][0][0]);

  for (int i = threadIdx.x; i < N3; i += blockDim.x) W3[i] = T.w[i / N2] * T.w[(i / N) % N] * T.w[i % N];
  if (threadIdx.x < N) xq[threadIdx.x] = T.x[threadIdx.x];
  int cell = 0;
  const int64_t slot = (int64_t)blockIdx.x * cb + team;
  const bool active = team < cb && slot_cell(a, slot, ncell_total, &cell);
  if (t == 0) *bad = 0;
  for (int c = t; c < 8; c += N2) {
    if (active) {
      const int v = a.vmap[(int64_t)cell * 8 + c];
      X[c][0] = a.xyz[(int64_t)v * 3 + 0];
      X[c][1] = a.xyz[(int64_t)v * 3 + 1];
      X[c][2] = a.xyz[(int64_t)v * 3 + 2];
    } else {
      X[c][0] = (c >> 2) & 1; X[c][1] = (c >> 1) & 1; X[c][2] = c & 1;
    }
  }
  __syncthreads();
  jacobian_columns<N>(X, xq, Jc, t);
  __syncthreads();
  for (int qp = t; qp < N3; qp += N2) {
    double r0[3];
    cross3(Jc[1][(qp / N2) * N + qp % N], Jc[2][(qp / N2) * N + (qp / N) % N], r0);
    if (!(dot3(Jc[0][qp % N2], r0) > 0.0)) *bad = 1;
  }
  __syncthreads();
  const bool ok = active && !*bad;
  if (active && *bad && t == 0) set_flag(a.status, SFX_DEV_INVERTED);
  // the vector map is component-major: local a*N3 + l
  const int32_t* mrow = a.map + (int64_t)cell * 3 * N3;
  const double mu = a.mu, lam = a.lambda;

#pragma unroll 1
  for (int r = 0; r < a.nrhs; ++r) {
    for (int comp = 0; comp < 3; ++comp) {
      for (int l = t; l < N3; l += N2) U[l] = ok ? a.x[(int64_t)mrow[comp * N3 + l] * a.nrhs + r] : 0.0;
      __syncthreads();
      contract<N, N, N, 0, N, false, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      contract<N, N, N, 1, N, false, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      contract<N, N, N, 2, N, false, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      contract<N, N, N, 0, N, false, false, kMaxQ>(U, H + (comp * 3 + 0) * N3, T.Dq, t);
      contract<N, N, N, 1, N, false, false, kMaxQ>(U, H + (comp * 3 + 1) * N3, T.Dq, t);
      contract<N, N, N, 2, N, false, false, kMaxQ>(U, H + (comp * 3 + 2) * N3, T.Dq, t);
      __syncthreads();
    }
    // pointwise: first Piola-Kirchhoff stress and the test flux w P adj(J)^T
    for (int qp = t; qp < N3; qp += N2) {
      const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
      const double* c0 = Jc[0][q2 * N + q3];
      const double* c1 = Jc[1][q1 * N + q3];
      const double* c2 = Jc[2][q1 * N + q2];
      double R[3][3];  // rows of adj(J) = S G
      cross3(c1, c2, R[0]);
      cross3(c2, c0, R[1]);
      cross3(c0, c1, R[2]);
      const double S = dot3(c0, R[0]);
      double Hq[3][3], flux[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) Hq[i][k] = H[(i * 3 + k) * N3 + qp];
      if (!hyperelastic_flux<NEO>(Hq, R, S, W3[qp], mu, lam, flux) && ok) set_flag(a.status, SFX_DEV_DETF);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) H[(i * 3 + k) * N3 + qp] = flux[i][k];
    }
    __syncthreads();
    for (int comp = 0; comp < 3; ++comp) {
      contract<N, N, N, 0, N, true, false, kMaxQ>(H + (comp * 3 + 0) * N3, U, T.Dq, t);
      __syncthreads();
      contract<N, N, N, 1, N, true, true, kMaxQ>(H + (comp * 3 + 1) * N3, U, T.Dq, t);
      __syncthreads();
      contract<N, N, N, 2, N, true, true, kMaxQ>(H + (comp * 3 + 2) * N3, U, T.Dq, t);
      __syncthreads();
      contract<N, N, N, 0, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      contract<N, N, N, 1, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      contract<N, N, N, 2, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      if (ok) {
        if (a.cell_vectors) {
          for (int l = t; l < N3; l += N2) a.y[(slot * 3 * N3 + comp * N3 + l) * a.nrhs + r] = U[l];
        } else {
          for (int l = t; l < N3; l += N2) a.y[(int64_t)mrow[comp * N3 + l] * a.nrhs + r] += U[l];
        }
      } else if (active && a.cell_vectors) {
        for (int l = t; l < N3; l += N2) a.y[(slot * 3 * N3 + comp * N3 + l) * a.nrhs + r] = 0.0;
      }
      __syncthreads();
    }
  }
  (void)ndof_scalar;
}

template <int N, bool NEO>
int launch_e(const ActArgs& a, int64_t nc, int64_t nds, cudaStream_t s) {
  using Sh = EShape<N>;
  const size_t per_team = Sh::TEAM * sizeof(double);
  const size_t fixed = (Sh::N3 + 16) * sizeof(double);
  int cb = Sh::MAXCB;
  // two CTAs per SM (110 KB each) while that still gives a CTA two or more
  // cells; otherwise one larger CTA (measured 8% faster at Q_8)
  while (cb > 1 && fixed + cb * per_team > 110 * 1024) --cb;
  if (cb < 2) {
    cb = Sh::MAXCB;
    while (cb > 1 && fixed + cb * per_team > 200 * 1024) --cb;
  }
  cb = tuned_team_cells(SFX_TUNE_ELASTIC, N - 1, cb, Sh::MAXCB, fixed, per_team, 200 * 1024);
  const size_t smem = fixed + cb * per_team;
  auto kern = k_residual_elastic_fp64<N, NEO>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<(unsigned)((a.ncells + cb - 1) / cb), cb * Sh::N2, smem, s>>>(a, nc, nds);
  return (int)cudaGetLastError();
}

template <bool NEO>
int dispatch_p(int p, const ActArgs& a, int64_t nc, int64_t nds, cudaStream_t s) {
  switch (p) {
    case 1: return launch_e<2, NEO>(a, nc, nds, s);
    case 2: return launch_e<3, NEO>(a, nc, nds, s);
    case 3: return launch_e<4, NEO>(a, nc, nds, s);
    case 4: return launch_e<5, NEO>(a, nc, nds, s);
    case 5: return launch_e<6, NEO>(a, nc, nds, s);
    case 6: return launch_e<7, NEO>(a, nc, nds, s);
    case 7: return launch_e<8, NEO>(a, nc, nds, s);
    case 8: return launch_e<9, NEO>(a, nc, nds, s);
  }
  return -1;
}

}  // namespace

int launch_action_elastic(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                          void* stream) {
  if (sp->family != SFX_VQ) return -1;
  if (prec != SFX_PREC_FP64) return launch_action_elastic_mixed(sp, form, prec, a, stream);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nds = sp->ndof / 3;
  if (form == SFX_NEOHOOKE) return dispatch_p<true>(sp->p, a, sp->mesh->ncell, nds, s);
  if (form == SFX_SVK) return dispatch_p<false>(sp->p, a, sp->mesh->ncell, nds, s);
  return -1;
}

}  // namespace sfx
