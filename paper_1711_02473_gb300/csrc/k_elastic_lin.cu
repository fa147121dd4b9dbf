// k_elastic_lin.cu -- action of the linearised hyperelastic operator on
// vector Q_p (GLL), FP64, sum-factorised:
//   y_(a,j) = sum_K int dP(F(u); dF) : grad(phi_j e_a),  F = I + grad u, dF = grad du,
// the Jacobian of the residual of k_elastic.cu (the operator whose action the
// paper's hyperelastic experiments time, Sec. 4.1, for the Saint Venant-
// Kirchhoff law; the neo-Hookean law is the same skeleton).
//
// Per cell: the state's reference gradient grad^ u (9 fields at the points) is
// formed once by the same per-component contractions as the residual (B along
// x, y, z, then the collocation derivative Dq), then for every direction du
// its gradient grad^ du, the pointwise linearised stress and the test flux
// w S dP G^T = w dP adj(J)^T, contracted back with Dq^T and B^T and added
// through the map (conflict-free per colour).  Pointwise, with G = adj(J)/S:
//   neo-Hookean  dP = mu dF + (mu - lambda ln J) F^{-T} dF^T F^{-T} + lambda tr(F^{-1} dF) F^{-T}
//   SVK          dP = dF S + F (lambda tr(dE) I + 2 mu dE),  dE = sym(F^T dF)
// A point with det F <= 0 (neo-Hookean) contributes zero and sets SFX_DEV_DETF.
//
// Element (tangent) matrices, a.unit_cols > 0: the directions are the cell's
// trial basis functions psi_j e_b themselves, and column (b,j) of A^K is the
// cell vector above for that direction.  Per CTA (its chunk of columns) the
// state's gradient and geometry are formed once, and so is the state-only
// part of the linearised stress at every point (neo-Hookean F^{-T} and
// mu - lambda ln J; SVK F and S), kept in shared memory.  Per direction: its
// reference gradient is the tensor product of the tabulated derivative and
// values (Dc x Bc x Bc, no forward contractions), its dF has one nonzero row,
// so dP costs a rank-one update of the cached state terms, and the transposed
// contractions run as for the action.  Cost per cell: 3 n^3 directions x
// O(n^4) = O(n^7), the order of the sum-factorised element matrices (Sec. 3.2).
#include "elastic_common.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_elastic_lin)

namespace {

template <int N>
struct LShape {
  static constexpr int N2 = N * N, N3 = N2 * N;
  // per team: U (N3 scratch), Hs (9 N3, state), Hd (9 N3, direction / flux),
  // corners, Jacobian columns, flag
  static constexpr int TEAM = N3 + 18 * N3 + 24 + 9 * N2 + 1;
  // element matrices: U, the state cache (16 per point, replacing Hs), Hd, ...
  static constexpr int MTEAM = N3 + 25 * N3 + 24 + 9 * N2 + 1;
  static constexpr int MAXCB = 256 / N2 > 0 ? 256 / N2 : 1;
};

// State-only terms of the linearised stress at one point (16 slots):
// neo-Hookean  C[0..8] = F^{-T}, C[9] = mu - lambda ln det F, C[10] = 1 (0 if det F <= 0);
// SVK          C[0..8] = F, C[9..14] = S (00, 11, 22, 01, 02, 12).
template <bool NEO>
__device__ __forceinline__ void state_terms(const double (*Hs)[3], const double (*R)[3], double S, double mu,
                                            double lam, double* C) {
  const double iS = recip_nr<2>(S);
  double F[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F[i][j] = (Hs[i][0] * R[0][j] + Hs[i][1] * R[1][j] + Hs[i][2] * R[2][j]) * iS + (i == j ? 1.0 : 0.0);
  if (NEO) {
    double Cf[3][3];
    cross3(F[1], F[2], Cf[0]);
    cross3(F[2], F[0], Cf[1]);
    cross3(F[0], F[1], Cf[2]);
    const double JF = dot3(F[0], Cf[0]);
    const bool good = JF > 0.0;
    const double iJ = good ? recip_nr<2>(JF) : 0.0, lnJ = good ? log(JF) : 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) C[i * 3 + j] = Cf[i][j] * iJ;
    C[9] = mu - lam * lnJ;
    C[10] = good ? 1.0 : 0.0;
  } else {
    double E[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        E[a][b] = 0.5 * (F[0][a] * F[0][b] + F[1][a] * F[1][b] + F[2][a] * F[2][b] - (a == b ? 1.0 : 0.0));
    const double trE = E[0][0] + E[1][1] + E[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) C[i * 3 + j] = F[i][j];
    C[9] = lam * trE + 2.0 * mu * E[0][0];
    C[10] = lam * trE + 2.0 * mu * E[1][1];
    C[11] = lam * trE + 2.0 * mu * E[2][2];
    C[12] = 2.0 * mu * E[0][1];
    C[13] = 2.0 * mu * E[0][2];
    C[14] = 2.0 * mu * E[1][2];
  }
}

// Linearised test flux for a direction whose displacement has only component
// bc, with reference gradient hd (3): dF = e_bc (x) v, v = hd adj(J) / S, so
//   neo-Hookean  dP = mu dF + c (F^{-T} v) (x) F^{-T}[bc] + lambda (F^{-T}[bc] . v) F^{-T}
//   SVK          dP = e_bc (x) (S v) + F (lambda tr dE I + 2 mu dE),
//                dE = (v (x) F[bc] + F[bc] (x) v) / 2,
// from the cached state terms C; out[i][k] = w sum_j dP[i][j] R[k][j].
// False (zero flux) where det F <= 0 (neo-Hookean).
template <bool NEO>
__device__ __forceinline__ bool unit_flux(const double* C, int bc, const double* hd, const double (*R)[3],
                                          double S, double w, double mu, double lam, double (*out)[3]) {
  const double iS = recip_nr<2>(S);
  double v[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) v[j] = (hd[0] * R[0][j] + hd[1] * R[1][j] + hd[2] * R[2][j]) * iS;
  double dP[3][3];
  bool good = true;
  // row bc of the cached F^{-T} (neo-Hookean) or F (SVK), selected in registers
  double Fb[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) Fb[j] = bc == 0 ? C[j] : (bc == 1 ? C[3 + j] : C[6 + j]);
  if (NEO) {
    good = C[10] != 0.0;
    double Fv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Fv[i] = C[i * 3 + 0] * v[0] + C[i * 3 + 1] * v[1] + C[i * 3 + 2] * v[2];
    const double tr = Fb[0] * v[0] + Fb[1] * v[1] + Fb[2] * v[2];
    const double c = C[9], lt = lam * tr;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double d = (i == bc ? mu * v[j] : 0.0) + c * Fv[i] * Fb[j] + lt * C[i * 3 + j];
        dP[i][j] = good ? d : 0.0;
      }
  } else {
    const double S2[3][3] = {{C[9], C[12], C[13]}, {C[12], C[10], C[14]}, {C[13], C[14], C[11]}};
    double dE[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) dE[a][b] = 0.5 * (v[a] * Fb[b] + Fb[a] * v[b]);
    const double ltr = lam * (dE[0][0] + dE[1][1] + dE[2][2]);
    double dS[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) dS[a][b] = (a == b ? ltr : 0.0) + 2.0 * mu * dE[a][b];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double d = C[i * 3 + 0] * dS[0][j] + C[i * 3 + 1] * dS[1][j] + C[i * 3 + 2] * dS[2][j];
        if (i == bc) d += v[0] * S2[0][j] + v[1] * S2[1][j] + v[2] * S2[2][j];
        dP[i][j] = d;
      }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) out[i][k] = w * dot3(dP[i], R[k]);
  return good;
}

// Reference gradient of component `comp` of the field v (component-major
// vector map mrow) into H[(comp*3 + k)*N3 + qp], via U.
template <int N>
__device__ __forceinline__ void component_gradient(const Tab1D& T, const double* v, int nrhs, int r,
                                                   const int32_t* mrow, bool ok, int comp, double* U, double* H,
                                                   int t) {
  constexpr int N2 = N * N, N3 = N2 * N;
  for (int l = t; l < N3; l += N2) U[l] = ok ? v[(int64_t)mrow[comp * N3 + l] * nrhs + r] : 0.0;
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

template <int N, bool NEO>
__global__ void __launch_bounds__(256) k_linearised_elastic_fp64(const ActArgs a, const int64_t ncell_total) {
  using Sh = LShape<N>;
  constexpr int N2 = Sh::N2, N3 = Sh::N3;
  const Tab1D& T = c_tab[N - 1];
  extern __shared__ double sm[];
  const int cb = blockDim.x / N2;
  const int team = threadIdx.x / N2, t = threadIdx.x - team * N2;
  const bool mat = a.unit_cols > 0;  // element matrices (see the file comment)
  double* W3 = sm;
  double* xq = sm + N3;
  double* Bs = xq + 16;  // element matrices: Bc and Dc (values and derivatives at the points)
  double* Ds = Bs + N2;
  double* base = sm + N3 + 16 + (mat ? 2 * N2 + team * Sh::MTEAM : team * Sh::TEAM);
  double* U = base;
  double* Hs = U + N3;                        // state gradient (element matrices: then the state terms)
  double* Hd = Hs + (mat ? 16 : 9) * N3;      // direction gradient, then the flux
  double(*X)[3] = reinterpret_cast<double(*)[3]>(Hd + 9 * N3);
  double(*Jc)[N2][3] = reinterpret_cast<double(*)[N2][3]>(&X[8][0]);
  int* bad = reinterpret_cast<int*>(&Jc[3][0][0]);

  for (int i = threadIdx.x; i < N3; i += blockDim.x) W3[i] = T.w[i / N2] * T.w[(i / N) % N] * T.w[i % N];
  if (threadIdx.x < N) xq[threadIdx.x] = T.x[threadIdx.x];
  if (mat)
    for (int i = threadIdx.x; i < N2; i += blockDim.x) {
      Bs[i] = T.Bc[i / N][i % N];
      Ds[i] = T.Dc[i / N][i % N];
    }
  int cell = 0;
  const int64_t slot = (int64_t)blockIdx.x * cb + team;
  const bool active = slot_cell(a, slot, ncell_total, &cell);
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
    double r0[3], r1[3], r2[3];
    if (!(point_rows<N, false>(Jc, qp, r0, r1, r2) > 0.0)) *bad = 1;
  }
  __syncthreads();
  const bool ok = active && !*bad;
  if (active && *bad && t == 0) set_flag(a.status, SFX_DEV_INVERTED);
  const int32_t* mrow = a.map + (int64_t)cell * 3 * N3;
  const double mu = a.mu, lam = a.lambda;

  // the state's reference gradient, once per cell
  for (int comp = 0; comp < 3; ++comp) component_gradient<N>(T, a.xs, 1, 0, mrow, ok, comp, U, Hs, t);

  // element matrices: the state-only terms of dP at every point, once (in
  // place of the state gradient: each point is read and rewritten by its owner)
  constexpr int NC = NEO ? 11 : 15;
  if (mat) {
    for (int qp = t; qp < N3; qp += N2) {
      double R[3][3], hs[3][3], C[16];
      const double S = point_rows<N, true>(Jc, qp, R[0], R[1], R[2]);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) hs[i][k] = Hs[(i * 3 + k) * N3 + qp];
      state_terms<NEO>(hs, R, S, mu, lam, C);
      if (NEO && C[10] == 0.0 && ok) set_flag(a.status, SFX_DEV_DETF);
#pragma unroll
      for (int k = 0; k < NC; ++k) Hs[k * N3 + qp] = C[k];
    }
    __syncthreads();
  }

  // action: the RHS r = 0..nrhs-1; element matrices: this CTA's chunk of
  // trial columns (the same for every team of the CTA)
  constexpr int NLOC = 3 * N3;
  const int rb = mat ? (int)blockIdx.y * a.unit_cols : 0;
  const int re = mat ? min(NLOC, rb + a.unit_cols) : a.nrhs;
#pragma unroll 1
  for (int r = rb; r < re; ++r) {
    if (mat) {
      // direction psi_j e_bc: reference gradient Dc (x) Bc (x) Bc at the points
      const int bc = r / N3, lj = r - bc * N3;
      const int j1 = lj / N2, j2 = (lj / N) % N, j3 = lj % N;
      for (int qp = t; qp < N3; qp += N2) {
        const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
        const double b1 = Bs[q1 * N + j1], b2 = Bs[q2 * N + j2], b3 = Bs[q3 * N + j3];
        const double hd[3] = {Ds[q1 * N + j1] * b2 * b3, b1 * Ds[q2 * N + j2] * b3, b1 * b2 * Ds[q3 * N + j3]};
        double R[3][3], C[16], flux[3][3];
        const double S = point_rows<N, true>(Jc, qp, R[0], R[1], R[2]);
#pragma unroll
        for (int k = 0; k < NC; ++k) C[k] = Hs[k * N3 + qp];
        unit_flux<NEO>(C, bc, hd, R, S, W3[qp], mu, lam, flux);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) Hd[(i * 3 + k) * N3 + qp] = flux[i][k];
      }
    } else {
      for (int comp = 0; comp < 3; ++comp) component_gradient<N>(T, a.x, a.nrhs, r, mrow, ok, comp, U, Hd, t);
      for (int qp = t; qp < N3; qp += N2) {
        double R[3][3];
        const double S = point_rows<N, true>(Jc, qp, R[0], R[1], R[2]);
        double hs[3][3], hd[3][3], flux[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            hs[i][k] = Hs[(i * 3 + k) * N3 + qp];
            hd[i][k] = Hd[(i * 3 + k) * N3 + qp];
          }
        if (!linearised_flux<NEO>(hs, hd, R, S, W3[qp], mu, lam, flux) && ok) set_flag(a.status, SFX_DEV_DETF);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) Hd[(i * 3 + k) * N3 + qp] = flux[i][k];
      }
    }
    __syncthreads();
    for (int comp = 0; comp < 3; ++comp) {
      contract<N, N, N, 0, N, true, false, kMaxQ>(Hd + (comp * 3 + 0) * N3, U, T.Dq, t);
      __syncthreads();
      contract<N, N, N, 1, N, true, true, kMaxQ>(Hd + (comp * 3 + 1) * N3, U, T.Dq, t);
      __syncthreads();
      contract<N, N, N, 2, N, true, true, kMaxQ>(Hd + (comp * 3 + 2) * N3, U, T.Dq, t);
      __syncthreads();
      contract<N, N, N, 0, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      contract<N, N, N, 1, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      contract<N, N, N, 2, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      if (mat) {
        if (active)
          for (int l = t; l < N3; l += N2) a.y[(slot * NLOC + comp * N3 + l) * NLOC + r] = ok ? U[l] : 0.0;
      } else if (ok) {
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
}

template <int N, bool NEO>
int launch_l(const ActArgs& a, int64_t nc, cudaStream_t s) {
  using Sh = LShape<N>;
  const bool mat = a.unit_cols > 0;
  const size_t per_team = (mat ? Sh::MTEAM : Sh::TEAM) * sizeof(double);
  const size_t fixed = (Sh::N3 + 16 + (mat ? 2 * Sh::N2 : 0)) * sizeof(double);
  int cb = Sh::MAXCB;
  // two CTAs per SM (110 KB each), even at one cell per CTA (measured faster
  // at Q_6 than one CTA of two cells)
  while (cb > 1 && fixed + cb * per_team > 110 * 1024) --cb;
  if (!mat) cb = tuned_team_cells(SFX_TUNE_LINEARISED, N - 1, cb, Sh::MAXCB, fixed, per_team, 200 * 1024);
  const size_t smem = fixed + cb * per_team;
  auto kern = k_linearised_elastic_fp64<N, NEO>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const unsigned chunks = a.unit_cols > 0 ? (unsigned)((3 * Sh::N3 + a.unit_cols - 1) / a.unit_cols) : 1u;
  kern<<<dim3((unsigned)((a.ncells + cb - 1) / cb), chunks), cb * Sh::N2, smem, s>>>(a, nc);
  return (int)cudaGetLastError();
}

template <bool NEO>
int dispatch_p(int p, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (p) {
    case 1: return launch_l<2, NEO>(a, nc, s);
    case 2: return launch_l<3, NEO>(a, nc, s);
    case 3: return launch_l<4, NEO>(a, nc, s);
    case 4: return launch_l<5, NEO>(a, nc, s);
    case 5: return launch_l<6, NEO>(a, nc, s);
    case 6: return launch_l<7, NEO>(a, nc, s);
    case 7: return launch_l<8, NEO>(a, nc, s);
    case 8: return launch_l<9, NEO>(a, nc, s);
  }
  return -1;
}

}  // namespace

int launch_linearised_elastic(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  if (sp->family != SFX_VQ) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  if (form == SFX_NEOHOOKE) return dispatch_p<true>(sp->p, a, sp->mesh->ncell, s);
  if (form == SFX_SVK) return dispatch_p<false>(sp->p, a, sp->mesh->ncell, s);
  return -1;
}

}  // namespace sfx
