// scalar_body.cuh -- device body of the FP64 scalar-form action (mass,
// Laplace, Helmholtz on Q_p / DQ_p), shared by the per-colour kernels
// (k_scalar.cu) and the persistent batched kernel (k_batched.cu).
//
// Per cell (Sec. 3.3, Eqs. coeff_def / coeff_eval / form_eval):
//   1. gather U^K through the cell-node map;
//   2. interpolate to the (p+1)^3 Gauss points with three 1D contractions by
//      the GLL->Gauss table B (x, then y, then z; Sec. 3.2 sum factorisation;
//      for DQ_p the nodes are the Gauss points and B = I, Sec. 2.5 Eq. colocated);
//   3. reference gradient at the points: one 1D contraction per axis with the
//      collocation derivative Dq on the Gauss points (exact: Q_p restricted to
//      a line is a degree-p polynomial, fixed by its p+1 Gauss values);
//   4. pointwise: geometry from the trilinear coordinate field (J, S = det J,
//      adj J) and the geometric factor P = w S G G^T (the P^(k,l) of Sec. 3.2);
//      flux f = P grad u (Laplace) and/or w S u (mass);
//   5. transposed contractions Dq^T then B^T;
//   6. add b^K into y through the map (conflict-free within one colour).
// Where the factors P and w S come from:
//   - geo_once (several right-hand sides): computed once per cell into shared
//     memory and reused for every RHS;
//   - otherwise at the point, when the flux is formed (no shared copy: a
//     smaller footprint, more resident warps);
//   - STORED: read from sfx_qdata instead of computed.
#pragma once
#include "kern_common.cuh"

namespace sfx {
namespace {

template <int N, int FORM, bool KAP = false>
struct ScalarShape {
  static constexpr int N2 = N * N, N3 = N * N * N;
  static constexpr bool LAP = FORM != SFX_MASS;
  static constexpr bool MAS = FORM != SFX_LAPLACE;
  // per-team shared doubles: U, G0..G2 (LAP), corners, Jacobian columns, flag
  static constexpr int LEAN = N3 + (LAP ? 3 * N3 : 0) + 24 + 9 * N2 + 1;
  // plus the staged factors K[6] (LAP) and WS (MAS) when geo_once
  static constexpr int FULL = LEAN + (LAP ? 6 * N3 : 0) + (MAS ? N3 : 0);
  static constexpr int TEAM = FULL + (KAP ? N3 : 0);
  static constexpr int MAXCB = (256 / N2) > 0 ? 256 / N2 : 1;
  // KAP: the coefficient kappa at the points follows (weighted Laplace)
  static constexpr int team_doubles(bool geo_once) { return (geo_once ? FULL : LEAN) + (KAP ? N3 : 0); }
};

// The factors at point qp of a cell: P (6 symmetric entries, scaled by alpha)
// and w S (scaled by beta), from the Jacobian column tables.  Returns S.
// 1/S is a two-step Newton reciprocal (FP64 rounding level).
template <int N, bool LAP, bool MAS>
__device__ __forceinline__ double point_factors(const double (*Jc)[N * N][3], const double* W3, int qp,
                                                double alpha, double beta, double* K, double* ws_mass) {
  double r0[3], r1[3], r2[3];
  const double S = point_rows<N, LAP>(Jc, qp, r0, r1, r2);
  if (LAP) {
    const double ws = alpha * W3[qp] * recip_nr<2>(S);  // P = w S G G^T = (w/S) adj(J) adj(J)^T
    K[0] = ws * dot3(r0, r0);
    K[1] = ws * dot3(r1, r1);
    K[2] = ws * dot3(r2, r2);
    K[3] = ws * dot3(r0, r1);
    K[4] = ws * dot3(r0, r2);
    K[5] = ws * dot3(r1, r2);
  }
  if (MAS) *ws_mass = beta * W3[qp] * S;
  return S;
}

// One tile: the cb cells of slots slot0 .. slot0+cb-1, one team of N^2 threads
// per cell (threads of teams >= cb idle but take part in the barriers).
// COLL: the collocated Gauss-Lobatto rule on the GLL nodes of Q_p (Sec. 2.5,
// "underintegration" in Sec. 4.1): the points are the nodes, so B = I as for
// DQ_p, the derivative table is the GLL collocation matrix and the geometry is
// evaluated at the GLL points with the GLL weights.
// KAP: the weighted Laplace form int kappa grad u . grad v (Sec. 1.1, Eq.
// weighted_laplace): kappa (a.kappa, dofs in the same space) is gathered once
// per cell, interpolated to the points by the same B contractions, and scales
// the geometric factor P at each point.
template <int N, bool DQ, int FORM, bool STORED = false, bool COLL = false, bool KAP = false>
__device__ __forceinline__ void scalar_tile_fp64(const ActArgs& a, const int64_t ncell_total, const int64_t slot0,
                                                 const int cb, double* sm, const bool geo_once) {
  using Sh = ScalarShape<N, FORM, KAP>;
  constexpr int N2 = Sh::N2, N3 = Sh::N3;
  constexpr bool LAP = Sh::LAP, MAS = Sh::MAS;
  const Tab1D& T = c_tab[N - 1];
  // Threads beyond the cb teams (the persistent kernel runs 256 threads for
  // every degree) only take part in the barriers: they alias team 0's shared
  // memory for pointer arithmetic but never read or write it.
  const int team_raw = threadIdx.x / N2;
  const bool member = team_raw < cb;
  const int team = member ? team_raw : 0;
  const int t = threadIdx.x - team_raw * N2;
  double* W3 = sm;              // 3D quadrature weights
  double* xq = sm + N3;         // 1D points (padded to 16)
  double* base = sm + N3 + 16 + team * Sh::team_doubles(geo_once);
  double* U = base;
  double* G0 = U + N3;
  double* G1 = G0 + N3;
  double* G2 = G1 + N3;
  double* X0 = LAP ? G2 + N3 : U + N3;
  double(*X)[3] = reinterpret_cast<double(*)[3]>(X0);
  double(*Jc)[N2][3] = reinterpret_cast<double(*)[N2][3]>(X0 + 24);
  int* bad = reinterpret_cast<int*>(X0 + 24 + 9 * N2);
  double* K = X0 + 24 + 9 * N2 + 1;                  // K[c][qp] (geo_once only)
  double* WS = K + (LAP ? 6 * N3 : 0);               // WS[qp]   (geo_once only)
  double* KA = base + Sh::team_doubles(geo_once) - (KAP ? N3 : 0);  // kappa at the points (KAP only)

  const double* tw = COLL ? T.wg : T.w;
  const double(*TD)[kMaxQ] = COLL ? T.Dg : T.Dq;  // derivative at the points
  for (int i = threadIdx.x; i < N3; i += blockDim.x) W3[i] = tw[i / N2] * tw[(i / N) % N] * tw[i % N];
  if (threadIdx.x < N) xq[threadIdx.x] = COLL ? T.xg[threadIdx.x] : T.x[threadIdx.x];

  int cell = 0;
  const int64_t slot = slot0 + team;
  const bool active = member && slot_cell(a, slot, ncell_total, &cell);
  if (member && t == 0) *bad = 0;
  const double alpha = FORM == SFX_HELMHOLTZ ? a.alpha : 1.0;
  const double beta = FORM == SFX_HELMHOLTZ ? a.beta : 1.0;
  const double* qd = STORED ? a.qd64 + (int64_t)cell * 7 * N3 : nullptr;
  if (!STORED) {
    for (int c = member ? t : 8; c < 8; c += N2) {  // a team may have fewer than 8 threads (p = 1)
      if (active) {
        const int v = a.vmap[(int64_t)cell * 8 + c];
        X[c][0] = a.xyz[(int64_t)v * 3 + 0];
        X[c][1] = a.xyz[(int64_t)v * 3 + 1];
        X[c][2] = a.xyz[(int64_t)v * 3 + 2];
      } else {  // idle team: unit cube keeps the arithmetic finite
        X[c][0] = (c >> 2) & 1; X[c][1] = (c >> 1) & 1; X[c][2] = c & 1;
      }
    }
  }
  __syncthreads();
  pdl_allow_next();
  if (!STORED && member) jacobian_columns<N>(X, xq, Jc, t);
  __syncthreads();
  if (KAP) {
    const int32_t* krow = a.map ? a.map + (int64_t)cell * N3 : nullptr;
    const int64_t koff = a.dq_off ? a.dq_off[cell] : 0;
    for (int l = member ? t : N3; l < N3; l += N2)
      KA[l] = active ? a.kappa[krow ? (int64_t)krow[l] : koff + l] : 0.0;
    __syncthreads();
    if (!DQ && !COLL) {
      if (member) contract<N, N, N, 0, N, false, false, kMaxN>(KA, KA, T.Bc, t);
      __syncthreads();
      if (member) contract<N, N, N, 1, N, false, false, kMaxN>(KA, KA, T.Bc, t);
      __syncthreads();
      if (member) contract<N, N, N, 2, N, false, false, kMaxN>(KA, KA, T.Bc, t);
      __syncthreads();
    }
  }
  if (geo_once) {
    // factors at the thread's points qp = k*N2 + t, staged for all RHS
#pragma unroll 1
    for (int k = 0; k < (member ? N : 0); ++k) {
      const int qp = k * N2 + t;
      if (STORED) {
        if (LAP)
          for (int j = 0; j < 6; ++j) K[j * N3 + qp] = active ? alpha * qd[j * N3 + qp] : 0.0;
        if (MAS) WS[qp] = active ? beta * qd[6 * N3 + qp] : 0.0;
      } else {
        double kk[6], wsm = 0.0;
        const double S = point_factors<N, LAP, MAS>(Jc, W3, qp, alpha, beta, kk, &wsm);
        if (!positive_finite(S)) *bad = 1;
        const double kap = KAP ? KA[qp] : 1.0;
        if (LAP)
          for (int j = 0; j < 6; ++j) K[j * N3 + qp] = KAP ? kap * kk[j] : kk[j];
        if (MAS) WS[qp] = wsm;
      }
    }
    __syncthreads();
  }
  const int tl = member ? t : N3;  // first index of this thread's strided loops (none for non-members)

  // dof of local l: the space's map, or cell offset + l for p-adaptive DQ
  const int32_t* mrow = a.map ? a.map + (int64_t)cell * N3 : nullptr;
  const int64_t doff = a.dq_off ? a.dq_off[cell] : 0;
  auto dof = [&](int l) -> int64_t { return mrow ? (int64_t)mrow[l] : doff + l; };
#pragma unroll 1
  for (int r = a.r0; r < a.r1; ++r) {
    for (int l = tl; l < N3; l += N2) U[l] = active ? a.x[dof(l) * a.nrhs + r] : 0.0;
    __syncthreads();
    if (!DQ && !COLL) {
      if (member) contract<N, N, N, 0, N, false, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      if (member) contract<N, N, N, 1, N, false, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      if (member) contract<N, N, N, 2, N, false, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
    }
    if (LAP) {
      if (member) {
        contract<N, N, N, 0, N, false, false, kMaxQ>(U, G0, TD, t);
        contract<N, N, N, 1, N, false, false, kMaxQ>(U, G1, TD, t);
        contract<N, N, N, 2, N, false, false, kMaxQ>(U, G2, TD, t);
      }
      __syncthreads();
    }
#pragma unroll 1
    for (int k = 0; k < (member ? N : 0); ++k) {
      const int qp = k * N2 + t;
      double kk[6] = {0, 0, 0, 0, 0, 0}, wsm = 0.0;
      if (geo_once) {
        if (LAP)
          for (int j = 0; j < 6; ++j) kk[j] = K[j * N3 + qp];
        if (MAS) wsm = WS[qp];
      } else if (STORED) {
        if (LAP)
          for (int j = 0; j < 6; ++j) kk[j] = active ? alpha * qd[j * N3 + qp] : 0.0;
        if (MAS) wsm = active ? beta * qd[6 * N3 + qp] : 0.0;
      } else {
        // at the point: the flux P g = (w/S) R R^T g with R the adjugate rows,
        // applied as R (t R^T g) without forming the six entries of P
        double r0[3], r1[3], r2[3];
        const double S = point_rows<N, LAP>(Jc, qp, r0, r1, r2);
        if (!positive_finite(S)) *bad = 1;
        if (LAP) {
          const double tw = (KAP ? alpha * W3[qp] * KA[qp] : alpha * W3[qp]) * recip_nr<2>(S);
          const double g0 = G0[qp], g1 = G1[qp], g2 = G2[qp];
          double v[3];
#pragma unroll
          for (int d = 0; d < 3; ++d) v[d] = tw * (r0[d] * g0 + r1[d] * g1 + r2[d] * g2);
          G0[qp] = dot3(r0, v);
          G1[qp] = dot3(r1, v);
          G2[qp] = dot3(r2, v);
        }
        if (MAS) U[qp] = (beta * W3[qp] * S) * U[qp];
        continue;
      }
      if (LAP) {
        const double g0 = G0[qp], g1 = G1[qp], g2 = G2[qp];
        G0[qp] = kk[0] * g0 + kk[3] * g1 + kk[4] * g2;
        G1[qp] = kk[3] * g0 + kk[1] * g1 + kk[5] * g2;
        G2[qp] = kk[4] * g0 + kk[5] * g1 + kk[2] * g2;
      }
      if (MAS) U[qp] = wsm * U[qp];
    }
    __syncthreads();
    if (LAP) {
      if (member) contract<N, N, N, 0, N, true, MAS, kMaxQ>(G0, U, TD, t);
      __syncthreads();
      if (member) contract<N, N, N, 1, N, true, true, kMaxQ>(G1, U, TD, t);
      __syncthreads();
      if (member) contract<N, N, N, 2, N, true, true, kMaxQ>(G2, U, TD, t);
      __syncthreads();
    }
    if (!DQ && !COLL) {
      if (member) contract<N, N, N, 0, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      if (member) contract<N, N, N, 1, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
      if (member) contract<N, N, N, 2, N, true, false, kMaxN>(U, U, T.Bc, t);
      __syncthreads();
    }
    // the inverted-cell flag is final here (set while forming the factors)
    if (r == a.r0) pdl_wait_prev();
    const bool ok = active && !*bad;
    if (ok) {
      if (a.cell_vectors) {
        for (int l = t; l < N3; l += N2) a.y[(slot * N3 + l) * a.nrhs + r] = U[l];
      } else {
        // reduction in L2 (red.global.add.f64): cells of one launch share no
        // dof, so each address is added to once per launch, in launch order;
        // in an overwriting action the dof's first pair stores instead
        for (int l = t; l < N3; l += N2) {
          double* yp = &a.y[dof(l) * a.nrhs + r];
          if (first_touch(a, cell, l, N3)) *yp = U[l]; else atomicAdd(yp, U[l]);
        }
      }
    } else if (active && a.cell_vectors) {
      for (int l = t; l < N3; l += N2) a.y[(slot * N3 + l) * a.nrhs + r] = 0.0;
    } else if (active) {
      for (int l = t; l < N3; l += N2)
        if (first_touch(a, cell, l, N3)) a.y[dof(l) * a.nrhs + r] = 0.0;
    }
    if (r == a.r0 && active && *bad && t == 0) set_flag(a.status, SFX_DEV_INVERTED);
    __syncthreads();
  }
}

}  // namespace
}  // namespace sfx
