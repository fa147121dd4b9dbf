// k_hdivcurl.cu -- operator actions on NCF_p (H(div)) and NCE_p (H(curl)), FP64.
//
// The elements are enriched sums of three HDiv/HCurl-wrapped tensor-product
// blocks (Sec. 2.6-2.7, Eq. rtcf_impl).  Splitting the Concatenate (Sec. 3.5,
// Eqs. rtcf_split_x/y) gives each block its own product structure, so each
// block is sum-factorised on its own, with anisotropic 1D tables:
//   NCF block c: P_p on GLL nodes (p+1) along axis c, dP_{p-1} on Gauss nodes (p)
//                across; value e_c and reference divergence d/dxi_c;
//   NCE block c: dP_{p-1} (p) along axis c, P_p (p+1) across; value e_c and the
//                reference curl, which needs the derivatives across.
// Pointwise (q = p+1 Gauss points, J from the trilinear coordinate field):
//   NCF: f_val = alpha w/S J^T J u^,  f_div = beta w/S div^ u^
//        (contravariant Piola u = J u^/S, div u = div^ u^/S)
//   NCE: f_curl = beta w/S J^T J curl^ u^,  f_val = alpha w S G G^T u^
//        (covariant Piola u = G^T u^, curl u = J curl^ u^/S)
// and the transposed contractions return b^K block by block.
#include "kern_common.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_hdivcurl)

namespace {

template <int P, bool NCF>
struct HShape {
  static constexpr int N = P + 1, Q = P + 1;
  static constexpr int N2 = N * N, Q3 = Q * Q * Q;
  static constexpr int BLK = NCF ? N * P * P : P * N * N;  // dofs per block
  static constexpr int NLOC = 3 * BLK;
  // per-team doubles: U (nloc), value arrays V0..2, derivative arrays
  // (NCF: DIV; NCE: C0..2), two temporaries, corners, Jacobian columns, flag
  static constexpr int NDER = NCF ? 1 : 3;
  static constexpr int TEAM = NLOC + 3 * Q3 + NDER * Q3 + 2 * Q3 + 24 + 9 * N2 + 1;
  static constexpr int MAXCB = 256 / N2 > 0 ? 256 / N2 : 1;
};

template <int P, bool NCF>
__global__ void __launch_bounds__(256) k_action_hdivcurl_fp64(const ActArgs a, const int64_t ncell_total) {
  using Sh = HShape<P, NCF>;
  constexpr int N = Sh::N, Q = Sh::Q, N2 = Sh::N2, Q3 = Sh::Q3, BLK = Sh::BLK, NLOC = Sh::NLOC;
  const Tab1D& T = c_tab[P];
  extern __shared__ double sm[];
  const int cb = blockDim.x / N2;
  const int team = threadIdx.x / N2, t = threadIdx.x - team * N2;
  double* W3 = sm;
  double* xq = sm + Q3;
  double* base = sm + Q3 + 16 + team * Sh::TEAM;
  double* U = base;
  double* V = U + NLOC;          // V[c*Q3 + qp]
  double* D = V + 3 * Q3;        // NCF: DIV; NCE: C0..C2
  double* T1 = D + Sh::NDER * Q3;
  double* T2 = T1 + Q3;
  double(*X)[3] = reinterpret_cast<double(*)[3]>(T2 + Q3);
  double(*Jc)[N2][3] = reinterpret_cast<double(*)[N2][3]>(&X[8][0]);
  int* bad = reinterpret_cast<int*>(&Jc[3][0][0]);

  for (int i = threadIdx.x; i < Q3; i += blockDim.x) W3[i] = T.w[i / (Q * Q)] * T.w[(i / Q) % Q] * T.w[i % Q];
  if (threadIdx.x < Q) xq[threadIdx.x] = T.x[threadIdx.x];
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
  // det J at every point (bad-cell check), before any arithmetic uses 1/S
  for (int qp = t; qp < Q3; qp += N2) {
    const int q1 = qp / (Q * Q), q2 = (qp / Q) % Q, q3 = qp % Q;
    double r0[3];
    cross3(Jc[1][q1 * Q + q3], Jc[2][q1 * Q + q2], r0);
    if (!(dot3(Jc[0][q2 * Q + q3], r0) > 0.0)) *bad = 1;
  }
  __syncthreads();
  const bool ok = active && !*bad;
  if (active && *bad && t == 0) set_flag(a.status, SFX_DEV_INVERTED);
  const int32_t* mrow = a.map + (int64_t)cell * NLOC;
  double* V0 = V;
  double* V1 = V + Q3;
  double* V2 = V + 2 * Q3;

#pragma unroll 1
  for (int r = 0; r < a.nrhs; ++r) {
    for (int l = t; l < NLOC; l += N2) U[l] = ok ? a.x[(int64_t)mrow[l] * a.nrhs + r] : 0.0;
    __syncthreads();
    if (NCF) {
      // block 0: (N,P,P) -> axis1 Bd -> (N,Q,P) -> axis2 Bd -> (N,Q,Q) -> axis0 Bc/Dc
      const double* u0 = U;
      const double* u1 = U + BLK;
      const double* u2 = U + 2 * BLK;
      if (t < N * P) contract<N, P, P, 1, Q, false, false, kMaxN>(u0, T1, T.Bd, t);
      __syncthreads();
      if (t < N * Q) contract<N, Q, P, 2, Q, false, false, kMaxN>(T1, T2, T.Bd, t);
      __syncthreads();
      if (t < Q * Q) {
        contract<N, Q, Q, 0, Q, false, false, kMaxN>(T2, V0, T.Bc, t);
        contract<N, Q, Q, 0, Q, false, false, kMaxN>(T2, D, T.Dc, t);
      }
      __syncthreads();
      // block 1: (P,N,P) -> axis0 Bd -> (Q,N,P) -> axis2 Bd -> (Q,N,Q) -> axis1 Bc/Dc
      if (t < N * P) contract<P, N, P, 0, Q, false, false, kMaxN>(u1, T1, T.Bd, t);
      __syncthreads();
      if (t < Q * N) contract<Q, N, P, 2, Q, false, false, kMaxN>(T1, T2, T.Bd, t);
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, N, Q, 1, Q, false, false, kMaxN>(T2, V1, T.Bc, t);
        contract<Q, N, Q, 1, Q, false, true, kMaxN>(T2, D, T.Dc, t);
      }
      __syncthreads();
      // block 2: (P,P,N) -> axis0 Bd -> (Q,P,N) -> axis1 Bd -> (Q,Q,N) -> axis2 Bc/Dc
      if (t < P * N) contract<P, P, N, 0, Q, false, false, kMaxN>(u2, T1, T.Bd, t);
      __syncthreads();
      if (t < Q * N) contract<Q, P, N, 1, Q, false, false, kMaxN>(T1, T2, T.Bd, t);
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, Q, N, 2, Q, false, false, kMaxN>(T2, V2, T.Bc, t);
        contract<Q, Q, N, 2, Q, false, true, kMaxN>(T2, D, T.Dc, t);
      }
      __syncthreads();
    } else {
      double* C0 = D;
      double* C1 = D + Q3;
      double* C2 = D + 2 * Q3;
      const double* u0 = U;
      const double* u1 = U + BLK;
      const double* u2 = U + 2 * BLK;
      // block 0: (P,N,N) -> axis0 Bd -> T1 (Q,N,N)
      //   axis1 Bc -> T2 (Q,Q,N): axis2 Bc -> V0, axis2 Dc -> d2u0 (+C1)
      //   axis1 Dc -> T2 (Q,Q,N): axis2 Bc -> d1u0 (-C2)
      if (t < N * N) contract<P, N, N, 0, Q, false, false, kMaxN>(u0, T1, T.Bd, t);
      __syncthreads();
      if (t < Q * N) contract<Q, N, N, 1, Q, false, false, kMaxN>(T1, T2, T.Bc, t);
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, Q, N, 2, Q, false, false, kMaxN>(T2, V0, T.Bc, t);
        contract<Q, Q, N, 2, Q, false, false, kMaxN>(T2, C1, T.Dc, t);
      }
      __syncthreads();
      if (t < Q * N) contract<Q, N, N, 1, Q, false, false, kMaxN>(T1, T2, T.Dc, t);
      __syncthreads();
      if (t < Q * Q) contract<Q, Q, N, 2, Q, false, false, kMaxN>(T2, C2, T.Bc, t);
      __syncthreads();
      for (int i = t; i < Q3; i += N2) C2[i] = -C2[i];
      // block 1: (N,P,N) -> axis1 Bd -> T1 (N,Q,N)
      //   axis0 Bc -> T2 (Q,Q,N): axis2 Bc -> V1, axis2 Dc -> d2u1 (-C0)
      //   axis0 Dc -> T2 (Q,Q,N): axis2 Bc -> d0u1 (+C2)
      if (t < N * N) contract<N, P, N, 1, Q, false, false, kMaxN>(u1, T1, T.Bd, t);
      __syncthreads();
      if (t < Q * N) contract<N, Q, N, 0, Q, false, false, kMaxN>(T1, T2, T.Bc, t);
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, Q, N, 2, Q, false, false, kMaxN>(T2, V1, T.Bc, t);
        contract<Q, Q, N, 2, Q, false, false, kMaxN>(T2, C0, T.Dc, t);
      }
      __syncthreads();
      for (int i = t; i < Q3; i += N2) C0[i] = -C0[i];
      if (t < Q * N) contract<N, Q, N, 0, Q, false, false, kMaxN>(T1, T2, T.Dc, t);
      __syncthreads();
      if (t < Q * Q) contract<Q, Q, N, 2, Q, false, true, kMaxN>(T2, C2, T.Bc, t);
      __syncthreads();
      // block 2: (N,N,P) -> axis2 Bd -> T1 (N,N,Q)
      //   axis0 Bc -> T2 (Q,N,Q): axis1 Bc -> V2, axis1 Dc -> d1u2 (+C0)
      //   axis0 Dc -> T2 (Q,N,Q): axis1 Bc -> d0u2 (-C1)
      if (t < N * N) contract<N, N, P, 2, Q, false, false, kMaxN>(u2, T1, T.Bd, t);
      __syncthreads();
      if (t < N * Q) contract<N, N, Q, 0, Q, false, false, kMaxN>(T1, T2, T.Bc, t);
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, N, Q, 1, Q, false, false, kMaxN>(T2, V2, T.Bc, t);
        contract<Q, N, Q, 1, Q, false, true, kMaxN>(T2, C0, T.Dc, t);
      }
      __syncthreads();
      if (t < N * Q) contract<N, N, Q, 0, Q, false, false, kMaxN>(T1, T2, T.Dc, t);
      __syncthreads();
      // C1 -= d0u2: negate, accumulate, negate back
      for (int i = t; i < Q3; i += N2) C1[i] = -C1[i];
      __syncthreads();
      if (t < Q * Q) contract<Q, N, Q, 1, Q, false, true, kMaxN>(T2, C1, T.Bc, t);
      __syncthreads();
      for (int i = t; i < Q3; i += N2) C1[i] = -C1[i];
    }
    __syncthreads();
    // pointwise
    for (int qp = t; qp < Q3; qp += N2) {
      const int q1 = qp / (Q * Q), q2 = (qp / Q) % Q, q3 = qp % Q;
      const double* c0 = Jc[0][q2 * Q + q3];
      const double* c1 = Jc[1][q1 * Q + q3];
      const double* c2 = Jc[2][q1 * Q + q2];
      double r0[3];
      cross3(c1, c2, r0);
      const double S = dot3(c0, r0);
      const double ws = W3[qp] / S;
      // J^T J (symmetric): m_ab = c_a . c_b
      const double m00 = dot3(c0, c0), m11 = dot3(c1, c1), m22 = dot3(c2, c2);
      const double m01 = dot3(c0, c1), m02 = dot3(c0, c2), m12 = dot3(c1, c2);
      if (NCF) {
        const double u0 = V0[qp], u1 = V1[qp], u2 = V2[qp];
        const double sa = a.alpha * ws;
        V0[qp] = sa * (m00 * u0 + m01 * u1 + m02 * u2);
        V1[qp] = sa * (m01 * u0 + m11 * u1 + m12 * u2);
        V2[qp] = sa * (m02 * u0 + m12 * u1 + m22 * u2);
        D[qp] = a.beta * ws * D[qp];
      } else {
        double* C0 = D;
        double* C1 = D + Q3;
        double* C2 = D + 2 * Q3;
        const double k0 = C0[qp], k1 = C1[qp], k2 = C2[qp];
        const double sb = a.beta * ws;
        C0[qp] = sb * (m00 * k0 + m01 * k1 + m02 * k2);
        C1[qp] = sb * (m01 * k0 + m11 * k1 + m12 * k2);
        C2[qp] = sb * (m02 * k0 + m12 * k1 + m22 * k2);
        // covariant mass: w S G G^T = (w/S) adj adj^T, adj rows r0, r1, r2
        double r1[3], r2[3];
        cross3(c2, c0, r1);
        cross3(c0, c1, r2);
        const double u0 = V0[qp], u1 = V1[qp], u2 = V2[qp];
        const double sa = a.alpha * ws;
        const double a00 = dot3(r0, r0), a11 = dot3(r1, r1), a22 = dot3(r2, r2);
        const double a01 = dot3(r0, r1), a02 = dot3(r0, r2), a12 = dot3(r1, r2);
        V0[qp] = sa * (a00 * u0 + a01 * u1 + a02 * u2);
        V1[qp] = sa * (a01 * u0 + a11 * u1 + a12 * u2);
        V2[qp] = sa * (a02 * u0 + a12 * u1 + a22 * u2);
      }
    }
    __syncthreads();
    double* y0 = U;
    double* y1 = U + BLK;
    double* y2 = U + 2 * BLK;
    if (NCF) {
      // block 0: axis0 Bc^T V0 + Dc^T DIV -> (N,Q,Q) -> axis1 Bd^T -> (N,P,Q) -> axis2 Bd^T -> (N,P,P)
      if (t < Q * Q) {
        contract<Q, Q, Q, 0, N, true, false, kMaxN>(V0, T2, T.Bc, t);
        contract<Q, Q, Q, 0, N, true, true, kMaxN>(D, T2, T.Dc, t);
      }
      __syncthreads();
      if (t < N * Q) contract<N, Q, Q, 1, P, true, false, kMaxN>(T2, T1, T.Bd, t);
      __syncthreads();
      if (t < N * P) contract<N, P, Q, 2, P, true, false, kMaxN>(T1, y0, T.Bd, t);
      __syncthreads();
      // block 1: axis1 Bc^T V1 + Dc^T DIV -> (Q,N,Q) -> axis0 Bd^T -> (P,N,Q) -> axis2 Bd^T
      if (t < Q * Q) {
        contract<Q, Q, Q, 1, N, true, false, kMaxN>(V1, T2, T.Bc, t);
        contract<Q, Q, Q, 1, N, true, true, kMaxN>(D, T2, T.Dc, t);
      }
      __syncthreads();
      if (t < N * Q) contract<Q, N, Q, 0, P, true, false, kMaxN>(T2, T1, T.Bd, t);
      __syncthreads();
      if (t < P * N) contract<P, N, Q, 2, P, true, false, kMaxN>(T1, y1, T.Bd, t);
      __syncthreads();
      // block 2: axis2 Bc^T V2 + Dc^T DIV -> (Q,Q,N) -> axis0 Bd^T -> (P,Q,N) -> axis1 Bd^T
      if (t < Q * Q) {
        contract<Q, Q, Q, 2, N, true, false, kMaxN>(V2, T2, T.Bc, t);
        contract<Q, Q, Q, 2, N, true, true, kMaxN>(D, T2, T.Dc, t);
      }
      __syncthreads();
      if (t < Q * N) contract<Q, Q, N, 0, P, true, false, kMaxN>(T2, T1, T.Bd, t);
      __syncthreads();
      if (t < P * N) contract<P, Q, N, 1, P, true, false, kMaxN>(T1, y2, T.Bd, t);
      __syncthreads();
    } else {
      double* C0 = D;
      double* C1 = D + Q3;
      double* C2 = D + 2 * Q3;
      // block 0 (v = phi e0, curl v = (0, d2 phi, -d1 phi)):
      //   axis2: T1 = Bc^T V0 + Dc^T C1 (Q,Q,N); T2 = -Bc^T C2 (Q,Q,N)
      //   axis1: T? = Bc^T T1 + Dc^T T2 -> (Q,N,N); axis0 Bd^T -> (P,N,N)
      for (int i = t; i < Q3; i += N2) C2[i] = -C2[i];
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, Q, Q, 2, N, true, false, kMaxN>(V0, T1, T.Bc, t);
        contract<Q, Q, Q, 2, N, true, true, kMaxN>(C1, T1, T.Dc, t);
        contract<Q, Q, Q, 2, N, true, false, kMaxN>(C2, T2, T.Bc, t);
      }
      __syncthreads();
      for (int i = t; i < Q3; i += N2) C2[i] = -C2[i];
      // reuse V0 as the (Q,N,N) buffer (V0 no longer needed)
      if (t < Q * N) {
        contract<Q, Q, N, 1, N, true, false, kMaxN>(T1, V0, T.Bc, t);
        contract<Q, Q, N, 1, N, true, true, kMaxN>(T2, V0, T.Dc, t);
      }
      __syncthreads();
      if (t < N * N) contract<Q, N, N, 0, P, true, false, kMaxN>(V0, y0, T.Bd, t);
      __syncthreads();
      // block 1 (v = phi e1, curl v = (-d2 phi, 0, d0 phi)):
      //   axis2: T1 = Bc^T V1 - Dc^T C0 (Q,Q,N); T2 = Bc^T C2 (Q,Q,N)
      //   axis0: V1buf = Bc^T T1 + Dc^T T2 -> (N,Q,N); axis1 Bd^T -> (N,P,N)
      for (int i = t; i < Q3; i += N2) C0[i] = -C0[i];
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, Q, Q, 2, N, true, false, kMaxN>(V1, T1, T.Bc, t);
        contract<Q, Q, Q, 2, N, true, true, kMaxN>(C0, T1, T.Dc, t);
        contract<Q, Q, Q, 2, N, true, false, kMaxN>(C2, T2, T.Bc, t);
      }
      __syncthreads();
      for (int i = t; i < Q3; i += N2) C0[i] = -C0[i];
      if (t < Q * N) {
        contract<Q, Q, N, 0, N, true, false, kMaxN>(T1, V1, T.Bc, t);
        contract<Q, Q, N, 0, N, true, true, kMaxN>(T2, V1, T.Dc, t);
      }
      __syncthreads();
      if (t < N * N) contract<N, Q, N, 1, P, true, false, kMaxN>(V1, y1, T.Bd, t);
      __syncthreads();
      // block 2 (v = phi e2, curl v = (d1 phi, -d0 phi, 0)):
      //   axis1: T1 = Bc^T V2 + Dc^T C0 (Q,N,Q); T2 = -Bc^T C1 (Q,N,Q)
      //   axis0: V2buf = Bc^T T1 + Dc^T T2 -> (N,N,Q); axis2 Bd^T -> (N,N,P)
      for (int i = t; i < Q3; i += N2) C1[i] = -C1[i];
      __syncthreads();
      if (t < Q * Q) {
        contract<Q, Q, Q, 1, N, true, false, kMaxN>(V2, T1, T.Bc, t);
        contract<Q, Q, Q, 1, N, true, true, kMaxN>(C0, T1, T.Dc, t);
        contract<Q, Q, Q, 1, N, true, false, kMaxN>(C1, T2, T.Bc, t);
      }
      __syncthreads();
      if (t < N * Q) {
        contract<Q, N, Q, 0, N, true, false, kMaxN>(T1, V2, T.Bc, t);
        contract<Q, N, Q, 0, N, true, true, kMaxN>(T2, V2, T.Dc, t);
      }
      __syncthreads();
      if (t < N * N) contract<N, N, Q, 2, P, true, false, kMaxN>(V2, y2, T.Bd, t);
      __syncthreads();
    }
    if (ok) {
      if (a.cell_vectors) {
        for (int l = t; l < NLOC; l += N2) a.y[(slot * NLOC + l) * a.nrhs + r] = U[l];
      } else {
        for (int l = t; l < NLOC; l += N2) a.y[(int64_t)mrow[l] * a.nrhs + r] += U[l];
      }
    } else if (active && a.cell_vectors) {
      for (int l = t; l < NLOC; l += N2) a.y[(slot * NLOC + l) * a.nrhs + r] = 0.0;
    }
    __syncthreads();
  }
}

template <int P, bool NCF>
int launch_h(const ActArgs& a, int64_t nc, cudaStream_t s) {
  using Sh = HShape<P, NCF>;
  const size_t per_team = Sh::TEAM * sizeof(double);
  const size_t fixed = (Sh::Q3 + 16) * sizeof(double);
  int cb = Sh::MAXCB;
  // two CTAs per SM (110 KB each) while that still gives a CTA two or more
  // cells; otherwise one larger CTA, as for the hyperelastic residual
  while (cb > 1 && fixed + cb * per_team > 110 * 1024) --cb;
  if (cb < 2) {
    cb = Sh::MAXCB;
    while (cb > 1 && fixed + cb * per_team > 200 * 1024) --cb;
  }
  cb = tuned_team_cells(SFX_TUNE_HDIVCURL, P, cb, Sh::MAXCB, fixed, per_team, 200 * 1024);
  const size_t smem = fixed + cb * per_team;
  auto kern = k_action_hdivcurl_fp64<P, NCF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kern<<<(unsigned)((a.ncells + cb - 1) / cb), cb * Sh::N2, smem, s>>>(a, nc);
  return (int)cudaGetLastError();
}

template <bool NCF>
int dispatch_p(int p, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (p) {
    case 1: return launch_h<1, NCF>(a, nc, s);
    case 2: return launch_h<2, NCF>(a, nc, s);
    case 3: return launch_h<3, NCF>(a, nc, s);
    case 4: return launch_h<4, NCF>(a, nc, s);
    case 5: return launch_h<5, NCF>(a, nc, s);
    case 6: return launch_h<6, NCF>(a, nc, s);
    case 7: return launch_h<7, NCF>(a, nc, s);
    case 8: return launch_h<8, NCF>(a, nc, s);
  }
  return -1;
}

}  // namespace

int launch_action_hdivcurl_mixed_tf32(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);
int launch_action_hdivcurl_mixed_bf16(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);

int launch_action_hdivcurl(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                           void* stream) {
  if (prec == SFX_PREC_TF32X3) return launch_action_hdivcurl_mixed_tf32(sp, form, a, stream);
  if (prec == SFX_PREC_BF16X3) return launch_action_hdivcurl_mixed_bf16(sp, form, a, stream);
  if (prec != SFX_PREC_FP64) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  if (sp->family == SFX_NCF && form == SFX_NCF_MASS_DIVDIV) return dispatch_p<true>(sp->p, a, sp->mesh->ncell, s);
  if (sp->family == SFX_NCE && form == SFX_NCE_CURLCURL) return dispatch_p<false>(sp->p, a, sp->mesh->ncell, s);
  return -1;
}

}  // namespace sfx
