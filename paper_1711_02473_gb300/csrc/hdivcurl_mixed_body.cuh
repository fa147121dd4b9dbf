#pragma once
// hdivcurl_mixed_body.cuh -- split-precision actions on NCF_p (mass + div-div)
// and NCE_p (mass + curl-curl).  Instantiated once per input format in
// k_hdivcurl_mixed_tf32.cu and k_hdivcurl_mixed_bf16.cu.
//
// Same algorithm as k_action_hdivcurl_fp64 (Secs. 2.6-2.7 and 3.5: each of
// the three HDiv / HCurl-wrapped blocks sum-factorised on its own, with the
// P_p factor on GLL nodes and the dP_{p-1} factor on Gauss nodes; Eq.
// curl_curl_form for NCE).  What changes is where the arithmetic runs:
//   - every 1D contraction (forward and transposed, 24 per RHS for NCF, 36 for
//     NCE) is a batched matrix product of a 1D table with the fibers of all
//     the CTA's cells on the tensor cores (tc_contract_g: split operands,
//     FP32 accumulation);
//   - J (from the trilinear coordinate field), S = det J, the rows of adj J
//     (NCE) and the weight scaling w/S are computed in FP64; the symmetric
//     products J^T J and adj J adj J^T, which only feed FP32 factors, run on
//     the FP32 pipe from the columns / rows rounded once, and the flux is
//     scaled by alpha w/S or beta w/S in FP64 before its final rounding;
//   - b^K is widened to FP64 and added into y in FP64.
// Pointwise (q = p+1 Gauss points):
//   NCF: f_val = alpha w/S J^T J u^,  f_div = beta w/S div^ u^
//   NCE: f_curl = beta w/S J^T J curl^ u^,  f_val = alpha w/S adj J adj J^T u^
// (contravariant Piola u = J u^ / S, div u = div^ u^ / S; covariant Piola
// u = J^-T u^, curl u = J curl^ u^ / S).
#include "mixed_common.cuh"

namespace sfx {
namespace {

template <int P, bool NCF>
struct HMShape {
  static constexpr int N = P + 1, Q = P + 1, N2 = N * N, Q3 = Q * Q * Q;
  static constexpr int BLK = NCF ? N * P * P : P * N * N;  // dofs per block
  static constexpr int NLOC = 3 * BLK;
  static constexpr int NDER = NCF ? 1 : 3;                 // derivative arrays: div, or curl
  // per-cell floats: U (dofs in, b^K out), V0..2, the derivative arrays, T1, T2
  static constexpr int CELLF = NLOC + (3 + NDER + 2) * Q3;
  // per-cell doubles: corners, Jacobian column tables Jc[3][N^2][3]
  static constexpr int CELLD = 24 + 9 * N2;
  static constexpr size_t fixed_bytes() { return 3 * sizeof(TabF) + (size_t)(Q3 + 16) * 8; }
  static constexpr size_t bytes(int cb) {
    return fixed_bytes() + (size_t)cb * CELLD * 8 + (size_t)cb * CELLF * 4 + (size_t)cb * 2 * 4;
  }
};

template <int P, bool NCF, int PREC>
__global__ void __launch_bounds__(kThreads) k_action_hdivcurl_mixed(const ActArgs a, const int64_t ncell_total,
                                                                    const int cb) {
  using Sh = HMShape<P, NCF>;
  constexpr int N = Sh::N, Q = Sh::Q, N2 = Sh::N2, Q3 = Sh::Q3, BLK = Sh::BLK, NLOC = Sh::NLOC;
  constexpr int NT = kThreads;
  const Tab1D& T = c_tab[P];
  extern __shared__ double smd[];
  // layout: [tabs Bc, Dc, Bd (FP32)][W3: Q3 doubles][xq: 16 doubles]
  //         [per cell doubles: X, Jc][float arrays, each cb x size][cell id, bad: cb ints each]
  TabF* tabs = reinterpret_cast<TabF*>(smd);
  double* W3 = reinterpret_cast<double*>(tabs + 3);
  double* xq = W3 + Q3;
  double* dd = xq + 16;
  float* U = reinterpret_cast<float*>(dd + (size_t)cb * Sh::CELLD);
  float* V0 = U + (size_t)cb * NLOC;
  float* V1 = V0 + (size_t)cb * Q3;
  float* V2 = V1 + (size_t)cb * Q3;
  float* D0 = V2 + (size_t)cb * Q3;  // NCF: div; NCE: curl components C0, C1, C2
  float* D1 = D0 + (size_t)cb * Q3;
  float* D2 = D1 + (size_t)cb * Q3;
  float* T1 = D0 + (size_t)cb * Sh::NDER * Q3;
  float* T2 = T1 + (size_t)cb * Q3;
  int* cid = reinterpret_cast<int*>(T2 + (size_t)cb * Q3);
  int* bad = cid + cb;
  const TabF& Bc = tabs[0];
  const TabF& Dc = tabs[1];
  const TabF& Bd = tabs[2];

  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * 256; i += NT) {
    const int m = i / 256, r = (i / 16) % 16, k = i % 16;
    float v = 0.f;
    if (r < Q) {
      if (m == 0 && k < N) v = (float)T.Bc[r][k];
      if (m == 1 && k < N) v = (float)T.Dc[r][k];
      if (m == 2 && k < P) v = (float)T.Bd[r][k];
    }
    tabs[m].v[r][k] = v;
  }
  for (int i = tid; i < Q3; i += NT) W3[i] = T.w[i / (Q * Q)] * T.w[(i / Q) % Q] * T.w[i % Q];
  if (tid < Q) xq[tid] = T.x[tid];
  for (int c = tid; c < cb; c += NT) {
    int cell = -1;
    if (!slot_cell(a, (int64_t)blockIdx.x * cb + c, ncell_total, &cell)) cell = -1;
    cid[c] = cell;
    bad[c] = 0;
  }
  __syncthreads();
  for (int i = tid; i < cb * 24; i += NT) {
    const int c = i / 24, v = (i % 24) / 3, k = i % 3;
    const int cell = cid[c];
    dd[(size_t)c * Sh::CELLD + v * 3 + k] =
        cell >= 0 ? a.xyz[(int64_t)a.vmap[(int64_t)cell * 8 + v] * 3 + k] : (double)((v >> (2 - k)) & 1);
  }
  __syncthreads();
  for (int i = tid; i < cb * N2; i += NT) {
    const int c = i / N2, t = i - c * N2;
    double* base = dd + (size_t)c * Sh::CELLD;
    jacobian_columns<N>(reinterpret_cast<const double(*)[3]>(base), xq,
                        reinterpret_cast<double(*)[N2][3]>(base + 24), t);
  }
  __syncthreads();
  const double alpha = a.alpha, beta = a.beta;

#pragma unroll 1
  for (int r = 0; r < a.nrhs; ++r) {
    for (int i = tid; i < cb * NLOC; i += NT) {
      const int c = i / NLOC, l = i - c * NLOC;
      const int cell = cid[c];
      U[i] = cell >= 0 ? d2f_int(__ldg(&a.x[(int64_t)__ldg(&a.map[(int64_t)cell * NLOC + l]) * a.nrhs + r])) : 0.f;
    }
    __syncthreads();
    // ---------------------------------------------------------------- forward
    if (NCF) {
      // block 0: (N,P,P) -axis1 Bd-> (N,Q,P) -axis2 Bd-> (N,Q,Q) -axis0 Bc/Dc-> V0, div
      tc_contract_g<N, P, P, 1, Q, NLOC, Q3, false, false, false, PREC>(U, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<N, Q, P, 2, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Bd, cb);
      __syncthreads();
      tc_contract_g<N, Q, Q, 0, Q, Q3, Q3, false, false, false, PREC>(T2, V0, Bc, cb);
      tc_contract_g<N, Q, Q, 0, Q, Q3, Q3, false, false, false, PREC>(T2, D0, Dc, cb);
      // block 1: (P,N,P) -axis0 Bd-> (Q,N,P) -axis2 Bd-> (Q,N,Q) -axis1 Bc/Dc-> V1, div +=
      tc_contract_g<P, N, P, 0, Q, NLOC, Q3, false, false, false, PREC>(U + BLK, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<Q, N, P, 2, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Bd, cb);
      __syncthreads();
      tc_contract_g<Q, N, Q, 1, Q, Q3, Q3, false, false, false, PREC>(T2, V1, Bc, cb);
      tc_contract_g<Q, N, Q, 1, Q, Q3, Q3, false, true, false, PREC>(T2, D0, Dc, cb);
      // block 2: (P,P,N) -axis0 Bd-> (Q,P,N) -axis1 Bd-> (Q,Q,N) -axis2 Bc/Dc-> V2, div +=
      tc_contract_g<P, P, N, 0, Q, NLOC, Q3, false, false, false, PREC>(U + 2 * BLK, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<Q, P, N, 1, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Bd, cb);
      __syncthreads();
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, false, false, PREC>(T2, V2, Bc, cb);
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, true, false, PREC>(T2, D0, Dc, cb);
      __syncthreads();
    } else {
      // reference curl of block c (value phi e_c): block 0 gives (0, d2, -d1),
      // block 1 (-d2, 0, d0), block 2 (d1, -d0, 0) of its scalar factor
      // block 0: (P,N,N) -axis0 Bd-> T1 (Q,N,N)
      tc_contract_g<P, N, N, 0, Q, NLOC, Q3, false, false, false, PREC>(U, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<Q, N, N, 1, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Bc, cb);  // (Q,Q,N)
      __syncthreads();
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, false, false, PREC>(T2, V0, Bc, cb);
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, false, false, PREC>(T2, D1, Dc, cb);  // C1 = d2
      __syncthreads();
      tc_contract_g<Q, N, N, 1, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Dc, cb);  // (Q,Q,N)
      __syncthreads();
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, false, true, PREC>(T2, D2, Bc, cb);  // C2 = -d1
      // block 1: (N,P,N) -axis1 Bd-> T1 (N,Q,N)
      tc_contract_g<N, P, N, 1, Q, NLOC, Q3, false, false, false, PREC>(U + BLK, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<N, Q, N, 0, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Bc, cb);  // (Q,Q,N)
      __syncthreads();
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, false, false, PREC>(T2, V1, Bc, cb);
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, false, true, PREC>(T2, D0, Dc, cb);  // C0 = -d2
      __syncthreads();
      tc_contract_g<N, Q, N, 0, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Dc, cb);  // (Q,Q,N)
      __syncthreads();
      tc_contract_g<Q, Q, N, 2, Q, Q3, Q3, false, true, false, PREC>(T2, D2, Bc, cb);  // C2 += d0
      // block 2: (N,N,P) -axis2 Bd-> T1 (N,N,Q)
      tc_contract_g<N, N, P, 2, Q, NLOC, Q3, false, false, false, PREC>(U + 2 * BLK, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<N, N, Q, 0, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Bc, cb);  // (Q,N,Q)
      __syncthreads();
      tc_contract_g<Q, N, Q, 1, Q, Q3, Q3, false, false, false, PREC>(T2, V2, Bc, cb);
      tc_contract_g<Q, N, Q, 1, Q, Q3, Q3, false, true, false, PREC>(T2, D0, Dc, cb);  // C0 += d1
      __syncthreads();
      tc_contract_g<N, N, Q, 0, Q, Q3, Q3, false, false, false, PREC>(T1, T2, Dc, cb);  // (Q,N,Q)
      __syncthreads();
      tc_contract_g<Q, N, Q, 1, Q, Q3, Q3, false, true, true, PREC>(T2, D1, Bc, cb);  // C1 -= d0
      __syncthreads();
    }
    // --------------------------------------------------------------- pointwise
    for (int i = tid; i < cb * Q3; i += NT) {
      const int c = i / Q3, qp = i - c * Q3;
      const int q1 = qp / (Q * Q), q2 = (qp / Q) % Q, q3 = qp % Q;
      const double(*Jc)[N2][3] = reinterpret_cast<const double(*)[N2][3]>(dd + (size_t)c * Sh::CELLD + 24);
      const double* c0 = Jc[0][q2 * Q + q3];
      const double* c1 = Jc[1][q1 * Q + q3];
      const double* c2 = Jc[2][q1 * Q + q2];
      double r0[3];
      cross3(c1, c2, r0);
      const double S = dot3(c0, r0);
      if (!positive_finite(S)) bad[c] = 1;
      const double ws = W3[qp] * recip_nr<1>(S);
      const double sa = alpha * ws, sb = beta * ws;
      float f0[3], f1[3], f2[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        f0[k] = d2f_int(c0[k]);
        f1[k] = d2f_int(c1[k]);
        f2[k] = d2f_int(c2[k]);
      }
      auto dotf = [](const float* u, const float* v) { return fmaf(u[0], v[0], fmaf(u[1], v[1], u[2] * v[2])); };
      // J^T J (FP32 from the rounded columns)
      const float m00 = dotf(f0, f0), m11 = dotf(f1, f1), m22 = dotf(f2, f2);
      const float m01 = dotf(f0, f1), m02 = dotf(f0, f2), m12 = dotf(f1, f2);
      if (NCF) {
        const float u0 = V0[i], u1 = V1[i], u2 = V2[i];
        V0[i] = d2f_int(sa * f2d_int(m00 * u0 + m01 * u1 + m02 * u2));
        V1[i] = d2f_int(sa * f2d_int(m01 * u0 + m11 * u1 + m12 * u2));
        V2[i] = d2f_int(sa * f2d_int(m02 * u0 + m12 * u1 + m22 * u2));
        D0[i] = d2f_int(sb * f2d_int(D0[i]));
      } else {
        const float k0 = D0[i], k1 = D1[i], k2 = D2[i];
        D0[i] = d2f_int(sb * f2d_int(m00 * k0 + m01 * k1 + m02 * k2));
        D1[i] = d2f_int(sb * f2d_int(m01 * k0 + m11 * k1 + m12 * k2));
        D2[i] = d2f_int(sb * f2d_int(m02 * k0 + m12 * k1 + m22 * k2));
        // covariant mass: w S G G^T = (w/S) adj J adj J^T, rows r0 = c1 x c2, r1 = c2 x c0, r2 = c0 x c1
        double r1[3], r2[3];
        cross3(c2, c0, r1);
        cross3(c0, c1, r2);
        float g0[3], g1[3], g2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          g0[k] = d2f_int(r0[k]);
          g1[k] = d2f_int(r1[k]);
          g2[k] = d2f_int(r2[k]);
        }
        const float a00 = dotf(g0, g0), a11 = dotf(g1, g1), a22 = dotf(g2, g2);
        const float a01 = dotf(g0, g1), a02 = dotf(g0, g2), a12 = dotf(g1, g2);
        const float u0 = V0[i], u1 = V1[i], u2 = V2[i];
        V0[i] = d2f_int(sa * f2d_int(a00 * u0 + a01 * u1 + a02 * u2));
        V1[i] = d2f_int(sa * f2d_int(a01 * u0 + a11 * u1 + a12 * u2));
        V2[i] = d2f_int(sa * f2d_int(a02 * u0 + a12 * u1 + a22 * u2));
      }
    }
    __syncthreads();
    // ------------------------------------------------------------- transposed
    if (NCF) {
      // block 0: axis0 Bc^T V0 + Dc^T div -> (N,Q,Q) -axis1 Bd^T-> (N,P,Q) -axis2 Bd^T-> (N,P,P)
      tc_contract_g<Q, Q, Q, 0, N, Q3, Q3, true, false, false, PREC>(V0, T2, Bc, cb);
      tc_contract_g<Q, Q, Q, 0, N, Q3, Q3, true, true, false, PREC>(D0, T2, Dc, cb);
      __syncthreads();
      tc_contract_g<N, Q, Q, 1, P, Q3, Q3, true, false, false, PREC>(T2, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<N, P, Q, 2, P, Q3, NLOC, true, false, false, PREC>(T1, U, Bd, cb);
      // block 1: axis1 Bc^T V1 + Dc^T div -> (Q,N,Q) -axis0 Bd^T-> (P,N,Q) -axis2 Bd^T-> (P,N,P)
      tc_contract_g<Q, Q, Q, 1, N, Q3, Q3, true, false, false, PREC>(V1, T2, Bc, cb);
      tc_contract_g<Q, Q, Q, 1, N, Q3, Q3, true, true, false, PREC>(D0, T2, Dc, cb);
      __syncthreads();
      tc_contract_g<Q, N, Q, 0, P, Q3, Q3, true, false, false, PREC>(T2, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<P, N, Q, 2, P, Q3, NLOC, true, false, false, PREC>(T1, U + BLK, Bd, cb);
      // block 2: axis2 Bc^T V2 + Dc^T div -> (Q,Q,N) -axis0 Bd^T-> (P,Q,N) -axis1 Bd^T-> (P,P,N)
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, false, false, PREC>(V2, T2, Bc, cb);
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, true, false, PREC>(D0, T2, Dc, cb);
      __syncthreads();
      tc_contract_g<Q, Q, N, 0, P, Q3, Q3, true, false, false, PREC>(T2, T1, Bd, cb);
      __syncthreads();
      tc_contract_g<P, Q, N, 1, P, Q3, NLOC, true, false, false, PREC>(T1, U + 2 * BLK, Bd, cb);
      __syncthreads();
    } else {
      // block 0 (test phi e0, curl (0, d2 phi, -d1 phi)):
      //   axis2: T1 = Bc^T V0 + Dc^T C1, T2 = -Bc^T C2 (Q,Q,N)
      //   axis1: V0 <- Bc^T T1 + Dc^T T2 (Q,N,N); axis0 Bd^T -> (P,N,N)
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, false, false, PREC>(V0, T1, Bc, cb);
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, true, false, PREC>(D1, T1, Dc, cb);
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, false, true, PREC>(D2, T2, Bc, cb);
      __syncthreads();
      tc_contract_g<Q, Q, N, 1, N, Q3, Q3, true, false, false, PREC>(T1, V0, Bc, cb);
      tc_contract_g<Q, Q, N, 1, N, Q3, Q3, true, true, false, PREC>(T2, V0, Dc, cb);
      __syncthreads();
      tc_contract_g<Q, N, N, 0, P, Q3, NLOC, true, false, false, PREC>(V0, U, Bd, cb);
      // block 1 (curl (-d2 phi, 0, d0 phi)):
      //   axis2: T1 = Bc^T V1 - Dc^T C0, T2 = Bc^T C2 (Q,Q,N)
      //   axis0: V1 <- Bc^T T1 + Dc^T T2 (N,Q,N); axis1 Bd^T -> (N,P,N)
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, false, false, PREC>(V1, T1, Bc, cb);
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, true, true, PREC>(D0, T1, Dc, cb);
      tc_contract_g<Q, Q, Q, 2, N, Q3, Q3, true, false, false, PREC>(D2, T2, Bc, cb);
      __syncthreads();
      tc_contract_g<Q, Q, N, 0, N, Q3, Q3, true, false, false, PREC>(T1, V1, Bc, cb);
      tc_contract_g<Q, Q, N, 0, N, Q3, Q3, true, true, false, PREC>(T2, V1, Dc, cb);
      __syncthreads();
      tc_contract_g<N, Q, N, 1, P, Q3, NLOC, true, false, false, PREC>(V1, U + BLK, Bd, cb);
      // block 2 (curl (d1 phi, -d0 phi, 0)):
      //   axis1: T1 = Bc^T V2 + Dc^T C0, T2 = -Bc^T C1 (Q,N,Q)
      //   axis0: V2 <- Bc^T T1 + Dc^T T2 (N,N,Q); axis2 Bd^T -> (N,N,P)
      tc_contract_g<Q, Q, Q, 1, N, Q3, Q3, true, false, false, PREC>(V2, T1, Bc, cb);
      tc_contract_g<Q, Q, Q, 1, N, Q3, Q3, true, true, false, PREC>(D0, T1, Dc, cb);
      tc_contract_g<Q, Q, Q, 1, N, Q3, Q3, true, false, true, PREC>(D1, T2, Bc, cb);
      __syncthreads();
      tc_contract_g<Q, N, Q, 0, N, Q3, Q3, true, false, false, PREC>(T1, V2, Bc, cb);
      tc_contract_g<Q, N, Q, 0, N, Q3, Q3, true, true, false, PREC>(T2, V2, Dc, cb);
      __syncthreads();
      tc_contract_g<N, N, Q, 2, P, Q3, NLOC, true, false, false, PREC>(V2, U + 2 * BLK, Bd, cb);
      __syncthreads();
    }
    // ----------------------------------------------------------------- scatter
    for (int i = tid; i < cb * NLOC; i += NT) {
      const int c = i / NLOC, l = i - c * NLOC;
      const int cell = cid[c];
      if (cell < 0) continue;
      const bool ok = !bad[c];
      if (a.cell_vectors) {
        const int64_t slot = (int64_t)blockIdx.x * cb + c;
        a.y[(slot * NLOC + l) * a.nrhs + r] = ok ? f2d_int(U[i]) : 0.0;
      } else if (ok) {
        // L2 reduction (red.global.add.f64); cells of one launch share no dof
        atomicAdd(&a.y[(int64_t)a.map[(int64_t)cell * NLOC + l] * a.nrhs + r], f2d_int(U[i]));
      }
    }
    if (r == 0)
      for (int c = tid; c < cb; c += NT)
        if (cid[c] >= 0 && bad[c]) set_flag(a.status, SFX_DEV_INVERTED);
    __syncthreads();
  }
}

template <int P, bool NCF, int PREC>
int launch_hm(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = HMShape<P, NCF>;
  // cells per CTA: the most (up to 32) for which two CTAs fit in one SM's
  // shared memory, else the most that fit 200 KB; when this launch's cells
  // then fill less than one wave of two CTAs per SM, the fewest that still fit
  // one wave (more CTAs, none in a second wave); the tuned value if set
  int cb = 32;
  while (cb > 1 && Sh::bytes(cb) > 110 * 1024) --cb;
  if (Sh::bytes(cb) > 110 * 1024) cb = 1;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int64_t slots = 2 * (int64_t)(nsm > 0 ? nsm : 1);
  if (a.ncells <= slots * cb) cb = (int)((a.ncells + slots - 1) / slots);
  cb = tuned_team_cells(SFX_TUNE_HDIVCURL_MIXED, P, cb, 32, Sh::bytes(0), Sh::bytes(1) - Sh::bytes(0), 200 * 1024);
  const size_t smem = Sh::bytes(cb);
  if (smem > 227 * 1024) return -1;
  auto kern = k_action_hdivcurl_mixed<P, NCF, PREC>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  kern<<<(unsigned)grid, kThreads, smem, s>>>(a, ncell_total, cb);
  return (int)cudaGetLastError();
}

template <bool NCF, int PREC>
int dispatch_hm(int p, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (p) {
    case 1: return launch_hm<1, NCF, PREC>(a, nc, s);
    case 2: return launch_hm<2, NCF, PREC>(a, nc, s);
    case 3: return launch_hm<3, NCF, PREC>(a, nc, s);
    case 4: return launch_hm<4, NCF, PREC>(a, nc, s);
    case 5: return launch_hm<5, NCF, PREC>(a, nc, s);
    case 6: return launch_hm<6, NCF, PREC>(a, nc, s);
    case 7: return launch_hm<7, NCF, PREC>(a, nc, s);
    case 8: return launch_hm<8, NCF, PREC>(a, nc, s);
  }
  return -1;
}

template <int PREC>
int launch_hdivcurl_mixed_prec(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (sp->family == SFX_NCF && form == SFX_NCF_MASS_DIVDIV) return dispatch_hm<true, PREC>(sp->p, a, sp->mesh->ncell, s);
  if (sp->family == SFX_NCE && form == SFX_NCE_CURLCURL) return dispatch_hm<false, PREC>(sp->p, a, sp->mesh->ncell, s);
  return -1;
}

}  // namespace
}  // namespace sfx
