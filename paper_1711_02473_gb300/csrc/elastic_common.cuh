#pragma once
// elastic_common.cuh -- pointwise linearised hyperelastic stress, shared by the
// FP64 (k_elastic_lin.cu) and split-precision (k_elastic_lin_mixed.cu)
// actions of the linearised operator (Sec. 4.1).
#include "kern_common.cuh"

namespace sfx {
namespace {

// Linearised test flux at one point: Hs = grad^ u, Hd = grad^ du (reference
// gradients, [i][k] = d u_i / d xi_k), R = rows of adj J, S = det J, w the
// weight; out[i][k] = w sum_j dP[i][j] R[k][j].  False (zero flux) if
// det F <= 0 for the neo-Hookean law.
template <bool NEO>
__device__ __forceinline__ bool linearised_flux(const double (*Hs)[3], const double (*Hd)[3], const double (*R)[3],
                                                double S, double w, double mu, double lam, double (*out)[3]) {
  const double iS = recip_nr<2>(S);
  double F[3][3], dF[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      F[i][j] = (Hs[i][0] * R[0][j] + Hs[i][1] * R[1][j] + Hs[i][2] * R[2][j]) * iS + (i == j ? 1.0 : 0.0);
      dF[i][j] = (Hd[i][0] * R[0][j] + Hd[i][1] * R[1][j] + Hd[i][2] * R[2][j]) * iS;
    }
  double dP[3][3];
  bool good = true;
  if (NEO) {
    double Cf[3][3];  // cofactor matrix of F: F^{-T} = Cf / det F
    cross3(F[1], F[2], Cf[0]);
    cross3(F[2], F[0], Cf[1]);
    cross3(F[0], F[1], Cf[2]);
    const double JF = dot3(F[0], Cf[0]);
    good = JF > 0.0;
    const double iJ = good ? recip_nr<2>(JF) : 0.0, lnJ = good ? log(JF) : 0.0;
    double FiT[3][3], T1[3][3];
    double tr = 0.0;  // tr(F^{-1} dF) = sum_ij F^{-T}_ij dF_ij
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        FiT[i][j] = Cf[i][j] * iJ;
        tr = fma(FiT[i][j], dF[i][j], tr);
      }
#pragma unroll
    for (int k = 0; k < 3; ++k)  // T1 = dF^T F^{-T}
#pragma unroll
      for (int j = 0; j < 3; ++j) T1[k][j] = dF[0][k] * FiT[0][j] + dF[1][k] * FiT[1][j] + dF[2][k] * FiT[2][j];
    const double c = mu - lam * lnJ, lt = lam * tr;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double m = FiT[i][0] * T1[0][j] + FiT[i][1] * T1[1][j] + FiT[i][2] * T1[2][j];
        dP[i][j] = good ? mu * dF[i][j] + c * m + lt * FiT[i][j] : 0.0;
      }
  } else {
    double E[3][3], dE[3][3], S2[3][3], dS[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        E[a][b] = 0.5 * (F[0][a] * F[0][b] + F[1][a] * F[1][b] + F[2][a] * F[2][b] - (a == b ? 1.0 : 0.0));
        dE[a][b] = 0.5 * (dF[0][a] * F[0][b] + dF[1][a] * F[1][b] + dF[2][a] * F[2][b] + F[0][a] * dF[0][b] +
                          F[1][a] * dF[1][b] + F[2][a] * dF[2][b]);
      }
    const double trE = E[0][0] + E[1][1] + E[2][2], trdE = dE[0][0] + dE[1][1] + dE[2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        S2[a][b] = (a == b ? lam * trE : 0.0) + 2.0 * mu * E[a][b];
        dS[a][b] = (a == b ? lam * trdE : 0.0) + 2.0 * mu * dE[a][b];
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        dP[i][j] = dF[i][0] * S2[0][j] + dF[i][1] * S2[1][j] + dF[i][2] * S2[2][j] + F[i][0] * dS[0][j] +
                   F[i][1] * dS[1][j] + F[i][2] * dS[2][j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) out[i][k] = w * dot3(dP[i], R[k]);
  return good;
}

}  // namespace
}  // namespace sfx
