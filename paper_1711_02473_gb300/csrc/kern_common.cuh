// kern_common.cuh -- device helpers shared by the kernel files: the per-degree
// 1D tables in constant memory, status flags, trilinear geometry and the
// per-team 1D contractions used by sum factorisation.
#pragma once
#include <cuda_runtime.h>

#include "sfx_internal.h"

namespace sfx {

// Per-translation-unit copy of the 1D tables, one per degree (index p).  The
// contents depend only on p, so every space uploads the same bytes.
static __constant__ Tab1D c_tab[kMaxDeg + 1];

#define SFX_DEFINE_TAB_UPLOAD(fn)                                                          \
  int fn(const Tab1D* t) {                                                                 \
    return (int)cudaMemcpyToSymbol(c_tab, t, sizeof(Tab1D), sizeof(Tab1D) * (size_t)t->p); \
  }

__device__ __forceinline__ void set_flag(uint32_t* st, uint32_t bit) { atomicOr(st, bit); }

// Resolve the cell handled by `slot`; false if the slot is idle or the
// caller's id is out of range (flagged).
__device__ __forceinline__ bool slot_cell(const ActArgs& a, int64_t slot, int64_t ncell_total, int* cell) {
  if (slot >= a.ncells) return false;
  if (a.cells) { *cell = a.cells[slot]; return true; }
  if (a.cells64) {
    int64_t c = a.cells64[slot];
    if (c < 0 || c >= ncell_total) { set_flag(a.status, SFX_DEV_BADCELL); return false; }
    *cell = (int)c;
    return true;
  }
  *cell = (int)slot;
  return true;
}

// Columns of the trilinear Jacobian on the tensor grid of quadrature points.
// Column d of J = dx/dxi_d does not depend on xi_d (Sec. 3.1: the coordinate
// field is vector-Q1 and its derivative tabulation factorises), so it is
// tabulated on the 2D grid of the other two coordinates:
//   Jc[0][(a,b)] = dx/dxi1 at (xi2, xi3) = (x_a, x_b)
//   Jc[1][(a,b)] = dx/dxi2 at (xi1, xi3) = (x_a, x_b)
//   Jc[2][(a,b)] = dx/dxi3 at (xi1, xi2) = (x_a, x_b)
// X holds the 8 corners, corner (a,b,c) at 4a+2b+c.  Thread t = (a,b) fills entry t.
template <int N>
__device__ __forceinline__ void jacobian_columns(const double (*X)[3], const double* xq, double (*Jc)[N * N][3],
                                                 int t) {
  const int a = t / N, b = t - (t / N) * N;
  const double ya = xq[a], yb = xq[b];
  const double w00 = (1.0 - ya) * (1.0 - yb), w01 = (1.0 - ya) * yb, w10 = ya * (1.0 - yb), w11 = ya * yb;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Jc[0][t][k] = w00 * (X[4][k] - X[0][k]) + w01 * (X[5][k] - X[1][k]) + w10 * (X[6][k] - X[2][k]) +
                  w11 * (X[7][k] - X[3][k]);
    Jc[1][t][k] = w00 * (X[2][k] - X[0][k]) + w01 * (X[3][k] - X[1][k]) + w10 * (X[6][k] - X[4][k]) +
                  w11 * (X[7][k] - X[5][k]);
    Jc[2][t][k] = w00 * (X[1][k] - X[0][k]) + w01 * (X[3][k] - X[2][k]) + w10 * (X[5][k] - X[4][k]) +
                  w11 * (X[7][k] - X[6][k]);
  }
}

// Conversions between double and float on the integer pipe (GB300's FP64
// pipe, which also runs the hardware conversions, is the scarce unit).
// float -> double is exact: re-bias the exponent, widen the mantissa.  Zero
// and subnormal floats map to a signed zero (values below 1.2e-38 do not
// matter here), infinities and NaNs take the hardware path.
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
  if (e == 0u) return __longlong_as_double((long long)sgn);
  if (e == 0xffu) return (double)f;
  const unsigned long long bits =
      sgn | ((unsigned long long)(e + (1023u - 127u)) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}
// double -> float, round to nearest even on the 52 -> 23 bit mantissa; a
// carry out of the mantissa increments the exponent field, as it should.
// Zero, results that would be subnormal or overflow, and non-finite values
// take the hardware path.
__device__ __forceinline__ float d2f_int(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
  if (e <= 0 || e >= 255) return (float)d;
  const unsigned long long m = b & 0xfffffffffffffull;
  const unsigned long long r = m + 0x0fffffffull + ((m >> 29) & 1ull);
  const uint32_t out = ((uint32_t)(b >> 63) << 31) | ((uint32_t)e << 23);
  return __uint_as_float(out + (uint32_t)(r >> 29));
}

__device__ __forceinline__ void cross3(const double* u, const double* v, double* w) {
  w[0] = u[1] * v[2] - u[2] * v[1];
  w[1] = u[2] * v[0] - u[0] * v[2];
  w[2] = u[0] * v[1] - u[1] * v[0];
}
__device__ __forceinline__ double dot3(const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

// Hyperelastic test flux at one point (Sec. 4.1 and the neo-Hookean variant).
// H = grad^ u (reference gradient, H[i][k] = d u_i / d xi_k), R = rows of
// adj(J) = S J^{-1}, S = det J, w the quadrature weight.  F = I + H R / S;
//   neo-Hookean  P = mu (F - F^{-T}) + lambda ln(det F) F^{-T}
//   SVK          P = F (lambda tr(E) I + 2 mu E),  E = (F^T F - I)/2
// and the flux w S P G^T = w P R^T is written to out[i][k].  Returns false
// (and a zero flux) if det F <= 0 for the neo-Hookean law.
template <bool NEO>
__device__ __forceinline__ bool hyperelastic_flux(const double (*H)[3], const double (*R)[3], double S, double w,
                                                  double mu, double lam, double (*out)[3]) {
  const double iS = 1.0 / S;
  double F[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F[i][j] = (H[i][0] * R[0][j] + H[i][1] * R[1][j] + H[i][2] * R[2][j]) * iS + (i == j ? 1.0 : 0.0);
  double Pk[3][3];
  bool good = true;
  if (NEO) {
    double Cf[3][3];  // cofactor matrix of F: F^{-T} = Cf / det F
    cross3(F[1], F[2], Cf[0]);
    cross3(F[2], F[0], Cf[1]);
    cross3(F[0], F[1], Cf[2]);
    const double JF = dot3(F[0], Cf[0]);
    good = JF > 0.0;
    const double iJ = good ? 1.0 / JF : 0.0, lnJ = good ? log(JF) : 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double FiT = Cf[i][j] * iJ;
        Pk[i][j] = good ? mu * (F[i][j] - FiT) + lam * lnJ * FiT : 0.0;
      }
  } else {
    double E[3][3], S2[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        E[i][j] = 0.5 * (F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j] - (i == j ? 1.0 : 0.0));
    const double trE = E[0][0] + E[1][1] + E[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) S2[i][j] = (i == j ? lam * trE : 0.0) + 2.0 * mu * E[i][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Pk[i][j] = F[i][0] * S2[0][j] + F[i][1] * S2[1][j] + F[i][2] * S2[2][j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) out[i][k] = w * dot3(Pk[i], R[k]);
  return good;
}


// One 1D contraction of an N0 x N1 x N2 array held in shared memory, along
// axis AX, for the fiber owned by thread `t` (fibers are indexed by the two
// other axes; t < product of their extents):
//   out[.., r, ..] = (ACC ? out[.., r, ..] : 0) + sum_k M[r][k] in[.., k, ..]
// TRANS uses M[k][r].  NIN / NOUT: extents of the contracted axis before and
// after; D0..D2 the full extents of the *input* array (the output has NOUT at
// AX).  In-place use (in == out, NIN == NOUT) is safe: a fiber is read whole
// into registers before it is written, and no other thread touches it.
template <int D0, int D1, int D2, int AX, int NOUT, bool TRANS, bool ACC, int LDM>
__device__ __forceinline__ void contract(const double* in, double* out, const double (*M)[LDM], int t) {
  constexpr int NIN = AX == 0 ? D0 : (AX == 1 ? D1 : D2);
  // output extents
  constexpr int E1 = AX == 1 ? NOUT : D1, E2 = AX == 2 ? NOUT : D2;
  int ib, ob, is, os;
  if (AX == 0) {
    const int f0 = t / D2, f1 = t - (t / D2) * D2;  // (i1, i2)
    ib = f0 * D2 + f1; is = D1 * D2;
    ob = f0 * E2 + f1; os = E1 * E2;
  } else if (AX == 1) {
    const int f0 = t / D2, f1 = t - (t / D2) * D2;  // (i0, i2)
    ib = f0 * D1 * D2 + f1; is = D2;
    ob = f0 * E1 * E2 + f1; os = E2;
  } else {
    const int f0 = t / D1, f1 = t - (t / D1) * D1;  // (i0, i1)
    ib = (f0 * D1 + f1) * D2; is = 1;
    ob = (f0 * E1 + f1) * E2; os = 1;
  }
  double v[NIN];
#pragma unroll
  for (int k = 0; k < NIN; ++k) v[k] = in[ib + k * is];
#pragma unroll
  for (int r = 0; r < NOUT; ++r) {
    double acc = ACC ? out[ob + r * os] : 0.0;
#pragma unroll
    for (int k = 0; k < NIN; ++k) acc = fma(TRANS ? M[k][r] : M[r][k], v[k], acc);
    out[ob + r * os] = acc;
  }
}

}  // namespace sfx
