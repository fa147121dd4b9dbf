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

// Programmatic dependent launch between the colour launches of one action.
// Launch k+1 may start while launch k drains (its CTAs take the SM slots that
// launch k's CTAs leave): the work before the scatter (gather, geometry,
// contractions) reads only inputs that no launch of the action writes.  Each
// thread of launch k+1 waits for launch k to complete, with its writes to y
// visible, before its first write to y, and every CTA passes that wait before
// it exits, so launch k+1 also completes after launch k.  In a kernel launched
// without the attribute both instructions do nothing.
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `k` on `s`, as a programmatic dependent of the previous launch on the
// stream when `overlap_prev` is set (the kernel must call pdl_wait_prev before
// its first write to y).
template <typename... P, typename... A>
cudaError_t launch_kernel(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                          bool overlap_prev, const A&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = overlap_prev ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Global dof of local index l of a cell: the space's cell-node map, or, for a
// p-adaptive DQ mesh (no map), the cell's dof offset + l.
__device__ __forceinline__ int64_t cell_dof(const ActArgs& a, int64_t cell, int l, int nloc) {
  return a.map ? (int64_t)__ldg(&a.map[cell * nloc + l]) : __ldg(&a.dq_off[cell]) + l;
}

// Whether (cell, l) writes its dof first in an overwriting action (ActArgs
// first / first_all): that pair stores its value (0 for a skipped cell), every
// later pair of the dof, in a later colour launch, adds to it.
__device__ __forceinline__ bool first_touch(const ActArgs& a, int64_t cell, int l, int nloc) {
  if (a.first_all) return true;
  if (!a.first) return false;
  const int words = (nloc + 31) >> 5;
  return (__ldg(&a.first[cell * words + (l >> 5)]) >> (l & 31)) & 1u;
}

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
  *cell = (int)(a.cell0 + slot);
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
// pipe, which also runs the hardware conversions, is the scarce unit).  The
// rare cases take the hardware conversion in an out-of-line call, so that it
// is a branch and not an FP64-pipe instruction issued under a predicate.
static __device__ __noinline__ float d2f_hw(double d) { return (float)d; }
static __device__ __noinline__ double f2d_hw(float f) { return (double)f; }
static __device__ __noinline__ double recip_div(double s) { return 1.0 / s; }

// float -> double is exact: re-bias the exponent, widen the mantissa.  Zero
// and subnormal floats map to a signed zero (values below 1.2e-38 do not
// matter here), infinities and NaNs take the hardware path.
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
  if (e == 0u) return __longlong_as_double((long long)sgn);
  if (e == 0xffu) return f2d_hw(f);
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
  if (e <= 0 || e >= 255) return d2f_hw(d);
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

// Rows r_k of adj J = S J^{-1} at point qp from the Jacobian column tables
// (r0 = c1 x c2, r1 = c2 x c0, r2 = c0 x c1); r1, r2 only when ROWS.  Returns
// S = det J = c0 . r0.
template <int N, bool ROWS>
__device__ __forceinline__ double point_rows(const double (*Jc)[N * N][3], int qp, double* r0, double* r1,
                                             double* r2) {
  constexpr int N2 = N * N;
  const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
  const double* c0 = Jc[0][q2 * N + q3];
  const double* c1 = Jc[1][q1 * N + q3];
  const double* c2 = Jc[2][q1 * N + q2];
  cross3(c1, c2, r0);
  if (ROWS) {
    cross3(c2, c0, r1);
    cross3(c0, c1, r2);
  }
  return dot3(c0, r0);
}

// s > 0 (and finite) decided on the integer bits of s, off the FP64 pipe:
// positive finite doubles are exactly the bit patterns in (0, 0x7ff0...0).
__device__ __forceinline__ bool positive_finite(double s) {
  const long long b = __double_as_longlong(s);
  return b > 0 && b < 0x7ff0000000000000LL;
}

// 1/s in FP64 by the Newton-Raphson iteration r <- r + r (1 - s r), seeded
// with the FP32 approximate reciprocal (PTX rcp.approx, relative error below
// 2^-22 including the rounding of s to FP32).  Each step squares the relative
// error: one step leaves < 2^-44, two steps reach FP64 rounding.  Two FMAs per
// step on the FP64 pipe instead of a full IEEE division; the conversions run
// on the integer pipe.  Outside the normal FP32 range of s the plain division
// is used.
template <int STEPS>
__device__ __forceinline__ double recip_nr(double s) {
  const float sf = d2f_int(s);
  const float af = fabsf(sf);
  if (!(af >= 1.0e-37f && af <= 1.0e37f)) return recip_div(s);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(sf));
  double r = f2d_int(rf);
#pragma unroll
  for (int k = 0; k < STEPS; ++k) r = fma(r, fma(-s, r, 1.0), r);
  return r;
}

// Adjugate rows of the trilinear Jacobian from per-cell tables.
//
// J = [c0 c1 c2] with c_d = dx/dxi_d; the rows of adj(J) = S J^{-1} are
// r0 = c1 x c2, r1 = c2 x c0, r2 = c0 x c1 (S = c0 . r0).  For the trilinear
// (vector-Q1) coordinate field (Sec. 3.1) each c_d is bilinear in the two
// other coordinates:
//   c0(xi2,xi3) = Pb + xi2 P2 + xi3 P3 + xi2 xi3 Pt
//   c1(xi1,xi3) = Qb + xi1 Q1 + xi3 Q3 + xi1 xi3 Qt
//   c2(xi1,xi2) = Rb + xi1 R1 + xi2 R2 + xi1 xi2 Rt
// with edge vectors from the 8 corners.  Expanding the cross products, each
// row is a bilinear combination, in the two coordinates it does not single
// out, of four vectors that depend on the third:
//   r0 = U0a(xi1) + xi2 U0b(xi1) + xi3 [U0c(xi1) + xi2 U0d(xi1)]
//   r1 = U1a(xi2) + xi3 U1b(xi2) + xi1 [U1c(xi2) + xi3 U1d(xi2)]
//   r2 = U2a(xi3) + xi2 U2b(xi3) + xi1 [U2c(xi3) + xi2 U2d(xi3)]
// (U0* = products of c1 = e0 + xi3 e1 and c2 = k0 + xi2 k1 at fixed xi1, and
// so on), the same sum factorisation as the basis functions get (Sec. 3.2).
// The tables are built in three stages per cell -- edge vectors (36 values),
// the 1D vectors U (one cross product per vector and point), then the 2D
// coefficient tables below with one FMA per component -- so that a point
// costs three FMAs per row instead of a cross product:
//   r0 = A0(q1,q2) + xi3 B0(q1,q2),  r1 = A1(q2,q3) + xi1 B1(q2,q3),
//   r2 = A2(q2,q3) + xi1 B2(q2,q3),  c0 = c0(q2,q3).
// The same sums as the direct cross products, in another rounding order.
//
// Layouts (per cell, doubles):
//   E[v*3 + k]        edge vectors, v = Pb P2 P3 Pt Qb Q1 Q3 Qt Rb R1 R2 Rt
//   T[q*42 + .]       1D vectors at point q: U0a..U0d (0..11), U1a..U1d, g0, g1
//                     (12..29; c0 = g0(xi2) + xi3 g1(xi2)), U2a..U2d (30..41)
//   R23[j*N^2 + (q2*N+q3)]  j = c0[0..2], then (REC23 = 16) A1[3], B1[3], A2[3],
//                     B2[3], and w2*w3 last; (REC23 = 4) c0[3], w2*w3
//   R12[j*N^2 + (q1*N+q2)]  j = A0[0..2], B0[0..2]
// Component-major 2D tables: threads at neighbouring points read neighbouring words.
constexpr int kAdjEdge = 36, kAdjT1D = 42;

// Stage 1: edge value j (< 36) from the corners X (corner (a,b,c) at 4a+2b+c).
__device__ __forceinline__ void adj_edges(const double (*X)[3], double* E, int j) {
  const int v = j / 3, k = j - (j / 3) * 3;
  const double x0 = X[0][k], x1 = X[1][k], x2 = X[2][k], x3 = X[3][k];
  const double x4 = X[4][k], x5 = X[5][k], x6 = X[6][k], x7 = X[7][k];
  const double tw = ((x7 - x6) - (x5 - x4)) - ((x3 - x2) - (x1 - x0));
  double e;
  switch (v) {
    case 0: e = x4 - x0; break;                  // Pb
    case 1: e = (x6 - x2) - (x4 - x0); break;    // P2
    case 2: e = (x5 - x1) - (x4 - x0); break;    // P3
    case 4: e = x2 - x0; break;                  // Qb
    case 5: e = (x6 - x4) - (x2 - x0); break;    // Q1
    case 6: e = (x3 - x1) - (x2 - x0); break;    // Q3
    case 8: e = x1 - x0; break;                  // Rb
    case 9: e = (x5 - x4) - (x1 - x0); break;    // R1
    case 10: e = (x3 - x2) - (x1 - x0); break;   // R2
    default: e = tw; break;                      // Pt = Qt = Rt
  }
  E[j] = e;
}

// Stage 2: the 1D vectors of axis `ax` at point q (one thread per (ax, q)).
// ROWS: all three rows (Laplace part); otherwise only r0 and c0 (det J).
template <bool ROWS>
__device__ __forceinline__ void adj_1d(const double* E, const double* xq, double* T, int ax, int q) {
  const double x = xq[q];
  const double* Pb = E + 0; const double* P2 = E + 3; const double* P3 = E + 6; const double* Pt = E + 9;
  const double* Qb = E + 12; const double* Q1 = E + 15; const double* Q3 = E + 18; const double* Qt = E + 21;
  const double* Rb = E + 24; const double* R1 = E + 27; const double* R2 = E + 30; const double* Rt = E + 33;
  double* o = T + q * kAdjT1D;
  double u[3], v[3], s[3], t[3];
  if (ax == 0) {  // r0 = (e0 + xi3 e1) x (k0 + xi2 k1) at xi1 = x
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      u[k] = fma(x, Q1[k], Qb[k]); v[k] = fma(x, Qt[k], Q3[k]);
      s[k] = fma(x, R1[k], Rb[k]); t[k] = fma(x, Rt[k], R2[k]);
    }
    cross3(u, s, o + 0); cross3(u, t, o + 3); cross3(v, s, o + 6); cross3(v, t, o + 9);
  } else if (ax == 1) {  // r1 = (f0 + xi1 f1) x (g0 + xi3 g1) at xi2 = x
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      u[k] = fma(x, R2[k], Rb[k]); v[k] = fma(x, Rt[k], R1[k]);
      s[k] = fma(x, P2[k], Pb[k]); t[k] = fma(x, Pt[k], P3[k]);
      o[24 + k] = s[k]; o[27 + k] = t[k];
    }
    if (ROWS) { cross3(u, s, o + 12); cross3(u, t, o + 15); cross3(v, s, o + 18); cross3(v, t, o + 21); }
  } else if (ROWS) {  // r2 = (h0 + xi2 h1) x (d0 + xi1 d1) at xi3 = x
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      u[k] = fma(x, P3[k], Pb[k]); v[k] = fma(x, Pt[k], P2[k]);
      s[k] = fma(x, Q3[k], Qb[k]); t[k] = fma(x, Qt[k], Q1[k]);
    }
    cross3(u, s, o + 30); cross3(v, s, o + 33); cross3(u, t, o + 36); cross3(v, t, o + 39);
  }
}

// Stage 3: entry t (< N^2) of both 2D tables.
template <int N, int REC23>
__device__ __forceinline__ void adj_2d(const double* T, const double* xq, const double* wq, double* R23, double* R12,
                                       int t) {
  constexpr int N2 = N * N;
  const int a = t / N, b = t - (t / N) * N;
  const double xa = xq[a], xb = xq[b];
  {  // (q2, q3) = (a, b)
    const double* ta = T + a * kAdjT1D;
    const double* tb = T + b * kAdjT1D;
#pragma unroll
    for (int k = 0; k < 3; ++k) R23[k * N2 + t] = fma(xb, ta[27 + k], ta[24 + k]);
    if (REC23 == 16) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        R23[(3 + k) * N2 + t] = fma(xb, ta[15 + k], ta[12 + k]);   // A1 = U1a + xi3 U1b
        R23[(6 + k) * N2 + t] = fma(xb, ta[21 + k], ta[18 + k]);   // B1 = U1c + xi3 U1d
        R23[(9 + k) * N2 + t] = fma(xa, tb[33 + k], tb[30 + k]);   // A2 = U2a + xi2 U2b
        R23[(12 + k) * N2 + t] = fma(xa, tb[39 + k], tb[36 + k]);  // B2 = U2c + xi2 U2d
      }
    }
    R23[(REC23 - 1) * N2 + t] = wq[a] * wq[b];
  }
  {  // (q1, q2) = (a, b)
    const double* ta = T + a * kAdjT1D;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      R12[k * N2 + t] = fma(xb, ta[3 + k], ta[0 + k]);        // A0 = U0a + xi2 U0b
      R12[(3 + k) * N2 + t] = fma(xb, ta[9 + k], ta[6 + k]);  // B0 = U0c + xi2 U0d
    }
  }
}

// Rows at point (q1,q2,q3) from the 2D tables of adj_2d: r0 always (with S),
// r1 and r2 when ROWS.  Returns S = det J; *w = w1 w2 w3.
template <int N, int REC23, bool ROWS>
__device__ __forceinline__ double adj_rows(const double* R23, const double* R12, const double* xq, const double* wq,
                                           int q1, int q2, int q3, double* r0, double* r1, double* r2, double* w) {
  constexpr int N2 = N * N;
  const double* o = R23 + (q2 * N + q3);
  const double* e = R12 + (q1 * N + q2);
  const double x1 = xq[q1], x3 = xq[q3];
#pragma unroll
  for (int k = 0; k < 3; ++k) r0[k] = fma(x3, e[(3 + k) * N2], e[k * N2]);
  if (ROWS) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r1[k] = fma(x1, o[(6 + k) * N2], o[(3 + k) * N2]);
      r2[k] = fma(x1, o[(12 + k) * N2], o[(9 + k) * N2]);
    }
  }
  *w = wq[q1] * o[(REC23 - 1) * N2];
  return o[0] * r0[0] + o[N2] * r0[1] + o[2 * N2] * r0[2];
}

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
