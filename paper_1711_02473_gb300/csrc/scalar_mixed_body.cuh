#pragma once
// scalar_mixed_body.cuh -- scalar-form actions (mass, Laplace, Helmholtz; Q_p
// and DQ_p) with the 1D contractions on the tensor cores as split-precision
// products, and the geometry / weight scaling / scatter in FP64.  Instantiated
// once per input format in k_scalar_mixed_tf32.cu and k_scalar_mixed_bf16.cu.
//
// Same algorithm as k_scalar.cu (Sec. 3.3, Eqs. coeff_eval and form_eval with
// the sum factorisation of Sec. 3.2).  What changes is where the arithmetic runs:
//   - J, det J, adj J and the weight scaling w/S are computed in FP64; the
//     six products of adjugate rows that form P = w S G G^T run in FP32 (they
//     only feed FP32 factors) and are scaled in FP64 before rounding;
//   - every 1D contraction (B, Dq and their transposes) is one batched matrix
//     product per CTA: the table (q x n, padded to 16 x 8k) times the fibers of
//     all cells held by the CTA (n x (cells*n^2)), on mma.sync with FP32
//     accumulation.  Each operand is split into a high and a low part in the
//     input format (TF32: 11 significant bits each; BF16: 8 each) and three
//     products hi*hi + hi*lo + lo*hi are accumulated (the lo*lo term is dropped);
//   - the flux P grad u is formed in FP32 from the rounded factors;
//   - b^K is widened to FP64 and added into y in FP64.
// Error model: each stage carries the FP32 accumulator's ~2^-24 relative
// rounding plus the split's representation error (TF32x3 ~2^-22, BF16x3 ~2^-16).
#include "mixed_common.cuh"

namespace sfx {
namespace {

template <int N, int FORM>
struct MixedShape {
  static constexpr int N2 = N * N, N3 = N2 * N;
  static constexpr bool LAP = FORM != SFX_MASS;
  static constexpr bool MAS = FORM != SFX_LAPLACE;
  // threads per CTA, chosen by measurement on the 64^3 sweep: 128 at n = 7
  // (smaller CTAs, more per SM, so one CTA's FP64 geometry overlaps another's
  // tensor-core phases: 7-16% faster), 256 elsewhere (128 was 5-12% slower
  // at n = 8, 9)
  static constexpr int NT = N == 7 ? 128 : 256;
  // Geometry tables: for N >= 4 the staged adjugate-row tables (see adj_rows;
  // 2D record per (q2,q3): all three rows for the Laplace part, only c0 for
  // mass); for N <= 3, where a cell has at most 27 points and the staged build
  // does not pay, the Jacobian column tables with cross products at the point.
  static constexpr bool HIER = N >= 4;
  static constexpr int REC23 = LAP ? 16 : 4;
  // per-cell floats: U, G0..G2 (LAP); plus the staged factors K[6] (LAP) and
  // WS (MAS) when geo_once
  static constexpr int cellf(bool geo_once) {
    return N3 + (LAP ? 3 * N3 : 0) + (geo_once ? (LAP ? 6 * N3 : 0) + (MAS ? N3 : 0) : 0);
  }
  // per-cell temporaries of the table build: corners, edge vectors, 1D vectors
  static constexpr int TMPD = HIER ? 24 + kAdjEdge + kAdjT1D * N : 24;
  // they live in the float area (free until the gather) when it is large enough
  static constexpr bool TMP_IN_F = HIER && 2 * TMPD <= N3 + (LAP ? 3 * N3 : 0);
  // per-cell doubles: [temporaries] + 2D tables R23, R12 (or the column
  // tables Jc[3][N^2][3]); on-the-fly geometry only
  static constexpr int TABD = HIER ? N2 * (REC23 + 6) : 9 * N2;
  static constexpr int celld(bool stored) { return stored ? 0 : (TMP_IN_F ? 0 : TMPD) + TABD; }
  // two FP32 tables, 1D points and weights (16 doubles each)
  static constexpr size_t fixed_bytes() { return 2 * sizeof(TabF) + 32 * 8; }
  static constexpr size_t bytes(int cb, bool geo_once, bool stored) {
    return fixed_bytes() + (size_t)cb * celld(stored) * 8 + (size_t)cb * cellf(geo_once) * 4 + (size_t)cb * 8 + 16;
  }
};

// Factors at point qp of a cell, from the cell's 2D adjugate-row tables (tab
// = R23 followed by R12).  The rows r_k of adj J = S J^{-1}, S = det J and the
// weight scaling w/S (Newton reciprocal, one step: < 2^-44 relative, far below
// the FP32 rounding of the factors) are computed in FP64; the six products
// r_k . r_l, which only feed FP32 factors, run on the FP32 pipe from the rows
// rounded once to FP32, and are scaled by w/S in FP64 before the final
// rounding.  Returns S.
template <int N, bool LAP, bool MAS>
__device__ __forceinline__ double mixed_point_factors(const double* tab, const double* xq, const double* wq, int qp,
                                                      double alpha, double beta, float* K, float* wsm) {
  constexpr int N2 = N * N;
  constexpr int REC23 = LAP ? 16 : 4;
  const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
  double r0[3], r1[3], r2[3], w, S;
  if (N >= 4) {
    S = adj_rows<N, REC23, LAP>(tab, tab + N2 * REC23, xq, wq, q1, q2, q3, r0, r1, r2, &w);
  } else {
    S = point_rows<N, LAP>(reinterpret_cast<const double(*)[N2][3]>(tab), qp, r0, r1, r2);
    w = wq[q1] * wq[q2] * wq[q3];
  }
  if (LAP) {
    const double ws = (alpha * w) * recip_nr<1>(S);
    float f0[3], f1[3], f2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      f0[k] = d2f_int(r0[k]);
      f1[k] = d2f_int(r1[k]);
      f2[k] = d2f_int(r2[k]);
    }
    auto dotf = [](const float* u, const float* v) { return fmaf(u[0], v[0], fmaf(u[1], v[1], u[2] * v[2])); };
    K[0] = d2f_int(ws * f2d_int(dotf(f0, f0)));
    K[1] = d2f_int(ws * f2d_int(dotf(f1, f1)));
    K[2] = d2f_int(ws * f2d_int(dotf(f2, f2)));
    K[3] = d2f_int(ws * f2d_int(dotf(f0, f1)));
    K[4] = d2f_int(ws * f2d_int(dotf(f0, f2)));
    K[5] = d2f_int(ws * f2d_int(dotf(f1, f2)));
  }
  if (MAS) *wsm = d2f_int((beta * w) * S);
  return S;
}

// Flux at point qp of a cell for one RHS, without forming the factors: the
// adjugate rows R (FP64, rounded once to FP32), S = det J and t = alpha w / S
// (FP64, one-step Newton reciprocal) give P g = t R R^T g, applied as R (t R^T g):
// R^T g and the final R v in FP32, the scaling of the three entries of R^T g
// by t in FP64.  g (in/out): the reference gradient, replaced by the flux;
// *u (in/out): the value, scaled by beta w S (mass part).  Returns S.
template <int N, bool LAP, bool MAS>
__device__ __forceinline__ double mixed_point_flux(const double* tab, const double* xq, const double* wq, int qp,
                                                   double alpha, double beta, float* g, float* u) {
  constexpr int N2 = N * N;
  constexpr int REC23 = LAP ? 16 : 4;
  const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
  double r0[3], r1[3], r2[3], w, S;
  if (N >= 4) {
    S = adj_rows<N, REC23, LAP>(tab, tab + N2 * REC23, xq, wq, q1, q2, q3, r0, r1, r2, &w);
  } else {
    S = point_rows<N, LAP>(reinterpret_cast<const double(*)[N2][3]>(tab), qp, r0, r1, r2);
    w = wq[q1] * wq[q2] * wq[q3];
  }
  if (LAP) {
    const double t = (alpha * w) * recip_nr<1>(S);
    float f0[3], f1[3], f2[3], v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      f0[k] = d2f_int(r0[k]);
      f1[k] = d2f_int(r1[k]);
      f2[k] = d2f_int(r2[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = d2f_int(t * f2d_int(fmaf(f0[k], g[0], fmaf(f1[k], g[1], f2[k] * g[2]))));
    g[0] = fmaf(f0[0], v[0], fmaf(f0[1], v[1], f0[2] * v[2]));
    g[1] = fmaf(f1[0], v[0], fmaf(f1[1], v[1], f1[2] * v[2]));
    g[2] = fmaf(f2[0], v[0], fmaf(f2[1], v[1], f2[2] * v[2]));
  }
  if (MAS) *u = d2f_int((beta * w) * S) * *u;
  return S;
}

// STORED: the FP32 factors come from a.qd32 (sfx_qdata) and no FP64 geometry
// runs in the kernel.  geo_once: stage the factors once per cell for all RHS.
// COLL: the collocated Gauss-Lobatto rule on the GLL nodes of Q_p (the points
// are the nodes: B = I, derivative table = GLL collocation matrix, geometry at
// the GLL points with the GLL weights; Sec. 2.5 and "underintegration" in 4.1).
// One tile: the cb cells of slots slot0 .. slot0+cb-1, run by the NT threads
// of the CTA (the per-colour kernel below, and the persistent p-adaptive batch
// with NT = its block size).  smd: the tile's shared memory (MixedShape::bytes).
template <int N, bool DQ, int FORM, int PREC, bool STORED, bool COLL, int NT>
__device__ __forceinline__ void scalar_tile_mixed(const ActArgs& a, const int64_t ncell_total, const int64_t slot0,
                                                  const int cb, const bool geo_once, double* smd) {
  using Sh = MixedShape<N, FORM>;
  constexpr int N2 = Sh::N2, N3 = Sh::N3;
  constexpr bool LAP = Sh::LAP, MAS = Sh::MAS;
  const Tab1D& T = c_tab[N - 1];
  // layout: [tables: 2 TabF][xq: 16 doubles][wq: 16 doubles][cells: doubles][cells: floats][flags]
  TabF* tabs = reinterpret_cast<TabF*>(smd);  // 0: B, 1: Dq
  double* xq = smd + (2 * sizeof(TabF)) / 8;
  double* wq = xq + 16;
  double* cd = wq + 16;                       // per-cell doubles (on-the-fly geometry)
  float* cf = reinterpret_cast<float*>(cd + (size_t)cb * Sh::celld(STORED));
  float* U = cf;
  float* G0 = U + cb * N3;
  float* G1 = G0 + cb * N3;
  float* G2 = G1 + cb * N3;
  float* K = (LAP ? G2 : U) + cb * N3;        // K[j][cell][qp]   (geo_once only)
  float* WS = K + (LAP ? 6 * cb * N3 : 0);   // WS[cell][qp]     (geo_once only)
  int* flags = reinterpret_cast<int*>(cf + (size_t)cb * Sh::cellf(geo_once));  // per cell: id or -1, bad

  const int tid = threadIdx.x;
  for (int i = tid; i < 16 * 16; i += NT) {
    const int r = i / 16, k = i % 16;
    tabs[0].v[r][k] = (r < N && k < N) ? (float)T.Bc[r][k] : 0.f;
    tabs[1].v[r][k] = (r < N && k < N) ? (float)(COLL ? T.Dg[r][k] : T.Dq[r][k]) : 0.f;
  }
  if (tid < N) {
    xq[tid] = COLL ? T.xg[tid] : T.x[tid];
    wq[tid] = COLL ? T.wg[tid] : T.w[tid];
  }
  for (int c = tid; c < cb; c += NT) {
    int cell = -1;
    if (!slot_cell(a, slot0 + c, ncell_total, &cell)) cell = -1;
    flags[2 * c] = cell;
    flags[2 * c + 1] = 0;
  }
  __syncthreads();
  pdl_allow_next();
  const double alpha = FORM == SFX_HELMHOLTZ ? a.alpha : 1.0;
  const double beta = FORM == SFX_HELMHOLTZ ? a.beta : 1.0;
  const float fa = (float)alpha, fb = (float)beta;
  // per-cell build temporaries and 2D tables (see adj_rows)
  auto tmp_of = [&](int c) -> double* {
    return Sh::TMP_IN_F ? reinterpret_cast<double*>(cf) + (size_t)c * Sh::TMPD : cd + (size_t)c * Sh::celld(false);
  };
  auto tab_of = [&](int c) -> const double* {
    return cd + (size_t)c * Sh::celld(false) + (Sh::TMP_IN_F ? 0 : Sh::TMPD);
  };
  if (!STORED) {
    for (int i = tid; i < cb * 24; i += NT) {
      const int c = i / 24, v = (i % 24) / 3, k = i % 3;
      const int cell = flags[2 * c];
      tmp_of(c)[v * 3 + k] =
          cell >= 0 ? a.xyz[(int64_t)a.vmap[(int64_t)cell * 8 + v] * 3 + k] : (double)((v >> (2 - k)) & 1);
    }
    __syncthreads();
    if (!Sh::HIER) {
      for (int i = tid; i < cb * N2; i += NT) {
        const int c = i / N2, t = i - c * N2;
        jacobian_columns<N>(reinterpret_cast<const double(*)[3]>(tmp_of(c)), xq,
                            reinterpret_cast<double(*)[N2][3]>(const_cast<double*>(tab_of(c))), t);
      }
      __syncthreads();
    } else {
      for (int i = tid; i < cb * kAdjEdge; i += NT) {
        const int c = i / kAdjEdge;
        double* X = tmp_of(c);
        adj_edges(reinterpret_cast<const double(*)[3]>(X), X + 24, i - c * kAdjEdge);
      }
      __syncthreads();
      for (int i = tid; i < cb * 3 * N; i += NT) {
        const int c = i / (3 * N), r = i - c * (3 * N);
        double* X = tmp_of(c);
        adj_1d<LAP>(X + 24, xq, X + 24 + kAdjEdge, r / N, r % N);
      }
      __syncthreads();
      for (int i = tid; i < cb * N2; i += NT) {
        const int c = i / N2, t = i - c * N2;
        double* R23 = const_cast<double*>(tab_of(c));
        adj_2d<N, Sh::REC23>(tmp_of(c) + 24 + kAdjEdge, xq, wq, R23, R23 + N2 * Sh::REC23, t);
      }
      __syncthreads();
    }
  }
  if (geo_once) {
    for (int i = tid; i < cb * N3; i += NT) {
      const int c = i / N3, qp = i - c * N3;
      const int cell = flags[2 * c];
      float kk[6], wsm = 0.f;
      if (STORED) {
        const float* qd = a.qd32 + (int64_t)(cell >= 0 ? cell : 0) * 7 * N3;
        if (LAP)
          for (int j = 0; j < 6; ++j) kk[j] = cell >= 0 ? fa * qd[j * N3 + qp] : 0.f;
        if (MAS) wsm = cell >= 0 ? fb * qd[6 * N3 + qp] : 0.f;
      } else {
        const double S = mixed_point_factors<N, LAP, MAS>(tab_of(c), xq, wq, qp, alpha, beta,
                                                          kk, &wsm);
        if (!positive_finite(S)) flags[2 * c + 1] = 1;
      }
      if (LAP)
        for (int j = 0; j < 6; ++j) K[(j * cb + c) * N3 + qp] = kk[j];
      if (MAS) WS[c * N3 + qp] = wsm;
    }
    __syncthreads();
  }

#pragma unroll 1
  for (int r = 0; r < a.nrhs; ++r) {
    for (int i = tid; i < cb * N3; i += NT) {
      const int c = i / N3, l = i - c * N3;
      const int cell = flags[2 * c];
      U[i] = cell >= 0 ? d2f_int(a.x[cell_dof(a, cell, l, N3) * a.nrhs + r]) : 0.f;
    }
    __syncthreads();
    if (!DQ && !COLL) {
      tc_contract<N, 0, false, false, PREC, NT>(U, U, tabs[0], cb);
      __syncthreads();
      tc_contract<N, 1, false, false, PREC, NT>(U, U, tabs[0], cb);
      __syncthreads();
      tc_contract<N, 2, false, false, PREC, NT>(U, U, tabs[0], cb);
      __syncthreads();
    }
    if (LAP) {
      tc_contract<N, 0, false, false, PREC, NT>(U, G0, tabs[1], cb);
      tc_contract<N, 1, false, false, PREC, NT>(U, G1, tabs[1], cb);
      tc_contract<N, 2, false, false, PREC, NT>(U, G2, tabs[1], cb);
      __syncthreads();
    }
    for (int i = tid; i < cb * N3; i += NT) {
      const int c = i / N3, qp = i - c * N3;
      const int cell = flags[2 * c];
      float kk[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, wsm = 0.f;
      if (geo_once) {
        if (LAP)
          for (int j = 0; j < 6; ++j) kk[j] = K[(j * cb + c) * N3 + qp];
        if (MAS) wsm = WS[c * N3 + qp];
      } else if (STORED) {
        if (cell >= 0) {
          const float* qd = a.qd32 + (int64_t)cell * 7 * N3;
          if (LAP)
            for (int j = 0; j < 6; ++j) kk[j] = fa * qd[j * N3 + qp];
          if (MAS) wsm = fb * qd[6 * N3 + qp];
        }
      } else {
        // factors at the point: flux R (t R^T g) without forming them
        float g[3] = {LAP ? G0[i] : 0.f, LAP ? G1[i] : 0.f, LAP ? G2[i] : 0.f}, u = U[i];
        const double S = mixed_point_flux<N, LAP, MAS>(tab_of(c), xq, wq, qp, alpha, beta, g, &u);
        if (!positive_finite(S)) flags[2 * c + 1] = 1;
        if (LAP) {
          G0[i] = g[0];
          G1[i] = g[1];
          G2[i] = g[2];
        }
        if (MAS) U[i] = u;
        continue;
      }
      if (LAP) {
        const float g0 = G0[i], g1 = G1[i], g2 = G2[i];
        G0[i] = kk[0] * g0 + kk[3] * g1 + kk[4] * g2;
        G1[i] = kk[3] * g0 + kk[1] * g1 + kk[5] * g2;
        G2[i] = kk[4] * g0 + kk[5] * g1 + kk[2] * g2;
      }
      if (MAS) U[i] = wsm * U[i];
    }
    __syncthreads();
    if (LAP) {
      tc_contract<N, 0, true, MAS, PREC, NT>(G0, U, tabs[1], cb);
      __syncthreads();
      tc_contract<N, 1, true, true, PREC, NT>(G1, U, tabs[1], cb);
      __syncthreads();
      tc_contract<N, 2, true, true, PREC, NT>(G2, U, tabs[1], cb);
      __syncthreads();
    }
    if (!DQ && !COLL) {
      tc_contract<N, 0, true, false, PREC, NT>(U, U, tabs[0], cb);
      __syncthreads();
      tc_contract<N, 1, true, false, PREC, NT>(U, U, tabs[0], cb);
      __syncthreads();
      tc_contract<N, 2, true, false, PREC, NT>(U, U, tabs[0], cb);
      __syncthreads();
    }
    if (r == 0) pdl_wait_prev();
    if (a.cell_vectors) {
      for (int i = tid; i < cb * N3; i += NT) {
        const int c = i / N3, l = i - c * N3;
        if (flags[2 * c] < 0) continue;
        const int64_t slot = slot0 + c;
        a.y[(slot * N3 + l) * a.nrhs + r] = !flags[2 * c + 1] ? f2d_int(U[i]) : 0.0;
      }
    } else {
      // reduction in L2 (red.global.add.f64), not on the SM's FP64 pipe; cells
      // of one launch share no dof, so every address is added to once per
      // launch and the order of the sums is that of the launches; in an
      // overwriting action the dof's first pair stores instead (0 if skipped).
      // GS map entries per thread are loaded before the first write.
      constexpr int GS = 4;
      for (int i0 = tid; i0 < cb * N3; i0 += GS * NT) {
        int64_t dof[GS];
#pragma unroll
        for (int g = 0; g < GS; ++g) {
          const int i = i0 + g * NT;
          const int c = i / N3;
          const int cell = i < cb * N3 ? flags[2 * c] : -1;
          dof[g] = cell >= 0 ? cell_dof(a, cell, i - c * N3, N3) : -1;
        }
#pragma unroll
        for (int g = 0; g < GS; ++g) {
          if (dof[g] < 0) continue;
          const int i = i0 + g * NT;
          const int c = i / N3;
          const bool ok = !flags[2 * c + 1];
          double* yp = &a.y[dof[g] * a.nrhs + r];
          if (first_touch(a, flags[2 * c], i - c * N3, N3)) *yp = ok ? f2d_int(U[i]) : 0.0;
          else if (ok) atomicAdd(yp, f2d_int(U[i]));
        }
      }
    }
    if (r == 0)
      for (int c = tid; c < cb; c += NT)
        if (flags[2 * c] >= 0 && flags[2 * c + 1]) set_flag(a.status, SFX_DEV_INVERTED);
    __syncthreads();
  }
}

template <int N, bool DQ, int FORM, int PREC, bool STORED, bool COLL = false>
__global__ void __launch_bounds__(MixedShape<N, FORM>::NT) k_action_scalar_mixed(const ActArgs a, const int64_t ncell_total,
                                                                  const int cb, const bool geo_once) {
  extern __shared__ double smd[];
  scalar_tile_mixed<N, DQ, FORM, PREC, STORED, COLL, MixedShape<N, FORM>::NT>(a, ncell_total, (int64_t)blockIdx.x * cb,
                                                                              cb, geo_once, smd);
}

// ------------------------------------------------------------------ launcher
template <int N, bool DQ, int FORM, int PREC>
int launch_mixed_one(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = MixedShape<N, FORM>;
  const bool stored = a.qd32 != nullptr;
  const bool geo_once = a.nrhs > 1;
  const size_t budget = 200 * 1024;
  // cells per CTA: the autotuned value, else enough fibers for dense tiles
  int cb = tuned_cells_per_cta(stored ? SFX_TUNE_SCALAR_MIXED_STORED : SFX_TUNE_SCALAR_MIXED, N - 1,
                               (N <= 3) ? 32 : 16);
  if (cb < 1) cb = 1;
  while (cb > 1 && Sh::bytes(cb, geo_once, stored) > budget) --cb;
  const size_t smem = Sh::bytes(cb, geo_once, stored);
  auto kern = stored ? k_action_scalar_mixed<N, DQ, FORM, PREC, true> : k_action_scalar_mixed<N, DQ, FORM, PREC, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  e = launch_kernel(kern, (unsigned)grid, Sh::NT, smem, s, a.overlap_prev != 0, a, ncell_total, cb, geo_once);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

template <int N, bool DQ, int PREC>
int mixed_dispatch_form(sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (form) {
    case SFX_MASS: return launch_mixed_one<N, DQ, SFX_MASS, PREC>(a, nc, s);
    case SFX_LAPLACE: return launch_mixed_one<N, DQ, SFX_LAPLACE, PREC>(a, nc, s);
    case SFX_HELMHOLTZ: return launch_mixed_one<N, DQ, SFX_HELMHOLTZ, PREC>(a, nc, s);
    default: return -1;
  }
}

template <int N, int PREC>
int mixed_dispatch(bool dq, sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  return dq ? mixed_dispatch_form<N, true, PREC>(form, a, nc, s) : mixed_dispatch_form<N, false, PREC>(form, a, nc, s);
}

// Launch of the split-precision scalar action in format PREC for one degree
// (one instantiation per translation unit): a colour of a space, or the cells
// of one degree of a p-adaptive plan (a.map null, a.dq_off set).
template <int PREC>
int launch_scalar_mixed_degree(int p, bool dq, sfx_form form, const ActArgs& a, int64_t nc, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  switch (p) {
    case 1: return mixed_dispatch<2, PREC>(dq, form, a, nc, s);
    case 2: return mixed_dispatch<3, PREC>(dq, form, a, nc, s);
    case 3: return mixed_dispatch<4, PREC>(dq, form, a, nc, s);
    case 4: return mixed_dispatch<5, PREC>(dq, form, a, nc, s);
    case 5: return mixed_dispatch<6, PREC>(dq, form, a, nc, s);
    case 6: return mixed_dispatch<7, PREC>(dq, form, a, nc, s);
    case 7: return mixed_dispatch<8, PREC>(dq, form, a, nc, s);
    case 8: return mixed_dispatch<9, PREC>(dq, form, a, nc, s);
  }
  return -1;
}

template <int PREC>
int launch_scalar_mixed_prec(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  return launch_scalar_mixed_degree<PREC>(sp->p, sp->family == SFX_DQ, form, a, sp->mesh->ncell, stream);
}

}  // namespace
}  // namespace sfx
