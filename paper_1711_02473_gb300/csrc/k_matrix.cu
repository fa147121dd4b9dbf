// k_matrix.cu -- local element matrices A^K (row = test, column = trial) of the
// bilinear forms, FP64, by argument factorisation and sum factorisation.
//
// Argument factorisation (Sec. 3.2, Eq. poisson_gem and the P^(k,l) factors)
// writes the integrand as a sum of terms, each the product of a per-point
// coefficient C(q), a test tensor-product factor and a trial tensor-product
// factor.  A term of the test block bt and trial block bs gives
//   A[(i1,i2,i3),(j1,j2,j3)] += sum_q X_t[q1][i1] Y_t[q2][i2] Z_t[q3][i3] C(q)
//                                     X_s[q1][j1] Y_s[q2][j2] Z_s[q3][j3]
// which is evaluated in the sum-factorised order of Eqs. opt1_product /
// opt2_product, one contraction index at a time (Algorithm 1's ordering q1,
// q2, q3 for every term):
//   T1[q2][q3]        = sum_q1 X_t X_s C                   (per fixed i1, j1)
//   T2[q3][i2][j2]    = sum_q2 Y_t Y_s T1
//   A[i2 i3][j2 j3]  += sum_q3 Z_t Z_s T2
// Terms sharing the (Z_t, Z_s) tables are summed in T2 before the last
// (O(n^7)) stage -- the factorisation by distributivity of pass (6).
// The H(div)/H(curl) forms are the same with one term list per block pair
// (split Concatenate, Sec. 3.5).  The naive variant evaluates every entry as a
// sum over all q^3 points (O(n^9)).
#include <algorithm>
#include <cstring>
#include <vector>

#include "kern_common.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_matrix)

namespace {

enum { TB_BC = 0, TB_DC = 1, TB_BD = 2, TB_DD = 3, TB_ID = 4, TB_DQ = 5, NTAB = 6 };
enum { CF_SCALAR = 0, CF_NCF = 1, CF_NCE = 2 };
constexpr int kMaxTerm = 48;
constexpr int kMaxCoef = 12;
constexpr int kMatThreads = 256;

struct MatTerm {
  int bt, bs, cid, zg;
  double sign;
  int tt[3], ts[3];
};

struct MatDesc {
  int nblk, nloc, kind, nterm;
  int dims[3][3];
  int off[3];
  int pair_begin[9], pair_end[9];  // term ranges of block pair bt*3+bs
  int pair_nzg[9];
  int zg_t[kMaxTerm], zg_s[kMaxTerm];  // Z tables of each z-group (global numbering)
  MatTerm term[kMaxTerm];
};

// sym index of (a,b) in {00,11,22,01,02,12}
__host__ __device__ inline int symi(int a, int b) {
  if (a == b) return a;
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// 1D table t, point q, basis i (q x 9 layout in shared memory)
__device__ __forceinline__ double tab(const double* tb, int t, int q, int i) { return tb[(t * kMaxQ + q) * kMaxN + i]; }

template <bool NAIVE>
__global__ void __launch_bounds__(kMatThreads) k_cell_matrices(const MatArgs a, const MatDesc d, const int p) {
  const Tab1D& T = c_tab[p];
  const int Q = p + 1, Q2 = Q * Q, Q3 = Q2 * Q;
  extern __shared__ double sm[];
  double* tb = sm;                                   // NTAB x 9 x 9
  double* coef = tb + NTAB * kMaxQ * kMaxN;          // kMaxCoef x Q3
  double* T1 = coef + kMaxCoef * Q3;                 // up to kMaxTerm x Q2
  double* T2 = T1 + kMaxTerm * Q2;                   // up to 4 x Q x 81
  double* X = T2 + 4 * Q * kMaxN * kMaxN;            // 24
  double* Jc = X + 24;                               // 3 x Q2 x 3
  double* KL = Jc + 9 * Q2;                          // kappa's dofs of the cell (weighted Laplace)
  int* bad = reinterpret_cast<int*>(KL + (a.kappa ? d.nloc : 0));
  const int tid = threadIdx.x;
  const int64_t cell = a.cell_begin + blockIdx.x;

  for (int i = tid; i < NTAB * kMaxQ * kMaxN; i += kMatThreads) {
    const int t = i / (kMaxQ * kMaxN), q = (i / kMaxN) % kMaxQ, j = i % kMaxN;
    double v = 0.0;
    if (q < Q) {
      switch (t) {
        case TB_BC: v = j <= p ? T.Bc[q][j] : 0.0; break;
        case TB_DC: v = j <= p ? T.Dc[q][j] : 0.0; break;
        case TB_BD: v = j < p ? T.Bd[q][j] : 0.0; break;
        case TB_DD: v = j < p ? T.Dd[q][j] : 0.0; break;
        case TB_ID: v = (j == q) ? 1.0 : 0.0; break;
        default: v = j < Q ? T.Dq[q][j] : 0.0; break;
      }
    }
    tb[i] = v;
  }
  if (tid < 24) {
    const int v = tid / 3, k = tid % 3;
    X[tid] = a.xyz[(int64_t)a.vmap[cell * 8 + v] * 3 + k];
  }
  if (tid == 0) *bad = 0;
  if (a.kappa)
    for (int l = tid; l < d.nloc; l += kMatThreads) KL[l] = a.kappa[a.map[cell * d.nloc + l]];
  __syncthreads();
  // Jacobian column tables (see jacobian_columns): Jc[(col*Q2 + ab)*3 + k]
  for (int i = tid; i < Q2; i += kMatThreads) {
    const int aa = i / Q, bb = i % Q;
    const double ya = T.x[aa], yb = T.x[bb];
    const double w00 = (1.0 - ya) * (1.0 - yb), w01 = (1.0 - ya) * yb, w10 = ya * (1.0 - yb), w11 = ya * yb;
    for (int k = 0; k < 3; ++k) {
      const double* Xc = X;
      Jc[(0 * Q2 + i) * 3 + k] = w00 * (Xc[12 + k] - Xc[0 + k]) + w01 * (Xc[15 + k] - Xc[3 + k]) +
                                 w10 * (Xc[18 + k] - Xc[6 + k]) + w11 * (Xc[21 + k] - Xc[9 + k]);
      Jc[(1 * Q2 + i) * 3 + k] = w00 * (Xc[6 + k] - Xc[0 + k]) + w01 * (Xc[9 + k] - Xc[3 + k]) +
                                 w10 * (Xc[18 + k] - Xc[12 + k]) + w11 * (Xc[21 + k] - Xc[15 + k]);
      Jc[(2 * Q2 + i) * 3 + k] = w00 * (Xc[3 + k] - Xc[0 + k]) + w01 * (Xc[9 + k] - Xc[6 + k]) +
                                 w10 * (Xc[15 + k] - Xc[12 + k]) + w11 * (Xc[21 + k] - Xc[18 + k]);
    }
  }
  __syncthreads();
  // per-point coefficients of the argument-factorised terms
  for (int qp = tid; qp < Q3; qp += kMatThreads) {
    const int q1 = qp / Q2, q2 = (qp / Q) % Q, q3 = qp % Q;
    const double w = T.w[q1] * T.w[q2] * T.w[q3];
    const double* c0 = Jc + (0 * Q2 + q2 * Q + q3) * 3;
    const double* c1 = Jc + (1 * Q2 + q1 * Q + q3) * 3;
    const double* c2 = Jc + (2 * Q2 + q1 * Q + q2) * 3;
    double r[3][3];
    cross3(c1, c2, r[0]);
    cross3(c2, c0, r[1]);
    cross3(c0, c1, r[2]);
    const double S = dot3(c0, r[0]);
    if (!(S > 0.0)) *bad = 1;
    const double* cc[3] = {c0, c1, c2};
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    if (d.kind == CF_SCALAR) {
      double kap = 1.0;  // weighted Laplace: kappa(xi_q) = sum_l kappa_l psi_l(xi_q)
      if (a.kappa) {
        const int tk = a.kappa_dq ? TB_ID : TB_BC;
        kap = 0.0;
        for (int l = 0; l < d.nloc; ++l) {
          const int i1 = l / Q2, i2 = (l / Q) % Q, i3 = l % Q;
          kap += KL[l] * tab(tb, tk, q1, i1) * tab(tb, tk, q2, i2) * tab(tb, tk, q3, i3);
        }
      }
      const double ws = kap * a.alpha * w / S;  // alpha = 1 for Laplace, 0 for mass
      for (int s = 0; s < 6; ++s) coef[s * Q3 + qp] = ws * dot3(r[pa[s]], r[pb[s]]);
      coef[6 * Q3 + qp] = a.beta * w * S;
    } else if (d.kind == CF_NCF) {
      const double sa = a.alpha * w / S;
      for (int s = 0; s < 6; ++s) coef[s * Q3 + qp] = sa * dot3(cc[pa[s]], cc[pb[s]]);
      coef[6 * Q3 + qp] = a.beta * w / S;
    } else {
      const double sb = a.beta * w / S, sa = a.alpha * w / S;
      for (int s = 0; s < 6; ++s) {
        coef[s * Q3 + qp] = sb * dot3(cc[pa[s]], cc[pb[s]]);
        coef[(6 + s) * Q3 + qp] = sa * dot3(r[pa[s]], r[pb[s]]);
      }
    }
  }
  __syncthreads();
  if (*bad) {
    if (tid == 0) set_flag(a.status, SFX_DEV_INVERTED);
    double* Ac = a.A + (int64_t)blockIdx.x * d.nloc * d.nloc;
    for (int i = tid; i < d.nloc * d.nloc; i += kMatThreads) Ac[i] = 0.0;
    return;
  }
  double* Ac = a.A + (int64_t)blockIdx.x * d.nloc * d.nloc;

  if constexpr (NAIVE) {
    // every entry as a full sum over the q^3 points: O(n^9) per cell
    for (int bt = 0; bt < d.nblk; ++bt)
      for (int bs = 0; bs < d.nblk; ++bs) {
        const int pr = bt * 3 + bs;
        const int* nt = d.dims[bt];
        const int* ns = d.dims[bs];
        const int mt = nt[0] * nt[1] * nt[2], ms = ns[0] * ns[1] * ns[2];
        for (int e = tid; e < mt * ms; e += kMatThreads) {
          const int it = e / ms, is = e % ms;
          const int i1 = it / (nt[1] * nt[2]), i2 = (it / nt[2]) % nt[1], i3 = it % nt[2];
          const int j1 = is / (ns[1] * ns[2]), j2 = (is / ns[2]) % ns[1], j3 = is % ns[2];
          double acc = 0.0;
          for (int tm = d.pair_begin[pr]; tm < d.pair_end[pr]; ++tm) {
            const MatTerm& m = d.term[tm];
            for (int qp = 0; qp < Q3; ++qp) {
              const int q1 = qp / Q2, q2 = (qp / Q) % Q, q3 = qp % Q;
              const double ft = tab(tb, m.tt[0], q1, i1) * tab(tb, m.tt[1], q2, i2) * tab(tb, m.tt[2], q3, i3);
              const double fs = tab(tb, m.ts[0], q1, j1) * tab(tb, m.ts[1], q2, j2) * tab(tb, m.ts[2], q3, j3);
              acc += m.sign * coef[m.cid * Q3 + qp] * ft * fs;
            }
          }
          Ac[(int64_t)(d.off[bt] + it) * d.nloc + d.off[bs] + is] = acc;
        }
      }
  } else {
    for (int bt = 0; bt < d.nblk; ++bt)
      for (int bs = 0; bs < d.nblk; ++bs) {
        const int pr = bt * 3 + bs;
        const int tb0 = d.pair_begin[pr], tb1 = d.pair_end[pr], nterm = tb1 - tb0, nzg = d.pair_nzg[pr];
        const int* nt = d.dims[bt];
        const int* ns = d.dims[bs];
        for (int i1 = 0; i1 < nt[0]; ++i1)
          for (int j1 = 0; j1 < ns[0]; ++j1) {
            // stage 1: T1[term][q2][q3] = sum_q1 X_t[q1][i1] X_s[q1][j1] C(q)
            for (int e = tid; e < nterm * Q2; e += kMatThreads) {
              const int tm = e / Q2, q23 = e % Q2;
              const MatTerm& m = d.term[tb0 + tm];
              double acc = 0.0;
              for (int q1 = 0; q1 < Q; ++q1)
                acc += tab(tb, m.tt[0], q1, i1) * tab(tb, m.ts[0], q1, j1) * coef[m.cid * Q3 + q1 * Q2 + q23];
              T1[e] = m.sign * acc;
            }
            __syncthreads();
            // stage 2: T2[zg][q3][i2][j2] = sum_{terms in zg} sum_q2 Y_t Y_s T1
            for (int e = tid; e < nzg * Q * nt[1] * ns[1]; e += kMatThreads) {
              const int zg = e / (Q * nt[1] * ns[1]);
              const int q3 = (e / (nt[1] * ns[1])) % Q;
              const int i2 = (e / ns[1]) % nt[1], j2 = e % ns[1];
              double acc = 0.0;
              for (int tm = 0; tm < nterm; ++tm) {
                const MatTerm& m = d.term[tb0 + tm];
                if (m.zg != zg) continue;
                for (int q2 = 0; q2 < Q; ++q2)
                  acc += tab(tb, m.tt[1], q2, i2) * tab(tb, m.ts[1], q2, j2) * T1[tm * Q2 + q2 * Q + q3];
              }
              T2[((zg * Q + q3) * kMaxN + i2) * kMaxN + j2] = acc;
            }
            __syncthreads();
            // stage 3: A[(i1,i2,i3),(j1,j2,j3)] = sum_zg sum_q3 Z_t Z_s T2 (j3 fastest: contiguous runs)
            const int nout = nt[1] * nt[2] * ns[1] * ns[2];
            for (int e = tid; e < nout; e += kMatThreads) {
              const int j3 = e % ns[2], j2 = (e / ns[2]) % ns[1];
              const int i3 = (e / (ns[1] * ns[2])) % nt[2], i2 = e / (ns[1] * ns[2] * nt[2]);
              double acc = 0.0;
              for (int zg = 0; zg < nzg; ++zg) {
                const int zt = d.zg_t[tb0 + zg], zs = d.zg_s[tb0 + zg];
                for (int q3 = 0; q3 < Q; ++q3)
                  acc += tab(tb, zt, q3, i3) * tab(tb, zs, q3, j3) * T2[((zg * Q + q3) * kMaxN + i2) * kMaxN + j2];
              }
              const int row = d.off[bt] + (i1 * nt[1] + i2) * nt[2] + i3;
              const int col = d.off[bs] + (j1 * ns[1] + j2) * ns[2] + j3;
              Ac[(int64_t)row * d.nloc + col] = acc;
            }
            __syncthreads();
          }
      }
  }
}

// Element matrices of the scalar forms on Q_p with the collocated Gauss-
// Lobatto rule (Sec. 4.1, "underintegration"): the points are the nodes, so a
// reference derivative of a basis function at a point is one 1D derivative
// table times two deltas,
//   d psi_r / d xi_1 (q) = D[q1][r1] delta(q2, r2) delta(q3, r3)   (cyclic),
// with D[a][b] = l_b'(x_a) the GLL collocation derivative.  Substituting this
// into A_rs = sum_q sum_kl C_kl(q) d_k psi_r(q) d_l psi_s(q) + M(q) psi_r psi_s
// cancels every sum but one (delta cancellation, Sec. 3.1 / 3.4):
//   k = l = 1:  [r2 = s2, r3 = s3]  sum_q1 C_11(q1,r2,r3) D[q1][r1] D[q1][s1]
//   k = l = 2:  [r1 = s1, r3 = s3]  sum_q2 C_22(r1,q2,r3) D[q2][r2] D[q2][s2]
//   k = l = 3:  [r1 = s1, r2 = s2]  sum_q3 C_33(r1,r2,q3) D[q3][r3] D[q3][s3]
//   k=1, l=2:   [r3 = s3]           C_12(s1,r2,r3) D[s1][r1] D[r2][s2]
//   k=2, l=1:   [r3 = s3]           C_12(r1,s2,r3) D[s2][r2] D[r1][s1]
//   (and the other off-diagonal pairs cyclically), mass:  [r = s]  M(r)
// with C = w S G G^T = (w/S) adj(J) adj(J)^T and M = w S at the GLL points:
// O(n^5) arithmetic per cell instead of the O(n^7) of the sum-factorised
// kernel above.  One CTA per (cell, r1).  It tabulates, for its r1, the three
// k = l sums (n^3 values each) and the six off-diagonal coefficients with one
// derivative factor folded in (n^3 each); each entry is then a sum of at most
// nine table terms.  The entries of its n^2 rows are enumerated class by class
// -- by which of r1 = s1, r2 = s2, r3 = s3 hold -- so that every warp applies
// one formula (the FP64 pipe issues per warp, so divergent branches would pay
// for all lanes); the all-unequal class, 70% of a dense Q_8 matrix, is zeros.
struct CollTabs {
  const double *T0, *T1, *T2;          // k = l sums: [s1][r2][r3], [r2][s2][r3], [r2][r3][s3]
  const double *a3, *b3, *a2, *b2, *a1, *b1;
  const double *D, *M;
};

// One entry of class (E1, E2, E3) = (r1 = s1, r2 = s2, r3 = s3).
template <int N, bool E1, bool E2, bool E3>
__device__ __forceinline__ double coll_entry(const CollTabs& t, int r1, int r2, int r3, int s1, int s2, int s3) {
  constexpr int N2 = N * N;
  auto d = [&](int q, int i) { return t.D[q * N + i]; };
  double acc = 0.0;
  if (E2 && E3) acc += t.T0[s1 * N2 + r2 * N + r3];
  if (E1 && E3) acc += t.T1[r2 * N2 + s2 * N + r3];
  if (E1 && E2) acc += t.T2[r2 * N2 + r3 * N + s3];
  if (E3) {  // (k, l) = (1, 2), (2, 1)
    acc = fma(t.a3[s1 * N2 + r2 * N + r3], d(r2, s2), acc);
    acc = fma(t.b3[r2 * N2 + s2 * N + r3], d(r1, s1), acc);
  }
  if (E2) {  // (1, 3), (3, 1)
    acc = fma(t.a2[s1 * N2 + r2 * N + r3], d(r3, s3), acc);
    acc = fma(t.b2[r2 * N2 + r3 * N + s3], d(r1, s1), acc);
  }
  if (E1) {  // (2, 3), (3, 2)
    acc = fma(t.a1[r2 * N2 + s2 * N + r3], d(r3, s3), acc);
    acc = fma(t.b1[r2 * N2 + r3 * N + s3], d(r2, s2), acc);
  }
  if (E1 && E2 && E3) acc += t.M[r2 * N + r3];
  return acc;
}

// All entries of class (E1, E2, E3) in the CTA's rows (r1, r2, r3): the
// unequal coordinates run over the N-1 values that skip the row's own.
template <int N, bool E1, bool E2, bool E3>
__device__ __forceinline__ void coll_class(const CollTabs& t, int r1, double* Ac, int tid, int nt) {
  constexpr int N2 = N * N, N3 = N2 * N, M1 = N - 1;
  constexpr int F1 = E1 ? 1 : M1, F2 = E2 ? 1 : M1, F3 = E3 ? 1 : M1;
  constexpr int SZ = F1 * F2 * F3;
  for (int k = tid; k < N2 * SZ; k += nt) {
    const int row = k / SZ, j = k - (k / SZ) * SZ;
    const int r2 = row / N, r3 = row - (row / N) * N;
    const int j1 = j / (F2 * F3), j2 = (j / F3) % F2, j3 = j % F3;
    const int s1 = E1 ? r1 : j1 + (j1 >= r1);
    const int s2 = E2 ? r2 : j2 + (j2 >= r2);
    const int s3 = E3 ? r3 : j3 + (j3 >= r3);
    const double v = (E1 || E2 || E3) ? coll_entry<N, E1, E2, E3>(t, r1, r2, r3, s1, s2, s3) : 0.0;
    Ac[(int64_t)row * N3 + (s1 * N + s2) * N + s3] = v;
  }
}

template <int N>
__global__ void __launch_bounds__(kMatThreads) k_cell_matrices_coll(const MatArgs a) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const Tab1D& T = c_tab[N - 1];
  extern __shared__ double sm[];
  double* D = sm;              // [a][b] = l_b'(x_a)
  double* xq = D + N2;         // 16
  double* wq = xq + 16;        // 16
  double* X = wq + 16;         // 24
  double* Jc = X + 24;         // [3][N2][3]
  double* C = Jc + 9 * N2;     // [6][N3]: C_00, C_11, C_22, C_01, C_02, C_12
  double* M = C + 6 * N3;      // [N2]: mass w S at (r1, r2, r3)
  double* Tt = M + N2;         // 9 tables of N3: T0, T1, T2, a3, b3, a2, b2, a1, b1
  int* bad = reinterpret_cast<int*>(Tt + 9 * N3);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t cell = a.cell_begin + blockIdx.x / N;
  const int r1 = blockIdx.x % N;
  for (int i = tid; i < N2; i += nt) D[i] = T.Dg[i / N][i % N];
  if (tid < N) {
    xq[tid] = T.xg[tid];
    wq[tid] = T.wg[tid];
  }
  if (tid < 24) X[tid] = a.xyz[(int64_t)a.vmap[cell * 8 + tid / 3] * 3 + tid % 3];
  if (tid == 0) *bad = 0;
  __syncthreads();
  for (int i = tid; i < N2; i += nt)
    jacobian_columns<N>(reinterpret_cast<const double(*)[3]>(X), xq, reinterpret_cast<double(*)[N2][3]>(Jc), i);
  __syncthreads();
  for (int qp = tid; qp < N3; qp += nt) {
    const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
    double r0[3], rr1[3], rr2[3];
    const double S = point_rows<N, true>(reinterpret_cast<const double(*)[N2][3]>(Jc), qp, r0, rr1, rr2);
    if (!(S > 0.0)) *bad = 1;
    const double w = wq[q1] * wq[q2] * wq[q3];
    const double ws = a.alpha * w * recip_nr<2>(S);
    C[0 * N3 + qp] = ws * dot3(r0, r0);
    C[1 * N3 + qp] = ws * dot3(rr1, rr1);
    C[2 * N3 + qp] = ws * dot3(rr2, rr2);
    C[3 * N3 + qp] = ws * dot3(r0, rr1);
    C[4 * N3 + qp] = ws * dot3(r0, rr2);
    C[5 * N3 + qp] = ws * dot3(rr1, rr2);
    if (q1 == r1) M[q2 * N + q3] = a.beta * w * S;
  }
  __syncthreads();
  auto at = [&](int k, int q1, int q2, int q3) { return C[k * N3 + (q1 * N + q2) * N + q3]; };
  auto d = [&](int q, int i) { return D[q * N + i]; };
  // the k = l sums and the folded off-diagonal coefficients of this r1
  for (int i = tid; i < N3; i += nt) {
    const int i0 = i / N2, i1 = (i / N) % N, i2 = i % N;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
#pragma unroll
    for (int q = 0; q < N; ++q) {
      t0 = fma(at(0, q, i1, i2), d(q, r1) * d(q, i0), t0);  // (s1, r2, r3) = (i0, i1, i2)
      t1 = fma(at(1, r1, q, i2), d(q, i0) * d(q, i1), t1);  // (r2, s2, r3)
      t2 = fma(at(2, r1, i0, q), d(q, i1) * d(q, i2), t2);  // (r2, r3, s3)
    }
    Tt[0 * N3 + i] = t0;
    Tt[1 * N3 + i] = t1;
    Tt[2 * N3 + i] = t2;
    Tt[3 * N3 + i] = at(3, i0, i1, i2) * d(i0, r1);  // a3[s1][r2][r3] = C_01(s1,r2,r3) D[s1][r1]
    Tt[4 * N3 + i] = at(3, r1, i1, i2) * d(i1, i0);  // b3[r2][s2][r3] = C_01(r1,s2,r3) D[s2][r2]
    Tt[5 * N3 + i] = at(4, i0, i1, i2) * d(i0, r1);  // a2[s1][r2][r3] = C_02(s1,r2,r3) D[s1][r1]
    Tt[6 * N3 + i] = at(4, r1, i0, i2) * d(i2, i1);  // b2[r2][r3][s3] = C_02(r1,r2,s3) D[s3][r3]
    Tt[7 * N3 + i] = at(5, r1, i1, i2) * d(i1, i0);  // a1[r2][s2][r3] = C_12(r1,s2,r3) D[s2][r2]
    Tt[8 * N3 + i] = at(5, r1, i0, i2) * d(i2, i1);  // b1[r2][r3][s3] = C_12(r1,r2,s3) D[s3][r3]
  }
  __syncthreads();
  double* Ac = a.A + ((int64_t)(blockIdx.x / N) * N3 + (int64_t)r1 * N2) * N3;  // rows (r1, *, *)
  if (*bad) {
    if (tid == 0 && r1 == 0) set_flag(a.status, SFX_DEV_INVERTED);
    for (int i = tid; i < N2 * N3; i += nt) Ac[i] = 0.0;
    return;
  }
  const CollTabs t{Tt, Tt + N3, Tt + 2 * N3, Tt + 3 * N3, Tt + 4 * N3, Tt + 5 * N3,
                   Tt + 6 * N3, Tt + 7 * N3, Tt + 8 * N3, D, M};
  coll_class<N, false, false, false>(t, r1, Ac, tid, nt);
  coll_class<N, false, false, true>(t, r1, Ac, tid, nt);
  coll_class<N, false, true, false>(t, r1, Ac, tid, nt);
  coll_class<N, true, false, false>(t, r1, Ac, tid, nt);
  coll_class<N, false, true, true>(t, r1, Ac, tid, nt);
  coll_class<N, true, false, true>(t, r1, Ac, tid, nt);
  coll_class<N, true, true, false>(t, r1, Ac, tid, nt);
  coll_class<N, true, true, true>(t, r1, Ac, tid, nt);
}

// ---------------------------------------------------------------- host side
void add_term(MatDesc& d, int bt, int bs, int cid, double sign, const int* tt, const int* ts) {
  MatTerm& m = d.term[d.nterm++];
  m.bt = bt; m.bs = bs; m.cid = cid; m.sign = sign; m.zg = -1;
  for (int k = 0; k < 3; ++k) { m.tt[k] = tt[k]; m.ts[k] = ts[k]; }
}

// Sort terms by block pair and assign z-groups (terms of one pair sharing the
// last-axis tables).  zg_t/zg_s are stored at index pair_begin + zg.
void finish_desc(MatDesc& d) {
  std::vector<MatTerm> all(d.term, d.term + d.nterm);
  int n = 0;
  for (int pr = 0; pr < 9; ++pr) {
    d.pair_begin[pr] = n;
    int nzg = 0;
    for (const MatTerm& m0 : all) {
      if (m0.bt * 3 + m0.bs != pr) continue;
      MatTerm m = m0;
      int zg = -1;
      for (int g = 0; g < nzg; ++g)
        if (d.zg_t[d.pair_begin[pr] + g] == m.tt[2] && d.zg_s[d.pair_begin[pr] + g] == m.ts[2]) zg = g;
      if (zg < 0) {
        zg = nzg++;
        d.zg_t[d.pair_begin[pr] + zg] = m.tt[2];
        d.zg_s[d.pair_begin[pr] + zg] = m.ts[2];
      }
      m.zg = zg;
      d.term[n++] = m;
    }
    d.pair_end[pr] = n;
    d.pair_nzg[pr] = nzg;
  }
}

bool build_desc(const sfx_space* sp, sfx_form form, MatDesc& d) {
  std::memset(&d, 0, sizeof(d));
  const int p = sp->p, n = p + 1;
  const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  (void)pa; (void)pb;
  if (sp->family == SFX_Q || sp->family == SFX_DQ) {
    if (form != SFX_MASS && form != SFX_LAPLACE && form != SFX_HELMHOLTZ) return false;
    const bool dq = sp->family == SFX_DQ;
    const int B = dq ? TB_ID : TB_BC, Dt = dq ? TB_DQ : TB_DC;
    d.kind = CF_SCALAR;
    d.nblk = 1;
    for (int k = 0; k < 3; ++k) d.dims[0][k] = n;
    d.nloc = n * n * n;
    if (form != SFX_MASS)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          int tt[3], ts[3];
          for (int ax = 0; ax < 3; ++ax) { tt[ax] = ax == k ? Dt : B; ts[ax] = ax == l ? Dt : B; }
          add_term(d, 0, 0, symi(k, l), 1.0, tt, ts);
        }
    if (form != SFX_LAPLACE) {
      int tt[3] = {B, B, B};
      add_term(d, 0, 0, 6, 1.0, tt, tt);
    }
  } else if (sp->family == SFX_NCF && form == SFX_NCF_MASS_DIVDIV) {
    d.kind = CF_NCF;
    d.nblk = 3;
    int off = 0;
    for (int b = 0; b < 3; ++b) {
      for (int ax = 0; ax < 3; ++ax) d.dims[b][ax] = ax == b ? n : p;
      d.off[b] = off;
      off += d.dims[b][0] * d.dims[b][1] * d.dims[b][2];
    }
    d.nloc = off;
    for (int bt = 0; bt < 3; ++bt)
      for (int bs = 0; bs < 3; ++bs) {
        int vt[3], vs[3], dt[3], ds[3];
        for (int ax = 0; ax < 3; ++ax) {
          vt[ax] = ax == bt ? TB_BC : TB_BD;
          vs[ax] = ax == bs ? TB_BC : TB_BD;
          dt[ax] = ax == bt ? TB_DC : TB_BD;
          ds[ax] = ax == bs ? TB_DC : TB_BD;
        }
        add_term(d, bt, bs, symi(bt, bs), 1.0, vt, vs);  // alpha w/S (J^T J)_{bt,bs}
        add_term(d, bt, bs, 6, 1.0, dt, ds);             // beta w/S div div
      }
  } else if (sp->family == SFX_NCE && form == SFX_NCE_CURLCURL) {
    d.kind = CF_NCE;
    d.nblk = 3;
    int off = 0;
    for (int b = 0; b < 3; ++b) {
      for (int ax = 0; ax < 3; ++ax) d.dims[b][ax] = ax == b ? p : n;
      d.off[b] = off;
      off += d.dims[b][0] * d.dims[b][1] * d.dims[b][2];
    }
    d.nloc = off;
    // curl of f e_b: (component, derivative axis, sign)
    const int ck[3][2] = {{1, 2}, {0, 2}, {0, 1}}, ce[3][2] = {{2, 1}, {2, 0}, {1, 0}};
    const double cs[3][2] = {{1.0, -1.0}, {-1.0, 1.0}, {1.0, -1.0}};
    for (int bt = 0; bt < 3; ++bt)
      for (int bs = 0; bs < 3; ++bs) {
        for (int u = 0; u < 2; ++u)
          for (int v = 0; v < 2; ++v) {
            int tt[3], ts[3];
            for (int ax = 0; ax < 3; ++ax) {
              tt[ax] = ax == bt ? TB_BD : (ax == ce[bt][u] ? TB_DC : TB_BC);
              ts[ax] = ax == bs ? TB_BD : (ax == ce[bs][v] ? TB_DC : TB_BC);
            }
            add_term(d, bt, bs, symi(ck[bt][u], ck[bs][v]), cs[bt][u] * cs[bs][v], tt, ts);
          }
        int vt[3], vs[3];
        for (int ax = 0; ax < 3; ++ax) {
          vt[ax] = ax == bt ? TB_BD : TB_BC;
          vs[ax] = ax == bs ? TB_BD : TB_BC;
        }
        add_term(d, bt, bs, 6 + symi(bt, bs), 1.0, vt, vs);  // alpha w S G G^T
      }
  } else {
    return false;
  }
  finish_desc(d);
  return true;
}

}  // namespace

int launch_cell_matrices(const sfx_space* sp, sfx_form form, sfx_algo algo, const MatArgs& a0, void* stream) {
  MatDesc d;
  if (!build_desc(sp, form, d)) return -1;
  for (int pr = 0; pr < 9; ++pr)
    if (d.pair_nzg[pr] > 4 || d.pair_end[pr] - d.pair_begin[pr] > kMaxTerm) return -1;
  MatArgs a = a0;
  if (sp->family == SFX_Q || sp->family == SFX_DQ) {
    // scalar coefficients: alpha scales the Laplace part, beta the mass part
    if (form == SFX_MASS) { a.alpha = 0.0; a.beta = 1.0; }
    if (form == SFX_LAPLACE) { a.alpha = 1.0; a.beta = 0.0; }
  }
  const int Q = sp->p + 1;
  const size_t smem = sizeof(double) * (NTAB * kMaxQ * kMaxN + kMaxCoef * Q * Q * Q + kMaxTerm * Q * Q +
                                        4 * Q * kMaxN * kMaxN + 24 + 9 * Q * Q + (a.kappa ? d.nloc : 0)) + 16;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (algo == SFX_ALGO_NAIVE) {
    e = cudaFuncSetAttribute(k_cell_matrices<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k_cell_matrices<true><<<(unsigned)a.ncells, kMatThreads, smem, s>>>(a, d, sp->p);
  } else {
    e = cudaFuncSetAttribute(k_cell_matrices<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    k_cell_matrices<false><<<(unsigned)a.ncells, kMatThreads, smem, s>>>(a, d, sp->p);
  }
  return (int)cudaGetLastError();
}

template <int N>
int launch_coll(const MatArgs& a, cudaStream_t s) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const size_t smem = sizeof(double) * (N2 + 32 + 24 + 9 * N2 + 6 * N3 + N2 + 9 * N3) + 16;
  cudaError_t e = cudaFuncSetAttribute(k_cell_matrices_coll<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  // one CTA per (cell, first test index r1); small degrees use fewer threads
  const int threads = N2 * N3 >= kMatThreads ? kMatThreads : ((N2 * N3 + 31) / 32) * 32;
  k_cell_matrices_coll<N><<<(unsigned)(a.ncells * N), threads, smem, s>>>(a);
  return (int)cudaGetLastError();
}

int launch_cell_matrices_coll(const sfx_space* sp, sfx_form form, const MatArgs& a0, void* stream) {
  if (sp->family != SFX_Q) return -1;
  if (form != SFX_MASS && form != SFX_LAPLACE && form != SFX_HELMHOLTZ) return -1;
  MatArgs a = a0;
  if (form == SFX_MASS) { a.alpha = 0.0; a.beta = 1.0; }
  if (form == SFX_LAPLACE) { a.alpha = 1.0; a.beta = 0.0; }
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 1: return launch_coll<2>(a, s);
    case 2: return launch_coll<3>(a, s);
    case 3: return launch_coll<4>(a, s);
    case 4: return launch_coll<5>(a, s);
    case 5: return launch_coll<6>(a, s);
    case 6: return launch_coll<7>(a, s);
    case 7: return launch_coll<8>(a, s);
    case 8: return launch_coll<9>(a, s);
  }
  return -1;
}

// Vector Q_p element matrices of the vector mass / Laplace / Helmholtz forms
// (Sec. 3.3): the component delta makes them block diagonal with the scalar
// matrix in every diagonal block.  One thread per output entry (coalesced
// writes); HBM-bound.
__global__ void k_vq_expand(const double* __restrict__ S, int64_t ncells, int n3, double* __restrict__ A) {
  const int64_t nl = 3 * (int64_t)n3, per = nl * nl, total = ncells * per;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / per, rc = e - c * per;
    const int64_t row = rc / nl, col = rc - row * nl;
    const int64_t a = row / n3, b = col / n3;
    A[e] = a == b ? S[(c * n3 + (row - a * n3)) * n3 + (col - b * n3)] : 0.0;
  }
}

int launch_vq_expand(const double* S, int64_t ncells, int n3, double* A, void* stream) {
  const int64_t total = ncells * 9 * (int64_t)n3 * n3;
  if (total == 0) return 0;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 152 * 32);
  k_vq_expand<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(S, ncells, n3, A);
  return (int)cudaGetLastError();
}

}  // namespace sfx
