/*
 * oracle.c -- plain FP64 CPU reference assembler (naive quadrature).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark
 * (CPU baseline, reference arm, sampled-error columns); never by the library.  Shares no code with the CUDA path.
 *
 * Every routine below follows the paper's definitions directly; nothing is
 * sum-factorised, blocked or fused:
 *   - 1D rules: Gauss-Legendre and Gauss-Lobatto-Legendre (Sec. 2.5, Eq. colocated),
 *     computed by Golub-Welsch (eigenvalues of the Jacobi matrix by Sturm
 *     bisection; Christoffel numbers for the Gauss weights).
 *   - Tensor-product bases psi_i(xi) = prod_d phi_{i_d}(xi_d) (Sec. 1.2, Eq. limits_tpe;
 *     Sec. 2.4, Eq. product_basis) and their concatenation into H(div)/H(curl)
 *     blocks (Sec. 2.6-2.7, Eq. rtcf_impl; Sec. 3.5, Eqs. rtcf_split_x/y).
 *   - Geometry: trilinear coordinate field, J = grad F_K, S = |J|, G = J^{-1}
 *     (Sec. 1.1; Sec. 3.1 for the coordinate element).
 *   - Integrals by quadrature, Eq. laplace_quadrature / laplace_prefiat, and the
 *     action as a linear form with coefficient u (Sec. 1.1; Sec. 3.3, Eqs.
 *     coeff_def, coeff_eval, form_eval).
 *   - Hyperelasticity (Sec. 4.1): F = I + grad u; SVK S = lambda tr(E) I + 2 mu E,
 *     P = F S; neo-Hookean P = mu (F - F^{-T}) + lambda ln(J) F^{-T}.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_plant = 0;
void orc_set_plant(int which) { g_plant = which; }

/* ------------------------------------------------------------------------ */
/* 1D quadrature: Golub-Welsch.                                              */
/* ------------------------------------------------------------------------ */

/* Number of eigenvalues of the symmetric tridiagonal matrix (zero diagonal,
 * off-diagonal e[0..m-2]) that are smaller than t (Sturm sequence count). */
static int sturm_count(int m, const double* e, double t) {
  int cnt = 0;
  double d = -t;
  if (d < 0) cnt++;
  for (int k = 1; k < m; ++k) {
    double prev = (d == 0.0) ? 1e-300 : d;
    d = -t - e[k - 1] * e[k - 1] / prev;
    if (d < 0) cnt++;
  }
  return cnt;
}

/* All eigenvalues (ascending) of that matrix; they lie in (-1, 1). */
static void tridiag_eigs(int m, const double* e, double* eig) {
  for (int k = 0; k < m; ++k) {
    double lo = -1.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(m, e, mid) > k) hi = mid; else lo = mid;
    }
    eig[k] = 0.5 * (lo + hi);
  }
}

/* Legendre P_k(x) for k = 0..m-1 by the three-term recurrence. */
static void legendre_all(int m, double x, double* P) {
  if (m > 0) P[0] = 1.0;
  if (m > 1) P[1] = x;
  for (int k = 1; k + 1 < m; ++k) P[k + 1] = ((2.0 * k + 1.0) * x * P[k] - k * P[k - 1]) / (k + 1.0);
}

int orc_gauss_legendre(int n, double* x, double* w) {
  if (n < 1 || n > 64) return -1;
  double e[64] = {0}, t[64], P[65];
  /* Jacobi matrix of the monic Legendre recurrence: beta_k = k^2/(4k^2-1). */
  for (int k = 1; k < n; ++k) e[k - 1] = k / sqrt(4.0 * k * k + (g_plant == 13 ? 1.0 : -1.0)); /* 13: planted */
  tridiag_eigs(n, e, t);
  for (int i = 0; i < n; ++i) {
    /* Christoffel number 1 / sum_k p~_k(t)^2, p~_k = sqrt((2k+1)/2) P_k. */
    legendre_all(n, t[i], P);
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += 0.5 * (2.0 * k + 1.0) * P[k] * P[k];
    x[i] = 0.5 * (t[i] + 1.0);
    w[i] = 0.5 * (1.0 / s);
  }
  return 0;
}

int orc_gauss_lobatto(int n, double* x, double* w) {
  if (n < 2 || n > 64) return -1;
  double e[64] = {0}, t[64], P[65];
  /* interior nodes: zeros of P'_{n-1}, i.e. of the Jacobi(1,1) polynomial of
   * degree n-2; monic recurrence beta_k = k(k+2)/((2k+1)(2k+3)). */
  int m = n - 2;
  for (int k = 1; k < m; ++k) e[k - 1] = sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
  tridiag_eigs(m, e, t + 1);
  t[0] = -1.0;
  t[n - 1] = 1.0;
  for (int i = 0; i < n; ++i) {
    legendre_all(n, t[i], P);
    double pn1 = P[n - 1];
    /* w_i = 2 / (n (n-1) P_{n-1}(t_i)^2) on [-1, 1] */
    double wi = 2.0 / (n * (n - 1.0) * pn1 * pn1);
    x[i] = 0.5 * (t[i] + 1.0);
    w[i] = 0.5 * wi;
  }
  return 0;
}

double orc_lagrange(const double* xn, int n, int i, double x) {
  double v = 1.0;
  for (int k = 0; k < n; ++k)
    if (k != i) v *= (x - xn[k]) / (xn[i] - xn[k]);
  return v;
}

double orc_lagrange_deriv(const double* xn, int n, int i, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double t = 1.0 / (xn[i] - xn[m]);
    int kend = (g_plant == 15 && n > 6) ? 6 : n; /* 15: planted: a fixed loop bound, wrong for n >= 7 only */
    for (int k = 0; k < kend; ++k)
      if (k != i && k != m) t *= (x - xn[k]) / (xn[i] - xn[k]);
    if (g_plant == 6 && m == n - 1) continue; /* planted: drops one term */
    s += t;
  }
  return s;
}

/* ------------------------------------------------------------------------ */
/* Element descriptions                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int comp;        /* vector component carried by the block; -1 = scalar   */
  int kind[3];     /* ORC_GLL (continuous factor) or ORC_GL (discontinuous) */
  int cnt[3];      /* 1D nodes per axis                                     */
  int loff;        /* local offset                                           */
  int64_t goff;    /* global offset                                          */
  int64_t gext[3]; /* global grid extent per axis                            */
} blk_t;

typedef struct {
  int family, p, nblk, nloc, cellmajor, vector;
  int64_t ndof;
  blk_t b[3];
} elem_t;

static int make_elem(int family, int p, int nx, int ny, int nz, elem_t* E) {
  memset(E, 0, sizeof(*E));
  if (p < 1 || p > 16 || nx < 1 || ny < 1 || nz < 1) return -1;
  E->family = family;
  E->p = p;
  int64_t N[3] = {nx, ny, nz};
  int n = p + 1;
  if (family == ORC_Q || family == ORC_DQ || family == ORC_VQ) {
    int nb = (family == ORC_VQ) ? 3 : 1;
    int kind = (family == ORC_DQ) ? ORC_GL : ORC_GLL;
    /* dofs per block: continuous grid (p N_d + 1 per axis), or cell-major
     * for the discontinuous DQ space (n^3 per cell) */
    int64_t per = 1;
    if (family == ORC_DQ) per = (int64_t)nx * ny * nz * n * n * n;
    else
      for (int d = 0; d < 3; ++d) per *= (int64_t)p * N[d] + 1;
    E->nblk = nb;
    for (int c = 0; c < nb; ++c) {
      blk_t* B = &E->b[c];
      B->comp = (family == ORC_VQ) ? c : -1;
      for (int d = 0; d < 3; ++d) {
        B->kind[d] = kind;
        B->cnt[d] = n;
        B->gext[d] = (int64_t)p * N[d] + 1;
      }
      B->loff = c * n * n * n;
      B->goff = c * per;
    }
    E->nloc = nb * n * n * n;
    E->ndof = nb * per;
    E->cellmajor = (family == ORC_DQ);
    E->vector = (family == ORC_VQ);
    return 0;
  }
  if (family == ORC_NCF || family == ORC_NCE) {
    E->nblk = 3;
    E->vector = 1;
    int loff = 0;
    int64_t goff = 0;
    for (int c = 0; c < 3; ++c) {
      blk_t* B = &E->b[c];
      B->comp = c;
      int64_t tot = 1;
      int cnt = 1;
      for (int d = 0; d < 3; ++d) {
        /* NCF: continuous P_p along its own axis, dP_{p-1} across;
         * NCE: dP_{p-1} along its own axis, continuous P_p across. */
        int cont = (family == ORC_NCF) ? (d == c) : (d != c);
        B->kind[d] = cont ? ORC_GLL : ORC_GL;
        B->cnt[d] = cont ? p + 1 : p;
        B->gext[d] = cont ? (int64_t)p * N[d] + 1 : (int64_t)p * N[d];
        tot *= B->gext[d];
        cnt *= B->cnt[d];
      }
      B->loff = loff;
      B->goff = goff;
      loff += cnt;
      goff += tot;
    }
    E->nloc = loff;
    E->ndof = goff;
    return 0;
  }
  return -1;
}

int orc_space_size(int family, int p, int nx, int ny, int nz, int64_t* ndof, int* nloc) {
  elem_t E;
  if (make_elem(family, p, nx, ny, nz, &E)) return -1;
  if (ndof) *ndof = E.ndof;
  if (nloc) *nloc = E.nloc;
  return 0;
}

static void cell_ijk(int ny, int nz, int64_t cell, int64_t* ci) {
  ci[2] = cell % nz;
  ci[1] = (cell / nz) % ny;
  ci[0] = cell / ((int64_t)ny * nz);
}

static void elem_cell_dofs(const elem_t* E, int ny, int nz, int64_t cell, int64_t* dofs) {
  int64_t ci[3];
  cell_ijk(ny, nz, cell, ci);
  if (E->cellmajor) {
    for (int l = 0; l < E->nloc; ++l) dofs[l] = cell * E->nloc + l;
    return;
  }
  for (int bi = 0; bi < E->nblk; ++bi) {
    const blk_t* B = &E->b[bi];
    int l = B->loff;
    for (int i1 = 0; i1 < B->cnt[0]; ++i1)
      for (int i2 = 0; i2 < B->cnt[1]; ++i2)
        for (int i3 = 0; i3 < B->cnt[2]; ++i3) {
          int ii[3] = {i1, i2, i3};
          int64_t g[3];
          for (int d = 0; d < 3; ++d) {
            /* continuous factor: p nodes advance per cell (shared endpoint);
             * discontinuous factor: cnt nodes per cell. */
            int64_t step = (B->kind[d] == ORC_GLL && g_plant != 14) ? (B->cnt[d] - 1) : B->cnt[d]; /* 14: planted */
            g[d] = step * ci[d] + ii[d];
          }
          dofs[l++] = B->goff + (g[0] * B->gext[1] + g[1]) * B->gext[2] + g[2];
        }
  }
}

int orc_cell_dofs(int family, int p, int nx, int ny, int nz, int64_t cell, int64_t* dofs) {
  elem_t E;
  if (make_elem(family, p, nx, ny, nz, &E)) return -1;
  if (cell < 0 || cell >= (int64_t)nx * ny * nz) return -1;
  elem_cell_dofs(&E, ny, nz, cell, dofs);
  return 0;
}

int orc_cell_map(int family, int p, int nx, int ny, int nz, int32_t* map) {
  elem_t E;
  if (make_elem(family, p, nx, ny, nz, &E)) return -1;
  if (E.ndof > 2147483647LL) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * E.nloc);
  for (int64_t c = 0; c < ncell; ++c) {
    elem_cell_dofs(&E, ny, nz, c, tmp);
    for (int l = 0; l < E.nloc; ++l) map[c * E.nloc + l] = (int32_t)tmp[l];
  }
  free(tmp);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dense tabulation of the reference basis at the 3D quadrature points       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nq, nq3, nloc;
  double* xq;     /* 1D points  */
  double* wq;     /* 1D weights */
  double* val;    /* [q][l]     value of the scalar factor product            */
  double* grad;   /* [q][l][3]  reference gradient of that product            */
  int* comp;      /* [l]        carried component (-1 scalar)                 */
} tab_t;

static void tab_free(tab_t* T) {
  free(T->xq); free(T->wq); free(T->val); free(T->grad); free(T->comp);
}

/* qrule: ORC_GL (Gauss-Legendre, the default of every form) or ORC_GLL
 * (Gauss-Lobatto-Legendre; with nq = p + 1 on a Q_p element the points are
 * the element's own nodes: the collocated rule of Sec. 2.5 that the
 * "underintegration" experiment of Sec. 4.1 uses). */
static int tabulate(const elem_t* E, int nq, int qrule, tab_t* T) {
  memset(T, 0, sizeof(*T));
  if (nq < 1 || nq > 32 || (qrule != ORC_GL && qrule != ORC_GLL) || (qrule == ORC_GLL && nq < 2)) return -1;
  T->nq = nq;
  T->nq3 = nq * nq * nq;
  T->nloc = E->nloc;
  T->xq = (double*)malloc(sizeof(double) * nq);
  T->wq = (double*)malloc(sizeof(double) * nq);
  if (qrule == ORC_GLL) orc_gauss_lobatto(nq, T->xq, T->wq);
  else orc_gauss_legendre(nq, T->xq, T->wq);
  T->val = (double*)malloc(sizeof(double) * T->nq3 * E->nloc);
  T->grad = (double*)malloc(sizeof(double) * T->nq3 * E->nloc * 3);
  T->comp = (int*)malloc(sizeof(int) * E->nloc);
  for (int bi = 0; bi < E->nblk; ++bi) {
    const blk_t* B = &E->b[bi];
    double nodes[3][33], wdum[33];
    for (int d = 0; d < 3; ++d) {
      if (B->kind[d] == ORC_GLL) orc_gauss_lobatto(B->cnt[d], nodes[d], wdum);
      else orc_gauss_legendre(B->cnt[d], nodes[d], wdum);
    }
    int l = B->loff;
    for (int i1 = 0; i1 < B->cnt[0]; ++i1)
      for (int i2 = 0; i2 < B->cnt[1]; ++i2)
        for (int i3 = 0; i3 < B->cnt[2]; ++i3, ++l) {
          T->comp[l] = B->comp;
          int ii[3] = {i1, i2, i3};
          for (int q1 = 0; q1 < nq; ++q1)
            for (int q2 = 0; q2 < nq; ++q2)
              for (int q3 = 0; q3 < nq; ++q3) {
                int qq[3] = {q1, q2, q3};
                int q = (q1 * nq + q2) * nq + q3;
                double f[3], df[3];
                for (int d = 0; d < 3; ++d) {
                  double xi = T->xq[qq[d]];
                  f[d] = orc_lagrange(nodes[d], B->cnt[d], ii[d], xi);
                  df[d] = orc_lagrange_deriv(nodes[d], B->cnt[d], ii[d], xi);
                }
                T->val[(size_t)q * E->nloc + l] = f[0] * f[1] * f[2];
                double* g = &T->grad[((size_t)q * E->nloc + l) * 3];
                g[0] = df[0] * f[1] * f[2];
                g[1] = f[0] * df[1] * f[2];
                g[2] = f[0] * f[1] * df[2];
              }
        }
  }
  return 0;
}

static double qweight(const tab_t* T, int q) {
  int q1 = q / (T->nq * T->nq), q2 = (q / T->nq) % T->nq, q3 = q % T->nq;
  if (g_plant == 4) return T->wq[q1] * T->wq[q1] * T->wq[q3]; /* planted */
  return T->wq[q1] * T->wq[q2] * T->wq[q3];
}

static void qpoint(const tab_t* T, int q, double* xi) {
  xi[0] = T->xq[q / (T->nq * T->nq)];
  xi[1] = T->xq[(q / T->nq) % T->nq];
  xi[2] = T->xq[q % T->nq];
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                   */
/* ------------------------------------------------------------------------ */

static void cell_vertices(int nx, int ny, int nz, const double* coords, int64_t cell, double X[8][3]) {
  (void)nx;
  int64_t ci[3];
  cell_ijk(ny, nz, cell, ci);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        int64_t v = ((ci[0] + a) * (ny + 1) + (ci[1] + b)) * (int64_t)(nz + 1) + (ci[2] + c);
        for (int k = 0; k < 3; ++k) X[4 * a + 2 * b + c][k] = coords[v * 3 + k];
      }
}

/* J_ij = d x_i / d xi_j of the trilinear map x(xi) = sum_v X_v N_v(xi). */
static void jacobian(const double X[8][3], const double* xi, double J[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) J[i][j] = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        double L0 = a ? xi[0] : 1.0 - xi[0], d0 = a ? 1.0 : -1.0;
        double L1 = b ? xi[1] : 1.0 - xi[1], d1 = b ? 1.0 : -1.0;
        double L2 = c ? xi[2] : 1.0 - xi[2], d2 = c ? 1.0 : -1.0;
        double dN[3] = {d0 * L1 * L2, L0 * d1 * L2, L0 * L1 * d2};
        const double* Xv = X[4 * a + 2 * b + c];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) J[i][j] += Xv[i] * dN[j];
      }
}

static void mapped_point(const double X[8][3], const double* xi, double* x) {
  x[0] = x[1] = x[2] = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) {
        double N = (a ? xi[0] : 1.0 - xi[0]) * (b ? xi[1] : 1.0 - xi[1]) * (c ? xi[2] : 1.0 - xi[2]);
        for (int i = 0; i < 3; ++i) x[i] += X[4 * a + 2 * b + c][i] * N;
      }
}

static double det3(double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* Inverse by Gauss-Jordan elimination with partial pivoting. */
static int inv3(double A[3][3], double R[3][3]) {
  double M[3][6];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      M[i][j] = A[i][j];
      M[i][3 + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (M[piv][c] == 0.0) return -1;
    if (piv != c)
      for (int j = 0; j < 6; ++j) { double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
    double d = M[c][c];
    for (int j = 0; j < 6; ++j) M[c][j] /= d;
    for (int r = 0; r < 3; ++r) {
      if (r == c) continue;
      double f = M[r][c];
      for (int j = 0; j < 6; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = M[i][3 + j];
  return 0;
}

typedef struct {
  double J[3][3], G[3][3], S;
} geo_t;

static int geometry(const double X[8][3], const double* xi, geo_t* g) {
  jacobian(X, xi, g->J);
  g->S = det3(g->J);
  if (!(g->S > 0.0)) return -1;
  return inv3(g->J, g->G);
}

/* physical gradient G^T v: (G^T v)_a = sum_k G_ka v_k */
static void push_grad(const geo_t* g, const double* v, double* out) {
  for (int a = 0; a < 3; ++a) {
    out[a] = 0.0;
    for (int k = 0; k < 3; ++k)
      out[a] += (g_plant == 1 ? g->G[a][k] : g->G[k][a]) * v[k];
  }
}

static void matvec(double A[3][3], const double* v, double* out) {
  for (int a = 0; a < 3; ++a) out[a] = A[a][0] * v[0] + A[a][1] * v[1] + A[a][2] * v[2];
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* reference curl of the block function f e_c, given grad f */
static void block_curl(int c, const double* gf, double* out) {
  if (c == 0) { out[0] = 0.0; out[1] = gf[2]; out[2] = -gf[1]; }
  else if (c == 1) { out[0] = -gf[2]; out[1] = 0.0; out[2] = gf[0]; }
  else { out[0] = gf[1]; out[1] = -gf[0]; out[2] = 0.0; }
  if (g_plant == 3) out[2] = -out[2]; /* planted */
}

static int form_ok(int family, int form) {
  switch (form) {
    case ORC_MASS: case ORC_LAPLACE: case ORC_HELMHOLTZ:
      return family == ORC_Q || family == ORC_DQ || family == ORC_VQ;
    case ORC_NCF_MASS_DIVDIV: return family == ORC_NCF;
    case ORC_NCE_CURLCURL: return family == ORC_NCE;
    case ORC_NEOHOOKE: case ORC_SVK: return family == ORC_VQ;
  }
  return 0;
}

/* stiffness / mass weights of the scalar forms */
static void scalar_weights(int form, const double* params, double* a_lap, double* b_mass) {
  if (form == ORC_MASS) { *a_lap = 0.0; *b_mass = 1.0; }
  else if (form == ORC_LAPLACE) { *a_lap = 1.0; *b_mass = 0.0; }
  else { *a_lap = params[0]; *b_mass = params[1]; }
}

/* First Piola-Kirchhoff stress for displacement gradient Hu = grad u.
 * Returns -1 if det F <= 0 (neo-Hookean only). */
static int piola(int form, const double* params, double Hu[3][3], double P[3][3], double* W) {
  double mu = params[2], lam = params[3];
  double F[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) F[a][b] = Hu[a][b] + (a == b ? 1.0 : 0.0);
  if (form == ORC_NEOHOOKE) {
    double JF = det3(F);
    if (!(JF > 0.0)) return -1;
    double Fi[3][3];
    if (inv3(F, Fi)) return -1;
    double lnJ = log(JF);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double FiT = (g_plant == 5) ? Fi[a][b] : Fi[b][a];
        P[a][b] = mu * (F[a][b] - FiT) + lam * lnJ * FiT;
      }
    if (W) {
      double trC = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) trC += F[a][b] * F[a][b];
      *W = 0.5 * mu * (trC - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ;
    }
    return 0;
  }
  /* Saint Venant-Kirchhoff */
  double E[3][3], S2[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double C = 0.0;
      for (int k = 0; k < 3; ++k) C += F[k][a] * F[k][b];
      E[a][b] = 0.5 * (C - (a == b ? 1.0 : 0.0));
    }
  double trE = E[0][0] + E[1][1] + E[2][2];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) S2[a][b] = lam * trE * (a == b ? 1.0 : 0.0) + 2.0 * mu * E[a][b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      P[a][b] = 0.0;
      for (int k = 0; k < 3; ++k) P[a][b] += F[a][k] * S2[k][b];
    }
  if (W) {
    double trE2 = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) trE2 += E[a][b] * E[b][a];
    *W = 0.5 * lam * trE * trE + mu * trE2;
  }
  return 0;
}

/* Directional derivative dP = (d/dt) P(I + Hu + t dH) at t = 0 of the two
 * stress laws (the linearisation of Sec. 4.1's residual, whose action the
 * paper benchmarks):
 *   neo-Hookean  dP = mu dF + (mu - lambda ln J) F^{-T} dF^T F^{-T}
 *                     + lambda tr(F^{-1} dF) F^{-T}
 *     (from d F^{-T} = -F^{-T} dF^T F^{-T} and d ln J = tr(F^{-1} dF));
 *   SVK          dE = (dF^T F + F^T dF)/2,  dS = lambda tr(dE) I + 2 mu dE,
 *                dP = dF S + F dS.
 * Returns -1 if det F <= 0 (neo-Hookean). */
static int dpiola(int form, const double* params, double Hu[3][3], double dF[3][3], double dP[3][3]) {
  double mu = params[2], lam = params[3];
  double F[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) F[a][b] = Hu[a][b] + (a == b ? 1.0 : 0.0);
  if (form == ORC_NEOHOOKE) {
    double JF = det3(F);
    if (!(JF > 0.0)) return -1;
    double Fi[3][3];
    if (inv3(F, Fi)) return -1;
    double lnJ = log(JF);
    double tr = 0.0; /* tr(F^{-1} dF) */
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) tr += Fi[a][b] * dF[b][a];
    double c = (g_plant == 8) ? mu : mu - lam * lnJ;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0.0; /* (F^{-T} dF^T F^{-T})_ij = sum_kl Fi[k][i] dF[l][k] Fi[j][l] */
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) t += Fi[k][i] * dF[l][k] * Fi[j][l];
        dP[i][j] = mu * dF[i][j] + c * t + lam * tr * Fi[j][i];
      }
    return 0;
  }
  double E[3][3], S2[3][3], dE[3][3], dS[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double C = 0.0, dC = 0.0;
      for (int k = 0; k < 3; ++k) {
        C += F[k][a] * F[k][b];
        dC += dF[k][a] * F[k][b] + F[k][a] * dF[k][b];
      }
      E[a][b] = 0.5 * (C - (a == b ? 1.0 : 0.0));
      dE[a][b] = 0.5 * dC;
    }
  double trE = E[0][0] + E[1][1] + E[2][2], trdE = dE[0][0] + dE[1][1] + dE[2][2];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      S2[a][b] = lam * trE * (a == b ? 1.0 : 0.0) + 2.0 * mu * E[a][b];
      dS[a][b] = lam * trdE * (a == b ? 1.0 : 0.0) + 2.0 * mu * dE[a][b];
    }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      dP[a][b] = 0.0;
      for (int k = 0; k < 3; ++k)
        dP[a][b] += (g_plant == 12 ? 0.0 : dF[a][k] * S2[k][b]) + F[a][k] * dS[k][b]; /* 12: planted */
    }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One cell: local vector b (nloc x nrhs) for coefficient xl (nloc x nrhs)    */
/* ------------------------------------------------------------------------ */

/* kap: the cell's dofs of the coefficient kappa of the weighted Laplace form
 * int kappa grad u . grad v (Sec. 1.1, Eq. weighted_laplace), interpolated in
 * the same space; NULL for every other form. */
static int cell_vector(const elem_t* E, const tab_t* T, int form, const double* params,
                       const double X[8][3], const double* xl, int nrhs, const double* kap, double* b) {
  int nloc = E->nloc;
  memset(b, 0, sizeof(double) * nloc * nrhs);
  for (int q = 0; q < T->nq3; ++q) {
    double xi[3];
    qpoint(T, q, xi);
    geo_t g;
    if (geometry(X, xi, &g)) return -2;
    double w = qweight(T, q);
    const double* val = &T->val[(size_t)q * nloc];
    const double* grd = &T->grad[(size_t)q * nloc * 3];
    for (int r = 0; r < nrhs; ++r) {
      if (E->family == ORC_Q || E->family == ORC_DQ) {
        double a_lap, b_mass;
        scalar_weights(form, params, &a_lap, &b_mass);
        if (kap) { /* kappa(xi_q) = sum_l kappa_l psi_l(xi_q) */
          a_lap = 0.0;
          for (int l = 0; l < nloc; ++l) a_lap += kap[l] * val[g_plant == 11 ? (l + 1) % nloc : l]; /* 11: planted */
          b_mass = 0.0;
        }
        /* coefficient evaluation, Eq. coeff_eval: u and reference gradient */
        double u = 0.0, gu[3] = {0, 0, 0};
        for (int l = 0; l < nloc; ++l) {
          double c = xl[l * nrhs + r];
          u += c * val[l];
          for (int k = 0; k < 3; ++k) gu[k] += c * grd[l * 3 + k];
        }
        double pg[3];
        push_grad(&g, gu, pg);
        double sw = (g_plant == 2) ? w : w * g.S;
        for (int l = 0; l < nloc; ++l) {
          double pv[3];
          push_grad(&g, &grd[l * 3], pv);
          b[l * nrhs + r] += sw * (a_lap * dot3(pg, pv) + b_mass * u * val[l]);
        }
      } else if (E->family == ORC_NCF) {
        double uh[3] = {0, 0, 0}, du = 0.0;
        for (int l = 0; l < nloc; ++l) {
          double c = xl[l * nrhs + r];
          int cc = T->comp[l];
          uh[cc] += c * val[l];
          du += c * grd[l * 3 + cc];
        }
        double Ju[3];
        matvec(g.J, uh, Ju);
        double inv = (g_plant == 7) ? 1.0 : 1.0 / g.S;
        for (int l = 0; l < nloc; ++l) {
          int cc = T->comp[l];
          double Jv[3] = {g.J[0][cc] * val[l], g.J[1][cc] * val[l], g.J[2][cc] * val[l]};
          b[l * nrhs + r] += w * (params[0] * inv * dot3(Ju, Jv) + params[1] / g.S * du * grd[l * 3 + cc]);
        }
      } else if (E->family == ORC_NCE) {
        double uh[3] = {0, 0, 0}, ch[3] = {0, 0, 0};
        for (int l = 0; l < nloc; ++l) {
          double c = xl[l * nrhs + r];
          int cc = T->comp[l];
          uh[cc] += c * val[l];
          double cl[3];
          block_curl(cc, &grd[l * 3], cl);
          for (int k = 0; k < 3; ++k) ch[k] += c * cl[k];
        }
        double Jc[3], pu[3];
        matvec(g.J, ch, Jc);
        push_grad(&g, uh, pu);
        for (int l = 0; l < nloc; ++l) {
          int cc = T->comp[l];
          double cl[3], Jcl[3], vh[3] = {0, 0, 0}, pv[3];
          block_curl(cc, &grd[l * 3], cl);
          matvec(g.J, cl, Jcl);
          vh[cc] = val[l];
          push_grad(&g, vh, pv);
          b[l * nrhs + r] += w * (params[1] / g.S * dot3(Jc, Jcl) + params[0] * g.S * dot3(pu, pv));
        }
      } else if (form == ORC_MASS || form == ORC_LAPLACE || form == ORC_HELMHOLTZ) {
        /* vector forms on vector Q_p (Sec. 3.3, Eq. vector_mass_form and its
         * Laplace analogue): a_lap int grad u : grad v + b_mass int u . v with
         * the basis psi_l e_comp(l); written with full vectors and 3x3
         * gradients, so the component delta follows from e_a . e_b */
        double a_lap, b_mass;
        scalar_weights(form, params, &a_lap, &b_mass);
        double u[3] = {0, 0, 0}, gu[3][3] = {{0}}; /* gu[a][.] = physical gradient of u_a */
        for (int l = 0; l < nloc; ++l) {
          double c = xl[l * nrhs + r], pg[3];
          int a = T->comp[l];
          push_grad(&g, &grd[l * 3], pg);
          u[a] += c * val[l];
          for (int k = 0; k < 3; ++k) gu[a][k] += c * pg[k];
        }
        for (int l = 0; l < nloc; ++l) {
          double v[3] = {0, 0, 0}, gv[3][3] = {{0}}, pg[3];
          int a = T->comp[l];
          push_grad(&g, &grd[l * 3], pg);
          v[a] = val[l];
          for (int k = 0; k < 3; ++k) gv[a][k] = pg[k];
          double dd = 0.0;
          for (int i = 0; i < 3; ++i) dd += dot3(gu[i], gv[i]);
          b[l * nrhs + r] += w * g.S * (a_lap * dd + b_mass * dot3(u, v));
        }
      } else { /* ORC_VQ hyperelastic residual */
        double H[3][3] = {{0}}; /* reference displacement gradient H_ac */
        for (int l = 0; l < nloc; ++l) {
          double c = xl[l * nrhs + r];
          int a = T->comp[l];
          for (int k = 0; k < 3; ++k) H[a][k] += c * grd[l * 3 + k];
        }
        double Hu[3][3], P[3][3], PGt[3][3];
        for (int a = 0; a < 3; ++a)
          for (int bb = 0; bb < 3; ++bb) {
            Hu[a][bb] = 0.0;
            for (int k = 0; k < 3; ++k) Hu[a][bb] += H[a][k] * g.G[k][bb];
          }
        if (piola(form, params, Hu, P, NULL)) return -3;
        for (int a = 0; a < 3; ++a)
          for (int k = 0; k < 3; ++k) {
            PGt[a][k] = 0.0;
            for (int bb = 0; bb < 3; ++bb) PGt[a][k] += P[a][bb] * g.G[k][bb];
          }
        for (int l = 0; l < nloc; ++l) {
          int a = T->comp[l];
          double s = 0.0;
          for (int k = 0; k < 3; ++k) s += PGt[a][k] * grd[l * 3 + k];
          b[l * nrhs + r] += w * g.S * s;
        }
      }
    }
  }
  return 0;
}

static int nthreads_of(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

int orc_cell_vectors(int family, int form, int p, int nq, const double* params,
                     int nx, int ny, int nz, const double* coords,
                     const double* x, int nrhs, const int64_t* cells, int64_t ncells,
                     double* b, int nthreads) {
  return orc_cell_vectors_rule(family, form, p, nq, ORC_GL, params, nx, ny, nz, coords, x, nrhs, cells, ncells, b,
                               nthreads);
}

static int cell_vectors_impl(int family, int form, int p, int nq, int qrule, const double* params,
                             int nx, int ny, int nz, const double* coords, const double* kappa,
                             const double* x, int nrhs, const int64_t* cells, int64_t ncells,
                             double* b, int nthreads);

int orc_cell_vectors_rule(int family, int form, int p, int nq, int qrule, const double* params,
                          int nx, int ny, int nz, const double* coords,
                          const double* x, int nrhs, const int64_t* cells, int64_t ncells,
                          double* b, int nthreads) {
  return cell_vectors_impl(family, form, p, nq, qrule, params, nx, ny, nz, coords, NULL, x, nrhs, cells, ncells,
                           b, nthreads);
}

int orc_weighted_cell_vectors(int family, int p, int nq, int nx, int ny, int nz, const double* coords,
                              const double* kappa, const double* x, int nrhs, const int64_t* cells,
                              int64_t ncells, double* b, int nthreads) {
  if (!kappa || (family != ORC_Q && family != ORC_DQ)) return -1;
  return cell_vectors_impl(family, ORC_LAPLACE, p, nq, ORC_GL, NULL, nx, ny, nz, coords, kappa, x, nrhs, cells,
                           ncells, b, nthreads);
}

static int cell_vectors_impl(int family, int form, int p, int nq, int qrule, const double* params,
                             int nx, int ny, int nz, const double* coords, const double* kappa,
                             const double* x, int nrhs, const int64_t* cells, int64_t ncells,
                             double* b, int nthreads) {
  elem_t E;
  if (make_elem(family, p, nx, ny, nz, &E) || !form_ok(family, form) || nrhs < 1) return -1;
  tab_t T;
  if (tabulate(&E, nq, qrule, &T)) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  int err = 0;
  int nt = nthreads_of(nthreads);
#pragma omp parallel num_threads(nt)
  {
    int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * E.nloc);
    double* xl = (double*)malloc(sizeof(double) * E.nloc * nrhs);
    double* kl = (double*)malloc(sizeof(double) * E.nloc);
#pragma omp for schedule(dynamic, 1)
    for (int64_t k = 0; k < ncells; ++k) {
      int64_t c = cells[k];
      if (c < 0 || c >= ncell) { err = -1; continue; }
      double X[8][3];
      cell_vertices(nx, ny, nz, coords, c, X);
      elem_cell_dofs(&E, ny, nz, c, dofs);
      for (int l = 0; l < E.nloc; ++l)
        for (int r = 0; r < nrhs; ++r) xl[l * nrhs + r] = x[dofs[l] * nrhs + r];
      if (kappa)
        for (int l = 0; l < E.nloc; ++l) kl[l] = kappa[dofs[l]];
      int e = cell_vector(&E, &T, form, params, X, xl, nrhs, kappa ? kl : NULL, &b[(size_t)k * E.nloc * nrhs]);
      if (e) err = e;
    }
    free(dofs);
    free(xl);
    free(kl);
  }
  tab_free(&T);
  return err;
}

int orc_action(int family, int form, int p, int nq, const double* params,
               int nx, int ny, int nz, const double* coords,
               const double* x, double* y, int nrhs, int nthreads) {
  return orc_action_rule(family, form, p, nq, ORC_GL, params, nx, ny, nz, coords, x, y, nrhs, nthreads);
}

static int action_impl(int family, int form, int p, int nq, int qrule, const double* params,
                       int nx, int ny, int nz, const double* coords, const double* kappa,
                       const double* x, double* y, int nrhs, int nthreads);

int orc_action_rule(int family, int form, int p, int nq, int qrule, const double* params,
                    int nx, int ny, int nz, const double* coords,
                    const double* x, double* y, int nrhs, int nthreads) {
  return action_impl(family, form, p, nq, qrule, params, nx, ny, nz, coords, NULL, x, y, nrhs, nthreads);
}

int orc_weighted_action(int family, int p, int nq, int nx, int ny, int nz, const double* coords,
                        const double* kappa, const double* x, double* y, int nrhs, int nthreads) {
  if (!kappa || (family != ORC_Q && family != ORC_DQ)) return -1;
  return action_impl(family, ORC_LAPLACE, p, nq, ORC_GL, NULL, nx, ny, nz, coords, kappa, x, y, nrhs, nthreads);
}

static int action_impl(int family, int form, int p, int nq, int qrule, const double* params,
                       int nx, int ny, int nz, const double* coords, const double* kappa,
                       const double* x, double* y, int nrhs, int nthreads) {
  elem_t E;
  if (make_elem(family, p, nx, ny, nz, &E) || !form_ok(family, form) || nrhs < 1) return -1;
  memset(y, 0, sizeof(double) * E.ndof * nrhs);
  int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t CH = 2048;
  int64_t* cells = (int64_t*)malloc(sizeof(int64_t) * CH);
  double* b = (double*)malloc(sizeof(double) * CH * E.nloc * nrhs);
  int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * E.nloc);
  int err = 0;
  for (int64_t c0 = 0; c0 < ncell && !err; c0 += CH) {
    int64_t m = (ncell - c0 < CH) ? ncell - c0 : CH;
    for (int64_t k = 0; k < m; ++k) cells[k] = c0 + k;
    err = cell_vectors_impl(family, form, p, nq, qrule, params, nx, ny, nz, coords, kappa, x, nrhs, cells, m, b,
                            nthreads);
    /* global assembly y += P_K^T b^K, cells in order */
    for (int64_t k = 0; k < m && !err; ++k) {
      elem_cell_dofs(&E, ny, nz, c0 + k, dofs);
      for (int l = 0; l < E.nloc; ++l)
        for (int r = 0; r < nrhs; ++r) y[dofs[l] * nrhs + r] += b[((size_t)k * E.nloc + l) * nrhs + r];
    }
  }
  free(cells);
  free(b);
  free(dofs);
  return err;
}

int orc_cell_matrices(int family, int form, int p, int nq, const double* params,
                      int nx, int ny, int nz, const double* coords,
                      int64_t cell_begin, int64_t cell_end, double* A, int nthreads) {
  return orc_cell_matrices_rule(family, form, p, nq, ORC_GL, params, nx, ny, nz, coords, cell_begin, cell_end, A,
                                nthreads);
}

static int cell_matrices_impl(int family, int form, int p, int nq, int qrule, const double* params,
                              int nx, int ny, int nz, const double* coords, const double* kappa,
                              const double* corners, int64_t cell_begin, int64_t cell_end, double* A,
                              int nthreads);

int orc_cell_matrices_rule(int family, int form, int p, int nq, int qrule, const double* params,
                           int nx, int ny, int nz, const double* coords,
                           int64_t cell_begin, int64_t cell_end, double* A, int nthreads) {
  return cell_matrices_impl(family, form, p, nq, qrule, params, nx, ny, nz, coords, NULL, NULL, cell_begin, cell_end, A,
                            nthreads);
}

int orc_weighted_cell_matrices(int family, int p, int nq, int nx, int ny, int nz, const double* coords,
                               const double* kappa, int64_t cell_begin, int64_t cell_end, double* A, int nthreads) {
  if (!kappa || (family != ORC_Q && family != ORC_DQ)) return -1;
  return cell_matrices_impl(family, ORC_LAPLACE, p, nq, ORC_GL, NULL, nx, ny, nz, coords, kappa, NULL, cell_begin,
                            cell_end, A, nthreads);
}

/* corners != NULL: any mesh, cell c's corner coordinates at corners[c*24 ..]
 * (corner (a,b,c) at 4a+2b+c), with nx = number of cells and ny = nz = 1. */
static int cell_matrices_impl(int family, int form, int p, int nq, int qrule, const double* params,
                              int nx, int ny, int nz, const double* coords, const double* kappa,
                              const double* corners, int64_t cell_begin, int64_t cell_end, double* A,
                              int nthreads) {
  elem_t E;
  if (make_elem(family, p, nx, ny, nz, &E) || !form_ok(family, form)) return -1;
  if (form == ORC_NEOHOOKE || form == ORC_SVK) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  if (cell_begin < 0 || cell_end > ncell || cell_begin > cell_end) return -1;
  tab_t T;
  if (tabulate(&E, nq, qrule, &T)) return -1;
  int nloc = E.nloc;
  int err = 0;
  int nt = nthreads_of(nthreads);
#pragma omp parallel num_threads(nt)
  {
    /* per-qp pushed quantities of every basis function */
    double* pv = (double*)malloc(sizeof(double) * nloc * 3);
    double* sv = (double*)malloc(sizeof(double) * nloc);
    double* pm = (double*)malloc(sizeof(double) * nloc * 3);
    double* kl = (double*)malloc(sizeof(double) * nloc);
    int64_t* kd = (int64_t*)malloc(sizeof(int64_t) * nloc);
#pragma omp for schedule(dynamic, 1)
    for (int64_t c = cell_begin; c < cell_end; ++c) {
      double* Ac = &A[(size_t)(c - cell_begin) * nloc * nloc];
      memset(Ac, 0, sizeof(double) * nloc * nloc);
      double X[8][3];
      if (corners) {
        for (int k = 0; k < 8; ++k)
          for (int d = 0; d < 3; ++d) X[k][d] = corners[((size_t)c * 8 + k) * 3 + d];
      } else {
        cell_vertices(nx, ny, nz, coords, c, X);
      }
      if (kappa) {
        elem_cell_dofs(&E, ny, nz, c, kd);
        for (int l = 0; l < nloc; ++l) kl[l] = kappa[kd[l]];
      }
      for (int q = 0; q < T.nq3; ++q) {
        double xi[3];
        qpoint(&T, q, xi);
        geo_t g;
        if (geometry(X, xi, &g)) { err = -2; break; }
        double w = qweight(&T, q);
        const double* val = &T.val[(size_t)q * nloc];
        const double* grd = &T.grad[(size_t)q * nloc * 3];
        double cA = 0.0, cB = 0.0; /* weights of the two parts of the form */
        for (int l = 0; l < nloc; ++l) {
          int cc = T.comp[l];
          if (E.family == ORC_Q || E.family == ORC_DQ || E.family == ORC_VQ) {
            push_grad(&g, &grd[l * 3], &pv[l * 3]);   /* physical gradient (of the component) */
            sv[l] = val[l];
          } else if (E.family == ORC_NCF) {
            double vh[3] = {0, 0, 0};
            vh[cc] = val[l];
            matvec(g.J, vh, &pv[l * 3]);              /* J v^ (Piola numerator) */
            sv[l] = grd[l * 3 + cc];                   /* reference divergence */
          } else {                                     /* NCE */
            double cl[3], vh[3] = {0, 0, 0};
            block_curl(cc, &grd[l * 3], cl);
            matvec(g.J, cl, &pv[l * 3]);              /* J curl^ v^ */
            vh[cc] = val[l];
            push_grad(&g, vh, &pm[l * 3]);            /* G^T v^ */
          }
        }
        if (E.family == ORC_Q || E.family == ORC_DQ) {
          double a_lap, b_mass;
          scalar_weights(form, params, &a_lap, &b_mass);
          if (kappa) { /* weighted Laplace: kappa(xi_q) = sum_l kappa_l psi_l(xi_q) */
            a_lap = 0.0;
            for (int l = 0; l < nloc; ++l) a_lap += kl[l] * val[l];
            b_mass = 0.0;
          }
          double sw = (g_plant == 2) ? w : w * g.S;
          cA = sw * a_lap;
          cB = sw * b_mass;
          for (int j = 0; j < nloc; ++j)
            for (int i = 0; i < nloc; ++i)
              Ac[(size_t)j * nloc + i] += cA * dot3(&pv[i * 3], &pv[j * 3]) + cB * sv[i] * sv[j];
        } else if (E.family == ORC_VQ) {
          /* vector forms (Sec. 3.3): basis psi_l e_comp(l); u . v and
           * grad u : grad v summed over the three components, no delta assumed */
          double a_lap, b_mass;
          scalar_weights(form, params, &a_lap, &b_mass);
          cA = w * g.S * a_lap;
          cB = w * g.S * b_mass;
          for (int j = 0; j < nloc; ++j)
            for (int i = 0; i < nloc; ++i) {
              double vv = 0.0, gg = 0.0;
              for (int k = 0; k < 3; ++k) {
                const double vik = (T.comp[i] == k) ? sv[i] : 0.0;
                const double vjk = (T.comp[g_plant == 10 ? i : j] == k) ? sv[j] : 0.0; /* 10: planted */
                vv += vik * vjk;
                for (int m = 0; m < 3; ++m)
                  gg += ((T.comp[i] == k) ? pv[i * 3 + m] : 0.0) * ((T.comp[j] == k) ? pv[j * 3 + m] : 0.0);
              }
              Ac[(size_t)j * nloc + i] += cA * gg + cB * vv;
            }
        } else if (E.family == ORC_NCF) {
          double inv = (g_plant == 7) ? 1.0 : 1.0 / g.S;
          cA = w * params[0] * inv;
          cB = w * params[1] / g.S;
          for (int j = 0; j < nloc; ++j)
            for (int i = 0; i < nloc; ++i)
              Ac[(size_t)j * nloc + i] += cA * dot3(&pv[i * 3], &pv[j * 3]) + cB * sv[i] * sv[j];
        } else {
          cA = w * params[1] / g.S;
          cB = w * params[0] * g.S;
          for (int j = 0; j < nloc; ++j)
            for (int i = 0; i < nloc; ++i)
              Ac[(size_t)j * nloc + i] += cA * dot3(&pv[i * 3], &pv[j * 3]) + cB * dot3(&pm[i * 3], &pm[j * 3]);
        }
      }
    }
    free(pv);
    free(sv);
    free(pm);
    free(kl);
    free(kd);
  }
  tab_free(&T);
  return err;
}

/* Linearised hyperelastic operator: b^K_(a,j) = sum_q w_q |J| dP(u_K; du_K) :
 * grad(psi_j e_a), with the state u (ndof, one vector) and the directions du
 * (ndof x nrhs); grad u = (grad^ u) G as in the residual. */
int orc_linearised_cell_vectors(int form, int p, int nq, const double* params,
                                int nx, int ny, int nz, const double* coords,
                                const double* u, const double* du, int nrhs,
                                const int64_t* cells, int64_t ncells, double* b, int nthreads) {
  elem_t E;
  if (make_elem(ORC_VQ, p, nx, ny, nz, &E) || !(form == ORC_NEOHOOKE || form == ORC_SVK) || nrhs < 1) return -1;
  tab_t T;
  if (tabulate(&E, nq, ORC_GL, &T)) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  int nloc = E.nloc;
  int err = 0;
  int nt = nthreads_of(nthreads);
#pragma omp parallel num_threads(nt)
  {
    int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * nloc);
    double* ul = (double*)malloc(sizeof(double) * nloc);
    double* dl = (double*)malloc(sizeof(double) * nloc * nrhs);
#pragma omp for schedule(dynamic, 1)
    for (int64_t kc = 0; kc < ncells; ++kc) {
      int64_t c = cells[kc];
      if (c < 0 || c >= ncell) { err = -1; continue; }
      double X[8][3];
      cell_vertices(nx, ny, nz, coords, c, X);
      elem_cell_dofs(&E, ny, nz, c, dofs);
      for (int l = 0; l < nloc; ++l) {
        ul[l] = u[dofs[l]];
        for (int r = 0; r < nrhs; ++r) dl[l * nrhs + r] = du[dofs[l] * nrhs + r];
      }
      double* bc = &b[(size_t)kc * nloc * nrhs];
      memset(bc, 0, sizeof(double) * nloc * nrhs);
      for (int q = 0; q < T.nq3; ++q) {
        double xi[3];
        qpoint(&T, q, xi);
        geo_t g;
        if (geometry(X, xi, &g)) { err = -2; break; }
        double w = qweight(&T, q);
        const double* grd = &T.grad[(size_t)q * nloc * 3];
        double Hr[3][3] = {{0}}, Hu[3][3];
        for (int l = 0; l < nloc; ++l) {
          int a = T.comp[l];
          for (int k = 0; k < 3; ++k) Hr[a][k] += ul[l] * grd[l * 3 + k];
        }
        for (int a = 0; a < 3; ++a)
          for (int bb = 0; bb < 3; ++bb) {
            Hu[a][bb] = 0.0;
            for (int k = 0; k < 3; ++k) Hu[a][bb] += Hr[a][k] * g.G[k][bb];
          }
        for (int r = 0; r < nrhs; ++r) {
          double Dr[3][3] = {{0}}, dF[3][3], dP[3][3], PGt[3][3];
          for (int l = 0; l < nloc; ++l) {
            int a = T.comp[l];
            for (int k = 0; k < 3; ++k) Dr[a][k] += dl[l * nrhs + r] * grd[l * 3 + k];
          }
          for (int a = 0; a < 3; ++a)
            for (int bb = 0; bb < 3; ++bb) {
              dF[a][bb] = 0.0;
              for (int k = 0; k < 3; ++k) dF[a][bb] += Dr[a][k] * g.G[k][bb];
            }
          if (dpiola(form, params, Hu, dF, dP)) { err = -3; break; }
          for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k) {
              PGt[a][k] = 0.0;
              for (int bb = 0; bb < 3; ++bb) PGt[a][k] += dP[a][bb] * g.G[k][bb];
            }
          for (int l = 0; l < nloc; ++l) {
            int a = T.comp[l];
            double sacc = 0.0;
            for (int k = 0; k < 3; ++k) sacc += PGt[a][k] * grd[l * 3 + k];
            bc[l * nrhs + r] += w * g.S * sacc;
          }
        }
      }
    }
    free(dofs);
    free(ul);
    free(dl);
  }
  tab_free(&T);
  return err;
}

/* Tangent (element) matrices of the hyperelastic residual at the state u
 * (Sec. 4.1: the linearised operator whose action the paper times, here
 * assembled per cell): row (a,i) = test psi_i e_a, column (b,j) = trial
 * psi_j e_b,
 *   A^K_((a,i),(b,j)) = sum_q w_q |J| dP(F(u); e_b (x) grad psi_j) : (e_a (x) grad psi_i),
 * i.e. the cell vector of the linearised operator for each trial basis
 * function as the direction.  Cells [cell_begin, cell_end), A row-major
 * (cell, nloc, nloc). */
int orc_linearised_cell_matrices(int form, int p, int nq, const double* params,
                                 int nx, int ny, int nz, const double* coords, const double* u,
                                 int64_t cell_begin, int64_t cell_end, double* A, int nthreads) {
  elem_t E;
  if (make_elem(ORC_VQ, p, nx, ny, nz, &E) || !(form == ORC_NEOHOOKE || form == ORC_SVK)) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  if (cell_begin < 0 || cell_end > ncell || cell_begin > cell_end) return -1;
  tab_t T;
  if (tabulate(&E, nq, ORC_GL, &T)) return -1;
  int nloc = E.nloc;
  int err = 0;
  int nt = nthreads_of(nthreads);
#pragma omp parallel num_threads(nt)
  {
    int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * nloc);
    double* ul = (double*)malloc(sizeof(double) * nloc);
    double* gx = (double*)malloc(sizeof(double) * nloc * 3); /* physical gradients of the basis at a point */
#pragma omp for schedule(dynamic, 1)
    for (int64_t c = cell_begin; c < cell_end; ++c) {
      double X[8][3];
      cell_vertices(nx, ny, nz, coords, c, X);
      elem_cell_dofs(&E, ny, nz, c, dofs);
      for (int l = 0; l < nloc; ++l) ul[l] = u[dofs[l]];
      double* Ac = &A[(size_t)(c - cell_begin) * nloc * nloc];
      memset(Ac, 0, sizeof(double) * nloc * nloc);
      for (int q = 0; q < T.nq3; ++q) {
        double xi[3];
        qpoint(&T, q, xi);
        geo_t g;
        if (geometry(X, xi, &g)) { err = -2; break; }
        double wS = qweight(&T, q) * g.S;
        const double* grd = &T.grad[(size_t)q * nloc * 3];
        for (int l = 0; l < nloc; ++l) /* grad psi_l = G^T grad^ psi_l */
          for (int bb = 0; bb < 3; ++bb) {
            double t = 0.0;
            for (int k = 0; k < 3; ++k) t += grd[l * 3 + k] * g.G[k][bb];
            gx[l * 3 + bb] = t;
          }
        double Hu[3][3] = {{0}};
        for (int l = 0; l < nloc; ++l)
          for (int bb = 0; bb < 3; ++bb) Hu[T.comp[l]][bb] += ul[l] * gx[l * 3 + bb];
        for (int j = 0; j < nloc; ++j) {
          double dF[3][3] = {{0}}, dP[3][3];
          for (int bb = 0; bb < 3; ++bb) {
            if (g_plant == 9) dF[bb][T.comp[j]] = gx[j * 3 + bb]; /* planted: transposed direction */
            else dF[T.comp[j]][bb] = gx[j * 3 + bb];
          }
          if (dpiola(form, params, Hu, dF, dP)) { err = -3; break; }
          for (int i = 0; i < nloc; ++i) {
            const int a = T.comp[i];
            Ac[(size_t)i * nloc + j] += wS * (dP[a][0] * gx[i * 3 + 0] + dP[a][1] * gx[i * 3 + 1] +
                                              dP[a][2] * gx[i * 3 + 2]);
          }
        }
      }
    }
    free(dofs);
    free(ul);
    free(gx);
  }
  tab_free(&T);
  return err;
}

int orc_linearised_action(int form, int p, int nq, const double* params,
                          int nx, int ny, int nz, const double* coords,
                          const double* u, const double* du, double* y, int nrhs, int nthreads) {
  elem_t E;
  if (make_elem(ORC_VQ, p, nx, ny, nz, &E) || nrhs < 1) return -1;
  memset(y, 0, sizeof(double) * E.ndof * nrhs);
  int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t CH = 2048;
  int64_t* cells = (int64_t*)malloc(sizeof(int64_t) * CH);
  double* b = (double*)malloc(sizeof(double) * CH * E.nloc * nrhs);
  int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * E.nloc);
  int err = 0;
  for (int64_t c0 = 0; c0 < ncell && !err; c0 += CH) {
    int64_t m = (ncell - c0 < CH) ? ncell - c0 : CH;
    for (int64_t k = 0; k < m; ++k) cells[k] = c0 + k;
    err = orc_linearised_cell_vectors(form, p, nq, params, nx, ny, nz, coords, u, du, nrhs, cells, m, b, nthreads);
    for (int64_t k = 0; k < m && !err; ++k) {
      elem_cell_dofs(&E, ny, nz, c0 + k, dofs);
      for (int l = 0; l < E.nloc; ++l)
        for (int r = 0; r < nrhs; ++r) y[dofs[l] * nrhs + r] += b[((size_t)k * E.nloc + l) * nrhs + r];
    }
  }
  free(cells);
  free(b);
  free(dofs);
  return err;
}

int orc_energy(int form, int p, int nq, const double* params,
               int nx, int ny, int nz, const double* coords,
               const double* x, double* energy) {
  elem_t E;
  if (make_elem(ORC_VQ, p, nx, ny, nz, &E) || !(form == ORC_NEOHOOKE || form == ORC_SVK)) return -1;
  tab_t T;
  if (tabulate(&E, nq, ORC_GL, &T)) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * E.nloc);
  double total = 0.0;
  int err = 0;
  for (int64_t c = 0; c < ncell && !err; ++c) {
    double X[8][3];
    cell_vertices(nx, ny, nz, coords, c, X);
    elem_cell_dofs(&E, ny, nz, c, dofs);
    for (int q = 0; q < T.nq3; ++q) {
      double xi[3];
      qpoint(&T, q, xi);
      geo_t g;
      if (geometry(X, xi, &g)) { err = -2; break; }
      const double* grd = &T.grad[(size_t)q * E.nloc * 3];
      double H[3][3] = {{0}}, Hu[3][3], P[3][3], W;
      for (int l = 0; l < E.nloc; ++l)
        for (int k = 0; k < 3; ++k) H[T.comp[l]][k] += x[dofs[l]] * grd[l * 3 + k];
      for (int a = 0; a < 3; ++a)
        for (int bb = 0; bb < 3; ++bb) {
          Hu[a][bb] = 0.0;
          for (int k = 0; k < 3; ++k) Hu[a][bb] += H[a][k] * g.G[k][bb];
        }
      if (piola(form, params, Hu, P, &W)) { err = -3; break; }
      total += qweight(&T, q) * g.S * W;
    }
  }
  free(dofs);
  tab_free(&T);
  *energy = total;
  return err;
}

/* ------------------------------------------------------------------------ */
/* Test helpers                                                               */
/* ------------------------------------------------------------------------ */

int orc_q_node_coords(int p, int nx, int ny, int nz, const double* coords, double* out) {
  elem_t E;
  if (make_elem(ORC_Q, p, nx, ny, nz, &E)) return -1;
  int n = p + 1;
  double xn[33], wd[33];
  orc_gauss_lobatto(n, xn, wd);
  int64_t ncell = (int64_t)nx * ny * nz;
  int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * E.nloc);
  for (int64_t c = 0; c < ncell; ++c) {
    double X[8][3];
    cell_vertices(nx, ny, nz, coords, c, X);
    elem_cell_dofs(&E, ny, nz, c, dofs);
    int l = 0;
    for (int i1 = 0; i1 < n; ++i1)
      for (int i2 = 0; i2 < n; ++i2)
        for (int i3 = 0; i3 < n; ++i3, ++l) {
          double xi[3] = {xn[i1], xn[i2], xn[i3]};
          mapped_point(X, xi, &out[dofs[l] * 3]);
        }
  }
  free(dofs);
  return 0;
}

/* Evaluate sum_l x_l * (factor product or its gradient) of a scalar tensor
 * block at a reference point. */
static void block_eval(const blk_t* B, const double* xl, const double* pt, double* val, double* grad) {
  double nodes[3][33], wd[33];
  for (int d = 0; d < 3; ++d) {
    if (B->kind[d] == ORC_GLL) orc_gauss_lobatto(B->cnt[d], nodes[d], wd);
    else orc_gauss_legendre(B->cnt[d], nodes[d], wd);
  }
  *val = 0.0;
  grad[0] = grad[1] = grad[2] = 0.0;
  int l = 0;
  for (int i1 = 0; i1 < B->cnt[0]; ++i1)
    for (int i2 = 0; i2 < B->cnt[1]; ++i2)
      for (int i3 = 0; i3 < B->cnt[2]; ++i3, ++l) {
        int ii[3] = {i1, i2, i3};
        double f[3], df[3];
        for (int d = 0; d < 3; ++d) {
          f[d] = orc_lagrange(nodes[d], B->cnt[d], ii[d], pt[d]);
          df[d] = orc_lagrange_deriv(nodes[d], B->cnt[d], ii[d], pt[d]);
        }
        *val += xl[l] * f[0] * f[1] * f[2];
        grad[0] += xl[l] * df[0] * f[1] * f[2];
        grad[1] += xl[l] * f[0] * df[1] * f[2];
        grad[2] += xl[l] * f[0] * f[1] * df[2];
      }
}

static void block_nodes(const blk_t* B, int d, double* xn) {
  double wd[33];
  if (B->kind[d] == ORC_GLL) orc_gauss_lobatto(B->cnt[d], xn, wd);
  else orc_gauss_legendre(B->cnt[d], xn, wd);
}

int orc_interp_grad_q_to_nce(int p, int nx, int ny, int nz, const double* xq, double* xnce) {
  elem_t Q, N;
  if (make_elem(ORC_Q, p, nx, ny, nz, &Q) || make_elem(ORC_NCE, p, nx, ny, nz, &N)) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  int64_t* dq = (int64_t*)malloc(sizeof(int64_t) * Q.nloc);
  int64_t* dn = (int64_t*)malloc(sizeof(int64_t) * N.nloc);
  double* xl = (double*)malloc(sizeof(double) * Q.nloc);
  for (int64_t c = 0; c < ncell; ++c) {
    elem_cell_dofs(&Q, ny, nz, c, dq);
    elem_cell_dofs(&N, ny, nz, c, dn);
    for (int l = 0; l < Q.nloc; ++l) xl[l] = xq[dq[l]];
    for (int bi = 0; bi < 3; ++bi) {
      const blk_t* B = &N.b[bi];
      double xn[3][33];
      for (int d = 0; d < 3; ++d) block_nodes(B, d, xn[d]);
      int l = B->loff;
      for (int i1 = 0; i1 < B->cnt[0]; ++i1)
        for (int i2 = 0; i2 < B->cnt[1]; ++i2)
          for (int i3 = 0; i3 < B->cnt[2]; ++i3, ++l) {
            double pt[3] = {xn[0][i1], xn[1][i2], xn[2][i3]}, v, gr[3];
            block_eval(&Q.b[0], xl, pt, &v, gr);
            xnce[dn[l]] = gr[B->comp];
          }
    }
  }
  free(dq); free(dn); free(xl);
  return 0;
}

int orc_interp_curl_nce_to_ncf(int p, int nx, int ny, int nz, const double* xnce, double* xncf) {
  elem_t Nc, Nf;
  if (make_elem(ORC_NCE, p, nx, ny, nz, &Nc) || make_elem(ORC_NCF, p, nx, ny, nz, &Nf)) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  int64_t* de = (int64_t*)malloc(sizeof(int64_t) * Nc.nloc);
  int64_t* df = (int64_t*)malloc(sizeof(int64_t) * Nf.nloc);
  double* xl = (double*)malloc(sizeof(double) * Nc.nloc);
  for (int64_t c = 0; c < ncell; ++c) {
    elem_cell_dofs(&Nc, ny, nz, c, de);
    elem_cell_dofs(&Nf, ny, nz, c, df);
    for (int l = 0; l < Nc.nloc; ++l) xl[l] = xnce[de[l]];
    for (int bi = 0; bi < 3; ++bi) {
      const blk_t* B = &Nf.b[bi];
      double xn[3][33];
      for (int d = 0; d < 3; ++d) block_nodes(B, d, xn[d]);
      int l = B->loff;
      for (int i1 = 0; i1 < B->cnt[0]; ++i1)
        for (int i2 = 0; i2 < B->cnt[1]; ++i2)
          for (int i3 = 0; i3 < B->cnt[2]; ++i3, ++l) {
            double pt[3] = {xn[0][i1], xn[1][i2], xn[2][i3]};
            double curl[3] = {0, 0, 0};
            for (int bj = 0; bj < 3; ++bj) {
              const blk_t* C = &Nc.b[bj];
              double v, gr[3], cl[3];
              block_eval(C, &xl[C->loff], pt, &v, gr);
              block_curl(C->comp, gr, cl);
              for (int k = 0; k < 3; ++k) curl[k] += cl[k];
            }
            xncf[df[l]] = curl[B->comp];
          }
    }
  }
  free(de); free(df); free(xl);
  return 0;
}

/* Interpolate the physical linear field u(x) = A x + b into NCE_p (covariant:
 * dof = (J^T u)_c at the block node) or NCF_p (contravariant: dof =
 * (|J| J^{-1} u)_c).  Exact whenever the pulled-back field lies in the space. */
int orc_interp_linear_field(int family, int p, int nx, int ny, int nz, const double* coords,
                            const double* A, const double* bvec, double* out) {
  elem_t E;
  if ((family != ORC_NCE && family != ORC_NCF) || make_elem(family, p, nx, ny, nz, &E)) return -1;
  int64_t ncell = (int64_t)nx * ny * nz;
  int64_t* dofs = (int64_t*)malloc(sizeof(int64_t) * E.nloc);
  for (int64_t c = 0; c < ncell; ++c) {
    double X[8][3];
    cell_vertices(nx, ny, nz, coords, c, X);
    elem_cell_dofs(&E, ny, nz, c, dofs);
    for (int bi = 0; bi < 3; ++bi) {
      const blk_t* B = &E.b[bi];
      double xn[3][33];
      for (int d = 0; d < 3; ++d) block_nodes(B, d, xn[d]);
      int l = B->loff;
      for (int i1 = 0; i1 < B->cnt[0]; ++i1)
        for (int i2 = 0; i2 < B->cnt[1]; ++i2)
          for (int i3 = 0; i3 < B->cnt[2]; ++i3, ++l) {
            double xi[3] = {xn[0][i1], xn[1][i2], xn[2][i3]}, x[3], u[3];
            geo_t g;
            if (geometry(X, xi, &g)) { free(dofs); return -2; }
            mapped_point(X, xi, x);
            for (int a = 0; a < 3; ++a) u[a] = A[a * 3] * x[0] + A[a * 3 + 1] * x[1] + A[a * 3 + 2] * x[2] + bvec[a];
            int cc = B->comp;
            double v = 0.0;
            if (family == ORC_NCE)
              for (int a = 0; a < 3; ++a) v += g.J[a][cc] * u[a];
            else
              for (int a = 0; a < 3; ++a) v += g.S * g.G[cc][a] * u[a];
            out[dofs[l]] = v;
          }
    }
  }
  free(dofs);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Any hexahedral mesh: the cells are given by their corner coordinates alone
 * (corner (a,b,c) at 4a+2b+c, ncells x 8 x 3), so the per-cell integrals do
 * not depend on any global numbering; the caller gathers and scatters through
 * its own cell-node map (Sec. 1.1: y = sum_K P_K^T b^K). */
int orc_local_vectors(int family, int form, int p, int nq, const double* params, int64_t ncells,
                      const double* corners, const double* xl, int nrhs, double* b, int nthreads) {
  elem_t E;
  if (ncells < 1 || !corners || make_elem(family, p, 1, 1, 1, &E) || !form_ok(family, form) || nrhs < 1) return -1;
  tab_t T;
  if (tabulate(&E, nq, ORC_GL, &T)) return -1;
  int err = 0;
  int nt = nthreads_of(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int64_t c = 0; c < ncells; ++c) {
    double X[8][3];
    for (int k = 0; k < 8; ++k)
      for (int d = 0; d < 3; ++d) X[k][d] = corners[((size_t)c * 8 + k) * 3 + d];
    int e = cell_vector(&E, &T, form, params, X, &xl[(size_t)c * E.nloc * nrhs], nrhs, NULL,
                        &b[(size_t)c * E.nloc * nrhs]);
    if (e) err = e;
  }
  tab_free(&T);
  return err;
}

int orc_local_matrices(int family, int form, int p, int nq, const double* params, int64_t ncells,
                       const double* corners, double* A, int nthreads) {
  if (ncells < 1 || ncells > 2000000000LL || !corners) return -1;
  return cell_matrices_impl(family, form, p, nq, ORC_GL, params, (int)ncells, 1, 1, NULL, NULL, corners, 0, ncells,
                            A, nthreads);
}
