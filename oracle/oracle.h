/*
 * oracle.h -- plain, slow, FP64 CPU reference for cell-local finite element
 * assembly on hexahedra (Homolya, Kirby & Ham, "Exposing and exploiting
 * structure: optimal code generation for high-order finite element methods").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this code; only the tests, the smoke check and the benchmark (its CPU
 * baseline, reference arm and sampled-error columns) use it.  It shares no source with the CUDA path.
 *
 * What it computes (naive quadrature, no sum factorisation):
 *   b^K_j = sum_q w_q I(u_K, psi_j, xi_q)          (Sec. 1.1, Eq. laplace_quadrature;
 *                                                   Sec. 3.3, Eqs. coeff_eval/form_eval)
 *   y     = sum_K P_K^T b^K                          (global assembly, Sec. 1.1)
 *   A^K_ji = sum_q w_q I(psi_i, psi_j, xi_q)         (Sec. 1.1, Eq. laplace_prefiat)
 * with every 3D basis function evaluated as a product of 1D Lagrange
 * polynomials at each 3D point (Sec. 1.2, Eq. limits_tpe) and the coefficient
 * u_K(xi_q) = sum_i U_i psi_i(xi_q) summed over all i (O(n^6) per cell).
 *
 * Conventions (readings of the paper):
 *   reference cell [0,1]^3; local index row-major over (i1,i2,i3), i3 fastest
 *   (Sec. 3.5, Eqs. rtcf_split_x/y); cell vertex v = 4a+2b+c for reference
 *   corner (a,b,c); structured nx*ny*nz box numbering (I,J,K), K fastest.
 */
#ifndef SFX_ORACLE_H
#define SFX_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* families */
enum { ORC_Q = 0, ORC_DQ = 1, ORC_NCF = 2, ORC_NCE = 3, ORC_VQ = 4 };
/* forms */
enum {
  ORC_MASS = 0, ORC_LAPLACE = 1, ORC_HELMHOLTZ = 2,
  ORC_NCF_MASS_DIVDIV = 3, ORC_NCE_CURLCURL = 4,
  ORC_NEOHOOKE = 5, ORC_SVK = 6
};
/* 1D node families */
enum { ORC_GLL = 0, ORC_GL = 1 };

/* Gauss-Legendre (n >= 1) and Gauss-Lobatto-Legendre (n >= 2) rules on [0,1]. */
int orc_gauss_legendre(int n, double* x, double* w);
int orc_gauss_lobatto(int n, double* x, double* w);
/* Lagrange polynomial i on nodes xn[0..n-1] and its derivative, at x. */
double orc_lagrange(const double* xn, int n, int i, double x);
double orc_lagrange_deriv(const double* xn, int n, int i, double x);

/* Space size: global dofs and local dofs per cell.  Returns 0 or -1. */
int orc_space_size(int family, int p, int nx, int ny, int nz, int64_t* ndof, int* nloc);
/* Global dof indices of one cell's local dofs, in local order. */
int orc_cell_dofs(int family, int p, int nx, int ny, int nz, int64_t cell, int64_t* dofs);
/* Whole cell-node map, ncell*nloc int32. */
int orc_cell_map(int family, int p, int nx, int ny, int nz, int32_t* map);

/* Per-cell local vectors b^K (no scatter) for the listed cells.
 *   coords: (nx+1)(ny+1)(nz+1) x 3 vertex coordinates, vertex (I,J,K) at
 *           ((I*(ny+1)+J)*(nz+1)+K).
 *   x: ndof x nrhs (rhs fastest).  b: ncells x nloc x nrhs.
 *   params: {alpha, beta, mu, lambda}.  nq: 1D Gauss points per direction.
 *   nthreads <= 0: OpenMP default. */
int orc_cell_vectors(int family, int form, int p, int nq, const double* params,
                     int nx, int ny, int nz, const double* coords,
                     const double* x, int nrhs, const int64_t* cells, int64_t ncells,
                     double* b, int nthreads);
/* Global action y = sum_K P_K^T b^K (y overwritten; cells in order). */
int orc_action(int family, int form, int p, int nq, const double* params,
               int nx, int ny, int nz, const double* coords,
               const double* x, double* y, int nrhs, int nthreads);
/* Local element matrices A[c][j][i] (row = test j, column = trial i) for
 * cells [cell_begin, cell_end).  Bilinear forms only (not NEOHOOKE/SVK). */
int orc_cell_matrices(int family, int form, int p, int nq, const double* params,
                      int nx, int ny, int nz, const double* coords,
                      int64_t cell_begin, int64_t cell_end, double* A, int nthreads);
/* The same three routines with the quadrature rule chosen: qrule = ORC_GL
 * (Gauss-Legendre, what the routines above use) or ORC_GLL (Gauss-Lobatto-
 * Legendre, nq >= 2).  With nq = p + 1 on Q_p the GLL points are the element's
 * nodes (collocated quadrature, Sec. 2.5, Eq. colocated; the "underintegration"
 * case of Sec. 4.1). */
int orc_cell_vectors_rule(int family, int form, int p, int nq, int qrule, const double* params,
                          int nx, int ny, int nz, const double* coords,
                          const double* x, int nrhs, const int64_t* cells, int64_t ncells,
                          double* b, int nthreads);
int orc_action_rule(int family, int form, int p, int nq, int qrule, const double* params,
                    int nx, int ny, int nz, const double* coords,
                    const double* x, double* y, int nrhs, int nthreads);
int orc_cell_matrices_rule(int family, int form, int p, int nq, int qrule, const double* params,
                           int nx, int ny, int nz, const double* coords,
                           int64_t cell_begin, int64_t cell_end, double* A, int nthreads);
/* Weighted Laplace form int kappa grad u . grad v (Sec. 1.1, Eq.
 * weighted_laplace) on Q_p / DQ_p, the coefficient kappa given by its dofs in
 * the same space (ndof values): per-cell vectors, action, element matrices. */
int orc_weighted_cell_vectors(int family, int p, int nq, int nx, int ny, int nz, const double* coords,
                              const double* kappa, const double* x, int nrhs, const int64_t* cells,
                              int64_t ncells, double* b, int nthreads);
int orc_weighted_action(int family, int p, int nq, int nx, int ny, int nz, const double* coords,
                        const double* kappa, const double* x, double* y, int nrhs, int nthreads);
int orc_weighted_cell_matrices(int family, int p, int nq, int nx, int ny, int nz, const double* coords,
                               const double* kappa, int64_t cell_begin, int64_t cell_end, double* A, int nthreads);
/* Linearised hyperelastic operator (NEOHOOKE or SVK) at the state u (ndof):
 * per-cell vectors and the assembled action on the directions du (ndof x
 * nrhs), b^K_(a,j) = sum_q w_q |J| dP(F(u); grad du) : grad(psi_j e_a). */
int orc_linearised_cell_vectors(int form, int p, int nq, const double* params,
                                int nx, int ny, int nz, const double* coords,
                                const double* u, const double* du, int nrhs,
                                const int64_t* cells, int64_t ncells, double* b, int nthreads);
int orc_linearised_action(int form, int p, int nq, const double* params,
                          int nx, int ny, int nz, const double* coords,
                          const double* u, const double* du, double* y, int nrhs, int nthreads);
/* Tangent matrices of the hyperelastic residual at the state u, cells
 * [cell_begin, cell_end), row = test (a,i), column = trial (b,j). */
int orc_linearised_cell_matrices(int form, int p, int nq, const double* params,
                                 int nx, int ny, int nz, const double* coords, const double* u,
                                 int64_t cell_begin, int64_t cell_end, double* A, int nthreads);
/* Hyperelastic stored energy W(u) (NEOHOOKE or SVK), summed over cells. */
int orc_energy(int form, int p, int nq, const double* params,
               int nx, int ny, int nz, const double* coords,
               const double* x, double* energy);

/* Test helpers: physical coordinates of the Q_p (GLL) nodes, ndof x 3. */
int orc_q_node_coords(int p, int nx, int ny, int nz, const double* coords, double* out);
/* Interpolate the reference gradient of a Q_p field into NCE_p dofs and the
 * reference curl of an NCE_p field into NCF_p dofs (exact for these spaces). */
int orc_interp_grad_q_to_nce(int p, int nx, int ny, int nz, const double* xq, double* xnce);
int orc_interp_curl_nce_to_ncf(int p, int nx, int ny, int nz, const double* xnce, double* xncf);

/* Interpolate the physical linear field u(x) = A x + b (A row-major 3x3)
 * into NCE_p (covariant) or NCF_p (contravariant) dofs. */
int orc_interp_linear_field(int family, int p, int nx, int ny, int nz, const double* coords,
                            const double* A, const double* b, double* out);

/* Any hexahedral mesh (no global numbering inside the oracle's C part): the
 * cells are given by their corner coordinates, corners[c][k][d] with corner
 * (a,b,c) at k = 4a+2b+c (ncells x 8 x 3).  Local vectors b (ncells x nloc x
 * nrhs) from local coefficients xl (ncells x nloc x nrhs), and local element
 * matrices A[c][j][i] (row = test); Gauss rule with nq points.  The caller
 * gathers and scatters through its own cell-node map. */
int orc_local_vectors(int family, int form, int p, int nq, const double* params, int64_t ncells,
                      const double* corners, const double* xl, int nrhs, double* b, int nthreads);
int orc_local_matrices(int family, int form, int p, int nq, const double* params, int64_t ncells,
                       const double* corners, double* A, int nthreads);

/* Deliberate-mistake switch used only by the tests that prove the pins catch
 * plausible errors.  0 = correct oracle. */
void orc_set_plant(int which);

#ifdef __cplusplus
}
#endif
#endif
