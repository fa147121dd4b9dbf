// sfx_internal.h -- objects and kernel-argument structs shared by the host code
// (sfx_host.cpp) and the CUDA kernels.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/sfx.h"

namespace sfx {

constexpr int kMaxDeg = 8;          // p <= 8
constexpr int kMaxN = kMaxDeg + 1;  // 1D nodes per axis
constexpr int kMaxQ = kMaxDeg + 1;  // 1D quadrature points per axis (q = p + 1)

// 1D tables on [0,1] for one degree, passed by value to kernels (constant bank).
//   w, x     Gauss rule with q = p+1 points
//   Bc, Dc   GLL Lagrange basis (p+1 nodes) values / derivatives at the points  [q][p+1]
//   Bd, Dd   Gauss-node Lagrange basis with p nodes (the dP_{p-1} factor)       [q][p]
//   Dq       collocation derivative on the Gauss points themselves              [q][q]
//            (Dq[a][b] = l_b'(x_a), l_b the Lagrange basis on the q points)
//   xg, wg   Gauss-Lobatto rule with p+1 points: the GLL nodes themselves
//            (the collocated rule of Sec. 2.5, "underintegration" in Sec. 4.1)
//   Dg       collocation derivative on the GLL nodes, Dg[a][b] = l_b'(xg_a)
struct Tab1D {
  int p, q;
  double w[kMaxQ], x[kMaxQ];
  double Bc[kMaxQ][kMaxN], Dc[kMaxQ][kMaxN];
  double Bd[kMaxQ][kMaxN], Dd[kMaxQ][kMaxN];
  double Dq[kMaxQ][kMaxQ];
  double wg[kMaxN], xg[kMaxN];
  double Dg[kMaxN][kMaxN];
};

// 1D rules and Lagrange tables (host, double).  Newton iteration on the
// Legendre recurrence; barycentric Lagrange evaluation.
void gauss_legendre(int n, double* x, double* w);
void gauss_lobatto(int n, double* x, double* w);
void lagrange_table(const double* nodes, int n, const double* pts, int q, int deriv, double* out /*q x n*/);
void make_tab1d(int p, Tab1D* t);

}  // namespace sfx

struct sfx_ctx {
  int device = 0;
  uint32_t* d_status = nullptr;  // device status word (SFX_DEV_* bits)
};

struct sfx_mesh {
  sfx_ctx* ctx = nullptr;
  int nx = 0, ny = 0, nz = 0;      // structured box; all 0 for a general mesh
  bool general = false;            // created by sfx_mesh_create (any hexahedral connectivity)
  int64_t nvert = 0, ncell = 0;
  std::vector<double> xyz;         // host, nvert x 3
  std::vector<int32_t> vmap;       // host, ncell x 8 (cell -> vertices, corner (a,b,c) at 4a+2b+c)
  double* d_xyz = nullptr;         // device copy
  int32_t* d_vmap = nullptr;       // device copy of vmap
};

struct sfx_space {
  const sfx_mesh* mesh = nullptr;
  sfx_family family = SFX_Q;
  int p = 1, nloc = 0;
  int64_t ndof = 0;
  std::vector<int32_t> map;        // host, ncell x nloc
  int32_t* d_map = nullptr;        // device copy
  // conflict-free scatter: cells grouped by colour (8 colours for shared-dof
  // families, 1 for DQ); d_cells holds the cell ids colour by colour.
  int ncolour = 1;
  double* d_naive = nullptr;       // dense 3D tabulation for the naive kernels (built on first use)
  std::vector<int64_t> colour_off; // ncolour + 1 offsets into d_cells
  std::vector<int32_t> cells;      // host copy of the cell ids, colour by colour
  int32_t* d_cells = nullptr;
  // scalar Q_p: bit l of cell c's row (nloc/32 words, rounded up) is set when
  // (c, l) is the first of its dof's cell-node pairs in colour order, so an
  // overwriting action stores that contribution and adds the later ones
  // instead of zeroing y first (DQ_p: every pair is first; no table)
  std::vector<uint32_t> first;     // host
  uint32_t* d_first = nullptr;     // device copy
  sfx::Tab1D tab;                  // 1D tables of degree p
  // vector Q_p only: the scalar Q_p space of one component (component a's
  // global dofs are a * scalar->ndof + the scalar numbering), built on first
  // use by the vector mass / Laplace / Helmholtz forms (delta structure)
  mutable sfx_space* scalar = nullptr;
};

// Geometric factors at the quadrature points of every cell, computed once in
// FP64: per cell 7 arrays of q^3 values, P = w S G G^T (00,11,22,01,02,12) and
// w S.  Kept in FP64 (d64) or rounded to FP32 (d32).
struct sfx_qdata {
  const sfx_space* space = nullptr;
  int fp32 = 0;
  double* d64 = nullptr;
  float* d32 = nullptr;
};

// ----------------------------------------------------------------- kernels
namespace sfx {

// Arguments of one action launch (one colour, or a cell list).
struct ActArgs {
  const int32_t* map;     // ncell x nloc
  const int32_t* cells;   // cell ids of this launch (colour list), or
  const int64_t* cells64; // caller's cell list (bounds-checked on the device); both null: slot == cell
  int64_t ncells;         // cells in this launch
  const int32_t* vmap;    // ncell x 8
  const double* xyz;      // nvert x 3
  const double* x;        // ndof x nrhs
  const double* xs;       // linearised operators: the state (ndof, one vector)
  const double* kappa;    // weighted Laplace: the coefficient's dofs (ndof, one vector)
  double* y;              // ndof x nrhs (scatter) or ncells x nloc x nrhs (cell vectors)
  int nrhs;
  int r0, r1;             // right-hand sides handled by this launch: [r0, r1)
  const int64_t* dq_off;  // p-adaptive DQ: dof of (cell, l) = dq_off[cell] + l (map unused)
  const double* qd64;     // stored geometric factors (FP64), [cell][7][q^3], or null
  const float* qd32;      // stored geometric factors (FP32), [cell][7][q^3], or null
  int cell_vectors;       // 1: write b^K per slot instead of scattering
  int unit_cols;          // linearised operator only: > 0 selects element matrices, this many
                          //    trial columns (unit directions) per CTA (blockIdx.y picks the chunk)
  int64_t cell0;          // no cell list: cell = cell0 + slot
  int stage_factors;      // 1: stage the per-point factors once per cell even for one RHS (the
                          //    arithmetic of the persistent batched kernel, for bitwise comparison)
  const uint32_t* first;  // overwrite mode, y not zeroed beforehand: the space's first-touch bits
  int first_all;          //    (d_first), or 1 here when every (cell, l) is its dof's only pair (DQ);
                          //    both unset: every contribution is added to y
  int overlap_prev;       // 1: not the first launch of its action on the stream; a launcher whose
                          //    kernel waits before writing y launches it as a programmatic
                          //    dependent of the previous launch (pdl_wait_prev)
  double alpha, beta, mu, lambda;
  uint32_t* status;
};

// Launchers (defined in the .cu files).  Return a cudaError_t as int.
int launch_action_scalar(const sfx_space* sp, sfx_form form, sfx_precision prec, sfx_algo algo,
                         const ActArgs& a, void* stream);
int launch_action_hdivcurl(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                           void* stream);
int launch_action_elastic(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                          void* stream);
int launch_action_elastic_mixed(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                                void* stream);
int launch_action_scalar_mixed(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                               void* stream);
int launch_action_scalar_naive(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);
// Linearised hyperelastic operator at the state a.xs on the directions a.x (FP64).
int launch_linearised_elastic(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);
int launch_linearised_elastic_mixed(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                                    void* stream);
// Q_p actions with the collocated GLL rule (B = I): FP64 and TF32x3.
int launch_action_scalar_coll(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);
int launch_action_scalar_mixed_coll(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream);
// Weighted Laplace action int kappa grad u . grad v on Q_p / DQ_p (FP64).
int launch_action_weighted(const sfx_space* sp, const ActArgs& a, void* stream);

struct MatArgs {
  const int32_t* vmap;
  const double* xyz;
  int64_t cell_begin, ncells;
  double* A;              // ncells x nloc x nloc
  double alpha, beta;
  const int32_t* map;     // weighted Laplace: the space's cell-node map, and
  const double* kappa;    // the coefficient's dofs (null: kappa = 1);
  int kappa_dq;           // 1 if the space is DQ_p (identity value table)
  uint32_t* status;
};
int launch_cell_matrices(const sfx_space* sp, sfx_form form, sfx_algo algo, const MatArgs& a, void* stream);
// Q_p element matrices with the collocated GLL rule, delta-cancelled (k_matrix.cu).
int launch_cell_matrices_coll(const sfx_space* sp, sfx_form form, const MatArgs& a, void* stream);

// FP64 scalar action over an explicit cell list for one degree (DQ, p-adaptive
// plans); also used by the per-launch comparison mode.
int launch_scalar_fp64_degree(int p, bool dq, sfx_form form, const ActArgs& a, int64_t ncell_total, void* stream);

// Sparse matrix kernels (k_csr.cu).
int launch_csr_scatter(const double* A, int64_t cell_begin, int64_t ncells, int nloc, const int32_t* map,
                       const int64_t* row_ptr, const int32_t* col, double* values, int colour, int ny, int nz,
                       uint32_t* status, void* stream);
int launch_csr_spmv(int lanes, int64_t nrows, const int64_t* row_ptr, const int32_t* col, const double* values,
                    const double* x, double* y, void* stream);

// Persistent batched launch over a tile list (k_batched.cu).
struct BatchTile {
  int32_t p, form, first, count;  // degree, form slot, range in the degree-sorted cell list
};
struct BatchArgs {
  ActArgs base;                   // x, vmap, xyz, nrhs, dq_off, status (cells/y/ncells per tile)
  const int32_t* sorted_cells;
  const BatchTile* tiles;
  int ntiles;
  const int* ntiles_dev;          // if set, the tile count is read from the device
  int* counter;                   // tile counter, zeroed before each launch
  double* y[4];
  double alpha[4], beta[4];
  int form_id[4];
  int64_t ncell_total;
};
// Vector Q_p element matrices of the linear vector forms from the scalar ones:
// A[c][(a,i)][(b,j)] = (a == b) S[c][i][j], all other entries zero (n3 = (p+1)^3).
int launch_vq_expand(const double* S, int64_t ncells, int n3, double* A, void* stream);
int batched_config(int* cb_per_degree /*[kMaxDeg+1]*/, size_t* smem, int* grid);
int batched_launch(const BatchArgs& b, int grid, size_t smem, void* stream);
int batched_tile_sizes(int* cb_per_degree /*[kMaxDeg+1]*/);
// The split-precision persistent batch (TF32x3 / BF16x3): tile sizes for the
// plan's forms (bit f of form_mask: form f, SFX_MASS = 0) and RHS count.
int batched_mixed_config_tf32(int form_mask, int nrhs, int* cb, size_t* smem, int* grid);
int batched_mixed_config_bf16(int form_mask, int nrhs, int* cb, size_t* smem, int* grid);
int batched_mixed_launch_tf32(const BatchArgs& b, int nrhs, int grid, size_t smem, void* stream);
int batched_mixed_launch_bf16(const BatchArgs& b, int nrhs, int grid, size_t smem, void* stream);
// One degree's cells of a split-precision scalar action (per-launch plan mode).
int launch_scalar_mixed_degree_tf32(int p, bool dq, sfx_form form, const ActArgs& a, int64_t ncell_total, void* stream);
int launch_scalar_mixed_degree_bf16(int p, bool dq, sfx_form form, const ActArgs& a, int64_t ncell_total, void* stream);
int launch_qdata(const sfx_space* sp, sfx_qdata* q, uint32_t* status, void* stream);

// Cells per CTA of the action kernels: the autotuner's choice per (kernel,
// degree) if one was set, else a built-in measured table, else the launcher's
// default.  Host-side tables.
enum {
  SFX_TUNE_SCALAR_FP64 = 0,
  SFX_TUNE_SCALAR_MIXED = 1,
  SFX_TUNE_SCALAR_MIXED_STORED = 2,
  SFX_TUNE_ELASTIC_MIXED = 3,
  SFX_TUNE_SCALAR_MIXED_WS = 4,
  SFX_TUNE_BATCHED = 5,  // cells per tile of the persistent p-adaptive batch (at most its layout's count)
  SFX_TUNE_HDIVCURL = 6,         // FP64 NCF / NCE actions
  SFX_TUNE_ELASTIC = 7,          // FP64 hyperelastic residual
  SFX_TUNE_LINEARISED = 8,       // FP64 linearised hyperelastic action
  SFX_TUNE_LINEARISED_MIXED = 9, // split-precision linearised hyperelastic action
  SFX_TUNE_HDIVCURL_MIXED = 10,  // split-precision NCF / NCE actions
  SFX_TUNE_BATCHED_MIXED = 11,   // cells per tile of the split-precision p-adaptive batch
  SFX_TUNE_NKERNEL = 12
};
// Tuned cells per CTA for the team-per-cell kernels: the tuned value if one
// is set (at most maxcb, and reduced until the shared memory fits `limit`),
// else `fallback`.
int tuned_team_cells(int kernel, int degree, int fallback, int maxcb, size_t fixed, size_t per_cell, size_t limit);
int tuned_cells_per_cta(int kernel, int degree, int fallback);
// Warp-specialised split-precision scalar action on (1) or off (0) by degree.
bool ws_enabled(int degree);
// Poll limit of the bounded waits between warp roles (sfx_set_wait_limit).
uint32_t ws_wait_cap();

// Each kernel file keeps its own constant-memory copy of the 1D tables.
int upload_tab_scalar(const Tab1D* t);
int upload_tab_scalar_mixed_tf32(const Tab1D* t);
int upload_tab_scalar_mixed_bf16(const Tab1D* t);
int upload_tab_scalar_mixed_ws_tf32(const Tab1D* t);
int upload_tab_scalar_mixed_ws_bf16(const Tab1D* t);
int upload_tab_hdivcurl(const Tab1D* t);
int upload_tab_hdivcurl_mixed_tf32(const Tab1D* t);
int upload_tab_hdivcurl_mixed_bf16(const Tab1D* t);
int upload_tab_batched_mixed_tf32(const Tab1D* t);
int upload_tab_batched_mixed_bf16(const Tab1D* t);
int upload_tab_elastic(const Tab1D* t);
int upload_tab_elastic_mixed(const Tab1D* t);
int upload_tab_matrix(const Tab1D* t);
int upload_tab_naive(const Tab1D* t);
int upload_tab_batched(const Tab1D* t);
int upload_tab_qdata(const Tab1D* t);
int upload_tab_scalar_coll(const Tab1D* t);
int upload_tab_scalar_mixed_coll(const Tab1D* t);
int upload_tab_elastic_lin(const Tab1D* t);
int upload_tab_elastic_lin_mixed(const Tab1D* t);
int upload_tab_scalar_kappa(const Tab1D* t);

}  // namespace sfx
