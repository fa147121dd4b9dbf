/*
 * sfx.h -- C ABI of the sum-factorised hexahedral assembly library (GB300, sm_103a).
 *
 * Implements cell-local finite element assembly by sum factorisation
 * (Homolya, Kirby & Ham, "Exposing and exploiting structure: optimal code
 * generation for high-order finite element methods"): matrix-free operator
 * actions (Sec. 1.1, the action as a parametrised linear form; Sec. 3.3, Eqs.
 * coeff_eval and form_eval) and local element matrices (Sec. 3.2, Eqs.
 * poisson_gem, opt1_product, opt2_product) on hexahedral meshes, for Q_p,
 * DQ_p, NCF_p (H(div)), NCE_p (H(curl)) and vector Q_p elements.
 *
 * Conventions used by every entry point:
 *   - Return value: SFX_OK (0) or a negative sfx_status.  No entry point throws,
 *     exits or prints.  Argument errors are detected on the host before any
 *     work is queued and leave outputs untouched.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the context's device (e.g. torch tensors' data_ptr()).
 *     The caller owns every array it passes; the library never frees them.
 *   - Objects (ctx, mesh, space) own their own host and device copies.
 *     Create/destroy calls are synchronous.  Assembly calls are asynchronous
 *     on the caller's stream (a cudaStream_t passed as void*, NULL = legacy
 *     default stream).
 *   - Reference cell [0,1]^3.  Local dofs are row-major over (i1,i2,i3) with
 *     i3 fastest (Sec. 3.5, Eqs. rtcf_split_x/y); H(div)/H(curl) blocks are
 *     concatenated x, y, z (Sec. 2.6, Eq. enriched_basis).
 *   - Floating point arrays are IEEE double.  Multi-RHS vectors are
 *     ndof x nrhs with the RHS index fastest.
 *   - Device-detected conditions (an inverted cell, det F <= 0) never trap:
 *     they set bits in the context's device status word, read by
 *     sfx_sync_status().
 */
#ifndef SFX_H
#define SFX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sfx_status;
#define SFX_OK 0
#define SFX_ERR_ARG (-1)         /* null pointer, bad size, bad enum, mismatch */
#define SFX_ERR_UNSUPPORTED (-2) /* valid but not implemented (degree, form/family) */
#define SFX_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define SFX_ERR_ALLOC (-4)       /* host or device allocation failed */
#define SFX_ERR_RANGE (-5)       /* sizes exceed 32-bit dof indexing */

/* device status bits (sfx_sync_status) */
#define SFX_DEV_INVERTED 1u /* det J <= 0 at a quadrature point; the cell's output is zero */
#define SFX_DEV_DETF 2u     /* det F <= 0 in a hyperelastic residual; that point contributes zero */
#define SFX_DEV_BADCELL 4u  /* a caller-supplied cell id is out of range; that slot is skipped */
#define SFX_DEV_TIMEOUT 8u  /* a kernel's bounded wait between its warp roles gave up; the output is not valid */

typedef enum { SFX_Q = 0, SFX_DQ = 1, SFX_NCF = 2, SFX_NCE = 3, SFX_VQ = 4 } sfx_family;

/* Forms (bilinear unless noted), with the integrand on cell K (J = dF_K/dX,
 * S = det J, G = J^{-1}; w the quadrature weight):
 *   SFX_MASS            S u v
 *   SFX_LAPLACE         S (G^T grad u).(G^T grad v)                 Sec. 1.1, Eq. laplace_prefiat
 *   SFX_HELMHOLTZ       alpha * LAPLACE + beta * MASS (beta = -k^2)
 *   SFX_NCF_MASS_DIVDIV (1/S) [alpha (J u^).(J v^) + beta div^u div^v]  contravariant Piola
 *   SFX_NCE_CURLCURL    beta (1/S)(J curl^u).(J curl^v) + alpha S (G^T u^).(G^T v^)
 *                                                         covariant Piola, Eq. curl_curl_form
 *   SFX_NEOHOOKE        residual (linear form in v): S P(F) : (grad^v G), F = I + grad^u G,
 *                       P = mu (F - F^{-T}) + lambda ln(det F) F^{-T}
 *   SFX_SVK             residual with P = F (lambda tr(E) I + 2 mu E), E = (F^T F - I)/2
 *                       (Sec. 4.1, Saint Venant-Kirchhoff)
 * On vector Q_p, SFX_MASS / SFX_LAPLACE / SFX_HELMHOLTZ are the vector forms
 * S u.v and S (grad u G):(grad v G) (Sec. 3.3, Eq. vector_mass_form): the
 * component delta makes them three copies of the scalar form, one per
 * component block (actions and element matrices; not the per-cell vectors). */
typedef enum {
  SFX_MASS = 0,
  SFX_LAPLACE = 1,
  SFX_HELMHOLTZ = 2,
  SFX_NCF_MASS_DIVDIV = 3,
  SFX_NCE_CURLCURL = 4,
  SFX_NEOHOOKE = 5,
  SFX_SVK = 6
} sfx_form;

typedef struct {
  double alpha, beta, mu, lambda;
} sfx_form_params;

typedef enum { SFX_NODES_GLL = 0, SFX_NODES_GL = 1 } sfx_nodes;

/* Arithmetic of the contractions.  FP64: all in double.  TF32X3 / BF16X3:
 * the 1D contractions run on the tensor cores as three split products
 * (hi*hi + hi*lo + lo*hi, FP32 accumulation); the geometry (J, det J, adj J)
 * and the quadrature-weight scaling are computed in double, and the scatter
 * adds in double.  Scalar forms round the scaled geometric factors once to
 * FP32 and apply them in FP32; the hyperelastic stress P(F) is evaluated in
 * double.  Available for Q_p / DQ_p (mass, Laplace, Helmholtz) and vector
 * Q_p (neo-Hookean, SVK); NCF/NCE accept FP64 only. */
typedef enum { SFX_PREC_FP64 = 0, SFX_PREC_TF32X3 = 1, SFX_PREC_BF16X3 = 2 } sfx_precision;

/* SUMFACT: sum-factorised kernels on the (p+1)-point Gauss rule.  NAIVE:
 * dense 3D tabulation, O(n^6) per cell for the action (the un-factorised form
 * of Sec. 3.2, for comparison).  COLLOCATED: Q_p mass / Laplace / Helmholtz
 * on the (p+1)-point Gauss-Lobatto rule, whose points are the GLL nodes of
 * Q_p (Sec. 2.5, Eq. colocated): the value tabulation is the identity, so
 * the action needs only the derivative contractions and the element matrix
 * is delta-cancelled to O(n^5) work (the "underintegration" case of Sec. 4.1;
 * the rule does not integrate these forms exactly, by design).  The action
 * accepts FP64 and TF32X3, the element matrices FP64. */
typedef enum { SFX_ALGO_SUMFACT = 0, SFX_ALGO_NAIVE = 1, SFX_ALGO_COLLOCATED = 2 } sfx_algo;

typedef struct sfx_ctx sfx_ctx;
typedef struct sfx_mesh sfx_mesh;
typedef struct sfx_space sfx_space;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (makes it current).  device = -1
 * gives a host-only context: meshes and spaces get no device copies (for
 * inspecting maps and coordinates without a GPU) and assembly calls on them
 * return SFX_ERR_ARG.  Allocates the
 * 4-byte device status word.  Errors: SFX_ERR_ARG (out NULL), SFX_ERR_CUDA. */
sfx_status sfx_ctx_create(int device, sfx_ctx** out);
void sfx_ctx_destroy(sfx_ctx* ctx);

/* Wait for `stream`, then copy the device status word (SFX_DEV_* bits) to
 * *bits and clear it.  Errors: SFX_ERR_ARG, SFX_ERR_CUDA. */
sfx_status sfx_sync_status(sfx_ctx* ctx, void* stream, uint32_t* bits);

const char* sfx_status_string(sfx_status s);

/* -------------------------------------------------------------------- mesh */

/* Structured nx*ny*nz hexahedral box on [0,1]^3.  Vertex (I,J,K) (K fastest,
 * v = (I*(ny+1)+J)*(nz+1)+K); cell (i,j,k) likewise; cell vertex 4a+2b+c is the
 * reference corner (a,b,c).  Each interior vertex is moved by
 * perturb*h_d*(2u-1) along each axis d, u from the SplitMix64 stream `seed`
 * (draw k = mix(seed + (k+1)*0x9E3779B97F4A7C15), u = (z>>11)*2^-53; three draws
 * per interior vertex in vertex order).  The trilinear coordinate field is the
 * vector-Q1 field of Sec. 3.1.  Errors: SFX_ERR_ARG (n < 1, |perturb| >= 0.5),
 * SFX_ERR_RANGE, SFX_ERR_ALLOC, SFX_ERR_CUDA. */
sfx_status sfx_mesh_create_box(sfx_ctx* ctx, int nx, int ny, int nz, double perturb, uint64_t seed,
                               sfx_mesh** out);
/* Same topology with caller-supplied vertex coordinates (host, nvert x 3,
 * copied).  Errors as above. */
sfx_status sfx_mesh_create_structured(sfx_ctx* ctx, int nx, int ny, int nz, const double* xyz_host,
                                      sfx_mesh** out);
/* General hexahedral mesh: any connectivity (Sec. 1.1: the domain is a union
 * of cells K, each the image F_K of the reference cell under its trilinear
 * map, and global assembly sums the cells' contributions through the
 * cell-node map).
 *   nvert, xyz      host, nvert x 3 vertex coordinates (copied)
 *   ncell, cell_vertices
 *                   host, ncell x 8 int32 vertex ids per cell in VTK
 *                   hexahedron order: the bottom face (reference z = 0)
 *                   counter-clockwise from the origin corner, then the top
 *                   face likewise; corners (0,0,0) (1,0,0) (1,1,0) (0,1,0)
 *                   (0,0,1) (1,0,1) (1,1,1) (0,1,1) of the reference cell.
 * Each cell must be positively oriented (det J > 0; the kernels flag
 * SFX_DEV_INVERTED otherwise).  Spaces on such a mesh: Q_p, DQ_p and vector
 * Q_p (NCF_p and NCE_p need face and edge orientation signs:
 * SFX_ERR_UNSUPPORTED).  The assembled CSR matrix needs a box mesh.
 * Errors: SFX_ERR_ARG (null, nvert < 8, ncell < 1, a vertex id out of range
 * or repeated within a cell), SFX_ERR_RANGE, SFX_ERR_ALLOC, SFX_ERR_CUDA. */
sfx_status sfx_mesh_create(sfx_ctx* ctx, int64_t nvert, const double* xyz_host, int64_t ncell,
                           const int32_t* cell_vertices_host, sfx_mesh** out);
/* Host view of the vertex coordinates (owned by the mesh). */
sfx_status sfx_mesh_info(const sfx_mesh* mesh, int64_t* nvert, int64_t* ncell, const double** xyz_host);
void sfx_mesh_destroy(sfx_mesh* mesh);

/* ------------------------------------------------------------------- space */

/* Function space of `family` and degree p (1 <= p <= 8) on `mesh` (Secs.
 * 2.3-2.7 for the families); builds the int32 cell-node map (ncell x nloc,
 * host and device: the P_K of global assembly, Sec. 1.1) and, for the
 * continuous families, the colour lists used by the conflict-free scatter.
 * Numbering on a box mesh: Q_p/vector-Q_p global node (I,J,K) on the
 * (pN+1)^3 GLL grid, vector-Q_p component-major; DQ_p cell-major
 * (cell*n^3 + l); NCF_p/NCE_p one lexicographic grid per block, block-major.
 * Colours on a box mesh: the 8 parity classes (i&1, j&1, k&1) of the cell
 * indices, colour 4(i&1) + 2(j&1) + (k&1), cells ascending within a colour.
 * On a general mesh (sfx_mesh_create), Q_p: vertex dofs first (the vertex
 * ids), then p-1 dofs per edge, (p-1)^2 per face and (p-1)^3 per cell, edges
 * and faces numbered in order of first appearance (cells in order); an
 * edge's nodes run from its smaller vertex id to its larger one, a face's
 * nodes first along the edge from its smallest-id corner to that corner's
 * neighbour of smaller id.  Colours: greedy first fit over the cells in order
 * (the smallest colour unused by earlier cells sharing a vertex).  DQ_p is
 * cell-major with one colour on either kind of mesh.
 * The mesh must outlive the space.
 * Errors: SFX_ERR_ARG, SFX_ERR_UNSUPPORTED (p out of range), SFX_ERR_RANGE,
 * SFX_ERR_ALLOC, SFX_ERR_CUDA. */
sfx_status sfx_space_create(const sfx_mesh* mesh, sfx_family family, int degree, sfx_space** out);
/* Sizes and a host view of the cell-node map (owned by the space). */
sfx_status sfx_space_info(const sfx_space* space, int64_t* ndof, int* nloc, int64_t* ncell,
                          const int32_t** host_map);
/* Host view of the colour lists (owned by the space): *ncolour colours;
 * cells[colour_off[k] .. colour_off[k+1]) are the cells of colour k.  Cells of
 * one colour share no dof, so one scatter launch per colour never adds twice
 * into one entry (Sec. 1.1, global assembly).  Any output may be NULL.
 * Errors: SFX_ERR_ARG. */
sfx_status sfx_space_colours(const sfx_space* space, int* ncolour, const int64_t** colour_off,
                             const int32_t** cells);
/* Host view of a scalar Q_p space's first-touch bits (owned by the space; an
 * ordering of the cellwise sum of Sec. 1.1, global assembly):
 * ncell rows of *words_per_cell words; bit l of cell c's row is set when
 * (c, l) is the first of its dof's cell-node pairs in colour order (the order
 * of the scatter launches).  Overwriting FP64 actions store that pair's
 * contribution and add the later ones instead of zeroing y first.  Other
 * families: *words_per_cell = 0, *bits = NULL.  Any output may be NULL.
 * Errors: SFX_ERR_ARG. */
sfx_status sfx_space_first_touch(const sfx_space* space, int* words_per_cell, const uint32_t** bits);
void sfx_space_destroy(sfx_space* space);

/* ------------------------------------------------------------ tabulation */

/* 1D rule and Lagrange table on [0,1] (Sec. 1.2, Eq. tpps; Sec. 2.5, Eq.
 * colocated): `points`/`weights` (host, nq each) receive the quadrature rule
 * `qrule` (GL: Gauss-Legendre, GLL: Gauss-Lobatto) with nq points; `table`
 * (host, nq x ndof1d row-major) receives phi_i(x_q) (deriv = 0) or phi_i'(x_q)
 * (deriv = 1) for the Lagrange basis on the ndof1d `nodes`.  Any output may be
 * NULL.  Errors: SFX_ERR_ARG (ndof1d < 1, GLL with < 2 points, nq < 1 or > 32). */
sfx_status sfx_tabulate_1d(sfx_nodes nodes, int ndof1d, sfx_nodes qrule, int nq, int deriv,
                           double* points, double* weights, double* table);

/* --------------------------------------------------------------- assembly */

/* Operator action / residual y = sum_K P_K^T b^K with
 * b^K_j = sum_q w_q I(u_K, psi_j)(xi_q) on the (p+1)^3 Gauss rule (Sec. 1.1;
 * Sec. 3.3, Eqs. coeff_def, coeff_eval, form_eval), u_K = sum_i x_{map(K,i)} psi_i.
 *   x, y   device, ndof x nrhs doubles (x read-only; must not alias y)
 *   nrhs   1 <= nrhs <= 64
 *   accumulate = 0: y is overwritten (every entry written, whatever it held:
 *   for DQ_p and the FP64 Q_p kernels with one right-hand side, and split-
 *   precision DQ_p with up to four, each dof's first contribution is stored;
 *   otherwise y is zeroed on `stream` first); 1: y += action.
 *   params may be NULL (defaults: Helmholtz alpha=1, beta=-1; NCF alpha=beta=1;
 *   NCE alpha=0, beta=1; hyperelastic mu=1, lambda=10).
 *   prec: FP64 for every form; TF32X3 / BF16X3 (split-precision tensor-core
 *   contractions, FP64 geometry, scaling and scatter) for the scalar forms on
 *   Q_p / DQ_p / vector Q_p, NCF_MASS_DIVDIV on NCF_p, NCE_CURLCURL on NCE_p
 *   and the hyperelastic residuals.
 * The scatter is deterministic (8 colour passes for shared-dof families; the
 * colour launches run in stream order, each one's scatter after the previous
 * one's has completed).
 * Errors: SFX_ERR_ARG (null, nrhs, form/family mismatch), SFX_ERR_UNSUPPORTED
 * (precision or algorithm not available for this form), SFX_ERR_CUDA. */
sfx_status sfx_assemble_action(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                               const sfx_space* space, const double* x, double* y, int nrhs,
                               int accumulate, sfx_precision prec, sfx_algo algo, void* stream);

/* Per-cell local vectors b^K (Sec. 3.3, Eq. form_eval; no scatter) for the
 * cells listed in `cells` (device int64, ncells entries, each in [0, ncell)),
 * written to b (device,
 * ncells x nloc x nrhs).  Same arithmetic as sfx_assemble_action.  Used to
 * compare sampled cells of large meshes.  Errors as sfx_assemble_action. */
sfx_status sfx_assemble_cell_vectors(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                     const sfx_space* space, const double* x, int nrhs,
                                     const int64_t* cells, int64_t ncells, double* b,
                                     sfx_precision prec, void* stream);

/* Weighted Laplace form a(u, v) = int kappa grad u . grad v (Sec. 1.1, Eq.
 * weighted_laplace) on Q_p / DQ_p, FP64: kappa is a coefficient given by its
 * dofs in the same space (device, ndof doubles, read-only), interpolated to
 * the Gauss points like u (Sec. 3.3, Eq. coeff_eval).
 * Action: x, y device, ndof x nrhs (y must alias neither x nor kappa);
 * accumulate as in sfx_assemble_action; deterministic colour passes.
 * Element matrices: A device, (cell_end - cell_begin) x nloc x nloc, row =
 * test, by sum factorisation (kappa evaluated at each point).
 * Errors: SFX_ERR_ARG (null, aliasing, family, range), SFX_ERR_UNSUPPORTED
 * (precision), SFX_ERR_CUDA. */
sfx_status sfx_assemble_weighted_action(sfx_ctx* ctx, const sfx_space* space, const double* kappa, const double* x,
                                        double* y, int nrhs, int accumulate, sfx_precision prec, void* stream);
sfx_status sfx_assemble_weighted_cell_matrices(sfx_ctx* ctx, const sfx_space* space, const double* kappa,
                                               int64_t cell_begin, int64_t cell_end, double* A, sfx_precision prec,
                                               void* stream);

/* Action of the linearised hyperelastic operator (the Jacobian of the
 * SFX_NEOHOOKE / SFX_SVK residual; Sec. 4.1 states the Saint Venant-Kirchhoff
 * law and times the assembly of this operator's matrices, Sec. 4.2 its action)
 * on vector Q_p:
 *   y_(a,j) = sum_K sum_q w_q S dP(F; dF) : (grad^ phi_j G) e_a,
 *   F = I + grad^u G (the state), dF = grad^du G (the direction),
 *   neo-Hookean dP = mu dF + (mu - lambda ln det F) F^{-T} dF^T F^{-T}
 *                    + lambda tr(F^{-1} dF) F^{-T};
 *   SVK dP = dF S + F (lambda tr(dE) I + 2 mu dE), dE = (dF^T F + F^T dF)/2.
 *   u    device, ndof doubles (one state, read-only)
 *   du   device, ndof x nrhs directions (read-only); y device, ndof x nrhs
 *        (must alias neither); accumulate as in sfx_assemble_action.
 * Deterministic colour-pass scatter.  A point with det F <= 0 (neo-Hookean)
 * contributes zero and sets SFX_DEV_DETF.  prec: FP64, or TF32X3 / BF16X3 for
 * the 1D contractions of both fields (u and du) on the tensor cores with the
 * geometry, F, dF, dP and the weight scaling in FP64.
 * Errors: SFX_ERR_ARG (null, aliasing, nrhs, family/form), SFX_ERR_CUDA. */
sfx_status sfx_assemble_linearised_action(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                          const sfx_space* space, const double* u, const double* du, double* y,
                                          int nrhs, int accumulate, sfx_precision prec, void* stream);

/* Per-cell vectors of the same operator (Sec. 4.1; no scatter) for the listed cells
 * (device int64, each in [0, ncell)), written to b (device, ncells x nloc x
 * nrhs).  Same arithmetic; errors as above. */
sfx_status sfx_assemble_linearised_cell_vectors(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                                const sfx_space* space, const double* u, const double* du,
                                                int nrhs, const int64_t* cells, int64_t ncells, double* b,
                                                sfx_precision prec, void* stream);

/* Element (tangent) matrices of the same operator at the state u: the
 * Jacobian of the cell residual, A^K = d b^K / d u_K, for cells
 * [cell_begin, cell_end) of the mesh:
 *   A^K_((a,i),(b,j)) = sum_q w_q S dP(F; e_b (x) grad^psi_j G) : (e_a (x) grad^psi_i G),
 * row = test (a,i), column = trial (b,j), local numbering component-major
 * (a * (p+1)^3 + i).  Column (b,j) is the per-cell vector of
 * sfx_assemble_linearised_cell_vectors for the unit local direction e_(b,j)
 * (bit for bit: same contractions).  Sum-factorised, O(p^7) per cell.
 *   u  device, ndof doubles (read-only)
 *   A  device, (cell_end - cell_begin) x nloc x nloc doubles, row-major per
 *      cell (nloc = 3 (p+1)^3; at p = 8, 38 MB per cell: callers chunk the range).
 * Cells with det J <= 0 get zero matrices and set SFX_DEV_INVERTED; points
 * with det F <= 0 (neo-Hookean) contribute zero and set SFX_DEV_DETF.
 * An empty range is a no-op (A may then be null).  FP64 only.
 * Errors: SFX_ERR_ARG (null, aliasing, family/form, range),
 * SFX_ERR_UNSUPPORTED (precision), SFX_ERR_CUDA. */
sfx_status sfx_assemble_linearised_cell_matrices(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                                 const sfx_space* space, const double* u, int64_t cell_begin,
                                                 int64_t cell_end, double* A, sfx_precision prec, void* stream);

/* Local element matrices A[c][j][i] (row = test j, column = trial i) of the
 * bilinear forms for cells [cell_begin, cell_end) (Sec. 3.2: argument
 * factorisation into P^(k,l) factors and sum factorisation, O(n^7) per cell;
 * Sec. 3.5 for the H(div)/H(curl) blocks).  A: device,
 * (cell_end - cell_begin) x nloc x nloc doubles.  algo NAIVE uses the dense
 * tabulation (O(n^9)).  Vector Q_p with the vector forms: the scalar block of
 * each cell (any algo available on Q_p) written to the three diagonal blocks,
 * the off-diagonal blocks zero (delta cancellation across the assignment,
 * Sec. 3.3); this path takes a stream-ordered scratch of at most 256 MB.
 * Errors: SFX_ERR_ARG (range, null, residual forms), SFX_ERR_UNSUPPORTED,
 * SFX_ERR_ALLOC (vector scratch), SFX_ERR_CUDA. */
sfx_status sfx_assemble_cell_matrices(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                      const sfx_space* space, int64_t cell_begin, int64_t cell_end,
                                      double* A, sfx_precision prec, sfx_algo algo, void* stream);

/* ------------------------------------------------------- assembled matrix */

/* Global sparse matrix of a scalar bilinear form (mass, Laplace, Helmholtz)
 * on Q_p or DQ_p in CSR format: A = sum_K P_K^T A^K P_K, the local tensors
 * added into the global matrix (Sec. 1.1), the assembled counterpart of the
 * matrix-free action that Sec. 4.2 compares with.
 * sfx_csr_create builds the sparsity pattern on the host (every pair of dofs
 * that share a cell; rows sorted; Q_p from the Kronecker product of the 1D
 * patterns of the structured mesh) and copies it to the device; it also holds
 * a device scratch for the element matrices of one chunk of cells (<= 512 MB).
 * Pattern: row_ptr int64 (nrows + 1), col int32 (nnz), host views owned by the
 * object.  With a host-only context only the host pattern is built.
 * Errors: SFX_ERR_ARG, SFX_ERR_UNSUPPORTED (family), SFX_ERR_ALLOC, SFX_ERR_CUDA. */
typedef struct sfx_csr sfx_csr;
sfx_status sfx_csr_create(const sfx_space* space, sfx_csr** out);
sfx_status sfx_csr_info(const sfx_csr* csr, int64_t* nrows, int64_t* nnz, const int64_t** row_ptr_host,
                        const int32_t** col_host);
/* Fill values (device, nnz doubles, caller-owned; overwritten) with the
 * assembled matrix of `form`: element matrices by sum factorisation (FP64, in
 * chunks), then a scatter colour by colour (conflict-free, deterministic).
 * Errors: SFX_ERR_ARG (null, form, host-only context), SFX_ERR_CUDA. */
sfx_status sfx_csr_assemble(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params, const sfx_csr* csr,
                            double* values, void* stream);
/* y = A x with the given values (device, nnz; the assembled operator that
 * Sec. 4.2 weighs against the matrix-free action); x, y device, nrows
 * doubles, must not alias.  A group of lanes per row, fixed-order reduction
 * (deterministic).  Errors: SFX_ERR_ARG, SFX_ERR_CUDA. */
sfx_status sfx_csr_spmv(sfx_ctx* ctx, const sfx_csr* csr, const double* values, const double* x, double* y,
                        void* stream);
void sfx_csr_destroy(sfx_csr* csr);

/* ----------------------------------------------- stored geometric factors */

/* Geometric factors at the quadrature points of every cell of a Q_p / DQ_p
 * space, computed once in FP64 (the argument-factorised P^(k,l) of Sec. 3.2
 * with weight and |J| folded in: P = w S G G^T, 6 symmetric entries, and w S)
 * and kept on the device, as double (SFX_QDATA_FP64) and/or float
 * (SFX_QDATA_FP32); 7 q^3 values per cell.  The stored actions read them
 * instead of recomputing J, det J and J^{-1} at every point: a trade of memory
 * traffic (56 or 28 bytes per point) for FP64 arithmetic, worthwhile when the
 * same operator is applied many times.  Synchronous.  The space must outlive
 * the factors.  Errors: SFX_ERR_ARG, SFX_ERR_UNSUPPORTED (family),
 * SFX_ERR_ALLOC, SFX_ERR_CUDA; an inverted cell sets SFX_DEV_INVERTED. */
typedef struct sfx_qdata sfx_qdata;
#define SFX_QDATA_FP64 1
#define SFX_QDATA_FP32 2
sfx_status sfx_qdata_create(sfx_ctx* ctx, const sfx_space* space, int formats, void* stream, sfx_qdata** out);
void sfx_qdata_destroy(sfx_qdata* qdata);

/* sfx_assemble_action for MASS / LAPLACE / HELMHOLTZ on the space of `qdata`
 * using the stored factors: prec FP64 needs SFX_QDATA_FP64 (same arithmetic as
 * the on-the-fly FP64 action), TF32X3 / BF16X3 need SFX_QDATA_FP32 (no FP64
 * geometry left in the kernel).  Other arguments and errors as
 * sfx_assemble_action. */
sfx_status sfx_assemble_action_stored(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                      const sfx_space* space, const sfx_qdata* qdata, const double* x, double* y,
                                      int nrhs, int accumulate, sfx_precision prec, void* stream);

/* ------------------------------------------------------------------ tuning */

/* Cells per CTA of the split-precision and FP64 action kernels, per kernel kind and degree
 * (1..8): 0 restores the built-in choice (for kinds 0-2 a table of the
 * autotuner's GB300 results; for kind 3 16 cells, 32 at p <= 2).  Kinds: 0 = FP64 (capped at the
 * 256-thread team limit, 256 / (p+1)^2), 1 = split precision with on-the-fly
 * geometry, 2 = split precision with stored factors, 3 = split-precision
 * hyperelastic residual (vector Q_p).  Every kernel reduces
 * the value further if its shared memory would not fit.  Values are chosen by
 * measurement (paper_1711_02473_gb300/autotune.py) and are process-wide.
 * Errors: SFX_ERR_ARG. */
sfx_status sfx_tune_set_cells_per_cta(int kernel, int degree, int cells);
sfx_status sfx_tune_get_cells_per_cta(int kernel, int degree, int* cells);

/* Kinds 6-10 of the table above: cells per CTA of the FP64 NCF / NCE actions
 * (6), the FP64 hyperelastic residual (7), the FP64 linearised hyperelastic
 * action (8), its split-precision version (9) and the split-precision NCF /
 * NCE actions (10); kind 11: cells per tile of the split-precision p-adaptive
 * batch (sfx_plan_create_padaptive_prec, at most its layout's count); 0 = the
 * launcher's rule
 * (the most cells for which two CTAs share an SM, else one larger CTA), and a
 * value that would not fit the kernel's team limit or shared memory is
 * reduced until it does.
 * Kind 5: cells per tile of the persistent p-adaptive
 * batch (sfx_plan_create_padaptive, sfx_padaptive_action_noalloc), at most the
 * count the kernel's shared-memory layout holds for that degree (larger values
 * are clamped); 0 = that count.  Takes effect for plans created afterwards.
 * Kind 4: cells per batch of the warp-specialised
 * split-precision action (0 = the launcher's choice: the most cells for
 * which two CTAs fit in one SM's shared memory).  That kernel computes the
 * Laplace and Helmholtz actions on Q_p / DQ_p, p >= 3, with geometry in the
 * flux (stored factors off): a persistent CTA whose producer warps build the
 * FP64 geometry factors of the next batch of cells while its consumer warps
 * run the tensor-core contractions, gathers and scatters of the current one.
 * Same arithmetic as the kernel kinds 1-2 use with staged factors.
 * sfx_tune_set_warp_specialised switches it per degree (1 = on; 0 = the kind-1
 * kernel; default on at p = 4, 5, 6, 8, where it measured faster on GB300).  Errors: SFX_ERR_ARG,
 * SFX_ERR_UNSUPPORTED (enable at p < 3). */
sfx_status sfx_tune_set_warp_specialised(int degree, int enable);
sfx_status sfx_tune_get_warp_specialised(int degree, int* enable);

/* ------------------------------------------------------------------ probes */

/* Throughput probes of the units the roofline divides by (no counterpart in
 * the paper: they measure this GPU).  One launch of `blocks` x `threads`
 * threads (threads a multiple of 32, <= 1024), each running `iters` rounds of
 * independent chains; `sink` (device, blocks*threads doubles, caller-owned)
 * receives one folded value per thread.  *ops receives the work of the
 * launch: FMAs for DFMA / FFMA (one FP64-pipe operation each for DFMA),
 * flops (2 M N K per mma) for the mma.sync forms.  Time it with CUDA events on
 * `stream`.  Errors: SFX_ERR_ARG, SFX_ERR_CUDA. */
typedef enum {
  SFX_PROBE_DFMA = 0,     /* FP64 FMA */
  SFX_PROBE_FFMA = 1,     /* FP32 FMA */
  SFX_PROBE_MMA_TF32 = 2, /* mma.sync m16n8k8 TF32, FP32 accumulate */
  SFX_PROBE_MMA_BF16 = 3, /* mma.sync m16n8k16 BF16, FP32 accumulate */
  SFX_PROBE_DMMA = 4      /* mma.sync m8n8k4 FP64 */
} sfx_probe_kind;
sfx_status sfx_probe_launch(int kind, int blocks, int threads, int iters, double* sink, void* stream, double* ops);

/* Poll limit of every bounded wait between the warp roles of one kernel
 * (mbarrier try_wait, each poll suspending for about 1 us; each wait also
 * gives up after 2 s).  A wait that gives up sets SFX_DEV_TIMEOUT; the kernel
 * still ends and its output is not valid.  Default 2^21; 0 makes every such
 * wait give up at once (for testing the timeout path).  Process-wide.
 * Errors: none. */
sfx_status sfx_set_wait_limit(uint32_t polls);

/* ------------------------------------------------------ batched execution */

/* A plan for repeated actions on a p-adaptive DQ mesh: cell c carries
 * DQ_{p_c} (1 <= p_c <= 8, Gauss nodes, cell-major numbering: cell c owns the
 * (p_c+1)^3 dofs starting at offset(c) = sum_{c' < c} (p_c'+1)^3), with up to 4
 * scalar forms (MASS / LAPLACE / HELMHOLTZ) applied to the same nrhs
 * right-hand sides.  Cells of different degree share no dofs, so the cells
 * are independent (no conforming hp constraints).
 *   degree   host, ncell int32 (copied);  forms/params host, nforms each
 *            (params may be NULL for the defaults).
 * The plan owns its tile list (cells sorted by degree, cut into one-CTA tiles,
 * largest degree first), a 4-byte tile counter and a private capture stream.
 * Errors: SFX_ERR_ARG, SFX_ERR_UNSUPPORTED (form), SFX_ERR_RANGE, SFX_ERR_ALLOC,
 * SFX_ERR_CUDA. */
typedef struct sfx_plan sfx_plan;
sfx_status sfx_plan_create_padaptive(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree, int nforms,
                                     const sfx_form* forms, const sfx_form_params* params, int nrhs,
                                     sfx_plan** out);
/* The same plan with the tile body in `prec`: FP64 (as above), or TF32X3 /
 * BF16X3, whose tiles run the split-precision scalar body (the 1D
 * contractions as split tensor-core products with FP32 accumulation; the
 * geometry, weight scaling and scatter in FP64; Sec. 3.3 with the
 * precision choice of sfx_assemble_action).  Its tile sizes are those of that
 * body's shared-memory layout for the plan's forms; kind 11 of
 * sfx_tune_set_cells_per_cta sets smaller ones.  PER_LAUNCH mode then runs one
 * launch per (form, degree) with all right-hand sides.  Errors as above, and
 * SFX_ERR_ARG for another precision. */
sfx_status sfx_plan_create_padaptive_prec(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree, int nforms,
                                          const sfx_form* forms, const sfx_form_params* params, int nrhs,
                                          sfx_precision prec, sfx_plan** out);
/* Total dofs, number of tiles and a host view of the ncell+1 dof offsets. */
sfx_status sfx_plan_info(const sfx_plan* plan, int64_t* ndof, int64_t* ntiles, const int64_t** cell_offset);

/* GRAPH: every tile of every form and all right-hand sides in ONE persistent
 * kernel launch (CTAs take tiles from the counter), captured once into a CUDA
 * graph per (x, y) pointer set and replayed.  PER_LAUNCH: one launch per
 * (form, degree, right-hand side), for comparison.
 *   x   device, ndof x nrhs;  y  host array of nforms device pointers, each
 *       ndof x nrhs (overwritten).
 * Launches of one plan must not overlap on the device (they share the tile
 * counter).  Errors: SFX_ERR_ARG, SFX_ERR_CUDA. */
typedef enum { SFX_EXEC_GRAPH = 0, SFX_EXEC_PER_LAUNCH = 1 } sfx_exec_mode;
sfx_status sfx_plan_execute(sfx_plan* plan, const double* x, double* const* y, sfx_exec_mode mode, void* stream);
void sfx_plan_destroy(sfx_plan* plan);

/* ------------------------------------------------- action without allocation */

/* The p-adaptive DQ action of one scalar form for callers that cannot
 * allocate device memory when they need it (a memory pool owns the device,
 * allocation is allowed only at start-up, or a solve phase forbids it).  It
 * does what sfx_plan_execute(GRAPH) does for one form, but builds the
 * degree-sorted cell list and tile list on the device, in a fixed scratch
 * array inside the library, and calls no cudaMalloc, cudaFree or allocating
 * routine.  The paper has no counterpart: this is an interface for callers.
 *   degree       device, ncell int32, each in 1..8
 *   cell_offset  device, ncell+1 int64: cell c owns dofs [off[c], off[c+1]),
 *                off[0] = 0, off[c+1] - off[c] = (degree[c]+1)^3
 *   x, y         device, ndof x nrhs with ndof = off[ncell] (y overwritten);
 *                1 <= nrhs <= 64
 * A cell whose degree or offsets break these rules is checked on the device,
 * flagged SFX_DEV_BADCELL (read it with sfx_sync_status) and skipped: its
 * block of y is left as it was, and no access goes through its offsets.
 * Limit: ncell <= 262144 (SFX_ERR_RANGE beyond).  The scratch (about 5 MB) is
 * a static device array that every GPU loading the library holds until exit;
 * it keeps the last call's contents, and the call clears what must start at
 * zero.  All calls share it, so calls that overlap on the GPU (different
 * streams, or threads) race: serialise them.  The first call on a device, with
 * that device current, looks up the scratch address and uploads the 1D
 * tables; make that first call before any stream capture.
 * Errors: SFX_ERR_ARG (also: ctx's device is not the current device; this is
 * checked on every call), SFX_ERR_UNSUPPORTED (form), SFX_ERR_RANGE,
 * SFX_ERR_CUDA. */
sfx_status sfx_padaptive_action_noalloc(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree,
                                        const int64_t* cell_offset, sfx_form form, const sfx_form_params* params,
                                        const double* x, double* y, int nrhs, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SFX_H */
