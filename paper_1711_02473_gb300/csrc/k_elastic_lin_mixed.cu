// k_elastic_lin_mixed.cu -- action of the linearised hyperelastic operator
// K(u) du on vector Q_p (neo-Hookean and Saint Venant-Kirchhoff) with the 1D
// contractions as split-precision tensor-core products (TF32x3 or BF16x3,
// FP32 accumulation).  This is the operator whose action the paper's
// hyperelastic experiments time (Sec. 4.1).
//
// Same algorithm as k_elastic_lin.cu (Sec. 3.3, Eqs. coeff_eval and
// form_eval, sum-factorised as in Sec. 3.2): per component a, interpolation to
// the Gauss points with B along x, y, z and the reference gradient with the
// collocation derivative Dq, for the state u (once per cell) and for each
// direction du; pointwise F = I + grad^u G, dF = grad^du G, the linearised
// stress dP(F; dF) and the test flux w dP adj(J)^T; then Dq^T and B^T back to
// the nodes.  Precision split:
//   - the 3 x 12 one-dimensional contractions per field run in tc_contract,
//     batched over all cells of the CTA;
//   - J, adj J, det J, F, dF, det F, ln det F, dP and the weight scaling run in
//     FP64 from the FP32 gradients (widened exactly); the flux is rounded once
//     to FP32 for the transposed contractions;
//   - the nodal result is widened to FP64 and added into y in FP64.
// Shared memory per cell: the state's nine gradient arrays Hs[a][k] and the
// direction's Hd[a][k] (FP32, n^3 each); component a's gather and
// interpolation live in Hd[a][2] (or Hs[a][2]), so no scratch array is needed.
#include "elastic_common.cuh"
#include "mixed_common.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_elastic_lin_mixed)

namespace {

template <int N>
struct LMShape {
  static constexpr int N2 = N * N, N3 = N2 * N;
  static constexpr int cellf = 18 * N3;       // Hs[9][cell][qp], Hd[9][cell][qp]
  static constexpr int celld = 24 + 9 * N2;   // corners + Jacobian column tables
  static constexpr size_t fixed_bytes() { return 2 * sizeof(TabF) + (N3 + 16) * 8; }
  static constexpr size_t bytes(int cb) {
    return fixed_bytes() + (size_t)cb * celld * 8 + (size_t)cb * cellf * 4 + (size_t)cb * 8 + 16;
  }
};

// Reference gradient of component `comp` of a field (x, stride nrhs, column
// r) into G[comp*3 + k] (k = 0, 1, 2) for every cell of the CTA: gather into
// G[comp*3+2], B along x, y, z in place, then Dq along each axis.
template <int N, int PREC>
__device__ __forceinline__ void mixed_component_gradient(const ActArgs& a, const double* x, int nrhs, int r, int comp,
                                                         const int* flags, int cb, const TabF* tabs, float* G,
                                                         int stride) {
  constexpr int N3 = N * N * N;
  float* G0 = G + (comp * 3 + 0) * stride;
  float* G1 = G0 + stride;
  float* G2 = G1 + stride;
  for (int i = threadIdx.x; i < cb * N3; i += kThreads) {
    const int c = i / N3, l = i - c * N3;
    const int cell = flags[2 * c];
    const bool ok = cell >= 0 && !flags[2 * c + 1];
    G2[i] = ok ? d2f_int(x[(int64_t)a.map[(int64_t)cell * 3 * N3 + comp * N3 + l] * nrhs + r]) : 0.f;
  }
  __syncthreads();
  tc_contract<N, 0, false, false, PREC>(G2, G2, tabs[0], cb);
  __syncthreads();
  tc_contract<N, 1, false, false, PREC>(G2, G2, tabs[0], cb);
  __syncthreads();
  tc_contract<N, 2, false, false, PREC>(G2, G2, tabs[0], cb);
  __syncthreads();
  tc_contract<N, 0, false, false, PREC>(G2, G0, tabs[1], cb);
  tc_contract<N, 1, false, false, PREC>(G2, G1, tabs[1], cb);
  __syncthreads();
  tc_contract<N, 2, false, false, PREC>(G2, G2, tabs[1], cb);
  __syncthreads();
}

template <int N, bool NEO, int PREC>
__global__ void __launch_bounds__(kThreads) k_linearised_elastic_mixed(const ActArgs a, const int64_t ncell_total,
                                                                       const int cb) {
  using Sh = LMShape<N>;
  constexpr int N2 = Sh::N2, N3 = Sh::N3;
  const Tab1D& T = c_tab[N - 1];
  extern __shared__ double smd[];
  // layout: [tables: 2 TabF][W3: N3 doubles][xq: 16 doubles][cells: doubles][Hs, Hd floats][flags]
  TabF* tabs = reinterpret_cast<TabF*>(smd);  // 0: B, 1: Dq
  double* W3 = smd + (2 * sizeof(TabF)) / 8;
  double* xq = W3 + N3;
  double* cd = xq + 16;
  float* Hs = reinterpret_cast<float*>(cd + (size_t)cb * Sh::celld);
  const int stride = cb * N3;  // distance between the gradient arrays
  float* Hd = Hs + 9 * stride;
  int* flags = reinterpret_cast<int*>(Hd + 9 * stride);  // per cell: id or -1, bad

  const int tid = threadIdx.x;
  for (int i = tid; i < 16 * 16; i += kThreads) {
    const int r = i / 16, k = i % 16;
    tabs[0].v[r][k] = (r < N && k < N) ? (float)T.Bc[r][k] : 0.f;
    tabs[1].v[r][k] = (r < N && k < N) ? (float)T.Dq[r][k] : 0.f;
  }
  for (int i = tid; i < N3; i += kThreads) W3[i] = T.w[i / N2] * T.w[(i / N) % N] * T.w[i % N];
  if (tid < N) xq[tid] = T.x[tid];
  for (int c = tid; c < cb; c += kThreads) {
    int cell = -1;
    if (!slot_cell(a, (int64_t)blockIdx.x * cb + c, ncell_total, &cell)) cell = -1;
    flags[2 * c] = cell;
    flags[2 * c + 1] = 0;
  }
  __syncthreads();
  for (int i = tid; i < cb * 24; i += kThreads) {
    const int c = i / 24, v = (i % 24) / 3, k = i % 3;
    const int cell = flags[2 * c];
    double* X = cd + (size_t)c * Sh::celld;
    X[v * 3 + k] = cell >= 0 ? a.xyz[(int64_t)a.vmap[(int64_t)cell * 8 + v] * 3 + k] : (double)((v >> (2 - k)) & 1);
  }
  __syncthreads();
  for (int i = tid; i < cb * N2; i += kThreads) {
    const int c = i / N2, t = i - c * N2;
    double* X = cd + (size_t)c * Sh::celld;
    jacobian_columns<N>(reinterpret_cast<const double(*)[3]>(X), xq, reinterpret_cast<double(*)[N2][3]>(X + 24), t);
  }
  __syncthreads();
  // a cell with det J <= 0 at any Gauss point contributes nothing
  for (int i = tid; i < cb * N3; i += kThreads) {
    const int c = i / N3, qp = i - c * N3;
    const double(*Jc)[N2][3] = reinterpret_cast<const double(*)[N2][3]>(cd + (size_t)c * Sh::celld + 24);
    double r0[3];
    cross3(Jc[1][(qp / N2) * N + qp % N], Jc[2][(qp / N2) * N + (qp / N) % N], r0);
    if (!(dot3(Jc[0][qp % N2], r0) > 0.0)) flags[2 * c + 1] = 1;
  }
  __syncthreads();
  for (int c = tid; c < cb; c += kThreads)
    if (flags[2 * c] >= 0 && flags[2 * c + 1]) set_flag(a.status, SFX_DEV_INVERTED);
  const double mu = a.mu, lam = a.lambda;
  // the state's reference gradient, once per cell
#pragma unroll 1
  for (int comp = 0; comp < 3; ++comp)
    mixed_component_gradient<N, PREC>(a, a.xs, 1, 0, comp, flags, cb, tabs, Hs, stride);

#pragma unroll 1
  for (int r = 0; r < a.nrhs; ++r) {
#pragma unroll 1
    for (int comp = 0; comp < 3; ++comp)
      mixed_component_gradient<N, PREC>(a, a.x, a.nrhs, r, comp, flags, cb, tabs, Hd, stride);
    // pointwise, FP64: the linearised stress and the test flux w dP adj(J)^T
    for (int i = tid; i < cb * N3; i += kThreads) {
      const int c = i / N3, qp = i - c * N3;
      const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
      const double(*Jc)[N2][3] = reinterpret_cast<const double(*)[N2][3]>(cd + (size_t)c * Sh::celld + 24);
      const double* c0 = Jc[0][q2 * N + q3];
      const double* c1 = Jc[1][q1 * N + q3];
      const double* c2 = Jc[2][q1 * N + q2];
      double R[3][3];  // rows of adj(J) = S G
      cross3(c1, c2, R[0]);
      cross3(c2, c0, R[1]);
      cross3(c0, c1, R[2]);
      const double S = dot3(c0, R[0]);
      double Hsq[3][3], Hdq[3][3], flux[3][3];
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        Hsq[j / 3][j % 3] = f2d_int(Hs[j * stride + i]);
        Hdq[j / 3][j % 3] = f2d_int(Hd[j * stride + i]);
      }
      const bool ok = flags[2 * c] >= 0 && !flags[2 * c + 1];
      if (!linearised_flux<NEO>(Hsq, Hdq, R, S, W3[qp], mu, lam, flux) && ok) set_flag(a.status, SFX_DEV_DETF);
#pragma unroll
      for (int j = 0; j < 9; ++j) Hd[j * stride + i] = ok ? d2f_int(flux[j / 3][j % 3]) : 0.f;
    }
    __syncthreads();
#pragma unroll 1
    for (int comp = 0; comp < 3; ++comp) {
      float* H0 = Hd + (comp * 3 + 0) * stride;
      float* H1 = H0 + stride;
      float* H2 = H1 + stride;
      tc_contract<N, 2, true, false, PREC>(H2, H2, tabs[1], cb);
      __syncthreads();
      tc_contract<N, 0, true, true, PREC>(H0, H2, tabs[1], cb);
      __syncthreads();
      tc_contract<N, 1, true, true, PREC>(H1, H2, tabs[1], cb);
      __syncthreads();
      tc_contract<N, 0, true, false, PREC>(H2, H2, tabs[0], cb);
      __syncthreads();
      tc_contract<N, 1, true, false, PREC>(H2, H2, tabs[0], cb);
      __syncthreads();
      tc_contract<N, 2, true, false, PREC>(H2, H2, tabs[0], cb);
      __syncthreads();
      for (int i = tid; i < cb * N3; i += kThreads) {
        const int c = i / N3, l = i - c * N3;
        const int cell = flags[2 * c];
        if (cell < 0) continue;
        const bool ok = !flags[2 * c + 1];
        const int64_t slot = (int64_t)blockIdx.x * cb + c;
        if (a.cell_vectors) {
          a.y[(slot * 3 * N3 + comp * N3 + l) * a.nrhs + r] = ok ? f2d_int(H2[i]) : 0.0;
        } else if (ok) {
          // reduction in L2 (red.global.add.f64): a launch adds to each address once
          atomicAdd(&a.y[(int64_t)a.map[(int64_t)cell * 3 * N3 + comp * N3 + l] * a.nrhs + r], f2d_int(H2[i]));
        }
      }
    }
    __syncthreads();
  }
}

template <int N, bool NEO, int PREC>
int launch_lm(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  using Sh = LMShape<N>;
  const size_t budget = 110 * 1024;  // two CTAs per SM
  int cb = (N <= 3) ? 16 : 8;
  while (cb > 1 && Sh::bytes(cb) > budget) --cb;
  cb = tuned_team_cells(SFX_TUNE_LINEARISED_MIXED, N - 1, cb, 64, Sh::bytes(0), Sh::bytes(1) - Sh::bytes(0),
                        200 * 1024);
  const size_t smem = Sh::bytes(cb);
  if (smem > 227 * 1024) return -1;
  auto kern = k_linearised_elastic_mixed<N, NEO, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  const int64_t grid = (a.ncells + cb - 1) / cb;
  kern<<<(unsigned)grid, kThreads, smem, s>>>(a, ncell_total, cb);
  return (int)cudaGetLastError();
}

template <bool NEO, int PREC>
int dispatch_p(int p, const ActArgs& a, int64_t nc, cudaStream_t s) {
  switch (p) {
    case 1: return launch_lm<2, NEO, PREC>(a, nc, s);
    case 2: return launch_lm<3, NEO, PREC>(a, nc, s);
    case 3: return launch_lm<4, NEO, PREC>(a, nc, s);
    case 4: return launch_lm<5, NEO, PREC>(a, nc, s);
    case 5: return launch_lm<6, NEO, PREC>(a, nc, s);
    case 6: return launch_lm<7, NEO, PREC>(a, nc, s);
    case 7: return launch_lm<8, NEO, PREC>(a, nc, s);
    case 8: return launch_lm<9, NEO, PREC>(a, nc, s);
  }
  return -1;
}

template <int PREC>
int dispatch_law(sfx_form form, int p, const ActArgs& a, int64_t nc, cudaStream_t s) {
  if (form == SFX_NEOHOOKE) return dispatch_p<true, PREC>(p, a, nc, s);
  if (form == SFX_SVK) return dispatch_p<false, PREC>(p, a, nc, s);
  return -1;
}

}  // namespace

int launch_linearised_elastic_mixed(const sfx_space* sp, sfx_form form, sfx_precision prec, const ActArgs& a,
                                    void* stream) {
  if (sp->family != SFX_VQ || a.unit_cols > 0) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nc = sp->mesh->ncell;
  if (prec == SFX_PREC_TF32X3) return dispatch_law<SFX_PREC_TF32X3>(form, sp->p, a, nc, s);
  if (prec == SFX_PREC_BF16X3) return dispatch_law<SFX_PREC_BF16X3>(form, sp->p, a, nc, s);
  return -1;
}

}  // namespace sfx
