// sfx_host.cpp -- host side of the C ABI: contexts, meshes, spaces (dof maps,
// colouring), 1D tabulation, argument validation and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <unordered_map>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>

#include "sfx_internal.h"

#include <nvtx3/nvToolsExt.h>

using namespace sfx;

namespace {

// Named range around a library entry point, for profilers and tracers (NVTX;
// a no-op unless a tool is attached to the process).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

template <class T>
sfx_status to_device(const T* h, size_t n, T** d) {
  *d = nullptr;
  if (n == 0) return SFX_OK;
  if (cudaMalloc((void**)d, n * sizeof(T)) != cudaSuccess) { *d = nullptr; return SFX_ERR_ALLOC; }
  if (cudaMemcpy(*d, h, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(*d); *d = nullptr; return SFX_ERR_CUDA;
  }
  return SFX_OK;
}

// SplitMix64 draw k of stream `seed` (Steele, Lea & Flood 2014, counter form).
inline uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Legendre P_n and P_n' at t by the three-term recurrence.
void legendre(int n, double t, double* P, double* dP) {
  double p0 = 1.0, p1 = t;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (t * p1 - p0) / (t * t - 1.0);  // valid for |t| < 1
}

bool family_ok(sfx_family f) { return f >= SFX_Q && f <= SFX_VQ; }
bool form_ok(sfx_family fam, sfx_form form) {
  switch (form) {
    case SFX_MASS: case SFX_LAPLACE: case SFX_HELMHOLTZ: return fam == SFX_Q || fam == SFX_DQ || fam == SFX_VQ;
    case SFX_NCF_MASS_DIVDIV: return fam == SFX_NCF;
    case SFX_NCE_CURLCURL: return fam == SFX_NCE;
    case SFX_NEOHOOKE: case SFX_SVK: return fam == SFX_VQ;
  }
  return false;
}

sfx_form_params default_params(sfx_form form) {
  switch (form) {
    case SFX_HELMHOLTZ: return {1.0, -1.0, 0.0, 0.0};
    case SFX_NCF_MASS_DIVDIV: return {1.0, 1.0, 0.0, 0.0};
    case SFX_NCE_CURLCURL: return {0.0, 1.0, 0.0, 0.0};
    case SFX_NEOHOOKE: case SFX_SVK: return {0.0, 0.0, 1.0, 10.0};
    default: return {0.0, 0.0, 0.0, 0.0};
  }
}

}  // namespace

// ------------------------------------------------------------------ 1D rules
namespace sfx {

void gauss_legendre(int n, double* x, double* w) {
  // roots of P_n by Newton from the asymptotic guesses cos(pi (i + 3/4)/(n + 1/2))
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    legendre(n, t, &P, &dP);
    // ascending order on [0,1]
    x[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dP * dP);  // 2/((1-t^2)P'^2) halved
  }
}

void gauss_lobatto(int n, double* x, double* w) {
  // interior nodes: roots of g(t) = P_{m-1}(t) - t P_m(t) (proportional to
  // (1-t^2) P_m'(t)), m = n-1, by Newton from Chebyshev-Lobatto guesses.
  int m = n - 1;
  x[0] = 0.0;
  x[n - 1] = 1.0;
  for (int i = 1; i < n - 1; ++i) {
    double t = -std::cos(M_PI * i / m);
    for (int it = 0; it < 100; ++it) {
      double Pm, dPm, Pm1, dPm1;
      legendre(m, t, &Pm, &dPm);
      legendre(m - 1, t, &Pm1, &dPm1);
      double g = Pm1 - t * Pm;
      double dg = dPm1 - Pm - t * dPm;
      double dt = g / dg;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    x[i] = 0.5 * (t + 1.0);
  }
  for (int i = 0; i < n; ++i) {
    double t = 2.0 * x[i] - 1.0, P, dP;
    if (i == 0 || i == n - 1) {
      P = (i == 0 && (m % 2)) ? -1.0 : 1.0;
    } else {
      legendre(m, t, &P, &dP);
    }
    w[i] = 1.0 / (n * (n - 1.0) * P * P);  // 2/(n(n-1)P_m^2) halved
  }
}

// Barycentric Lagrange evaluation (Berrut & Trefethen 2004): values or first
// derivatives of the n basis functions on `nodes` at q points.
void lagrange_table(const double* nodes, int n, const double* pts, int q, int deriv, double* out) {
  double lam[64];
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= nodes[j] - nodes[k];
    lam[j] = 1.0 / prod;
  }
  for (int a = 0; a < q; ++a) {
    double t = pts[a];
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (t == nodes[j]) hit = j;
    double* row = out + (size_t)a * n;
    if (hit >= 0) {
      for (int j = 0; j < n; ++j) {
        if (!deriv) { row[j] = (j == hit) ? 1.0 : 0.0; continue; }
        if (j != hit) {
          row[j] = (lam[j] / lam[hit]) / (nodes[hit] - nodes[j]);
        } else {
          double s = 0.0;
          for (int k = 0; k < n; ++k)
            if (k != hit) s += 1.0 / (nodes[hit] - nodes[k]);
          row[j] = s;
        }
      }
      continue;
    }
    double den = 0.0, s = 0.0;
    for (int k = 0; k < n; ++k) {
      den += lam[k] / (t - nodes[k]);
      s += 1.0 / (t - nodes[k]);
    }
    for (int j = 0; j < n; ++j) {
      double l = (lam[j] / (t - nodes[j])) / den;
      row[j] = deriv ? l * (s - 1.0 / (t - nodes[j])) : l;
    }
  }
}

void make_tab1d(int p, Tab1D* t) {
  std::memset(t, 0, sizeof(*t));
  int n = p + 1, q = p + 1;
  t->p = p;
  t->q = q;
  gauss_legendre(q, t->x, t->w);
  double xc[kMaxN], wc[kMaxN], xd[kMaxN], wd[kMaxN], tmp[kMaxQ * kMaxN];
  gauss_lobatto(n, xc, wc);
  lagrange_table(xc, n, t->x, q, 0, tmp);
  for (int a = 0; a < q; ++a) for (int j = 0; j < n; ++j) t->Bc[a][j] = tmp[a * n + j];
  lagrange_table(xc, n, t->x, q, 1, tmp);
  for (int a = 0; a < q; ++a) for (int j = 0; j < n; ++j) t->Dc[a][j] = tmp[a * n + j];
  gauss_legendre(p, xd, wd);
  lagrange_table(xd, p, t->x, q, 0, tmp);
  for (int a = 0; a < q; ++a) for (int j = 0; j < p; ++j) t->Bd[a][j] = tmp[a * p + j];
  lagrange_table(xd, p, t->x, q, 1, tmp);
  for (int a = 0; a < q; ++a) for (int j = 0; j < p; ++j) t->Dd[a][j] = tmp[a * p + j];
  lagrange_table(t->x, q, t->x, q, 1, tmp);
  for (int a = 0; a < q; ++a) for (int j = 0; j < q; ++j) t->Dq[a][j] = tmp[a * q + j];
  // collocated Gauss-Lobatto rule on the GLL nodes
  for (int a = 0; a < n; ++a) { t->xg[a] = xc[a]; t->wg[a] = wc[a]; }
  lagrange_table(xc, n, xc, n, 1, tmp);
  for (int a = 0; a < n; ++a) for (int j = 0; j < n; ++j) t->Dg[a][j] = tmp[a * n + j];
}

}  // namespace sfx

// Copy the 1D tables of one degree into every kernel file's constant memory.
static int upload_tables(const Tab1D* t) {
  int e = upload_tab_scalar(t);
  if (!e) e = upload_tab_scalar_mixed_tf32(t);
  if (!e) e = upload_tab_scalar_mixed_bf16(t);
  if (!e) e = upload_tab_scalar_mixed_ws_tf32(t);
  if (!e) e = upload_tab_scalar_mixed_ws_bf16(t);
  if (!e) e = upload_tab_qdata(t);
  if (!e) e = upload_tab_hdivcurl(t);
  if (!e) e = upload_tab_hdivcurl_mixed_tf32(t);
  if (!e) e = upload_tab_hdivcurl_mixed_bf16(t);
  if (!e) e = upload_tab_batched_mixed_tf32(t);
  if (!e) e = upload_tab_batched_mixed_bf16(t);
  if (!e) e = upload_tab_elastic(t);
  if (!e) e = upload_tab_elastic_mixed(t);
  if (!e) e = upload_tab_matrix(t);
  if (!e) e = upload_tab_naive(t);
  if (!e) e = upload_tab_batched(t);
  if (!e) e = upload_tab_scalar_coll(t);
  if (!e) e = upload_tab_scalar_mixed_coll(t);
  if (!e) e = upload_tab_elastic_lin(t);
  if (!e) e = upload_tab_elastic_lin_mixed(t);
  if (!e) e = upload_tab_scalar_kappa(t);
  return e;
}

namespace sfx {
// Tables of every degree into every kernel file (used by the no-alloc entry
// point, which has no space or plan to trigger the upload).
int upload_all_tables() {
  for (int p = 1; p <= kMaxDeg; ++p) {
    Tab1D t;
    make_tab1d(p, &t);
    if (upload_tables(&t) != 0) return 1;
  }
  return 0;
}
}  // namespace sfx

// ------------------------------------------------------------------- tuning
namespace {
int g_tune[SFX_TUNE_NKERNEL][kMaxDeg + 1] = {{0}};
// Built-in cells per CTA by degree 1..8: the autotuner's choice on GB300
// (Q_p Laplace, 32^3 tuning mesh), the same in repeated tunings up to one
// entry.  0 = the launcher's own default.
constexpr int kBuiltinCells[SFX_TUNE_NKERNEL][kMaxDeg + 1] = {
    {0, 16, 7, 2, 10, 7, 5, 4, 3},  // FP64
    {0, 8, 6, 8, 4, 4, 2, 2, 2},    // split precision, geometry at the point
    {0, 8, 6, 6, 6, 3, 3, 3, 3},    // split precision, stored factors
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // split-precision hyperelastic residual
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // warp-specialised split precision (launcher default)
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // p-adaptive batch tiles (the layout's full count)
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // FP64 NCF / NCE actions (launcher's shared-memory rule)
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // FP64 hyperelastic residual (same)
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // FP64 linearised hyperelastic action (same)
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // split-precision linearised hyperelastic action (same)
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // split-precision NCF / NCE actions (same)
    {0, 0, 0, 0, 0, 0, 0, 0, 0},    // split-precision p-adaptive batch tiles (the layout's full count)
};
// by degree (needs n = p + 1 >= 4): on where it measured faster than the
// one-role kernel on the 64^3 Laplace and Helmholtz actions (p = 4, 5, 6, 8:
// 4-14% on Q_p); at p = 3 and 7 the two are within a few per cent either way
int g_ws[kMaxDeg + 1] = {0, 0, 0, 0, 1, 1, 1, 0, 1};
uint32_t g_wait_cap = 1u << 21;
}
namespace sfx {
bool ws_enabled(int degree) { return degree >= 3 && degree <= kMaxDeg && g_ws[degree] != 0; }
uint32_t ws_wait_cap() { return g_wait_cap; }
int tuned_team_cells(int kernel, int degree, int fallback, int maxcb, size_t fixed, size_t per_cell, size_t limit) {
  const int t = kernel >= 0 && kernel < SFX_TUNE_NKERNEL && degree >= 1 && degree <= kMaxDeg ? g_tune[kernel][degree] : 0;
  if (t <= 0) return fallback;
  int cb = t < maxcb ? t : maxcb;
  while (cb > 1 && fixed + (size_t)cb * per_cell > limit) --cb;
  return cb;
}
int tuned_cells_per_cta(int kernel, int degree, int fallback) {
  if (kernel < 0 || kernel >= SFX_TUNE_NKERNEL || degree < 1 || degree > kMaxDeg) return fallback;
  if (g_tune[kernel][degree] > 0) return g_tune[kernel][degree];
  if (kBuiltinCells[kernel][degree] > 0) return kBuiltinCells[kernel][degree];
  return fallback;
}
}  // namespace sfx

extern "C" sfx_status sfx_tune_set_cells_per_cta(int kernel, int degree, int cells) {
  if (kernel < 0 || kernel >= SFX_TUNE_NKERNEL || degree < 1 || degree > kMaxDeg || cells < 0 || cells > 64)
    return SFX_ERR_ARG;
  g_tune[kernel][degree] = cells;
  return SFX_OK;
}

extern "C" sfx_status sfx_tune_set_warp_specialised(int degree, int enable) {
  if (degree < 1 || degree > kMaxDeg || (enable != 0 && enable != 1)) return SFX_ERR_ARG;
  if (enable && degree < 3) return SFX_ERR_UNSUPPORTED;
  g_ws[degree] = enable;
  return SFX_OK;
}

extern "C" sfx_status sfx_tune_get_warp_specialised(int degree, int* enable) {
  if (degree < 1 || degree > kMaxDeg || !enable) return SFX_ERR_ARG;
  *enable = ws_enabled(degree) ? 1 : 0;
  return SFX_OK;
}

extern "C" sfx_status sfx_set_wait_limit(uint32_t polls) {
  g_wait_cap = polls;
  return SFX_OK;
}

extern "C" sfx_status sfx_tune_get_cells_per_cta(int kernel, int degree, int* cells) {
  if (kernel < 0 || kernel >= SFX_TUNE_NKERNEL || degree < 1 || degree > kMaxDeg || !cells) return SFX_ERR_ARG;
  *cells = g_tune[kernel][degree];
  return SFX_OK;
}

// ------------------------------------------------------------------ context
extern "C" sfx_status sfx_ctx_create(int device, sfx_ctx** out) {
  if (!out || device < -1) return SFX_ERR_ARG;
  *out = nullptr;
  sfx_ctx* c = new (std::nothrow) sfx_ctx;
  if (!c) return SFX_ERR_ALLOC;
  c->device = device;
  if (device < 0) {  // host-only: meshes and spaces without device copies
    *out = c;
    return SFX_OK;
  }
  if (cudaSetDevice(device) != cudaSuccess) { delete c; return SFX_ERR_CUDA; }
  if (cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess) { delete c; return SFX_ERR_ALLOC; }
  if (cudaMemset(c->d_status, 0, sizeof(uint32_t)) != cudaSuccess) {
    cudaFree(c->d_status); delete c; return SFX_ERR_CUDA;
  }
  *out = c;
  return SFX_OK;
}

extern "C" void sfx_ctx_destroy(sfx_ctx* c) {
  if (!c) return;
  if (c->d_status) cudaFree(c->d_status);
  delete c;
}

extern "C" sfx_status sfx_sync_status(sfx_ctx* c, void* stream, uint32_t* bits) {
  if (!c || !bits || c->device < 0) return SFX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t h = 0;
  if (cudaMemcpyAsync(&h, c->d_status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SFX_ERR_CUDA;
  if (cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), s) != cudaSuccess) return SFX_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SFX_ERR_CUDA;
  *bits = h;
  return SFX_OK;
}

extern "C" const char* sfx_status_string(sfx_status s) {
  switch (s) {
    case SFX_OK: return "ok";
    case SFX_ERR_ARG: return "invalid argument";
    case SFX_ERR_UNSUPPORTED: return "unsupported combination";
    case SFX_ERR_CUDA: return "CUDA runtime error";
    case SFX_ERR_ALLOC: return "allocation failed";
    case SFX_ERR_RANGE: return "size exceeds 32-bit indexing";
  }
  return "unknown status";
}

// --------------------------------------------------------------------- mesh
static sfx_status mesh_finish(sfx_mesh* m) {
  if (!m->general) {
    const int ny = m->ny, nz = m->nz;
    try { m->vmap.resize((size_t)m->ncell * 8); } catch (...) { return SFX_ERR_ALLOC; }
    for (int64_t c = 0; c < m->ncell; ++c) {
      int64_t k = c % nz, j = (c / nz) % ny, i = c / ((int64_t)ny * nz);
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
          for (int cc = 0; cc < 2; ++cc)
            m->vmap[c * 8 + 4 * a + 2 * b + cc] =
                (int32_t)(((i + a) * (ny + 1) + (j + b)) * (int64_t)(nz + 1) + (k + cc));
    }
  }
  if (m->ctx->device < 0) return SFX_OK;
  sfx_status st = to_device(m->xyz.data(), m->xyz.size(), &m->d_xyz);
  if (st) return st;
  return to_device(m->vmap.data(), m->vmap.size(), &m->d_vmap);
}

static sfx_status mesh_alloc(sfx_ctx* ctx, int nx, int ny, int nz, sfx_mesh** out) {
  if (!ctx || !out || nx < 1 || ny < 1 || nz < 1) return SFX_ERR_ARG;
  *out = nullptr;
  int64_t nvert = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  if (nvert > 2000000000LL) return SFX_ERR_RANGE;
  sfx_mesh* m = new (std::nothrow) sfx_mesh;
  if (!m) return SFX_ERR_ALLOC;
  m->ctx = ctx;
  m->nx = nx; m->ny = ny; m->nz = nz;
  m->nvert = nvert;
  m->ncell = (int64_t)nx * ny * nz;
  try { m->xyz.resize((size_t)nvert * 3); } catch (...) { delete m; return SFX_ERR_ALLOC; }
  *out = m;
  return SFX_OK;
}

extern "C" sfx_status sfx_mesh_create_box(sfx_ctx* ctx, int nx, int ny, int nz, double perturb, uint64_t seed,
                                          sfx_mesh** out) {
  if (!(std::fabs(perturb) < 0.5)) return SFX_ERR_ARG;
  sfx_mesh* m;
  sfx_status st = mesh_alloc(ctx, nx, ny, nz, &m);
  if (st) return st;
  const double h[3] = {1.0 / nx, 1.0 / ny, 1.0 / nz};
  uint64_t draw = 0;
  for (int64_t I = 0; I <= nx; ++I)
    for (int64_t J = 0; J <= ny; ++J)
      for (int64_t K = 0; K <= nz; ++K) {
        double* v = &m->xyz[(size_t)(((I * (ny + 1) + J) * (nz + 1) + K) * 3)];
        v[0] = (double)I / nx;
        v[1] = (double)J / ny;
        v[2] = (double)K / nz;
        bool interior = I > 0 && I < nx && J > 0 && J < ny && K > 0 && K < nz;
        if (interior && perturb != 0.0) {
          for (int d = 0; d < 3; ++d) {
            double u = (double)(splitmix64_at(seed, draw++) >> 11) * 0x1.0p-53;
            v[d] += perturb * h[d] * (2.0 * u - 1.0);
          }
        }
      }
  st = mesh_finish(m);
  if (st) { sfx_mesh_destroy(m); return st; }
  *out = m;
  return SFX_OK;
}

extern "C" sfx_status sfx_mesh_create_structured(sfx_ctx* ctx, int nx, int ny, int nz, const double* xyz,
                                                 sfx_mesh** out) {
  if (!xyz) return SFX_ERR_ARG;
  sfx_mesh* m;
  sfx_status st = mesh_alloc(ctx, nx, ny, nz, &m);
  if (st) return st;
  std::memcpy(m->xyz.data(), xyz, m->xyz.size() * sizeof(double));
  st = mesh_finish(m);
  if (st) { sfx_mesh_destroy(m); return st; }
  *out = m;
  return SFX_OK;
}

// Local corner 4a+2b+c (reference corner (a,b,c)) -> position in the VTK
// hexahedron's vertex list (bottom face z = 0 counter-clockwise from the
// origin, then the top face likewise).
static const int kVtkOfCorner[8] = {0, 4, 3, 7, 1, 5, 2, 6};

extern "C" sfx_status sfx_mesh_create(sfx_ctx* ctx, int64_t nvert, const double* xyz, int64_t ncell,
                                      const int32_t* cell_vertices, sfx_mesh** out) {
  if (!ctx || !out || !xyz || !cell_vertices || nvert < 8 || ncell < 1) return SFX_ERR_ARG;
  *out = nullptr;
  if (nvert > 2000000000LL || ncell > 2000000000LL) return SFX_ERR_RANGE;
  for (int64_t c = 0; c < ncell; ++c) {
    const int32_t* v = cell_vertices + c * 8;
    for (int k = 0; k < 8; ++k) {
      if (v[k] < 0 || v[k] >= nvert) return SFX_ERR_ARG;
      for (int l = 0; l < k; ++l)
        if (v[l] == v[k]) return SFX_ERR_ARG;  // a degenerate hexahedron
    }
  }
  sfx_mesh* m = new (std::nothrow) sfx_mesh;
  if (!m) return SFX_ERR_ALLOC;
  m->ctx = ctx;
  m->general = true;
  m->nvert = nvert;
  m->ncell = ncell;
  try {
    m->xyz.assign(xyz, xyz + nvert * 3);
    m->vmap.resize((size_t)ncell * 8);
  } catch (...) { delete m; return SFX_ERR_ALLOC; }
  for (int64_t c = 0; c < ncell; ++c)
    for (int k = 0; k < 8; ++k) m->vmap[c * 8 + k] = cell_vertices[c * 8 + kVtkOfCorner[k]];
  sfx_status st = mesh_finish(m);
  if (st) { sfx_mesh_destroy(m); return st; }
  *out = m;
  return SFX_OK;
}

extern "C" sfx_status sfx_mesh_info(const sfx_mesh* m, int64_t* nvert, int64_t* ncell, const double** xyz) {
  if (!m) return SFX_ERR_ARG;
  if (nvert) *nvert = m->nvert;
  if (ncell) *ncell = m->ncell;
  if (xyz) *xyz = m->xyz.data();
  return SFX_OK;
}

extern "C" void sfx_mesh_destroy(sfx_mesh* m) {
  if (!m) return;
  if (m->d_xyz) cudaFree(m->d_xyz);
  if (m->d_vmap) cudaFree(m->d_vmap);
  delete m;
}

// -------------------------------------------------------------------- space
namespace {

// One tensor-product block of a family: per-axis node count and whether the
// factor is continuous (shared between neighbouring cells).
struct Block {
  int cnt[3];
  bool cont[3];
  int64_t ext[3];  // global grid extent per axis
  int loff;
  int64_t goff;
};

int blocks_of(sfx_family fam, int p, const int64_t N[3], Block* B, int64_t* ndof, int* nloc) {
  int n = p + 1;
  if (fam == SFX_Q || fam == SFX_VQ) {
    int nb = fam == SFX_VQ ? 3 : 1;
    int64_t per = 1;
    for (int d = 0; d < 3; ++d) per *= p * N[d] + 1;
    for (int c = 0; c < nb; ++c) {
      for (int d = 0; d < 3; ++d) { B[c].cnt[d] = n; B[c].cont[d] = true; B[c].ext[d] = p * N[d] + 1; }
      B[c].loff = c * n * n * n;
      B[c].goff = c * per;
    }
    *ndof = nb * per;
    *nloc = nb * n * n * n;
    return nb;
  }
  if (fam == SFX_DQ) {
    *nloc = n * n * n;
    *ndof = N[0] * N[1] * N[2] * (int64_t)(*nloc);
    return 0;  // cell-major, no grid blocks
  }
  int64_t goff = 0;
  int loff = 0;
  for (int c = 0; c < 3; ++c) {
    int64_t tot = 1;
    int cnt = 1;
    for (int d = 0; d < 3; ++d) {
      bool cont = (fam == SFX_NCF) ? (d == c) : (d != c);
      B[c].cont[d] = cont;
      B[c].cnt[d] = cont ? p + 1 : p;
      B[c].ext[d] = cont ? p * N[d] + 1 : p * N[d];
      tot *= B[c].ext[d];
      cnt *= B[c].cnt[d];
    }
    B[c].loff = loff;
    B[c].goff = goff;
    loff += cnt;
    goff += tot;
  }
  *ndof = goff;
  *nloc = loff;
  return 3;
}

}  // namespace

namespace {

// Corner index 4a+2b+c of the reference corner with bits b[0..2] = (a,b,c).
inline int corner_of(const int b[3]) { return 4 * b[0] + 2 * b[1] + b[2]; }

// Global numbering of Q_p (ncomp = 1) or vector Q_p (ncomp = 3, component-
// major) on a general hexahedral mesh, from the mesh's topology alone:
//   vertex dofs  = the vertex ids                          [0, nvert)
//   edge dofs    = nvert + edge * (p-1) + k                 edges numbered in order of first appearance
//   face dofs    = ... + face * (p-1)^2 + k                 faces likewise
//   cell dofs    = ... + cell * (p-1)^3 + k                 interior nodes, local order
// Two cells sharing an edge or a face must agree on the order of its interior
// nodes, whatever their local axes.  The order is taken from the global vertex
// ids: an edge runs from its smaller vertex id to its larger one; a face's
// nodes run first along the face edge from its smallest-id corner to that
// corner's neighbour with the smaller id, then along the other edge.  Since
// the GLL nodes are symmetric (x_{p-i} = 1 - x_i), this identifies the same
// physical points from either cell (Sec. 1.1: the global basis is the union
// of the cells' bases, glued through shared entities).
sfx_status general_q_map(const sfx_mesh* m, int p, int ncomp, std::vector<int32_t>& map, int64_t* ndof_out) {
  const int n = p + 1, n3 = n * n * n, nloc = ncomp * n3;
  const int64_t ncell = m->ncell, nvert = m->nvert;
  const int32_t* V = m->vmap.data();
  std::unordered_map<uint64_t, int64_t> edges;
  std::map<std::array<int32_t, 4>, int64_t> faces;
  if (p >= 2) {
    for (int64_t c = 0; c < ncell; ++c) {
      const int32_t* v = V + c * 8;
      for (int d = 0; d < 3; ++d)      // 12 edges: along axis d, the other two bits free
        for (int o = 0; o < 4; ++o) {
          int b0[3], b1[3], k = 0;
          for (int e = 0; e < 3; ++e) {
            if (e == d) { b0[e] = 0; b1[e] = 1; continue; }
            b0[e] = b1[e] = (o >> k++) & 1;
          }
          const uint32_t ga = (uint32_t)v[corner_of(b0)], gb = (uint32_t)v[corner_of(b1)];
          const uint64_t key = ((uint64_t)std::min(ga, gb) << 32) | std::max(ga, gb);
          edges.emplace(key, (int64_t)edges.size());
        }
      for (int f = 0; f < 3; ++f)      // 6 faces: axis f fixed at 0 or 1
        for (int side = 0; side < 2; ++side) {
          std::array<int32_t, 4> key;
          int q = 0;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
              int bits[3], k = 0;
              for (int e = 0; e < 3; ++e) bits[e] = e == f ? side : (k++ == 0 ? a : b);
              key[q++] = v[corner_of(bits)];
            }
          std::sort(key.begin(), key.end());
          faces.emplace(key, (int64_t)faces.size());
        }
    }
  }
  const int64_t pe = p - 1, pf = pe * pe, pc = pe * pe * pe;
  const int64_t off_e = nvert, off_f = off_e + (int64_t)edges.size() * pe,
                off_c = off_f + (int64_t)faces.size() * pf, per = off_c + ncell * pc;
  if (ncomp * per >= (1LL << 31) - 1) return SFX_ERR_RANGE;
  try { map.resize((size_t)ncell * nloc); } catch (...) { return SFX_ERR_ALLOC; }
  for (int64_t c = 0; c < ncell; ++c) {
    const int32_t* v = V + c * 8;
    int32_t* row = &map[(size_t)c * nloc];
    int l = 0;
    for (int i1 = 0; i1 < n; ++i1)
      for (int i2 = 0; i2 < n; ++i2)
        for (int i3 = 0; i3 < n; ++i3, ++l) {
          const int ii[3] = {i1, i2, i3};
          int bnd[3], nb = 0;
          for (int d = 0; d < 3; ++d) { bnd[d] = ii[d] == 0 || ii[d] == p; nb += bnd[d]; }
          int64_t g;
          if (nb == 3) {
            const int bits[3] = {i1 / p, i2 / p, i3 / p};
            g = v[corner_of(bits)];
          } else if (nb == 2) {
            int d = !bnd[0] ? 0 : (!bnd[1] ? 1 : 2);
            int b0[3], b1[3];
            for (int e = 0; e < 3; ++e) { b0[e] = e == d ? 0 : ii[e] / p; b1[e] = e == d ? 1 : ii[e] / p; }
            const uint32_t ga = (uint32_t)v[corner_of(b0)], gb = (uint32_t)v[corner_of(b1)];
            const uint64_t key = ((uint64_t)std::min(ga, gb) << 32) | std::max(ga, gb);
            const int64_t t = ii[d], pos = ga < gb ? t - 1 : p - t - 1;
            g = off_e + edges.at(key) * pe + pos;
          } else if (nb == 1) {
            const int f = bnd[0] ? 0 : (bnd[1] ? 1 : 2);
            const int d1 = f == 0 ? 1 : 0, d2 = f == 2 ? 1 : 2;
            int32_t cv[2][2];
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) {
                int bits[3];
                bits[f] = ii[f] / p;
                bits[d1] = a;
                bits[d2] = b;
                cv[a][b] = v[corner_of(bits)];
              }
            int a0 = 0, b0 = 0;
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b)
                if (cv[a][b] < cv[a0][b0]) { a0 = a; b0 = b; }
            const int64_t s1 = a0 ? p - ii[d1] : ii[d1], s2 = b0 ? p - ii[d2] : ii[d2];
            const bool first_d1 = cv[1 - a0][b0] < cv[a0][1 - b0];
            const int64_t u = first_d1 ? s1 : s2, w = first_d1 ? s2 : s1;
            std::array<int32_t, 4> key = {cv[0][0], cv[0][1], cv[1][0], cv[1][1]};
            std::sort(key.begin(), key.end());
            g = off_f + faces.at(key) * pf + (u - 1) * pe + (w - 1);
          } else {
            g = off_c + c * pc + ((i1 - 1) * pe + (i2 - 1)) * pe + (i3 - 1);
          }
          for (int cmp = 0; cmp < ncomp; ++cmp) row[cmp * n3 + l] = (int32_t)(cmp * per + g);
        }
  }
  *ndof_out = ncomp * per;
  return SFX_OK;
}

// Greedy first-fit colouring: cells in order, each takes the smallest colour
// that no earlier cell sharing one of its vertices has.  Cells of one colour
// then share no vertex, hence no dof of Q_p or vector Q_p.
void greedy_colour(const sfx_mesh* m, std::vector<int>& col, int* ncol) {
  const int64_t ncell = m->ncell, nvert = m->nvert;
  const int32_t* V = m->vmap.data();
  std::vector<int64_t> start((size_t)nvert + 1, 0);
  for (int64_t i = 0; i < ncell * 8; ++i) start[V[i] + 1]++;
  for (int64_t v = 0; v < nvert; ++v) start[v + 1] += start[v];
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  std::vector<int32_t> cells_of((size_t)ncell * 8);
  for (int64_t c = 0; c < ncell; ++c)
    for (int k = 0; k < 8; ++k) cells_of[fill[V[c * 8 + k]]++] = (int32_t)c;
  col.assign((size_t)ncell, -1);
  std::vector<int64_t> seen;
  *ncol = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    for (int k = 0; k < 8; ++k) {
      const int32_t v = V[c * 8 + k];
      for (int64_t i = start[v]; i < start[v + 1]; ++i) {
        const int32_t o = cells_of[i];
        if (o < c) seen[col[o]] = c;
      }
    }
    int k = 0;
    while (k < *ncol && seen[k] == c) ++k;
    if (k == *ncol) { seen.push_back(-1); ++*ncol; }
    col[c] = k;
  }
}

}  // namespace

extern "C" sfx_status sfx_space_create(const sfx_mesh* mesh, sfx_family fam, int p, sfx_space** out) {
  if (!mesh || !out || !family_ok(fam)) return SFX_ERR_ARG;
  *out = nullptr;
  if (p < 1 || p > kMaxDeg) return SFX_ERR_UNSUPPORTED;
  if (mesh->general && (fam == SFX_NCF || fam == SFX_NCE)) return SFX_ERR_UNSUPPORTED;
  const int64_t N[3] = {mesh->nx, mesh->ny, mesh->nz};
  Block B[3];
  int64_t ndof;
  int nloc;
  int nb = 0;
  const int64_t ncell = mesh->ncell;
  std::vector<int32_t> gmap;
  if (!mesh->general) {
    nb = blocks_of(fam, p, N, B, &ndof, &nloc);
  } else if (fam == SFX_DQ) {
    nloc = (p + 1) * (p + 1) * (p + 1);
    ndof = ncell * nloc;
  } else {
    sfx_status st = general_q_map(mesh, p, fam == SFX_VQ ? 3 : 1, gmap, &ndof);
    if (st) return st;
    nloc = (fam == SFX_VQ ? 3 : 1) * (p + 1) * (p + 1) * (p + 1);
  }
  if (ndof >= (1LL << 31) - 1) return SFX_ERR_RANGE;
  sfx_space* s = new (std::nothrow) sfx_space;
  if (!s) return SFX_ERR_ALLOC;
  s->mesh = mesh;
  s->family = fam;
  s->p = p;
  s->nloc = nloc;
  s->ndof = ndof;
  if (!gmap.empty()) {
    s->map.swap(gmap);
  } else {
    try { s->map.resize((size_t)ncell * nloc); } catch (...) { delete s; return SFX_ERR_ALLOC; }
  }
  for (int64_t c = 0; c < ncell && (fam == SFX_DQ || !mesh->general); ++c) {
    int32_t* row = &s->map[(size_t)c * nloc];
    if (fam == SFX_DQ) {
      for (int l = 0; l < nloc; ++l) row[l] = (int32_t)(c * nloc + l);
      continue;
    }
    int64_t ci[3] = {c / (N[1] * N[2]), (c / N[2]) % N[1], c % N[2]};
    for (int b = 0; b < nb; ++b) {
      int l = B[b].loff;
      for (int i1 = 0; i1 < B[b].cnt[0]; ++i1)
        for (int i2 = 0; i2 < B[b].cnt[1]; ++i2)
          for (int i3 = 0; i3 < B[b].cnt[2]; ++i3) {
            int ii[3] = {i1, i2, i3};
            int64_t g[3];
            for (int d = 0; d < 3; ++d) g[d] = (B[b].cont[d] ? B[b].cnt[d] - 1 : B[b].cnt[d]) * ci[d] + ii[d];
            row[l++] = (int32_t)(B[b].goff + (g[0] * B[b].ext[1] + g[1]) * B[b].ext[2] + g[2]);
          }
    }
  }
  // colouring: cells with the same parity in every axis share no vertex
  // (structured box); greedy first-fit on a general mesh
  std::vector<int32_t>& cells = s->cells;
  try { cells.resize((size_t)ncell); } catch (...) { delete s; return SFX_ERR_ALLOC; }
  if (fam == SFX_DQ) {
    s->ncolour = 1;
    for (int64_t c = 0; c < ncell; ++c) cells[c] = (int32_t)c;
    s->colour_off = {0, ncell};
  } else if (mesh->general) {
    std::vector<int> col;
    greedy_colour(mesh, col, &s->ncolour);
    s->colour_off.assign((size_t)s->ncolour + 1, 0);
    for (int64_t c = 0; c < ncell; ++c) s->colour_off[col[c] + 1]++;
    for (int k = 0; k < s->ncolour; ++k) s->colour_off[k + 1] += s->colour_off[k];
    std::vector<int64_t> pos(s->colour_off.begin(), s->colour_off.end() - 1);
    for (int64_t c = 0; c < ncell; ++c) cells[pos[col[c]]++] = (int32_t)c;
  } else {
    s->ncolour = 8;
    s->colour_off.assign(9, 0);
    for (int64_t c = 0; c < ncell; ++c) {
      int col = (int)(((c / (N[1] * N[2])) & 1) * 4 + (((c / N[2]) % N[1]) & 1) * 2 + ((c % N[2]) & 1));
      s->colour_off[col + 1]++;
    }
    for (int k = 0; k < 8; ++k) s->colour_off[k + 1] += s->colour_off[k];
    std::vector<int64_t> pos(s->colour_off.begin(), s->colour_off.end() - 1);
    for (int64_t c = 0; c < ncell; ++c) {
      int col = (int)(((c / (N[1] * N[2])) & 1) * 4 + (((c / N[2]) % N[1]) & 1) * 2 + ((c % N[2]) & 1));
      cells[pos[col]++] = (int32_t)c;
    }
  }
  make_tab1d(p, &s->tab);
  if (fam == SFX_Q) {
    // first-touch bits: walk the cells colour by colour (the order of the
    // launches) and mark each dof's first cell-node pair
    const int words = (nloc + 31) / 32;
    std::vector<uint8_t> seen;
    try {
      s->first.assign((size_t)ncell * words, 0u);
      seen.assign((size_t)ndof, 0);
    } catch (...) {
      delete s;
      return SFX_ERR_ALLOC;
    }
    for (size_t k = 0; k < cells.size(); ++k) {
      const int64_t c = cells[k];
      const int32_t* row = &s->map[(size_t)c * nloc];
      uint32_t* bits = &s->first[(size_t)c * words];
      for (int l = 0; l < nloc; ++l)
        if (!seen[(size_t)row[l]]) {
          seen[(size_t)row[l]] = 1;
          bits[l >> 5] |= 1u << (l & 31);
        }
    }
  }
  if (mesh->ctx->device < 0) {
    *out = s;
    return SFX_OK;
  }
  if (upload_tables(&s->tab) != 0) { sfx_space_destroy(s); return SFX_ERR_CUDA; }
  sfx_status st = to_device(s->map.data(), s->map.size(), &s->d_map);
  if (!st) st = to_device(cells.data(), cells.size(), &s->d_cells);
  if (!st && !s->first.empty()) st = to_device(s->first.data(), s->first.size(), &s->d_first);
  if (st) { sfx_space_destroy(s); return st; }
  *out = s;
  return SFX_OK;
}

extern "C" sfx_status sfx_space_info(const sfx_space* s, int64_t* ndof, int* nloc, int64_t* ncell,
                                     const int32_t** host_map) {
  if (!s) return SFX_ERR_ARG;
  if (ndof) *ndof = s->ndof;
  if (nloc) *nloc = s->nloc;
  if (ncell) *ncell = s->mesh->ncell;
  if (host_map) *host_map = s->map.data();
  return SFX_OK;
}

extern "C" sfx_status sfx_space_colours(const sfx_space* s, int* ncolour, const int64_t** colour_off,
                                        const int32_t** cells) {
  if (!s) return SFX_ERR_ARG;
  if (ncolour) *ncolour = s->ncolour;
  if (colour_off) *colour_off = s->colour_off.data();
  if (cells) *cells = s->cells.data();
  return SFX_OK;
}

extern "C" sfx_status sfx_space_first_touch(const sfx_space* s, int* words_per_cell, const uint32_t** bits) {
  if (!s) return SFX_ERR_ARG;
  const bool has = !s->first.empty();
  if (words_per_cell) *words_per_cell = has ? (s->nloc + 31) / 32 : 0;
  if (bits) *bits = has ? s->first.data() : nullptr;
  return SFX_OK;
}

namespace {
std::mutex g_scalar_mutex;

bool linear_form(sfx_form f) { return f == SFX_MASS || f == SFX_LAPLACE || f == SFX_HELMHOLTZ; }

// The scalar Q_p space of a vector Q_p space's components, created on first use.
sfx_status vq_scalar(const sfx_space* sp, const sfx_space** out) {
  std::lock_guard<std::mutex> lock(g_scalar_mutex);
  if (!sp->scalar) {
    sfx_space* s = nullptr;
    const sfx_status st = sfx_space_create(sp->mesh, SFX_Q, sp->p, &s);
    if (st) return st;
    sp->scalar = s;
  }
  *out = sp->scalar;
  return SFX_OK;
}
}  // namespace

extern "C" void sfx_space_destroy(sfx_space* s) {
  if (!s) return;
  if (s->scalar) sfx_space_destroy(s->scalar);
  if (s->d_map) cudaFree(s->d_map);
  if (s->d_cells) cudaFree(s->d_cells);
  if (s->d_first) cudaFree(s->d_first);
  if (s->d_naive) cudaFree(s->d_naive);
  delete s;
}

// --------------------------------------------------------------- tabulation
extern "C" sfx_status sfx_tabulate_1d(sfx_nodes nodes, int ndof1d, sfx_nodes qrule, int nq, int deriv,
                                      double* points, double* weights, double* table) {
  if (ndof1d < 1 || ndof1d > 32 || nq < 1 || nq > 32) return SFX_ERR_ARG;
  if ((nodes != SFX_NODES_GLL && nodes != SFX_NODES_GL) || (qrule != SFX_NODES_GLL && qrule != SFX_NODES_GL))
    return SFX_ERR_ARG;
  if ((nodes == SFX_NODES_GLL && ndof1d < 2) || (qrule == SFX_NODES_GLL && nq < 2)) return SFX_ERR_ARG;
  if (deriv != 0 && deriv != 1) return SFX_ERR_ARG;
  double xq[32], wq[32], xn[32], wn[32];
  if (qrule == SFX_NODES_GL) gauss_legendre(nq, xq, wq); else gauss_lobatto(nq, xq, wq);
  if (nodes == SFX_NODES_GL) gauss_legendre(ndof1d, xn, wn); else gauss_lobatto(ndof1d, xn, wn);
  if (points) std::memcpy(points, xq, nq * sizeof(double));
  if (weights) std::memcpy(weights, wq, nq * sizeof(double));
  if (table) lagrange_table(xn, ndof1d, xq, nq, deriv, table);
  return SFX_OK;
}

// ----------------------------------------------------------------- assembly
// Overwriting scalar actions skip the memset of y where that measured faster
// on GB300: DQ_p (every contribution is its dof's only one: plain stores, no
// table), and Q_p in the FP64 kernels (the first contribution to each dof is
// stored, the later ones added; see d_first).  The split-precision Q_p kernels
// keep the memset: there the per-dof table lookup and the split between stores
// and reductions within a warp cost more than the memset saves (2-7% at p = 7,
// 8).  With several right-hand sides (y is dof-major, RHS fastest) each store
// covers part of a DRAM sector, which costs more than the memset's full
// sectors once y does not fit in L2: stores only for one RHS in FP64 (DQ_8,
// 16 RHS: 58.5 ms against 57.9 with the memset) and up to four in split
// precision (4 RHS: 4.06 against 4.18; 16 RHS: 20.35 against 20.17).
static bool first_touch_pays(sfx_precision prec, int nrhs) {
  return nrhs == 1 || (prec != SFX_PREC_FP64 && nrhs <= 4);
}
static void set_first_touch(const sfx_space* sp, sfx_precision prec, int nrhs, ActArgs* a) {
  if (!first_touch_pays(prec, nrhs)) return;
  if (sp->family == SFX_DQ) a->first_all = 1;
  else if (sp->family == SFX_Q && prec == SFX_PREC_FP64) a->first = sp->d_first;
}

extern "C" sfx_status sfx_assemble_action(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                          const sfx_space* sp, const double* x, double* y, int nrhs,
                                          int accumulate, sfx_precision prec, sfx_algo algo, void* stream) {
  Range range("sfx_assemble_action");
  if (!ctx || !sp || !x || !y || nrhs < 1 || nrhs > 64 || ctx->device < 0 || !sp->d_map) return SFX_ERR_ARG;
  if (!form_ok(sp->family, form)) return SFX_ERR_ARG;
  if (x == y) return SFX_ERR_ARG;
  if (prec < SFX_PREC_FP64 || prec > SFX_PREC_BF16X3 ||
      (algo != SFX_ALGO_SUMFACT && algo != SFX_ALGO_NAIVE && algo != SFX_ALGO_COLLOCATED))
    return SFX_ERR_ARG;
  if (sp->family == SFX_VQ && linear_form(form)) {
    // vector forms (Sec. 3.3): the component delta leaves one scalar action per
    // component, on the component's contiguous slice of x and y
    const sfx_space* S = nullptr;
    const sfx_status st = vq_scalar(sp, &S);
    if (st) return st;
    for (int c = 0; c < 3; ++c) {
      const int64_t off = (int64_t)c * S->ndof * nrhs;
      const sfx_status e = sfx_assemble_action(ctx, form, params, S, x + off, y + off, nrhs, accumulate, prec,
                                               algo, stream);
      if (e) return e;
    }
    return SFX_OK;
  }
  if (algo == SFX_ALGO_COLLOCATED &&
      (sp->family != SFX_Q || (prec != SFX_PREC_FP64 && prec != SFX_PREC_TF32X3)))
    return SFX_ERR_UNSUPPORTED;
  sfx_form_params pr = params ? *params : default_params(form);
  cudaStream_t s = (cudaStream_t)stream;
  ActArgs a{};
  // overwrite without a memset where the kernels store each dof's first
  // contribution (the scalar sum-factorised and collocated kernels)
  if (!accumulate && algo != SFX_ALGO_NAIVE) set_first_touch(sp, prec, nrhs, &a);
  if (!accumulate && !a.first && !a.first_all) {
    if (cudaMemsetAsync(y, 0, (size_t)sp->ndof * nrhs * sizeof(double), s) != cudaSuccess) return SFX_ERR_CUDA;
  }
  a.map = sp->d_map;
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.x = x;
  a.y = y;
  a.nrhs = nrhs;
  a.r0 = 0;
  a.r1 = nrhs;
  a.cell_vectors = 0;
  a.alpha = pr.alpha; a.beta = pr.beta; a.mu = pr.mu; a.lambda = pr.lambda;
  a.status = ctx->d_status;
  bool launched = false;
  for (int col = 0; col < sp->ncolour; ++col) {
    a.cells = sp->d_cells + sp->colour_off[col];
    a.ncells = sp->colour_off[col + 1] - sp->colour_off[col];
    if (a.ncells == 0) continue;
    // later colours may start while the previous one drains (see pdl_wait_prev)
    a.overlap_prev = launched ? 1 : 0;
    launched = true;
    int e;
    if (algo == SFX_ALGO_COLLOCATED)
      e = prec == SFX_PREC_FP64 ? launch_action_scalar_coll(sp, form, a, stream)
                                : launch_action_scalar_mixed_coll(sp, form, a, stream);
    else if (sp->family == SFX_Q || sp->family == SFX_DQ) e = launch_action_scalar(sp, form, prec, algo, a, stream);
    else if (algo != SFX_ALGO_SUMFACT) return SFX_ERR_UNSUPPORTED;
    else if (sp->family == SFX_VQ) e = launch_action_elastic(sp, form, prec, a, stream);
    else e = launch_action_hdivcurl(sp, form, prec, a, stream);
    if (e == -1) return SFX_ERR_UNSUPPORTED;
    if (e) return SFX_ERR_CUDA;
  }
  return SFX_OK;
}

extern "C" sfx_status sfx_assemble_cell_vectors(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                                const sfx_space* sp, const double* x, int nrhs,
                                                const int64_t* cells, int64_t ncells, double* b,
                                                sfx_precision prec, void* stream) {
  Range range("sfx_assemble_cell_vectors");
  if (!ctx || !sp || !x || !b || nrhs < 1 || nrhs > 64 || ncells < 0 || ctx->device < 0 || !sp->d_map)
    return SFX_ERR_ARG;
  if (ncells > 0 && !cells) return SFX_ERR_ARG;
  if (!form_ok(sp->family, form)) return SFX_ERR_ARG;
  if (prec < SFX_PREC_FP64 || prec > SFX_PREC_BF16X3) return SFX_ERR_ARG;
  if (sp->family == SFX_VQ && linear_form(form)) return SFX_ERR_UNSUPPORTED;
  if (ncells == 0) return SFX_OK;
  sfx_form_params pr = params ? *params : default_params(form);
  ActArgs a{};
  a.map = sp->d_map;
  a.cells = nullptr;
  a.cells64 = cells;
  a.ncells = ncells;
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.x = x;
  a.y = b;
  a.nrhs = nrhs;
  a.r0 = 0;
  a.r1 = nrhs;
  a.cell_vectors = 1;
  a.alpha = pr.alpha; a.beta = pr.beta; a.mu = pr.mu; a.lambda = pr.lambda;
  a.status = ctx->d_status;
  int e;
  if (sp->family == SFX_Q || sp->family == SFX_DQ) e = launch_action_scalar(sp, form, prec, SFX_ALGO_SUMFACT, a, stream);
  else if (sp->family == SFX_VQ) e = launch_action_elastic(sp, form, prec, a, stream);
  else e = launch_action_hdivcurl(sp, form, prec, a, stream);
  if (e == -1) return SFX_ERR_UNSUPPORTED;
  return e ? SFX_ERR_CUDA : SFX_OK;
}

// Weighted Laplace form int kappa grad u . grad v (Sec. 1.1, Eq. weighted_laplace).
extern "C" sfx_status sfx_assemble_weighted_action(sfx_ctx* ctx, const sfx_space* sp, const double* kappa,
                                                   const double* x, double* y, int nrhs, int accumulate,
                                                   sfx_precision prec, void* stream) {
  Range range("sfx_assemble_weighted_action");
  if (!ctx || !sp || !kappa || !x || !y || nrhs < 1 || nrhs > 64 || ctx->device < 0 || !sp->d_map)
    return SFX_ERR_ARG;
  if (sp->family != SFX_Q && sp->family != SFX_DQ) return SFX_ERR_ARG;
  if (y == x || y == kappa) return SFX_ERR_ARG;
  if (prec < SFX_PREC_FP64 || prec > SFX_PREC_BF16X3) return SFX_ERR_ARG;
  if (prec != SFX_PREC_FP64) return SFX_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  ActArgs a{};
  if (!accumulate) set_first_touch(sp, prec, nrhs, &a);
  if (!accumulate && !a.first && !a.first_all) {
    if (cudaMemsetAsync(y, 0, (size_t)sp->ndof * nrhs * sizeof(double), s) != cudaSuccess) return SFX_ERR_CUDA;
  }
  a.map = sp->d_map;
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.x = x;
  a.kappa = kappa;
  a.y = y;
  a.nrhs = nrhs;
  a.r0 = 0;
  a.r1 = nrhs;
  a.alpha = 1.0;
  a.beta = 0.0;
  a.status = ctx->d_status;
  for (int col = 0; col < sp->ncolour; ++col) {
    a.cells = sp->d_cells + sp->colour_off[col];
    a.ncells = sp->colour_off[col + 1] - sp->colour_off[col];
    if (a.ncells == 0) continue;
    const int e = launch_action_weighted(sp, a, stream);
    if (e == -1) return SFX_ERR_UNSUPPORTED;
    if (e) return SFX_ERR_CUDA;
  }
  return SFX_OK;
}

extern "C" sfx_status sfx_assemble_weighted_cell_matrices(sfx_ctx* ctx, const sfx_space* sp, const double* kappa,
                                                          int64_t cell_begin, int64_t cell_end, double* A,
                                                          sfx_precision prec, void* stream) {
  Range range("sfx_assemble_weighted_cell_matrices");
  if (!ctx || !sp || !kappa || !A || ctx->device < 0 || !sp->d_map) return SFX_ERR_ARG;
  if (sp->family != SFX_Q && sp->family != SFX_DQ) return SFX_ERR_ARG;
  if (cell_begin < 0 || cell_end > sp->mesh->ncell || cell_begin > cell_end) return SFX_ERR_ARG;
  if (prec != SFX_PREC_FP64) return SFX_ERR_UNSUPPORTED;
  if (cell_end == cell_begin) return SFX_OK;
  MatArgs a{};
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.cell_begin = cell_begin;
  a.ncells = cell_end - cell_begin;
  a.A = A;
  a.alpha = 1.0;
  a.beta = 0.0;
  a.map = sp->d_map;
  a.kappa = kappa;
  a.kappa_dq = sp->family == SFX_DQ;
  a.status = ctx->d_status;
  const int e = launch_cell_matrices(sp, SFX_LAPLACE, SFX_ALGO_SUMFACT, a, stream);
  if (e == -1) return SFX_ERR_UNSUPPORTED;
  return e ? SFX_ERR_CUDA : SFX_OK;
}

// Linearised hyperelastic operator: per colour, or per listed cell (cells != null).
static sfx_status linearised(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params, const sfx_space* sp,
                             const double* u, const double* du, double* y, int nrhs, int accumulate,
                             const int64_t* cells, int64_t ncells, sfx_precision prec, void* stream) {
  if (!ctx || !sp || !u || !du || !y || nrhs < 1 || nrhs > 64 || ctx->device < 0 || !sp->d_map) return SFX_ERR_ARG;
  if (sp->family != SFX_VQ || (form != SFX_NEOHOOKE && form != SFX_SVK)) return SFX_ERR_ARG;
  if (y == du || y == u) return SFX_ERR_ARG;
  if (prec < SFX_PREC_FP64 || prec > SFX_PREC_BF16X3) return SFX_ERR_ARG;
  if (ncells < 0 || (ncells > 0 && !cells)) return SFX_ERR_ARG;
  auto launch = [&](const ActArgs& aa) {
    return prec == SFX_PREC_FP64 ? launch_linearised_elastic(sp, form, aa, stream)
                                 : launch_linearised_elastic_mixed(sp, form, prec, aa, stream);
  };
  sfx_form_params pr = params ? *params : default_params(form);
  cudaStream_t s = (cudaStream_t)stream;
  ActArgs a{};
  a.map = sp->d_map;
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.x = du;
  a.xs = u;
  a.y = y;
  a.nrhs = nrhs;
  a.r0 = 0;
  a.r1 = nrhs;
  a.alpha = pr.alpha; a.beta = pr.beta; a.mu = pr.mu; a.lambda = pr.lambda;
  a.status = ctx->d_status;
  if (cells) {
    if (ncells == 0) return SFX_OK;
    a.cells64 = cells;
    a.ncells = ncells;
    a.cell_vectors = 1;
    const int e = launch(a);
    if (e == -1) return SFX_ERR_UNSUPPORTED;
    return e ? SFX_ERR_CUDA : SFX_OK;
  }
  if (!accumulate) {
    if (cudaMemsetAsync(y, 0, (size_t)sp->ndof * nrhs * sizeof(double), s) != cudaSuccess) return SFX_ERR_CUDA;
  }
  for (int col = 0; col < sp->ncolour; ++col) {
    a.cells = sp->d_cells + sp->colour_off[col];
    a.ncells = sp->colour_off[col + 1] - sp->colour_off[col];
    if (a.ncells == 0) continue;
    const int e = launch(a);
    if (e == -1) return SFX_ERR_UNSUPPORTED;
    if (e) return SFX_ERR_CUDA;
  }
  return SFX_OK;
}

extern "C" sfx_status sfx_assemble_linearised_action(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                                     const sfx_space* sp, const double* u, const double* du,
                                                     double* y, int nrhs, int accumulate, sfx_precision prec,
                                                     void* stream) {
  Range range("sfx_assemble_linearised_action");
  return linearised(ctx, form, params, sp, u, du, y, nrhs, accumulate, nullptr, 0, prec, stream);
}

extern "C" sfx_status sfx_assemble_linearised_cell_vectors(sfx_ctx* ctx, sfx_form form,
                                                           const sfx_form_params* params, const sfx_space* sp,
                                                           const double* u, const double* du, int nrhs,
                                                           const int64_t* cells, int64_t ncells, double* b,
                                                           sfx_precision prec, void* stream) {
  Range range("sfx_assemble_linearised_cell_vectors");
  if (ncells > 0 && !cells) return SFX_ERR_ARG;
  if (ncells == 0) return (ctx && sp && u && du && b) ? SFX_OK : SFX_ERR_ARG;
  return linearised(ctx, form, params, sp, u, du, b, nrhs, 0, cells, ncells, prec, stream);
}

extern "C" sfx_status sfx_assemble_linearised_cell_matrices(sfx_ctx* ctx, sfx_form form,
                                                            const sfx_form_params* params, const sfx_space* sp,
                                                            const double* u, int64_t cell_begin, int64_t cell_end,
                                                            double* A, sfx_precision prec, void* stream) {
  Range range("sfx_assemble_linearised_cell_matrices");
  if (!ctx || !sp || !u || ctx->device < 0 || !sp->d_map) return SFX_ERR_ARG;
  if (sp->family != SFX_VQ || (form != SFX_NEOHOOKE && form != SFX_SVK)) return SFX_ERR_ARG;
  if (cell_begin < 0 || cell_end > sp->mesh->ncell || cell_begin > cell_end) return SFX_ERR_ARG;
  if (prec < SFX_PREC_FP64 || prec > SFX_PREC_BF16X3) return SFX_ERR_ARG;
  if (prec != SFX_PREC_FP64) return SFX_ERR_UNSUPPORTED;
  if (cell_begin == cell_end) return SFX_OK;  // nothing written: A may be null
  if (!A || A == u) return SFX_ERR_ARG;
  const sfx_form_params pr = params ? *params : default_params(form);
  const int n3 = (sp->p + 1) * (sp->p + 1) * (sp->p + 1);
  ActArgs a{};
  a.map = sp->d_map;
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.xs = u;
  a.y = A;
  a.nrhs = 1;
  a.r0 = 0;
  a.r1 = 1;
  a.ncells = cell_end - cell_begin;
  a.cell0 = cell_begin;
  // trial columns per CTA: at least three chunks (one per component), more
  // when few cells are asked for, so that cells x chunks fills the GPU
  // (>= 16 per SM); at least 8 columns per chunk to amortise the state's
  // gradient and the geometry, which every chunk forms again.  Each column's
  // arithmetic is the same whatever the chunking.
  const int64_t ncells = cell_end - cell_begin;
  int64_t chunks = std::max<int64_t>(3, (152 * 16 + ncells - 1) / ncells);
  chunks = std::min<int64_t>(chunks, std::max(3, 3 * n3 / 8));
  a.unit_cols = (int)((3 * n3 + chunks - 1) / chunks);
  a.alpha = pr.alpha; a.beta = pr.beta; a.mu = pr.mu; a.lambda = pr.lambda;
  a.status = ctx->d_status;
  const int e = launch_linearised_elastic(sp, form, a, stream);
  if (e == -1) return SFX_ERR_UNSUPPORTED;
  return e ? SFX_ERR_CUDA : SFX_OK;
}

extern "C" sfx_status sfx_assemble_cell_matrices(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                                 const sfx_space* sp, int64_t cell_begin, int64_t cell_end,
                                                 double* A, sfx_precision prec, sfx_algo algo, void* stream) {
  Range range("sfx_assemble_cell_matrices");
  if (!ctx || !sp || !A || ctx->device < 0 || !sp->d_map) return SFX_ERR_ARG;
  if (!form_ok(sp->family, form) || form == SFX_NEOHOOKE || form == SFX_SVK) return SFX_ERR_ARG;
  if (cell_begin < 0 || cell_end > sp->mesh->ncell || cell_begin > cell_end) return SFX_ERR_ARG;
  if (prec != SFX_PREC_FP64) return SFX_ERR_UNSUPPORTED;
  if (algo != SFX_ALGO_SUMFACT && algo != SFX_ALGO_NAIVE && algo != SFX_ALGO_COLLOCATED) return SFX_ERR_ARG;
  if (algo == SFX_ALGO_COLLOCATED && sp->family != SFX_Q && sp->family != SFX_VQ) return SFX_ERR_UNSUPPORTED;
  if (cell_end == cell_begin) return SFX_OK;
  if (sp->family == SFX_VQ) {
    // vector forms: delta cancellation across the assignment (Sec. 3.3) -- the
    // scalar block once per cell, written to the three diagonal blocks of the
    // cleared matrix.  Scalar blocks go through a stream-ordered scratch of at
    // most 256 MB, chunk by chunk.
    const sfx_space* S = nullptr;
    sfx_status st = vq_scalar(sp, &S);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int n3 = S->nloc;
    const size_t per_cell = (size_t)n3 * n3 * sizeof(double);
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(cell_end - cell_begin, (256 << 20) / per_cell));
    double* scratch = nullptr;
    if (cudaMallocAsync((void**)&scratch, (size_t)chunk * per_cell, s) != cudaSuccess) return SFX_ERR_ALLOC;
    for (int64_t c0 = cell_begin; c0 < cell_end && !st; c0 += chunk) {
      const int64_t m = std::min(chunk, cell_end - c0);
      st = sfx_assemble_cell_matrices(ctx, form, params, S, c0, c0 + m, scratch, prec, algo, stream);
      if (!st && launch_vq_expand(scratch, m, n3, A + (size_t)(c0 - cell_begin) * 9 * n3 * n3, stream))
        st = SFX_ERR_CUDA;
    }
    if (cudaFreeAsync(scratch, s) != cudaSuccess && !st) st = SFX_ERR_CUDA;
    return st;
  }
  sfx_form_params pr = params ? *params : default_params(form);
  MatArgs a{};
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.cell_begin = cell_begin;
  a.ncells = cell_end - cell_begin;
  a.A = A;
  a.alpha = pr.alpha;
  a.beta = pr.beta;
  a.status = ctx->d_status;
  int e = algo == SFX_ALGO_COLLOCATED ? launch_cell_matrices_coll(sp, form, a, stream)
                                      : launch_cell_matrices(sp, form, algo, a, stream);
  if (e == -1) return SFX_ERR_UNSUPPORTED;
  return e ? SFX_ERR_CUDA : SFX_OK;
}

// ------------------------------------------------------------ sparse matrix
struct sfx_csr {
  const sfx_space* space = nullptr;
  int64_t nrows = 0, nnz = 0;
  std::vector<int64_t> row_ptr;  // host, nrows + 1
  std::vector<int32_t> col;      // host, nnz (sorted within each row)
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_scratch = nullptr;   // element matrices of one chunk of cells
  int64_t chunk = 0;             // cells per chunk
  int lanes = 32;                // lanes per row in the product
};

namespace {
// Column range [lo, hi] of 1D Q_p node I on a line of ncell cells: the nodes
// of the cells that contain I (two cells for a vertex node inside the line).
inline void q_range_1d(int64_t I, int p, int64_t ncell, int64_t* lo, int64_t* hi) {
  int64_t cmin = I / p, cmax = I / p;
  if (I % p == 0) cmin -= 1;
  if (cmin < 0) cmin = 0;
  if (cmax > ncell - 1) cmax = ncell - 1;
  *lo = (int64_t)p * cmin;
  *hi = (int64_t)p * (cmax + 1);
}
}  // namespace

extern "C" sfx_status sfx_csr_create(const sfx_space* sp, sfx_csr** out) {
  if (!sp || !out) return SFX_ERR_ARG;
  *out = nullptr;
  if (sp->family != SFX_Q && sp->family != SFX_DQ) return SFX_ERR_UNSUPPORTED;
  if (sp->mesh->general) return SFX_ERR_UNSUPPORTED;  // the pattern below uses the box's grid structure
  const sfx_mesh* m = sp->mesh;
  const int p = sp->p, n = p + 1, nloc = sp->nloc;
  sfx_csr* c = new (std::nothrow) sfx_csr;
  if (!c) return SFX_ERR_ALLOC;
  c->space = sp;
  c->nrows = sp->ndof;
  const int64_t N[3] = {m->nx, m->ny, m->nz};
  const int64_t M[3] = {p * N[0] + 1, p * N[1] + 1, p * N[2] + 1};
  try {
    c->row_ptr.resize((size_t)c->nrows + 1);
  } catch (...) { delete c; return SFX_ERR_ALLOC; }
  // row lengths: Q_p -- the pattern is the Kronecker product of the 1D
  // patterns (two nodes share a cell iff they share a 1D cell along every
  // axis), each a contiguous range; DQ_p -- the dofs of the row's own cell
  c->row_ptr[0] = 0;
  for (int64_t r = 0; r < c->nrows; ++r) {
    int64_t len;
    if (sp->family == SFX_DQ) {
      len = nloc;
    } else {
      const int64_t I[3] = {r / (M[1] * M[2]), (r / M[2]) % M[1], r % M[2]};
      len = 1;
      for (int d = 0; d < 3; ++d) {
        int64_t lo, hi;
        q_range_1d(I[d], p, N[d], &lo, &hi);
        len *= hi - lo + 1;
      }
    }
    c->row_ptr[r + 1] = c->row_ptr[r] + len;
  }
  c->nnz = c->row_ptr[c->nrows];
  try {
    c->col.resize((size_t)c->nnz);
  } catch (...) { delete c; return SFX_ERR_ALLOC; }
  const unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nth; ++t) {
    pool.emplace_back([&, t]() {
      for (int64_t r = t; r < c->nrows; r += nth) {
        int32_t* o = &c->col[(size_t)c->row_ptr[r]];
        if (sp->family == SFX_DQ) {
          const int64_t b = (r / nloc) * nloc;
          for (int l = 0; l < nloc; ++l) o[l] = (int32_t)(b + l);
          continue;
        }
        const int64_t I[3] = {r / (M[1] * M[2]), (r / M[2]) % M[1], r % M[2]};
        int64_t lo[3], hi[3];
        for (int d = 0; d < 3; ++d) q_range_1d(I[d], p, N[d], &lo[d], &hi[d]);
        for (int64_t a = lo[0]; a <= hi[0]; ++a)
          for (int64_t b = lo[1]; b <= hi[1]; ++b)
            for (int64_t k = lo[2]; k <= hi[2]; ++k) *o++ = (int32_t)((a * M[1] + b) * M[2] + k);
      }
    });
  }
  for (auto& th : pool) th.join();
  // lanes per row, by measurement: few for short rows, because on this GPU an
  // FP64 add of a whole warp costs 16 clocks of the SM's FP64 pipe and the
  // tree reduction over L lanes adds log2(L) of them per row; long rows (Q_5,
  // Q_6) gain more from the extra loads in flight than the reduction costs
  const double avg = c->nrows ? (double)c->nnz / (double)c->nrows : 0.0;
  c->lanes = avg < 32 ? 4 : (avg < 160 ? 8 : (avg < 400 ? 16 : 32));
  (void)n;
  if (m->ctx->device < 0) {
    *out = c;
    return SFX_OK;
  }
  sfx_status st = to_device(c->row_ptr.data(), c->row_ptr.size(), &c->d_row_ptr);
  if (!st) st = to_device(c->col.data(), c->col.size(), &c->d_col);
  if (!st) {
    const int64_t per = (int64_t)nloc * nloc * (int64_t)sizeof(double);
    c->chunk = std::max<int64_t>(1, std::min<int64_t>(m->ncell, (512LL << 20) / per));
    if (cudaMalloc((void**)&c->d_scratch, (size_t)(c->chunk * per)) != cudaSuccess) {
      c->d_scratch = nullptr;
      st = SFX_ERR_ALLOC;
    }
  }
  if (st) { sfx_csr_destroy(c); return st; }
  *out = c;
  return SFX_OK;
}

extern "C" sfx_status sfx_csr_info(const sfx_csr* c, int64_t* nrows, int64_t* nnz, const int64_t** row_ptr,
                                   const int32_t** col) {
  if (!c) return SFX_ERR_ARG;
  if (nrows) *nrows = c->nrows;
  if (nnz) *nnz = c->nnz;
  if (row_ptr) *row_ptr = c->row_ptr.data();
  if (col) *col = c->col.data();
  return SFX_OK;
}

extern "C" sfx_status sfx_csr_assemble(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                       const sfx_csr* c, double* values, void* stream) {
  Range range("sfx_csr_assemble");
  if (!ctx || !c || !values || ctx->device < 0 || !c->d_col) return SFX_ERR_ARG;
  const sfx_space* sp = c->space;
  if (form != SFX_MASS && form != SFX_LAPLACE && form != SFX_HELMHOLTZ) return SFX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(values, 0, (size_t)c->nnz * sizeof(double), s) != cudaSuccess) return SFX_ERR_CUDA;
  const int64_t ncell = sp->mesh->ncell;
  for (int64_t b = 0; b < ncell; b += c->chunk) {
    const int64_t e = std::min(ncell, b + c->chunk);
    const sfx_status st = sfx_assemble_cell_matrices(ctx, form, params, sp, b, e, c->d_scratch, SFX_PREC_FP64,
                                                     SFX_ALGO_SUMFACT, stream);
    if (st) return st;
    // colour by colour: cells of one colour share no dof, so no row
    const int ncol = sp->family == SFX_DQ ? 1 : 8;
    for (int col = 0; col < ncol; ++col)
      if (launch_csr_scatter(c->d_scratch, b, e - b, sp->nloc, sp->d_map, c->d_row_ptr, c->d_col, values,
                             sp->family == SFX_DQ ? -1 : col, sp->mesh->ny, sp->mesh->nz, ctx->d_status, stream))
        return SFX_ERR_CUDA;
  }
  return SFX_OK;
}

extern "C" sfx_status sfx_csr_spmv(sfx_ctx* ctx, const sfx_csr* c, const double* values, const double* x,
                                   double* y, void* stream) {
  Range range("sfx_csr_spmv");
  if (!ctx || !c || !values || !x || !y || x == y || ctx->device < 0 || !c->d_col) return SFX_ERR_ARG;
  return launch_csr_spmv(c->lanes, c->nrows, c->d_row_ptr, c->d_col, values, x, y, stream) ? SFX_ERR_CUDA : SFX_OK;
}

extern "C" void sfx_csr_destroy(sfx_csr* c) {
  if (!c) return;
  if (c->d_row_ptr) cudaFree(c->d_row_ptr);
  if (c->d_col) cudaFree(c->d_col);
  if (c->d_scratch) cudaFree(c->d_scratch);
  delete c;
}

// -------------------------------------------------------------------- plans
struct sfx_plan {
  sfx_ctx* ctx = nullptr;
  const sfx_mesh* mesh = nullptr;
  int nforms = 0, nrhs = 1;
  sfx_precision prec = SFX_PREC_FP64;  // tile body: FP64, or the split-precision body
  sfx_form forms[4];
  sfx_form_params params[4];
  int64_t ndof = 0;
  std::vector<int64_t> off;          // host dof offset of every cell (ncell + 1)
  int64_t* d_off = nullptr;
  int32_t* d_sorted = nullptr;       // cells sorted by degree
  int64_t deg_begin[kMaxDeg + 2] = {0}, deg_end[kMaxDeg + 2] = {0};
  std::vector<BatchTile> tiles;
  BatchTile* d_tiles = nullptr;
  int* d_counter = nullptr;
  int cb[kMaxDeg + 1] = {0};
  size_t smem = 0;
  int grid = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double* gx = nullptr;
  double* gy[4] = {nullptr, nullptr, nullptr, nullptr};
};

extern "C" void sfx_plan_destroy(sfx_plan* pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  if (pl->d_off) cudaFree(pl->d_off);
  if (pl->d_sorted) cudaFree(pl->d_sorted);
  if (pl->d_tiles) cudaFree(pl->d_tiles);
  if (pl->d_counter) cudaFree(pl->d_counter);
  delete pl;
}

extern "C" sfx_status sfx_plan_create_padaptive(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree,
                                                int nforms, const sfx_form* forms, const sfx_form_params* params,
                                                int nrhs, sfx_plan** out) {
  return sfx_plan_create_padaptive_prec(ctx, mesh, degree, nforms, forms, params, nrhs, SFX_PREC_FP64, out);
}

extern "C" sfx_status sfx_plan_create_padaptive_prec(sfx_ctx* ctx, const sfx_mesh* mesh, const int32_t* degree,
                                                     int nforms, const sfx_form* forms,
                                                     const sfx_form_params* params, int nrhs, sfx_precision prec,
                                                     sfx_plan** out) {
  if (!ctx || !mesh || !degree || !forms || !out || nforms < 1 || nforms > 4 || nrhs < 1 || nrhs > 64)
    return SFX_ERR_ARG;
  if (prec != SFX_PREC_FP64 && prec != SFX_PREC_TF32X3 && prec != SFX_PREC_BF16X3) return SFX_ERR_ARG;
  if (ctx->device < 0 || mesh->ctx != ctx || !mesh->d_vmap) return SFX_ERR_ARG;
  *out = nullptr;
  for (int f = 0; f < nforms; ++f)
    if (forms[f] != SFX_MASS && forms[f] != SFX_LAPLACE && forms[f] != SFX_HELMHOLTZ) return SFX_ERR_UNSUPPORTED;
  const int64_t ncell = mesh->ncell;
  for (int64_t c = 0; c < ncell; ++c)
    if (degree[c] < 1 || degree[c] > kMaxDeg) return SFX_ERR_ARG;
  sfx_plan* pl = new (std::nothrow) sfx_plan;
  if (!pl) return SFX_ERR_ALLOC;
  pl->ctx = ctx;
  pl->mesh = mesh;
  pl->nforms = nforms;
  pl->nrhs = nrhs;
  pl->prec = prec;
  for (int f = 0; f < nforms; ++f) {
    pl->forms[f] = forms[f];
    pl->params[f] = params ? params[f] : default_params(forms[f]);
  }
  // dof offsets (cell-major DQ numbering: cell c owns (p_c+1)^3 consecutive dofs)
  pl->off.resize((size_t)ncell + 1);
  pl->off[0] = 0;
  for (int64_t c = 0; c < ncell; ++c) {
    const int64_t n = degree[c] + 1;
    pl->off[c + 1] = pl->off[c] + n * n * n;
  }
  pl->ndof = pl->off[ncell];
  if (pl->ndof * nrhs >= (1LL << 40)) { sfx_plan_destroy(pl); return SFX_ERR_RANGE; }
  // cells sorted by degree (stable), per-degree ranges
  std::vector<int32_t> sorted;
  sorted.reserve((size_t)ncell);
  for (int p = 1; p <= kMaxDeg; ++p) {
    pl->deg_begin[p] = (int64_t)sorted.size();
    for (int64_t c = 0; c < ncell; ++c)
      if (degree[c] == p) sorted.push_back((int32_t)c);
    pl->deg_end[p] = (int64_t)sorted.size();
  }
  sfx_status st = SFX_OK;
  int form_mask = 0;
  for (int f = 0; f < nforms; ++f) form_mask |= 1 << (int)forms[f];
  int ce = 0;
  if (prec == SFX_PREC_FP64) ce = batched_config(pl->cb, &pl->smem, &pl->grid);
  else if (prec == SFX_PREC_TF32X3) ce = batched_mixed_config_tf32(form_mask, nrhs, pl->cb, &pl->smem, &pl->grid);
  else ce = batched_mixed_config_bf16(form_mask, nrhs, pl->cb, &pl->smem, &pl->grid);
  if (ce != 0) st = SFX_ERR_CUDA;
  // tiles: largest degree first, then form, then cells
  for (int p = kMaxDeg; p >= 1 && !st; --p)
    for (int f = 0; f < nforms; ++f)
      for (int64_t c0 = pl->deg_begin[p]; c0 < pl->deg_end[p]; c0 += pl->cb[p]) {
        BatchTile t;
        t.p = p;
        t.form = f;
        t.first = (int32_t)c0;
        t.count = (int32_t)std::min<int64_t>(pl->cb[p], pl->deg_end[p] - c0);
        pl->tiles.push_back(t);
      }
  if (!st) st = to_device(pl->off.data(), pl->off.size(), &pl->d_off);
  if (!st) st = to_device(sorted.data(), sorted.size(), &pl->d_sorted);
  if (!st && !pl->tiles.empty()) st = to_device(pl->tiles.data(), pl->tiles.size(), &pl->d_tiles);
  if (!st && cudaMalloc(&pl->d_counter, sizeof(int)) != cudaSuccess) st = SFX_ERR_ALLOC;
  if (!st && cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) != cudaSuccess) st = SFX_ERR_CUDA;
  if (!st) {
    for (int p = 1; p <= kMaxDeg && !st; ++p) {  // constant tables for every degree
      Tab1D t;
      make_tab1d(p, &t);
      if (upload_tables(&t) != 0) st = SFX_ERR_CUDA;
    }
  }
  if (st) { sfx_plan_destroy(pl); return st; }
  *out = pl;
  return SFX_OK;
}

extern "C" sfx_status sfx_plan_info(const sfx_plan* pl, int64_t* ndof, int64_t* ntiles, const int64_t** cell_offset) {
  if (!pl) return SFX_ERR_ARG;
  if (ndof) *ndof = pl->ndof;
  if (ntiles) *ntiles = (int64_t)pl->tiles.size();
  if (cell_offset) *cell_offset = pl->off.data();
  return SFX_OK;
}

static ActArgs plan_args(const sfx_plan* pl, const double* x) {
  ActArgs a{};
  a.map = nullptr;
  a.dq_off = pl->d_off;
  a.vmap = pl->mesh->d_vmap;
  a.xyz = pl->mesh->d_xyz;
  a.x = x;
  a.nrhs = pl->nrhs;
  a.r0 = 0;
  a.r1 = pl->nrhs;
  a.status = pl->ctx->d_status;
  // every (cell, l) of a p-adaptive DQ space is its dof's only pair: with one
  // right-hand side the kernels store b^K into y, which then needs no memset
  // (with several, y is zeroed and added to; see first_touch_pays)
  a.first_all = first_touch_pays(pl->prec, pl->nrhs) ? 1 : 0;
  return a;
}

extern "C" sfx_status sfx_plan_execute(sfx_plan* pl, const double* x, double* const* y, sfx_exec_mode mode,
                                       void* stream) {
  Range range("sfx_plan_execute");
  if (!pl || !x || !y) return SFX_ERR_ARG;
  for (int f = 0; f < pl->nforms; ++f)
    if (!y[f] || y[f] == x) return SFX_ERR_ARG;
  const size_t ybytes = (size_t)pl->ndof * pl->nrhs * sizeof(double);
  const bool zero = !first_touch_pays(pl->prec, pl->nrhs);
  cudaStream_t s = (cudaStream_t)stream;
  if (mode == SFX_EXEC_PER_LAUNCH) {
    for (int f = 0; f < pl->nforms; ++f) {
      if (zero && cudaMemsetAsync(y[f], 0, ybytes, s) != cudaSuccess) return SFX_ERR_CUDA;
      for (int p = 1; p <= kMaxDeg; ++p) {
        const int64_t cnt = pl->deg_end[p] - pl->deg_begin[p];
        if (cnt == 0) continue;
        if (pl->prec != SFX_PREC_FP64) {
          // split precision: one launch per (form, degree), all right-hand sides
          ActArgs a = plan_args(pl, x);
          a.cells = pl->d_sorted + pl->deg_begin[p];
          a.ncells = cnt;
          a.y = y[f];
          a.alpha = pl->params[f].alpha;
          a.beta = pl->params[f].beta;
          const int e = pl->prec == SFX_PREC_TF32X3
                            ? launch_scalar_mixed_degree_tf32(p, true, pl->forms[f], a, pl->mesh->ncell, stream)
                            : launch_scalar_mixed_degree_bf16(p, true, pl->forms[f], a, pl->mesh->ncell, stream);
          if (e != 0) return SFX_ERR_CUDA;
          continue;
        }
        for (int r = 0; r < pl->nrhs; ++r) {
          ActArgs a = plan_args(pl, x);
          a.cells = pl->d_sorted + pl->deg_begin[p];
          a.ncells = cnt;
          a.y = y[f];
          a.r0 = r;
          a.r1 = r + 1;
          a.stage_factors = 1;  // same per-point arithmetic as the persistent kernel
          a.alpha = pl->params[f].alpha;
          a.beta = pl->params[f].beta;
          if (launch_scalar_fp64_degree(p, true, pl->forms[f], a, pl->mesh->ncell, stream) != 0) return SFX_ERR_CUDA;
        }
      }
    }
    return SFX_OK;
  }
  if (mode != SFX_EXEC_GRAPH) return SFX_ERR_ARG;
  bool same = pl->exec && pl->gx == x;
  for (int f = 0; f < pl->nforms && same; ++f) same = pl->gy[f] == y[f];
  if (!same) {
    if (pl->exec) { cudaGraphExecDestroy(pl->exec); pl->exec = nullptr; }
    BatchArgs b{};
    b.base = plan_args(pl, x);
    b.sorted_cells = pl->d_sorted;
    b.tiles = pl->d_tiles;
    b.ntiles = (int)pl->tiles.size();
    b.counter = pl->d_counter;
    b.ncell_total = pl->mesh->ncell;
    for (int f = 0; f < pl->nforms; ++f) {
      b.y[f] = y[f];
      b.alpha[f] = pl->params[f].alpha;
      b.beta[f] = pl->params[f].beta;
      b.form_id[f] = pl->forms[f];
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SFX_ERR_CUDA;
    int e = 0;
    for (int f = 0; f < pl->nforms && zero && !e; ++f) e = (int)cudaMemsetAsync(y[f], 0, ybytes, pl->cap);
    if (!e) e = (int)cudaMemsetAsync(pl->d_counter, 0, sizeof(int), pl->cap);
    if (!e && b.ntiles > 0) {
      if (pl->prec == SFX_PREC_FP64) e = batched_launch(b, pl->grid, pl->smem, pl->cap);
      else if (pl->prec == SFX_PREC_TF32X3) e = batched_mixed_launch_tf32(b, pl->nrhs, pl->grid, pl->smem, pl->cap);
      else e = batched_mixed_launch_bf16(b, pl->nrhs, pl->grid, pl->smem, pl->cap);
    }
    cudaError_t ee = cudaStreamEndCapture(pl->cap, &g);
    if (e || ee != cudaSuccess || !g) { if (g) cudaGraphDestroy(g); return SFX_ERR_CUDA; }
    ee = cudaGraphInstantiate(&pl->exec, g, 0);
    cudaGraphDestroy(g);
    if (ee != cudaSuccess) { pl->exec = nullptr; return SFX_ERR_CUDA; }
    pl->gx = x;
    for (int f = 0; f < pl->nforms; ++f) pl->gy[f] = y[f];
  }
  return cudaGraphLaunch(pl->exec, s) == cudaSuccess ? SFX_OK : SFX_ERR_CUDA;
}

// ---------------------------------------------------- stored geometry factors
extern "C" void sfx_qdata_destroy(sfx_qdata* q) {
  if (!q) return;
  if (q->d64) cudaFree(q->d64);
  if (q->d32) cudaFree(q->d32);
  delete q;
}

extern "C" sfx_status sfx_qdata_create(sfx_ctx* ctx, const sfx_space* sp, int formats, void* stream, sfx_qdata** out) {
  Range range("sfx_qdata_create");
  if (!ctx || !sp || !out || ctx->device < 0 || !sp->d_map) return SFX_ERR_ARG;
  if ((formats & ~(SFX_QDATA_FP64 | SFX_QDATA_FP32)) || !formats) return SFX_ERR_ARG;
  *out = nullptr;
  if (sp->family != SFX_Q && sp->family != SFX_DQ) return SFX_ERR_UNSUPPORTED;
  sfx_qdata* q = new (std::nothrow) sfx_qdata;
  if (!q) return SFX_ERR_ALLOC;
  q->space = sp;
  const int64_t n = sp->p + 1;
  const size_t cnt = (size_t)sp->mesh->ncell * 7 * n * n * n;
  if ((formats & SFX_QDATA_FP64) && cudaMalloc(&q->d64, cnt * sizeof(double)) != cudaSuccess) {
    q->d64 = nullptr; sfx_qdata_destroy(q); return SFX_ERR_ALLOC;
  }
  if ((formats & SFX_QDATA_FP32) && cudaMalloc(&q->d32, cnt * sizeof(float)) != cudaSuccess) {
    q->d32 = nullptr; sfx_qdata_destroy(q); return SFX_ERR_ALLOC;
  }
  q->fp32 = (formats & SFX_QDATA_FP32) != 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (launch_qdata(sp, q, ctx->d_status, stream) != 0 || cudaStreamSynchronize(s) != cudaSuccess) {
    sfx_qdata_destroy(q);
    return SFX_ERR_CUDA;
  }
  *out = q;
  return SFX_OK;
}

extern "C" sfx_status sfx_assemble_action_stored(sfx_ctx* ctx, sfx_form form, const sfx_form_params* params,
                                                 const sfx_space* sp, const sfx_qdata* q, const double* x, double* y,
                                                 int nrhs, int accumulate, sfx_precision prec, void* stream) {
  Range range("sfx_assemble_action_stored");
  if (!ctx || !sp || !q || !x || !y || x == y || nrhs < 1 || nrhs > 64 || ctx->device < 0 || !sp->d_map)
    return SFX_ERR_ARG;
  if (q->space != sp) return SFX_ERR_ARG;
  if (form != SFX_MASS && form != SFX_LAPLACE && form != SFX_HELMHOLTZ) return SFX_ERR_ARG;
  if (prec < SFX_PREC_FP64 || prec > SFX_PREC_BF16X3) return SFX_ERR_ARG;
  if ((prec == SFX_PREC_FP64 && !q->d64) || (prec != SFX_PREC_FP64 && !q->d32)) return SFX_ERR_ARG;
  sfx_form_params pr = params ? *params : default_params(form);
  cudaStream_t s = (cudaStream_t)stream;
  ActArgs a{};
  if (!accumulate) set_first_touch(sp, prec, nrhs, &a);
  if (!accumulate && !a.first && !a.first_all &&
      cudaMemsetAsync(y, 0, (size_t)sp->ndof * nrhs * sizeof(double), s) != cudaSuccess)
    return SFX_ERR_CUDA;
  a.map = sp->d_map;
  a.vmap = sp->mesh->d_vmap;
  a.xyz = sp->mesh->d_xyz;
  a.x = x;
  a.y = y;
  a.nrhs = nrhs;
  a.r0 = 0;
  a.r1 = nrhs;
  a.alpha = pr.alpha;
  a.beta = pr.beta;
  a.status = ctx->d_status;
  if (prec == SFX_PREC_FP64) a.qd64 = q->d64; else a.qd32 = q->d32;
  bool launched = false;
  for (int col = 0; col < sp->ncolour; ++col) {
    a.cells = sp->d_cells + sp->colour_off[col];
    a.ncells = sp->colour_off[col + 1] - sp->colour_off[col];
    if (a.ncells == 0) continue;
    a.overlap_prev = launched ? 1 : 0;
    launched = true;
    const int e = launch_action_scalar(sp, form, prec, SFX_ALGO_SUMFACT, a, stream);
    if (e == -1) return SFX_ERR_UNSUPPORTED;
    if (e) return SFX_ERR_CUDA;
  }
  return SFX_OK;
}
