#pragma once
// scalar_mixed_ws.cuh -- warp-specialised split-precision scalar action
// (Laplace and Helmholtz on Q_p and DQ_p, n >= 4).
//
// Same algorithm as k_action_scalar_mixed (Sec. 3.3, Eqs. coeff_eval and
// form_eval, with the sum factorisation of Sec. 3.2), with the per-point
// geometry staged once per cell of a batch.  What changes is who
// does it and when.  On this GPU the FP64 pipe (geometry: adjugate-row tables,
// det J, the weight scaling) and the other units (tensor-core contractions,
// shared-memory traffic, gathers and scatters) can run at the same time, but a
// kernel whose warps all go through the phases together uses them one after
// the other.  Here a persistent CTA splits its warps in two roles:
//   producers (NPW warps): for batch j of cb cells, the adjugate-row tables,
//     then, once the factor buffer is free, at every point t = alpha w / S
//     (FP64), the row products D = R R^T of adj J (six FP32 values) and
//     beta w S;
//   consumers (NCW warps): gather, forward contractions, the flux t (D g)
//     (the scaling by t in FP64: three operations per point, all the FP64
//     work they do), transposed contractions and scatter of batch j.
// One factor buffer is enough: the consumers read it only in their flux
// phase, so the producers fill it for batch j+1 while the consumers run the
// transposed contractions and scatter of batch j and the gather and forward
// contractions of batch j+1.
//
// Hand-off: two mbarriers in shared memory.  `full` counts the producer
// threads' arrivals (factors of a batch written), `empty` the consumer
// threads' arrivals (factors of a batch read).  Every wait polls
// mbarrier.try_wait with a suspend hint of about 1 us, at most `cap` times and
// for at most 2 s; a wait that gives up sets SFX_DEV_TIMEOUT and a shared
// abort word, after which every wait returns at once.  No thread leaves early:
// each role still passes all of its own barriers (named barrier 1 for the
// producers, 2 for the consumers, whole warps only), so the kernel always
// ends; after a timeout its output is not valid.
#include "scalar_mixed_body.cuh"

namespace sfx {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\t"
      "mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Bounded wait for the phase of `bar` with parity `parity` (see the header).
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, uint32_t cap, volatile int* abort_word,
                                        uint32_t* status) {
  if (*abort_word) return false;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < cap; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_word) return false;
    if (global_ns() - t0 > 2000000000ull) break;
  }
  *abort_word = 1;
  set_flag(status, SFX_DEV_TIMEOUT);
  return false;
}

// Producer work at point qp of a cell, from its 2D adjugate-row tables: the
// rows r_k of adj J, S = det J and t = alpha w / S (one-step Newton
// reciprocal) in FP64; the six row products D = (r_k . r_l) in FP32 from the
// rows rounded once (they only feed FP32 factors); beta w S rounded to FP32.
// The consumer applies t R R^T g as t (D g), the scaling by t in FP64, so the
// FP64 work here is the geometry alone.  Returns S.
template <int N, bool LAP, bool MAS>
__device__ __forceinline__ double ws_point_factors(const double* tab, const double* xq, const double* wq, int qp,
                                                   double alpha, double beta, float* D, double* t, float* wsm) {
  constexpr int N2 = N * N;
  constexpr int REC23 = LAP ? 16 : 4;
  const int q1 = qp / N2, q2 = (qp / N) % N, q3 = qp % N;
  double r0[3], r1[3], r2[3], w;
  const double S = adj_rows<N, REC23, LAP>(tab, tab + N2 * REC23, xq, wq, q1, q2, q3, r0, r1, r2, &w);
  if (LAP) {
    *t = (alpha * w) * recip_nr<1>(S);
    float f0[3], f1[3], f2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      f0[k] = d2f_int(r0[k]);
      f1[k] = d2f_int(r1[k]);
      f2[k] = d2f_int(r2[k]);
    }
    auto dotf = [](const float* u, const float* v) { return fmaf(u[0], v[0], fmaf(u[1], v[1], u[2] * v[2])); };
    D[0] = dotf(f0, f0);
    D[1] = dotf(f1, f1);
    D[2] = dotf(f2, f2);
    D[3] = dotf(f0, f1);
    D[4] = dotf(f0, f2);
    D[5] = dotf(f1, f2);
  }
  if (MAS) *wsm = d2f_int((beta * w) * S);
  return S;
}

template <int N, int FORM, int NPW, int NCW>
struct WsShape {
  using Sh = MixedShape<N, FORM>;
  static constexpr int N2 = N * N, N3 = N2 * N;
  static constexpr bool LAP = FORM != SFX_MASS, MAS = FORM != SFX_LAPLACE;
  static constexpr int NPT = NPW * 32, NCT = NCW * 32, NT = NPT + NCT;
  static constexpr int NK = (LAP ? 6 : 0) + (MAS ? 1 : 0);  // staged FP32 factors per point
  static constexpr int NT64 = LAP ? 1 : 0;                  // staged FP64 factors per point (t = alpha w / S)
  static constexpr int NC = LAP ? 4 : 1;                    // consumer arrays per point (U, G0..G2)
  // map entries kept in shared memory from the gather to the scatter, when
  // there is room: not with the mass factor of the Helmholtz form, which would
  // leave only one n = 9 cell per batch at two CTAs per SM
  static constexpr bool CMAP = !MAS;
  static constexpr int TMPD = 24 + kAdjEdge + kAdjT1D * N;  // corners, edge vectors, 1D vectors
  static constexpr int TABD = N2 * (Sh::REC23 + 6);         // 2D tables R23, R12
  static constexpr int PD = TMPD + TABD;                    // producer doubles per cell
  static constexpr size_t kHead = 64;                       // two mbarriers, the abort word
  static constexpr size_t bytes(int cb) {
    return kHead + 2 * sizeof(TabF) + 32 * 8 + (size_t)cb * (PD + NT64 * N3) * 8 + (size_t)cb * N3 * (NK + NC) * 4 +
           (CMAP ? (size_t)cb * N3 * 4 : 0) + (size_t)cb * 6 * 4;
  }
};

// Producer / consumer warps of a 512-thread CTA by degree and family, from
// measurement on the 64^3 Laplace and Helmholtz actions (TF32x3, ms, 8+8 ->
// chosen): 8 + 8 where the two roles bind together (Q_8); more producers where
// the FP64 geometry binds (DQ_8: 12.18 -> 12.02 Helmholtz; p = 5: 4.70 -> 4.63)
// or where 7 consumer warps still take each contraction stage's fiber tiles in
// as many rounds as 8 (p = 6: 7.10 -> 6.87; Q_4: 3.24 -> 3.21).  SFX_WS_NPW /
// SFX_WS_NCW, when defined, override the table.
constexpr int ws_npw_of(int N, bool DQ) {
  return N == 5 ? (DQ ? 8 : 9) : N == 6 ? 10 : N == 7 ? 9 : N == 9 ? (DQ ? 10 : 8) : 8;
}
#ifdef SFX_WS_NPW
constexpr int ws_npw(int, bool) { return SFX_WS_NPW; }
constexpr int ws_ncw(int, bool) { return SFX_WS_NCW; }
#else
constexpr int ws_npw(int N, bool DQ) { return ws_npw_of(N, DQ); }
constexpr int ws_ncw(int N, bool DQ) { return 16 - ws_npw_of(N, DQ); }
#endif
#ifndef SFX_WS_CTAS
#define SFX_WS_CTAS 2
#endif
#ifndef SFX_WS_PUNROLL
#define SFX_WS_PUNROLL 1
#endif

template <int N, bool DQ, int FORM, int PREC, int NPW, int NCW>
__global__ void __launch_bounds__((NPW + NCW) * 32, SFX_WS_CTAS)
    k_action_scalar_mixed_ws(const ActArgs a, const int64_t ncell_total, const int cb, const int64_t nbatch,
                             const uint32_t cap) {
  static_assert(FORM != SFX_MASS && N >= 4, "Laplace part and the staged adjugate tables (n >= 4) only");
  using W = WsShape<N, FORM, NPW, NCW>;
  constexpr int N2 = W::N2, N3 = W::N3, NPT = W::NPT, NCT = W::NCT, NT = W::NT;
  constexpr bool LAP = W::LAP, MAS = W::MAS;
  constexpr int REC23 = W::Sh::REC23;
  const Tab1D& T = c_tab[N - 1];
  extern __shared__ double smd[];
  // layout: [full, empty mbarriers; abort word][2 TabF][xq 16][wq 16]
  //         [producer doubles: cb x PD][t: cb x N3 doubles][factors: NK x cb x N3 floats]
  //         [consumer floats: NC x cb x N3][map: cb x N3 ints if CMAP][bad: cb, ccid: 2 cb, pcid: cb,
  //         cbad: 2 cb ints (the consumers' cell ids and flags alternate between two slots by batch)]
  unsigned char* base = reinterpret_cast<unsigned char*>(smd);
  uint64_t* full = reinterpret_cast<uint64_t*>(base);
  uint64_t* empty = full + 1;
  volatile int* abort_word = reinterpret_cast<volatile int*>(base + 16);
  TabF* tabs = reinterpret_cast<TabF*>(base + W::kHead);  // 0: B, 1: Dq
  double* xq = reinterpret_cast<double*>(tabs + 2);
  double* wq = xq + 16;
  double* pd = wq + 16;
  double* td = pd + (size_t)cb * W::PD;
  float* kf = reinterpret_cast<float*>(td + (size_t)cb * N3 * W::NT64);
  float* cf = kf + (size_t)cb * N3 * W::NK;
  int* cmap = reinterpret_cast<int*>(cf + (size_t)cb * N3 * W::NC);
  int* bad = cmap + (W::CMAP ? (size_t)cb * N3 : 0);
  int* ccid = bad + cb;
  int* pcid = ccid + 2 * cb;
  int* cbad = pcid + cb;

  const int tid = threadIdx.x;
  for (int i = tid; i < 16 * 16; i += NT) {
    const int r = i / 16, k = i % 16;
    tabs[0].v[r][k] = (r < N && k < N) ? (float)T.Bc[r][k] : 0.f;
    tabs[1].v[r][k] = (r < N && k < N) ? (float)T.Dq[r][k] : 0.f;
  }
  if (tid < N) {
    xq[tid] = T.x[tid];
    wq[tid] = T.w[tid];
  }
  if (tid == 0) {
    mbar_init(full, NPT);
    mbar_init(empty, NCT);
    *abort_word = 0;
  }
  __syncthreads();
  pdl_allow_next();
  const double alpha = FORM == SFX_HELMHOLTZ ? a.alpha : 1.0;
  const double beta = FORM == SFX_HELMHOLTZ ? a.beta : 1.0;

  if (tid < NPT) {
    // ------------------------------------------------------------ producers
    const int pt = tid;
    constexpr int PU = SFX_WS_PUNROLL;
    auto tmp_of = [&](int c) -> double* { return pd + (size_t)c * W::PD; };
    auto tab_of = [&](int c) -> double* { return pd + (size_t)c * W::PD + W::TMPD; };
    int j = 0;
    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x, ++j) {
      for (int c = pt; c < cb; c += NPT) {
        int cell = -1;
        if (!slot_cell(a, b * cb + c, ncell_total, &cell)) cell = -1;
        pcid[c] = cell;
      }
      named_sync(1, NPT);
      for (int i = pt; i < cb * 24; i += NPT) {
        const int c = i / 24, v = (i % 24) / 3, k = i % 3;
        const int cell = pcid[c];
        tmp_of(c)[v * 3 + k] =
            cell >= 0 ? a.xyz[(int64_t)a.vmap[(int64_t)cell * 8 + v] * 3 + k] : (double)((v >> (2 - k)) & 1);
      }
      named_sync(1, NPT);
      for (int i = pt; i < cb * kAdjEdge; i += NPT) {
        const int c = i / kAdjEdge;
        double* X = tmp_of(c);
        adj_edges(reinterpret_cast<const double(*)[3]>(X), X + 24, i - c * kAdjEdge);
      }
      named_sync(1, NPT);
      for (int i = pt; i < cb * 3 * N; i += NPT) {
        const int c = i / (3 * N), r = i - c * (3 * N);
        double* X = tmp_of(c);
        adj_1d<LAP>(X + 24, xq, X + 24 + kAdjEdge, r / N, r % N);
      }
      named_sync(1, NPT);
      for (int i = pt; i < cb * N2; i += NPT) {
        const int c = i / N2, t = i - c * N2;
        double* R23 = tab_of(c);
        adj_2d<N, REC23>(tmp_of(c) + 24 + kAdjEdge, xq, wq, R23, R23 + N2 * REC23, t);
      }
      // the factor buffer is free once the consumers have read batch j-1's
      if (j > 0) ws_wait(empty, (uint32_t)((j - 1) & 1), cap, abort_word, a.status);
      for (int c = pt; c < cb; c += NPT) bad[c] = 0;
      named_sync(1, NPT);  // also: the 2D tables of every cell are complete
      // PU points per thread per step: independent dependency chains for the
      // latency-bound FP64 / conversion sequence of each point
      for (int i0 = pt; i0 < cb * N3; i0 += PU * NPT) {
#pragma unroll
        for (int u = 0; u < PU; ++u) {
          const int i = i0 + u * NPT;
          if (i < cb * N3) {
            const int c = i / N3, qp = i - c * N3;
            float kk[6], wsm = 0.f;
            double t = 0.0;
            const double S = ws_point_factors<N, LAP, MAS>(tab_of(c), xq, wq, qp, alpha, beta, kk, &t, &wsm);
            if (!positive_finite(S)) bad[c] = 1;
            if (LAP) {
#pragma unroll
              for (int q = 0; q < 6; ++q) kf[((size_t)q * cb + c) * N3 + qp] = kk[q];
              td[(size_t)c * N3 + qp] = t;
            }
            if (MAS) kf[((size_t)(LAP ? 6 : 0) * cb + c) * N3 + qp] = wsm;
          }
        }
      }
      mbar_arrive(full);
    }
  } else {
    // ------------------------------------------------------------ consumers
    constexpr int G = 8;  // gathers in flight per thread
    const int ct = tid - NPT;
    float* U = cf;
    float* G0 = U + (size_t)cb * N3;
    float* G1 = G0 + (size_t)cb * N3;
    float* G2 = G1 + (size_t)cb * N3;
    bool waited = false;  // pdl_wait_prev passed
    int j = 0;
    for (int64_t b = blockIdx.x; b < nbatch; b += gridDim.x, ++j) {
      // this batch's slot of the cell ids and flags: threads still scattering
      // the previous batch read the other slot, so no barrier is needed
      // between that scatter and these writes
      int* const cid = ccid + (j & 1) * cb;
      int* const cfl = cbad + (j & 1) * cb;
      for (int c = ct; c < cb; c += NCT) {
        int cell = -1;
        if (!slot_cell(a, b * cb + c, ncell_total, &cell)) cell = -1;
        cid[c] = cell;
      }
      named_sync(2, NCT);
      const int tot = cb * N3;
#pragma unroll 1
      for (int r = 0; r < a.nrhs; ++r) {
        // gather: G independent (map, x) load pairs per thread in flight; the
        // map entries are kept in shared memory for the scatter (CMAP)
        auto gather = [&](const int* idx) {
          int dof[G];
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int i = idx[g];
            const int c = i / N3;
            const int cell = i >= 0 ? cid[c] : -1;
            dof[g] = cell >= 0 ? ((r == 0 || !W::CMAP) ? __ldg(&a.map[(int64_t)cell * N3 + (i - c * N3)]) : cmap[i])
                               : -1;
          }
          double xv[G];
#pragma unroll
          for (int g = 0; g < G; ++g) xv[g] = dof[g] >= 0 ? __ldg(&a.x[(int64_t)dof[g] * a.nrhs + r]) : 0.0;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const int i = idx[g];
            if (i >= 0) {
              U[i] = d2f_int(xv[g]);
              if (W::CMAP && r == 0) cmap[i] = dof[g];
            }
          }
        };
        for (int i0 = ct; i0 < tot; i0 += G * NCT) {
          int idx[G];
#pragma unroll
          for (int g = 0; g < G; ++g) idx[g] = i0 + g * NCT < tot ? i0 + g * NCT : -1;
          gather(idx);
        }
        named_sync(2, NCT);
        if (!DQ) {
          tc_contract<N, 0, false, false, PREC, NCT, NPW>(U, U, tabs[0], cb);
          named_sync(2, NCT);
          tc_contract<N, 1, false, false, PREC, NCT, NPW>(U, U, tabs[0], cb);
          named_sync(2, NCT);
          tc_contract<N, 2, false, false, PREC, NCT, NPW>(U, U, tabs[0], cb);
          named_sync(2, NCT);
        }
        tc_contract<N, 0, false, false, PREC, NCT, NPW>(U, G0, tabs[1], cb);
        tc_contract<N, 1, false, false, PREC, NCT, NPW>(U, G1, tabs[1], cb);
        tc_contract<N, 2, false, false, PREC, NCT, NPW>(U, G2, tabs[1], cb);
        if (r == 0) {
          ws_wait(full, (uint32_t)(j & 1), cap, abort_word, a.status);
          for (int c = ct; c < cb; c += NCT) cfl[c] = bad[c];
        }
        named_sync(2, NCT);
        for (int i = ct; i < tot; i += NCT) {
          const int c = i / N3, qp = i - c * N3;
          const float* kc = kf + (size_t)c * N3 + qp;
          const size_t ks = (size_t)cb * N3;
          // flux t (R R^T) g: the row products D = R R^T in FP32, the scaling
          // by t = alpha w / S in FP64
          const float g0 = G0[i], g1 = G1[i], g2 = G2[i];
          const double t = td[(size_t)c * N3 + qp];
          const float v0 = kc[0] * g0 + kc[3 * ks] * g1 + kc[4 * ks] * g2;
          const float v1 = kc[3 * ks] * g0 + kc[ks] * g1 + kc[5 * ks] * g2;
          const float v2 = kc[4 * ks] * g0 + kc[5 * ks] * g1 + kc[2 * ks] * g2;
          G0[i] = d2f_int(t * f2d_int(v0));
          G1[i] = d2f_int(t * f2d_int(v1));
          G2[i] = d2f_int(t * f2d_int(v2));
          if (MAS) U[i] = kc[6 * ks] * U[i];
        }
        if (r == a.nrhs - 1) mbar_arrive(empty);
        named_sync(2, NCT);
        // transposed derivative stages in place, one per array (no barrier
        // between them: they touch different arrays); their sum, plus the
        // mass term in U, is formed where it is read next -- in the first
        // transposed B stage (Q_p) or in the scatter (DQ_p)
        tc_contract<N, 0, true, false, PREC, NCT, NPW>(G0, G0, tabs[1], cb);
        tc_contract<N, 1, true, false, PREC, NCT, NPW>(G1, G1, tabs[1], cb);
        tc_contract<N, 2, true, false, PREC, NCT, NPW>(G2, G2, tabs[1], cb);
        named_sync(2, NCT);
        if (!DQ) {
          tc_contract<N, 0, true, false, PREC, NCT, NPW, 3, MAS>(G0, U, tabs[0], cb, cb * N3);
          named_sync(2, NCT);
          tc_contract<N, 1, true, false, PREC, NCT, NPW>(U, U, tabs[0], cb);
          named_sync(2, NCT);
          tc_contract<N, 2, true, false, PREC, NCT, NPW>(U, U, tabs[0], cb);
          named_sync(2, NCT);
        }
        // b^K at local index i: U (Q_p), or the sum of the stages (DQ_p)
        auto bk = [&](int i) -> float {
          if (!DQ) return U[i];
          const float v = G0[i] + G1[i] + G2[i];
          return MAS ? v + U[i] : v;
        };
        if (!waited) {
          pdl_wait_prev();
          waited = true;
        }
        if (a.cell_vectors) {
          for (int i = ct; i < tot; i += NCT) {
            const int c = i / N3, l = i - c * N3;
            if (cid[c] < 0) continue;
            const int64_t slot = b * cb + c;
            a.y[(slot * N3 + l) * a.nrhs + r] = !cfl[c] ? f2d_int(bk(i)) : 0.0;
          }
        } else {
          // L2 reduction (red.global.add.f64); cells of one launch share no
          // dof; in an overwriting action the dof's first pair stores instead.
          // G map entries per thread are loaded before the first write, so
          // their latencies overlap (the map is re-read from L2 unless kept
          // in shared memory)
          for (int i0 = ct; i0 < tot; i0 += G * NCT) {
            int dof[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
              const int i = i0 + g * NCT;
              const int c = i / N3;
              const int cell = i < tot ? cid[c] : -1;
              dof[g] = cell >= 0 ? (W::CMAP ? cmap[i] : __ldg(&a.map[(int64_t)cell * N3 + (i - c * N3)])) : -1;
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
              if (dof[g] < 0) continue;
              const int i = i0 + g * NCT;
              const int c = i / N3;
              const bool ok = !cfl[c];
              const bool fst = first_touch(a, cid[c], i - c * N3, N3);
              double* yp = &a.y[(int64_t)dof[g] * a.nrhs + r];
              if (fst) *yp = ok ? f2d_int(bk(i)) : 0.0;
              else if (ok) atomicAdd(yp, f2d_int(bk(i)));
            }
          }
        }
        if (r == 0)
          for (int c = ct; c < cb; c += NCT)
            if (cid[c] >= 0 && cfl[c]) set_flag(a.status, SFX_DEV_INVERTED);
        // no barrier here: a thread gathers the next right-hand side (or the
        // next batch) into the same local indices i it has just scattered, and
        // the next batch's cell ids go to the other slot
      }
    }
    if (!waited) pdl_wait_prev();
  }
}

// Host side: cells per batch (the tuned value, else the most for which two
// CTAs fit in one SM's shared memory), a persistent grid of as many CTAs as fit
// on the GPU (at most one per batch).  Returns -1 if the case is not one this
// kernel covers.
template <int N, bool DQ, int FORM, int PREC>
int launch_ws_one(const ActArgs& a, int64_t ncell_total, cudaStream_t s) {
  constexpr int NPW = ws_npw(N, DQ), NCW = ws_ncw(N, DQ);
  using W = WsShape<N, FORM, NPW, NCW>;
  const size_t max_smem = 227 * 1024, per_cta = (228 * 1024) / SFX_WS_CTAS - 1024;
  int cb = tuned_cells_per_cta(SFX_TUNE_SCALAR_MIXED_WS, N - 1, 0);
  if (cb <= 0) {
    cb = 1;
    while (cb < 32 && W::bytes(cb + 1) <= per_cta) ++cb;
  }
  while (cb > 1 && W::bytes(cb) > max_smem) --cb;
  const size_t smem = W::bytes(cb);
  if (smem > max_smem) return -1;
  auto kern = k_action_scalar_mixed_ws<N, DQ, FORM, PREC, NPW, NCW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, nsm = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return (int)e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return (int)e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W::NT, smem)) != cudaSuccess) return (int)e;
  if (per_sm < 1) per_sm = 1;
  const int64_t nbatch = (a.ncells + cb - 1) / cb;
  if (nbatch == 0) return 0;
  const int64_t grid = nbatch < (int64_t)nsm * per_sm ? nbatch : (int64_t)nsm * per_sm;
  const uint32_t cap = ws_wait_cap();
  e = launch_kernel(kern, (unsigned)grid, W::NT, smem, s, a.overlap_prev != 0, a, ncell_total, cb, nbatch, cap);
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

template <int N, int PREC>
int launch_ws_n(bool dq, sfx_form form, const ActArgs& a, int64_t nc, cudaStream_t s) {
  if (form == SFX_LAPLACE)
    return dq ? launch_ws_one<N, true, SFX_LAPLACE, PREC>(a, nc, s) : launch_ws_one<N, false, SFX_LAPLACE, PREC>(a, nc, s);
  if (form == SFX_HELMHOLTZ)
    return dq ? launch_ws_one<N, true, SFX_HELMHOLTZ, PREC>(a, nc, s)
              : launch_ws_one<N, false, SFX_HELMHOLTZ, PREC>(a, nc, s);
  return -1;
}

template <int PREC>
int launch_ws_prec(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  if (a.qd32 || a.qd64 || !ws_enabled(sp->p)) return -1;
  if (form != SFX_LAPLACE && form != SFX_HELMHOLTZ) return -1;
  const bool dq = sp->family == SFX_DQ;
  const int64_t nc = sp->mesh->ncell;
  cudaStream_t s = (cudaStream_t)stream;
  switch (sp->p) {
    case 3: return launch_ws_n<4, PREC>(dq, form, a, nc, s);
    case 4: return launch_ws_n<5, PREC>(dq, form, a, nc, s);
    case 5: return launch_ws_n<6, PREC>(dq, form, a, nc, s);
    case 6: return launch_ws_n<7, PREC>(dq, form, a, nc, s);
    case 7: return launch_ws_n<8, PREC>(dq, form, a, nc, s);
    case 8: return launch_ws_n<9, PREC>(dq, form, a, nc, s);
  }
  return -1;
}

}  // namespace
}  // namespace sfx
