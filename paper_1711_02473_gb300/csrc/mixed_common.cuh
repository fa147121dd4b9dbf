#pragma once
// mixed_common.cuh -- split-precision 1D contractions on the tensor cores,
// shared by the scalar and the hyperelastic split-precision actions.
//
// A contraction out = M in along one axis of a [cells][N][N][N] array is one
// batched matrix product per CTA: the 1D table (padded to 16 x 8k) times the
// fibers of all the CTA's cells, on mma.sync with FP32 accumulation.  Each
// operand is split into a high and a low part in the input format (TF32: 11
// significant bits each; BF16: 8 each) and the three products hi*hi + hi*lo +
// lo*hi are accumulated (lo*lo is dropped).
#include <cuda_bf16.h>

#include "kern_common.cuh"

namespace sfx {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ uint32_t tf32_bits(float v) { return __float_as_uint(v) & 0xffffe000u; }

// split v into tf32 hi + tf32 lo (both as b32 registers)
__device__ __forceinline__ void split_tf32(float v, uint32_t& hi, uint32_t& lo) {
  hi = tf32_bits(v);
  lo = tf32_bits(v - __uint_as_float(hi));
}
// split v into bf16 hi + bf16 lo (returned in the high 16 bits of a b32)
__device__ __forceinline__ void split_bf16(float v, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(v) & 0xffff0000u;
  lo = __float_as_uint(v - __uint_as_float(hi)) & 0xffff0000u;
}
__device__ __forceinline__ uint32_t pack_bf16(uint32_t first, uint32_t second) {
  return (first >> 16) | (second & 0xffff0000u);
}

__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// FP32 copy of a 1D table, zero-padded to 16 x 16, row = output index.
struct TabF {
  float v[16][16];
};

// Address of element (fiber f of cell c, index k along AX) in a [cells][N][N][N] array.
template <int N, int AX>
__device__ __forceinline__ int faddr(int c, int f, int k) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int f0 = f / N, f1 = f - (f / N) * N;
  if (AX == 0) return c * N3 + k * N2 + f0 * N + f1;
  if (AX == 1) return c * N3 + f0 * N2 + k * N + f1;
  return c * N3 + f0 * N2 + f1 * N + k;
}

// out[c, .., r, ..] (+)= sum_k M[r][k] in[c, .., k, ..] along axis AX for every
// fiber of every cell in the CTA (TRANS: M[k][r]).  One warp owns 8 fibers at a
// time (the n dimension of the mma); in-place use is safe because a warp reads
// all of its fibers before writing them and no other warp touches them.
// NT: threads taking part (whole warps, starting at warp WOFF of the CTA).
// NSUM > 1: the input is the sum of NSUM arrays `sstride` floats apart (in,
// in + sstride, ...), plus the array sstride before `in` when PRE, summed in
// FP32 as the values are loaded; in-place use (out = in or out = in - sstride)
// stays safe for the same reason.
template <int N, int AX, bool TRANS, bool ACC, int PREC, int NT = kThreads, int WOFF = 0, int NSUM = 1,
          bool PRE = false>
__device__ __forceinline__ void tc_contract(const float* in, float* out, const TabF& M, int ncell, int sstride = 0) {
  constexpr int NW = NT / 32;
  constexpr int N2 = N * N;
  const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - WOFF;
  const int g = lane >> 2, tq = lane & 3;
  const int nfib = ncell * N2;
  const int ntiles = (nfib + 7) >> 3;
  auto A = [&](int r, int k) -> float { return TRANS ? M.v[k][r] : M.v[r][k]; };
  auto ld = [&](int a) -> float {
    float v = in[a];
#pragma unroll
    for (int s = 1; s < NSUM; ++s) v += in[a + s * sstride];
    if (PRE) v += in[a - sstride];
    return v;
  };
  if (PREC == SFX_PREC_TF32X3) {
    constexpr int KS = (N + 7) / 8;
    uint32_t ah[KS][4], al[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const int k0 = ks * 8 + tq;
      split_tf32(A(g, k0), ah[ks][0], al[ks][0]);
      split_tf32(A(g + 8, k0), ah[ks][1], al[ks][1]);
      split_tf32(A(g, k0 + 4), ah[ks][2], al[ks][2]);
      split_tf32(A(g + 8, k0 + 4), ah[ks][3], al[ks][3]);
    }
    for (int tile = warp; tile < ntiles; tile += NW) {
      const int fb = tile * 8 + g;
      const bool vb = fb < nfib;
      const int cb = vb ? fb / N2 : 0, lb = vb ? fb - cb * N2 : 0;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int k0 = ks * 8 + tq, k1 = k0 + 4;
        const float v0 = (vb && k0 < N) ? ld(faddr<N, AX>(cb, lb, k0)) : 0.f;
        const float v1 = (vb && k1 < N) ? ld(faddr<N, AX>(cb, lb, k1)) : 0.f;
        uint32_t h0, l0, h1, l1;
        split_tf32(v0, h0, l0);
        split_tf32(v1, h1, l1);
        mma_tf32(c, ah[ks], h0, h1);
        mma_tf32(c, ah[ks], l0, l1);
        mma_tf32(c, al[ks], h0, h1);
      }
      __syncwarp();
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = g + ((e >> 1) << 3);
        const int fc = tile * 8 + 2 * tq + (e & 1);
        if (r < N && fc < nfib) {
          const int cc = fc / N2, lc = fc - cc * N2;
          const int ad = faddr<N, AX>(cc, lc, r);
          out[ad] = ACC ? out[ad] + c[e] : c[e];
        }
      }
    }
  } else {  // BF16x3, m16n8k16: one k-step covers n <= 16
    uint32_t ah[4], al[4];
    {
      uint32_t h[8], l[8];
      const int rr[8] = {g, g, g + 8, g + 8, g, g, g + 8, g + 8};
      const int kk[8] = {2 * tq, 2 * tq + 1, 2 * tq, 2 * tq + 1, 2 * tq + 8, 2 * tq + 9, 2 * tq + 8, 2 * tq + 9};
#pragma unroll
      for (int e = 0; e < 8; ++e) split_bf16(A(rr[e], kk[e]), h[e], l[e]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ah[q] = pack_bf16(h[2 * q], h[2 * q + 1]);
        al[q] = pack_bf16(l[2 * q], l[2 * q + 1]);
      }
    }
    for (int tile = warp; tile < ntiles; tile += NW) {
      const int fb = tile * 8 + g;
      const bool vb = fb < nfib;
      const int cb = vb ? fb / N2 : 0, lb = vb ? fb - cb * N2 : 0;
      float v[4];
      const int kk[4] = {2 * tq, 2 * tq + 1, 2 * tq + 8, 2 * tq + 9};
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (vb && kk[e] < N) ? ld(faddr<N, AX>(cb, lb, kk[e])) : 0.f;
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) split_bf16(v[e], h[e], l[e]);
      const uint32_t bh0 = pack_bf16(h[0], h[1]), bh1 = pack_bf16(h[2], h[3]);
      const uint32_t bl0 = pack_bf16(l[0], l[1]), bl1 = pack_bf16(l[2], l[3]);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c, ah, bh0, bh1);
      mma_bf16(c, ah, bl0, bl1);
      mma_bf16(c, al, bh0, bh1);
      __syncwarp();
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = g + ((e >> 1) << 3);
        const int fc = tile * 8 + 2 * tq + (e & 1);
        if (r < N && fc < nfib) {
          const int cc = fc / N2, lc = fc - cc * N2;
          const int ad = faddr<N, AX>(cc, lc, r);
          out[ad] = ACC ? out[ad] + c[e] : c[e];
        }
      }
    }
  }
}

// The same contraction on a [cells][I0][I1][I2] array whose axis AX changes
// length, K = I_AX -> R (the anisotropic blocks of NCF_p / NCE_p, Sec. 3.5:
// tables of the P_p factor, q x (p+1), and of the dP_{p-1} factor, q x p).
// The fibers are the other two axes; CSI / CSO are the cell strides of in and
// out (floats).  NEG negates the product before it is stored or added.
template <int I0, int I1, int I2, int AX, int R, int CSI, int CSO, bool TRANS, bool ACC, bool NEG, int PREC,
          int NT = kThreads>
__device__ __forceinline__ void tc_contract_g(const float* in, float* out, const TabF& M, int ncell) {
  constexpr int NW = NT / 32;
  constexpr int K = AX == 0 ? I0 : (AX == 1 ? I1 : I2);
  constexpr int F = I0 * I1 * I2 / K;  // fibers per cell
  constexpr int O1 = AX == 1 ? R : I1, O2 = AX == 2 ? R : I2;
  static_assert(K <= 16 && R <= 16, "1D tables are at most 16 x 16");
  auto ain = [](int c, int f, int k) -> int {
    if (AX == 0) return c * CSI + k * (I1 * I2) + f;
    if (AX == 1) {
      const int f0 = f / I2, f1 = f - (f / I2) * I2;
      return c * CSI + f0 * (I1 * I2) + k * I2 + f1;
    }
    return c * CSI + f * I2 + k;
  };
  auto aout = [](int c, int f, int r) -> int {
    if (AX == 0) return c * CSO + r * (O1 * O2) + f;
    if (AX == 1) {
      const int f0 = f / O2, f1 = f - (f / O2) * O2;
      return c * CSO + f0 * (O1 * O2) + r * O2 + f1;
    }
    return c * CSO + f * R + r;
  };
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int nfib = ncell * F;
  const int ntiles = (nfib + 7) >> 3;
  auto A = [&](int r, int k) -> float { return TRANS ? M.v[k][r] : M.v[r][k]; };
  auto store = [&](int tile, const float* c) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = g + ((e >> 1) << 3);
      const int fc = tile * 8 + 2 * tq + (e & 1);
      if (r < R && fc < nfib) {
        const int cc = fc / F, lc = fc - cc * F;
        const int ad = aout(cc, lc, r);
        const float v = NEG ? -c[e] : c[e];
        out[ad] = ACC ? out[ad] + v : v;
      }
    }
  };
  if (PREC == SFX_PREC_TF32X3) {
    constexpr int KS = (K + 7) / 8;
    uint32_t ah[KS][4], al[KS][4];
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const int k0 = ks * 8 + tq;
      split_tf32(A(g, k0), ah[ks][0], al[ks][0]);
      split_tf32(A(g + 8, k0), ah[ks][1], al[ks][1]);
      split_tf32(A(g, k0 + 4), ah[ks][2], al[ks][2]);
      split_tf32(A(g + 8, k0 + 4), ah[ks][3], al[ks][3]);
    }
    for (int tile = warp; tile < ntiles; tile += NW) {
      const int fb = tile * 8 + g;
      const bool vb = fb < nfib;
      const int cb = vb ? fb / F : 0, lb = vb ? fb - cb * F : 0;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const int k0 = ks * 8 + tq, k1 = k0 + 4;
        const float v0 = (vb && k0 < K) ? in[ain(cb, lb, k0)] : 0.f;
        const float v1 = (vb && k1 < K) ? in[ain(cb, lb, k1)] : 0.f;
        uint32_t h0, l0, h1, l1;
        split_tf32(v0, h0, l0);
        split_tf32(v1, h1, l1);
        mma_tf32(c, ah[ks], h0, h1);
        mma_tf32(c, ah[ks], l0, l1);
        mma_tf32(c, al[ks], h0, h1);
      }
      __syncwarp();
      store(tile, c);
    }
  } else {  // BF16x3, m16n8k16: one k-step covers K <= 16
    uint32_t ah[4], al[4];
    {
      uint32_t h[8], l[8];
      const int rr[8] = {g, g, g + 8, g + 8, g, g, g + 8, g + 8};
      const int kk[8] = {2 * tq, 2 * tq + 1, 2 * tq, 2 * tq + 1, 2 * tq + 8, 2 * tq + 9, 2 * tq + 8, 2 * tq + 9};
#pragma unroll
      for (int e = 0; e < 8; ++e) split_bf16(A(rr[e], kk[e]), h[e], l[e]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ah[q] = pack_bf16(h[2 * q], h[2 * q + 1]);
        al[q] = pack_bf16(l[2 * q], l[2 * q + 1]);
      }
    }
    for (int tile = warp; tile < ntiles; tile += NW) {
      const int fb = tile * 8 + g;
      const bool vb = fb < nfib;
      const int cb = vb ? fb / F : 0, lb = vb ? fb - cb * F : 0;
      float v[4];
      const int kk[4] = {2 * tq, 2 * tq + 1, 2 * tq + 8, 2 * tq + 9};
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (vb && kk[e] < K) ? in[ain(cb, lb, kk[e])] : 0.f;
      uint32_t h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) split_bf16(v[e], h[e], l[e]);
      const uint32_t bh0 = pack_bf16(h[0], h[1]), bh1 = pack_bf16(h[2], h[3]);
      const uint32_t bl0 = pack_bf16(l[0], l[1]), bl1 = pack_bf16(l[2], l[3]);
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c, ah, bh0, bh1);
      mma_bf16(c, ah, bl0, bl1);
      mma_bf16(c, al, bh0, bh1);
      __syncwarp();
      store(tile, c);
    }
  }
}

}  // namespace
}  // namespace sfx
