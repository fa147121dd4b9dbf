// k_probe.cu -- throughput probes of the execution units the roofline divides
// by: FP64 FMA (the binding unit of the geometry and of the FP64 kernels),
// FP32 FMA, and the tensor-core forms the split-precision contractions use
// (mma.sync TF32 m16n8k8, BF16 m16n8k16) plus FP64 mma.sync (m8n8k4).
//
// Each probe runs independent dependency chains (many per thread, many warps
// per SM) so that the unit, not latency, sets the rate.  The result is folded
// into one value per thread and written to `sink` so the work cannot be
// removed.  The caller times a launch with CUDA events; *ops receives the
// operations of one launch (an FMA or a multiply-add of an mma counts 2
// flops, i.e. 2 * M * N * K per mma; for DFMA/FFMA the count is FMAs, one
// FP64-pipe operation each, matching the roofline's FP64-operation unit).
#include <cuda_runtime.h>

#include "sfx_internal.h"

namespace sfx {
namespace {

constexpr int kChains = 8;

__global__ void k_probe_dfma(int iters, double seed, double* sink) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + threadIdx.x * 1e-7 + k * 1e-3;
  const double m = 0.999999999, c = 1e-9;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_ffma(int iters, double seed, double* sink) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)seed + threadIdx.x * 1e-5f + k * 1e-3f;
  const float m = 0.9999999f, c = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Tensor-core probes: kChains independent accumulators per warp, the same
// operand registers (values are irrelevant to the rate).
__global__ void k_probe_mma_tf32(int iters, double seed, double* sink) {
  uint32_t a[4], b[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = __float_as_uint((float)seed + k) & 0xffffe000u;
  b[0] = a[1];
  b[1] = a[2];
  float c[kChains][4] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      asm volatile(
          "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_mma_bf16(int iters, double seed, double* sink) {
  uint32_t a[4], b[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = 0x3f803f80u + (uint32_t)k + (uint32_t)(seed > 2.0);
  b[0] = a[1];
  b[1] = a[2];
  float c[kChains][4] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k][0] + c[k][1] + c[k][2] + c[k][3];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_probe_dmma(int iters, double seed, double* sink) {
  const double a = seed * 1e-3, b = seed * 2e-3;
  double c[kChains][2] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += c[k][0] + c[k][1];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace sfx

using namespace sfx;

extern "C" sfx_status sfx_probe_launch(int kind, int blocks, int threads, int iters, double* sink, void* stream,
                                       double* ops) {
  if (blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1 || !sink || !ops)
    return SFX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const double nthr = (double)blocks * threads, nwarp = nthr / 32.0;
  switch (kind) {
    case SFX_PROBE_DFMA:
      k_probe_dfma<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
      *ops = nthr * iters * 16.0 * kChains;
      break;
    case SFX_PROBE_FFMA:
      k_probe_ffma<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
      *ops = nthr * iters * 16.0 * kChains;
      break;
    case SFX_PROBE_MMA_TF32:
      k_probe_mma_tf32<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
      *ops = nwarp * iters * kChains * 2.0 * 16 * 8 * 8;
      break;
    case SFX_PROBE_MMA_BF16:
      k_probe_mma_bf16<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
      *ops = nwarp * iters * kChains * 2.0 * 16 * 8 * 16;
      break;
    case SFX_PROBE_DMMA:
      k_probe_dmma<<<blocks, threads, 0, s>>>(iters, 1.0, sink);
      *ops = nwarp * iters * kChains * 2.0 * 8 * 8 * 4;
      break;
    default:
      return SFX_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? SFX_OK : SFX_ERR_CUDA;
}
