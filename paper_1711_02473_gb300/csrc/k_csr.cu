// k_csr.cu -- global sparse matrix of a scalar bilinear form (CSR) and its
// product with a vector, the assembled counterpart of the matrix-free action
// (Sec. 1.1: the local tensors are added into the global matrix; Sec. 4.2
// compares the action with a product by the assembled matrix).
//
// Assembly: element matrices of a chunk of cells (k_matrix.cu, by sum
// factorisation) land in a scratch buffer; the scatter adds entry (i, j) of
// cell K into the row map(K, i) at the position of column map(K, j), found by
// binary search in the row's sorted column list.  Cells are added colour by
// colour (cells of one colour share no dof, hence no row), so the sums are
// conflict-free and run-to-run deterministic.
//
// Product y = A x: a group of L lanes per row (4 to 32 by row length: the
// reduction's FP64 adds cost a full warp slot of the FP64 pipe each, so short
// rows take few lanes), each lane striding over the row, then a butterfly
// reduction inside the group (fixed order).
#include "kern_common.cuh"

namespace sfx {

namespace {

constexpr int kCsrThreads = 256;

__global__ void __launch_bounds__(kCsrThreads)
    k_csr_scatter(const double* __restrict__ A, int64_t cell_begin, int64_t ncells, int nloc,
                  const int32_t* __restrict__ map, const int64_t* __restrict__ row_ptr,
                  const int32_t* __restrict__ col, double* __restrict__ values, int colour, int ny, int nz,
                  uint32_t* status) {
  const int64_t nl2 = (int64_t)nloc * nloc;
  const int64_t e = (int64_t)blockIdx.x * kCsrThreads + threadIdx.x;
  if (e >= ncells * nl2) return;
  const int64_t cell = cell_begin + e / nl2;
  if (colour >= 0) {
    const int64_t ci = cell / ((int64_t)ny * nz), cj = (cell / nz) % ny, ck = cell % nz;
    if ((int)((ci & 1) * 4 + (cj & 1) * 2 + (ck & 1)) != colour) return;
  }
  const int i = (int)((e / nloc) % nloc), j = (int)(e % nloc);
  const int32_t r = map[cell * nloc + i], c = map[cell * nloc + j];
  int64_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
  while (lo < hi) {  // first position with col >= c
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (col[mid] < c) lo = mid + 1; else hi = mid;
  }
  if (col[lo] != c) {  // not in the pattern: cannot happen for a pattern built from the same map
    atomicOr(status, SFX_DEV_BADCELL);
    return;
  }
  values[lo] += A[e];
}

template <int L>
__global__ void __launch_bounds__(kCsrThreads)
    k_csr_spmv(int64_t nrows, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const double* __restrict__ values, const double* __restrict__ x, double* __restrict__ y) {
  const int64_t g = ((int64_t)blockIdx.x * kCsrThreads + threadIdx.x);
  const int64_t row = g / L;
  const int lane = (int)(g % L);
  double acc = 0.0;
  if (row < nrows) {
    const int64_t b = row_ptr[row], end = row_ptr[row + 1];
    for (int64_t k = b + lane; k < end; k += L) acc = fma(values[k], x[col[k]], acc);
  }
#pragma unroll
  for (int off = L / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off, L);
  if (row < nrows && lane == 0) y[row] = acc;
}

}  // namespace

int launch_csr_scatter(const double* A, int64_t cell_begin, int64_t ncells, int nloc, const int32_t* map,
                       const int64_t* row_ptr, const int32_t* col, double* values, int colour, int ny, int nz,
                       uint32_t* status, void* stream) {
  const int64_t n = ncells * (int64_t)nloc * nloc;
  if (n == 0) return 0;
  k_csr_scatter<<<(unsigned)((n + kCsrThreads - 1) / kCsrThreads), kCsrThreads, 0, (cudaStream_t)stream>>>(
      A, cell_begin, ncells, nloc, map, row_ptr, col, values, colour, ny, nz, status);
  return (int)cudaGetLastError();
}

int launch_csr_spmv(int lanes, int64_t nrows, const int64_t* row_ptr, const int32_t* col, const double* values,
                    const double* x, double* y, void* stream) {
  const int64_t threads = nrows * lanes;
  const unsigned grid = (unsigned)((threads + kCsrThreads - 1) / kCsrThreads);
  cudaStream_t s = (cudaStream_t)stream;
  switch (lanes) {
    case 4: k_csr_spmv<4><<<grid, kCsrThreads, 0, s>>>(nrows, row_ptr, col, values, x, y); break;
    case 8: k_csr_spmv<8><<<grid, kCsrThreads, 0, s>>>(nrows, row_ptr, col, values, x, y); break;
    case 16: k_csr_spmv<16><<<grid, kCsrThreads, 0, s>>>(nrows, row_ptr, col, values, x, y); break;
    default: k_csr_spmv<32><<<grid, kCsrThreads, 0, s>>>(nrows, row_ptr, col, values, x, y); break;
  }
  return (int)cudaGetLastError();
}

}  // namespace sfx
