// k_batched_mixed_bf16.cu -- BF16x3 instantiation of the split-precision persistent
// p-adaptive batch (body in batched_mixed_body.cuh); one translation unit per
// format so that the build compiles them in parallel.
#include "batched_mixed_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_batched_mixed_bf16)

int batched_mixed_config_bf16(int form_mask, int nrhs, int* cb, size_t* smem, int* grid) {
  return batched_mixed_config_prec<SFX_PREC_BF16X3>(form_mask, nrhs, cb, smem, grid);
}

int batched_mixed_launch_bf16(const BatchArgs& b, int nrhs, int grid, size_t smem, void* stream) {
  return batched_mixed_launch_prec<SFX_PREC_BF16X3>(b, nrhs, grid, smem, stream);
}

}  // namespace sfx
