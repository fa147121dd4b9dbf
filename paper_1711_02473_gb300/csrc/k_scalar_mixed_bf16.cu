// k_scalar_mixed_bf16.cu -- BF16x3 instantiation of the split-precision scalar
// actions (body and launcher in scalar_mixed_body.cuh).  The two formats are
// separate translation units so that the build compiles them in parallel.
#include "scalar_mixed_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_scalar_mixed_bf16)

int launch_action_scalar_mixed_bf16(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  return launch_scalar_mixed_prec<SFX_PREC_BF16X3>(sp, form, a, stream);
}

int launch_scalar_mixed_degree_bf16(int p, bool dq, sfx_form form, const ActArgs& a, int64_t ncell_total,
                                   void* stream) {
  return launch_scalar_mixed_degree<SFX_PREC_BF16X3>(p, dq, form, a, ncell_total, stream);
}

}  // namespace sfx
