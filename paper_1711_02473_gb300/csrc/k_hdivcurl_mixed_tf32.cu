// k_hdivcurl_mixed_tf32.cu -- TF32x3 instantiation of the split-precision
// NCF_p / NCE_p actions (body in hdivcurl_mixed_body.cuh); one translation
// unit per format so that the build compiles them in parallel.
#include "hdivcurl_mixed_body.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_hdivcurl_mixed_tf32)

int launch_action_hdivcurl_mixed_tf32(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  return launch_hdivcurl_mixed_prec<SFX_PREC_TF32X3>(sp, form, a, stream);
}

}  // namespace sfx
