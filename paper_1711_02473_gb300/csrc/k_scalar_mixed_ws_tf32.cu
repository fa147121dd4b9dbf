// k_scalar_mixed_ws_tf32.cu -- TF32x3 instantiation of the warp-specialised
// split-precision scalar action (body in scalar_mixed_ws.cuh); one translation
// unit per format so that the build compiles them in parallel.
#include "scalar_mixed_ws.cuh"

namespace sfx {

SFX_DEFINE_TAB_UPLOAD(upload_tab_scalar_mixed_ws_tf32)

int launch_action_scalar_mixed_ws_tf32(const sfx_space* sp, sfx_form form, const ActArgs& a, void* stream) {
  return launch_ws_prec<SFX_PREC_TF32X3>(sp, form, a, stream);
}

}  // namespace sfx
