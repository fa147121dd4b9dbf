// k_stubs.cu -- launchers not implemented yet report "unsupported" (-1).
#include "kern_common.cuh"
namespace sfx {
int launch_action_scalar_naive(const sfx_space*, sfx_form, const ActArgs&, void*) { return -1; }
int launch_cell_matrices(const sfx_space*, sfx_form, sfx_algo, const MatArgs&, void*) { return -1; }
}  // namespace sfx
