// ANCF3443 shell tangent passes in the float32 element form (kernels in tl_ancf_impl.cuh).
#include "tl_ancf_impl.cuh"

namespace tl {

tl_status ancf_launch_shell_f32(tl_mesh* m, const double* q_n, const double* v, double h, double alpha,
                              double beta, double mass_scale, bool do_force, double* f, float* values,
                              float* K_elem) {
  return ancf::launch_kind<float, ancf::kShell>(m, q_n, v, h, alpha, beta, mass_scale, do_force, true, f, values,
                                             K_elem);
}

}  // namespace tl
