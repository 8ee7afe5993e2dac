// ANCF3243 beam element passes in float64 (kernels in tl_ancf_impl.cuh).
#include "tl_ancf_impl.cuh"

namespace tl {

tl_status ancf_launch_beam(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                        double mass_scale, bool do_force, bool do_tangent, double* f, double* values,
                        double* K_elem) {
  return ancf::launch_kind<double, ancf::kBeam>(m, q_n, v, h, alpha, beta, mass_scale, do_force, do_tangent, f,
                                              values, K_elem);
}

}  // namespace tl
