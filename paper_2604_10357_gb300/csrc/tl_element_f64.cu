// Force-only and tangent-only passes of the element kernels, float64.
#include "tl_element_impl.cuh"

namespace tl {

tl_status elem_tangent_f64_fused(tl_mesh* m, const double* q_n, const double* v, double h, double alpha,
                                  double beta, double mass_scale, double* f, void* values, void* K_elem);

tl_status elem_force_f64(tl_mesh* m, const double* q_n, const double* v, double h, double* f) {
  return elem::launch_all<double, true, false>(m, q_n, v, h, 0.0, 0.0, 0.0, f, nullptr, nullptr);
}

tl_status elem_tangent_f64(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                            double mass_scale, bool do_force, double* f, void* values, void* K_elem) {
  if (do_force) return elem_tangent_f64_fused(m, q_n, v, h, alpha, beta, mass_scale, f, values, K_elem);
  return elem::launch_all<double, false, true>(m, q_n, v, h, alpha, beta, mass_scale, f, values, K_elem);
}

}  // namespace tl
