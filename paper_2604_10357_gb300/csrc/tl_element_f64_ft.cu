// Fused force + tangent pass of the element kernels, float64.
#include "tl_element_impl.cuh"

namespace tl {

tl_status elem_tangent_f64_fused(tl_mesh* m, const double* q_n, const double* v, double h, double alpha,
                                  double beta, double mass_scale, double* f, void* values, void* K_elem) {
  return elem::launch_all<double, true, true>(m, q_n, v, h, alpha, beta, mass_scale, f, values, K_elem);
}

}  // namespace tl
