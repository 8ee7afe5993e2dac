// Force-only pass of the element kernels in double-float arithmetic (float32
// pairs, 48-bit significands): the float64-class internal force of the
// residual for float32 handles, at float32 instruction rates.
#include "tl_element_impl.cuh"

namespace tl {

tl_status elem_force_df(tl_mesh* m, const double* q_n, const double* v, double h, double* f) {
  return elem::launch_all<dfl, true, false>(m, q_n, v, h, 0.0, 0.0, 0.0, f, nullptr, nullptr);
}

}  // namespace tl
