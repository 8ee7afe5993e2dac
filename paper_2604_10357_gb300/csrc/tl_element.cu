// Dispatch of the element passes (force, tangent, fused) to the T10 kernels of
// tl_element_impl.cuh, instantiated per precision and pass in tl_element_*.cu,
// or to the ANCF kernels (tl_ancf.cu).
#include "tl_internal.cuh"

namespace tl {

tl_status elem_force_f32(tl_mesh*, const double*, const double*, double, double*);
tl_status elem_force_f64(tl_mesh*, const double*, const double*, double, double*);
tl_status elem_force_df(tl_mesh*, const double*, const double*, double, double*);
tl_status elem_tangent_f32(tl_mesh*, const double*, const double*, double, double, double, double, bool, double*,
                           void*, void*);
tl_status elem_tangent_f64(tl_mesh*, const double*, const double*, double, double, double, double, bool, double*,
                           void*, void*);

tl_status launch_force(tl_mesh* m, const double* q_n, const double* v, double h, double* f) {
  TL_CUDA(m, cudaMemsetAsync(f, 0, sizeof(double) * 3 * m->nn, m->stream));
  if (m->etype != TL_ELEM_T10) return ancf_launch(m, q_n, v, h, 1.0, 0.0, 0.0, true, false, f, nullptr, nullptr);
  if (m->precision == TL_FP32_ELEM) return elem_force_f32(m, q_n, v, h, f);
  return elem_force_f64(m, q_n, v, h, f);
}

tl_status launch_force_prec(tl_mesh* m, const double* q_n, const double* v, double h, double* f, bool fp64) {
  TL_CUDA(m, cudaMemsetAsync(f, 0, sizeof(double) * 3 * m->nn, m->stream));
  if (m->etype != TL_ELEM_T10) return ancf_launch(m, q_n, v, h, 1.0, 0.0, 0.0, true, false, f, nullptr, nullptr);
  if (m->precision == TL_FP32_ELEM && !fp64) return elem_force_f32(m, q_n, v, h, f);
  // float32 handles: the float64-class force in double-float arithmetic
  if (m->precision == TL_FP32_ELEM && m->tune.force_split && m->d_geo_df) return elem_force_df(m, q_n, v, h, f);
  return elem_force_f64(m, q_n, v, h, f);
}

tl_status launch_tangent(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                         double mass_scale, bool do_force, double* f, void* values, void* K_elem) {
  if (do_force) TL_CUDA(m, cudaMemsetAsync(f, 0, sizeof(double) * 3 * m->nn, m->stream));
  if (m->etype != TL_ELEM_T10)
    return ancf_launch(m, q_n, v, h, alpha, beta, mass_scale, do_force, true, f, values, K_elem);
  if (m->precision == TL_FP32_ELEM)
    return elem_tangent_f32(m, q_n, v, h, alpha, beta, mass_scale, do_force, f, values, K_elem);
  return elem_tangent_f64(m, q_n, v, h, alpha, beta, mass_scale, do_force, f, values, K_elem);
}

}  // namespace tl
