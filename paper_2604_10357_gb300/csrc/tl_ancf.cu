// ANCF elements: the exact consistent mass (node-level CSR, gravity weights
// and the per-element mass folded into the Hessian) and the dispatch of the
// element passes to the beam / shell kernels (float64; the tangent passes of
// float32 handles in the float32 element form, their residual forces in
// float64).
//
// Paper: arxiv 2604.10357 Sec. 4.1 (m_ij = int rho S_i S_j dV, constant,
// M_e = [m_ij I3]) and Sec. 4.3 (element passes).  The mass is integrated by
// a rule exact for straight, rectangular elements (4 Gauss points along each
// cubic direction, 2 along each linear one); the gravity load uses the
// weights int rho S_a dV (the gradient shape functions do not sum to one, so
// the row sums of M are not the load).
#include "tl_ancf.cuh"
#include "tl_internal.cuh"

namespace tl {

tl_status ancf_launch_beam(tl_mesh*, const double*, const double*, double, double, double, double, bool, bool,
                           double*, double*, double*);
tl_status ancf_launch_shell(tl_mesh*, const double*, const double*, double, double, double, double, bool, bool,
                            double*, double*, double*);
tl_status ancf_launch_beam_f32(tl_mesh*, const double*, const double*, double, double, double, double, bool,
                               double*, float*, float*);
tl_status ancf_launch_shell_f32(tl_mesh*, const double*, const double*, double, double, double, double, bool,
                                double*, float*, float*);

namespace {

// Thread per (element, a): row a of the element mass and the weight of a.
template <int ET>
__global__ void ancf_mass(const int32_t* conn, const double* geo, const double* X, const uint8_t* blk,
                          const int32_t* node_ptr, int64_t e_begin, int64_t e_end, double rho, double* mass,
                          double* mrow, double* me) {
  constexpr int NEN = ancf::Traits<ET>::NEN, NMQ = ancf::Traits<ET>::NMQ, NP = NEN * (NEN + 1) / 2;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t e = e_begin + t / NEN;
  if (e >= e_end) return;
  const int a = (int)(t % NEN);
  const int32_t* c = conn + e * NEN;
  const double dims[3] = {geo[e * 16], geo[e * 16 + 1], geo[e * 16 + 2]};
  double row[NEN];
#pragma unroll
  for (int b = 0; b < NEN; ++b) row[b] = 0.0;
  double wa = 0.0;
  for (int mq = 0; mq < NMQ; ++mq) {
    double p[3], w;
    ancf::mass_point<ET>(mq, p, w);
    double S[NEN], J0[3][3] = {};
#pragma unroll
    for (int b = 0; b < NEN; ++b) {
      double d[3];
      ancf::shape<ET, double>(b, p, dims, &S[b], d);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) J0[i][j] += X[3 * c[b] + i] * d[j];
    }
    double Ji[3][3];
    const double dv = rho * w * ancf::inv3<double>(J0, Ji);
    const double sa = dv * S[a];
    wa += sa;
#pragma unroll
    for (int b = 0; b < NEN; ++b) row[b] += sa * S[b];
  }
  const int I = c[a];
  const int pI = node_ptr[I];
  const uint8_t* bk = blk + e * (NEN * NEN) + a * NEN;
  const int rbase = a * NEN - a * (a - 1) / 2;     // pair index of (a, a)
#pragma unroll
  for (int b = 0; b < NEN; ++b) {
    atomicAdd(&mass[pI + bk[b]], row[b]);
    if (b >= a) me[e * NP + rbase + (b - a)] = row[b];
  }
  atomicAdd(&mrow[I], wa);
}

inline unsigned nblocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

// Node-level mass, gravity weights and the element mass table of an ANCF
// handle (after the slot blocks exist; mass and mrow zeroed by the caller).
tl_status ancf_build_mass(tl_mesh* m) {
  const int nen = m->nen;
  const int np = nen * (nen + 1) / 2;
  TL_CUDA(m, cudaMalloc(&m->d_ancf_me, sizeof(double) * np * std::max<int64_t>(m->ne_pad, 1)));
  TL_CUDA(m, cudaMemsetAsync(m->d_ancf_me, 0, sizeof(double) * np * std::max<int64_t>(m->ne_pad, 1), m->stream));
  for (const Segment& sg : m->segs) {
    const int64_t cnt = (sg.end - sg.begin) * nen;
    if (cnt == 0) continue;
    const double rho = m->mats[sg.mat].rho;
    if (m->etype == TL_ELEM_ANCF3243)
      ancf_mass<ancf::kBeam><<<nblocks(cnt, 128), 128, 0, m->stream>>>(
          m->d_conn, m->d_geo64, m->d_X, m->d_blk, m->d_node_ptr, sg.begin, sg.end, rho, m->d_mass, m->d_mrow,
          m->d_ancf_me);
    else
      ancf_mass<ancf::kShell><<<nblocks(cnt, 128), 128, 0, m->stream>>>(
          m->d_conn, m->d_geo64, m->d_X, m->d_blk, m->d_node_ptr, sg.begin, sg.end, rho, m->d_mass, m->d_mrow,
          m->d_ancf_me);
    TL_CUDA(m, cudaGetLastError());
  }
  return TL_OK;
}

tl_status ancf_launch(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                      double mass_scale, bool do_force, bool do_tangent, double* f, void* values, void* K_elem) {
  if (do_tangent && !m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  cudaEvent_t t0 = timer_open(m);
  tl_status s;
  if (m->precision == TL_FP32_ELEM && do_tangent) {     // the float32 element form: float values / K_elem
    if (m->etype == TL_ELEM_ANCF3243)
      s = ancf_launch_beam_f32(m, q_n, v, h, alpha, beta, mass_scale, do_force, f,
                               reinterpret_cast<float*>(values), reinterpret_cast<float*>(K_elem));
    else
      s = ancf_launch_shell_f32(m, q_n, v, h, alpha, beta, mass_scale, do_force, f,
                                reinterpret_cast<float*>(values), reinterpret_cast<float*>(K_elem));
  } else if (m->etype == TL_ELEM_ANCF3243)
    s = ancf_launch_beam(m, q_n, v, h, alpha, beta, mass_scale, do_force, do_tangent, f,
                         reinterpret_cast<double*>(values), reinterpret_cast<double*>(K_elem));
  else
    s = ancf_launch_shell(m, q_n, v, h, alpha, beta, mass_scale, do_force, do_tangent, f,
                          reinterpret_cast<double*>(values), reinterpret_cast<double*>(K_elem));
  timer_close(m, t0, kTimeElement);
  return s;
}

}  // namespace tl
