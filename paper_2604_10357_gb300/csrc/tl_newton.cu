// One backward-Euler time step by Newton's method inside the augmented
// Lagrangian loop (Algorithm 3 without line search; Algorithm 1 for the
// multiplier update, eq. lambda_update).
//
// Per inner iteration: residual g and ||g|| (eq. residual) on the device, the
// norm to the host for the convergence test, Hessian assembly (eq. hessian),
// numeric factorization + solve (eq. newton_linear_system, vendor solver),
// v += dv.  After the inner loop: c(q) for the clamp rows, lambda += rho c if
// the inner loop converged, ||c|| to the host for the outer test.
//
// Readings: the inner target is max(atol, rtol * ||g(v_n; lambda)||) with the
// residual at the plain start v_n, whatever start is used; lambda persists in
// the caller's array across steps.  For the FP32 element form the Hessian,
// its factorization and the direction are float32, while the residual used in
// the convergence test keeps a float64 force evaluation (flag below), since a
// float32 force has a noise floor of ~1e-7 of the element force scale, above a
// 1e-8 relative target in steps close to equilibrium.
#include <chrono>
#include <cmath>

#include "tl_internal.cuh"

namespace tl {

tl_status solver_setup(tl_mesh* m);
tl_status solver_factor_solve(tl_mesh* m, const void* values, const double* g, double* dv);

namespace {

__global__ void axpy_kernel(double* y, const double* x, double a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void q_from_v(const double* q_n, const double* v, double h, int64_t n, double* q) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) q[i] = q_n[i] + h * v[i];
}

// c_j = q_n + h v - X at every clamped DOF (the j-th fixed node's d-th DOF is
// constraint 3j+d); optionally lambda += rho c; ||c||^2 into out (one block).
__global__ void clamp_constraint(const int32_t* fixed_of_node, const double* X,
                                 const double* q_n, const double* v, double h, int64_t nn, double rho,
                                 int update_lambda, double* lambda, double* out) {
  __shared__ double red[32];
  double sq = 0.0;
  for (int64_t I = threadIdx.x; I < nn; I += blockDim.x) {
    const int j = fixed_of_node[I];
    if (j < 0) continue;
    for (int d = 0; d < 3; ++d) {
      const int64_t r = 3 * I + d;
      const double c = (q_n[r] + h * v[r]) - X[r];
      sq += c * c;
      if (update_lambda) lambda[3 * j + d] += rho * c;
    }
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *out = sqrt(t);
  }
}

}  // namespace

tl_status launch_force_prec(tl_mesh* m, const double* q_n, const double* v, double h, double* f, bool fp64);

}  // namespace tl

using namespace tl;

extern "C" tl_status tl_newton_step(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n,
                                    const double* v_init, const double* f_ext, double* lambda, double* v_out,
                                    double* q_out, tl_newton_stats* stats) {
  if (!m || !p || !q_n || !v_n || !v_out || !q_out || !(p->h > 0.0) || p->max_inner < 1 || p->max_outer < 1)
    return TL_ERR_INVALID_ARG;
  if (m->nfixed > 0 && !lambda) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  const auto t_start = std::chrono::steady_clock::now();
  const bool use_pcg = p->linear_solver == TL_SOLVER_PCG;
  if (!use_pcg) {
    tl_status st = solver_setup(m);
    if (st != TL_OK) return st;
  }
  const double lin_rtol = p->lin_rtol > 0.0 ? p->lin_rtol : 1e-10;
  const int lin_max = p->lin_max_iter > 0 ? p->lin_max_iter : 5000;
  int lin_total = 0;
  const int64_t ndof = 3 * m->nn;
  const size_t vb = (m->precision == TL_FP32_ELEM ? sizeof(float) : sizeof(double));
  // work buffers: allocated on the first call, owned by the handle
  if (!m->nw_g) {
    TL_CUDA(m, cudaMalloc(&m->nw_g, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_f, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_dv, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_scal, sizeof(double) * 4));
    TL_CUDA(m, cudaMalloc(&m->nw_values, vb * m->nnz));
  }
  struct {
    double *g, *f, *dv, *scal;
    void* values;
  } w = {m->nw_g, m->nw_f, m->nw_dv, m->nw_scal, m->nw_values};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  auto cleanup = [&]() {
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  };
#define NTRY(call)                         \
  do {                                     \
    tl_status _s = (call);                 \
    if (_s != TL_OK) {                     \
      cleanup();                           \
      return _s;                           \
    }                                      \
  } while (0)
#define NCUDA(call)                        \
  do {                                     \
    cudaError_t _e = (call);               \
    if (_e != cudaSuccess) {               \
      cleanup();                           \
      return cuda_fail(m, _e, #call);      \
    }                                      \
  } while (0)
  cudaStream_t s = m->stream;
  const unsigned nb = (unsigned)((ndof + 255) / 256);
  double* v = v_out;
  NCUDA(cudaMemcpyAsync(v, v_init ? v_init : v_n, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
  const bool fp64_force = true;   // residual force in float64 for both element forms
  double ms_asm = 0.0, ms_sol = 0.0;
  for (auto& e : ev) NCUDA(cudaEventCreate(&e));
  auto residual = [&](const double* vv, double* gnorm_host) -> tl_status {
    tl_status r = launch_force_prec(m, q_n, vv, p->h, w.f, fp64_force);
    if (r != TL_OK) return r;
    r = launch_residual(m, p, q_n, v_n, vv, w.f, f_ext, lambda, w.g, w.scal);
    if (r != TL_OK) return r;
    if (cudaMemcpyAsync(gnorm_host, w.scal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(m, TL_ERR_CUDA, "residual norm transfer");
    if (!std::isfinite(*gnorm_host)) return fail(m, TL_ERR_NONFINITE, "non-finite residual");
    return TL_OK;
  };
  // reference norm at the plain start v_n
  double g_ref = 0.0;
  NTRY(residual(v_n, &g_ref));
  const double target = std::max(p->atol, p->rtol * g_ref);
  int inner_total = 0, outer = 0;
  bool converged = false;
  double gn = 0.0, cn = 0.0, g_init = -1.0;
  for (outer = 1; outer <= p->max_outer; ++outer) {
    bool inner_ok = false;
    for (int l = 0; l < p->max_inner; ++l) {
      cudaEventRecord(ev[0], s);
      NTRY(residual(v, &gn));
      if (g_init < 0.0) g_init = gn;
      if (gn <= target) {
        inner_ok = true;
        cudaEventRecord(ev[1], s);
        cudaEventSynchronize(ev[1]);
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[0], ev[1]);
        ms_asm += t;
        break;
      }
      NCUDA(cudaMemsetAsync(w.values, 0, vb * m->nnz, s));
      NTRY(launch_tangent(m, q_n, v, p->h, p->h, 1.0, 1.0 / p->h, false, nullptr, w.values, nullptr));
      NTRY(launch_add_penalty(m, p->h * p->h * p->rho_alm, w.values));
      cudaEventRecord(ev[1], s);
      if (use_pcg) {
        int it = 0;
        // inexact Newton: the linear residual only needs to be well below the
        // Newton target (g_{k+1} ~ linear residual + O(|dv|^2))
        const double eta = p->lin_adaptive ? std::min(0.5, std::max(lin_rtol, 0.1 * target / gn)) : lin_rtol;
        NTRY(pcg_solve(m, w.values, w.g, w.dv, eta, lin_max, &it));
        lin_total += it;
      } else {
        NTRY(solver_factor_solve(m, w.values, w.g, w.dv));
      }
      axpy_kernel<<<nb, 256, 0, s>>>(v, w.dv, 1.0, ndof);
      NCUDA(cudaGetLastError());
      ++m->launches;
      cudaEventRecord(ev[2], s);
      cudaEventSynchronize(ev[2]);
      float t1 = 0.f, t2 = 0.f;
      cudaEventElapsedTime(&t1, ev[0], ev[1]);
      cudaEventElapsedTime(&t2, ev[1], ev[2]);
      ms_asm += t1;
      ms_sol += t2;
      ++inner_total;
    }
    clamp_constraint<<<1, 1024, 0, s>>>(m->d_fixed_of_node, m->d_X, q_n, v, p->h, m->nn, p->rho_alm,
                                         inner_ok ? 1 : 0, lambda, w.scal + 1);
    NCUDA(cudaGetLastError());
    ++m->launches;
    NCUDA(cudaMemcpyAsync(&cn, w.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    NCUDA(cudaStreamSynchronize(s));
    if (inner_ok && cn <= p->eps_out) {
      converged = true;
      break;
    }
  }
  if (outer > p->max_outer) outer = p->max_outer;
  q_from_v<<<nb, 256, 0, s>>>(q_n, v, p->h, ndof, q_out);
  NCUDA(cudaGetLastError());
  ++m->launches;
  NCUDA(cudaStreamSynchronize(s));
  cleanup();
#undef NTRY
#undef NCUDA
  if (stats) {
    stats->inner_iters = inner_total;
    stats->outer_iters = outer;
    stats->converged = converged ? 1 : 0;
    stats->g_ref = g_ref;
    stats->g_norm = gn;
    stats->c_norm = cn;
    stats->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    stats->ms_assembly = ms_asm;
    stats->ms_solver = ms_sol;
    stats->lin_iters = lin_total;
    stats->g_init = g_init;
  }
  return converged ? TL_OK : fail(m, TL_ERR_NOT_CONVERGED, "Newton / ALM iteration caps reached");
}
