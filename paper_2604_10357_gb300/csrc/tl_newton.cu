// One backward-Euler time step by Newton's method inside the augmented
// Lagrangian loop (Algorithm 3, with the optional Armijo line search of eq.
// armijo; Algorithm 1 for the multiplier update, eq. lambda_update), and the
// same step with the first-order AdamW inner solver (Algorithm 2).
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
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "tl_internal.cuh"

namespace tl {

tl_status solver_setup(tl_mesh* m);
tl_status solver_factor_solve(tl_mesh* m, const void* values, const double* g, double* dv);

namespace {

__global__ void axpy_kernel(double* y, const double* x, double a, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// AdamW update of Algorithm 2 per DOF: moments from the previous gradient,
// bias correction (bc1 = 1 - beta1^l, bc2 = 1 - beta2^l), velocity update with
// decoupled weight decay.
__global__ void adamw_update(double* v, double* m1, double* m2, const double* g, int64_t n, double beta1,
                             double beta2, double bc1, double bc2, double lr, double wd, double eps) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = g[i];
  const double a = beta1 * m1[i] + (1.0 - beta1) * gi;
  const double b = beta2 * m2[i] + (1.0 - beta2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  v[i] = (1.0 - lr * wd) * v[i] - lr * (a / bc1) / (sqrt(b / bc2) + eps);
}

// ||x||_2 in one block (deterministic order); the AdamW absolute test needs |v|
__global__ void norm_one_block(const double* x, int64_t n, double* out) {
  __shared__ double red[32];
  double sq = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) sq += x[i] * x[i];
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *out = sqrt(t);
  }
}

// y = v + a dx (line-search trial point)
__global__ void axpby_kernel(const double* v, const double* dx, double a, int64_t n, double* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = v[i] + a * dx[i];
}

__global__ void q_from_v(const double* q_n, const double* v, double h, int64_t n, double* q) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) q[i] = q_n[i] + h * v[i];
}

// c_j = q_n + h v - X at every clamped DOF (the j-th fixed node's d-th DOF is
// constraint 3j+d); optionally lambda += rho c; ||c||^2 into out (one block).
// (update_flag, when given, is read on the device instead of update_lambda.)
__global__ void clamp_constraint(const int32_t* fixed_of_node, const double* X,
                                 const double* q_n, const double* v, double h, int64_t nn, double rho,
                                 int update_lambda, const int32_t* update_flag, double* lambda, double* out,
                                 const double* extra_sq) {
  __shared__ double red[32];
  if (update_flag) update_lambda = *update_flag;
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
    if (threadIdx.x == 0) *out = sqrt(t + (extra_sq ? *extra_sq : 0.0));   // + the general rows
  }
}

// ---------------------------------------------------------------------------
// Captured Newton step (tl_params.use_graph): the loops of Algorithm 3 run as
// conditional nodes of one CUDA graph, and the convergence tests that the
// host makes in the loop above (the ||g|| and ||c|| transfers) are made by
// one-thread control kernels that set the loop conditions.  Every loop is
// bounded by its own counter (max_outer, max_inner, lin_max_iter), so the
// graph always ends.

struct NewtonCtl {
  double g_ref, target, gn, g_init, cn, tol2, eta;
  double ls_alpha, ls_phi0;                       // line search: current step, phi(0)
  int32_t l, inner_total, outer, inner_ok, converged, lin_total, pcg_it, abort;
  int32_t ls_j, ls_ok, ls_trials, _pad;
};

__global__ void ctl_reset(NewtonCtl* c) {
  NewtonCtl z = {};
  z.g_init = -1.0;
  *c = z;
}

// reference norm at v_n -> inner target; arm the outer loop
__global__ void ctl_target(NewtonCtl* c, const double* gnorm, double atol, double rtol,
                           cudaGraphConditionalHandle h_out) {
  const double g = *gnorm;
  c->g_ref = g;
  c->target = fmax(atol, rtol * g);
  const bool ok = isfinite(g);
  if (!ok) c->abort = 1;
  cudaGraphSetConditional(h_out, ok ? 1u : 0u);
}

__global__ void ctl_outer_begin(NewtonCtl* c, cudaGraphConditionalHandle h_in) {
  c->l = 0;
  c->inner_ok = 0;
  cudaGraphSetConditional(h_in, 1u);
}

// inner test: stop on ||g|| <= target (or a non-finite norm); otherwise take
// a Newton step, counted against max_inner
__global__ void ctl_inner(NewtonCtl* c, const double* gnorm, int max_inner, double lin_rtol, int adaptive,
                          double eta_min, cudaGraphConditionalHandle h_in, cudaGraphConditionalHandle h_step) {
  const double g = *gnorm;
  c->gn = g;
  if (!isfinite(g) || c->abort) {
    c->abort = 1;
    cudaGraphSetConditional(h_step, 0u);
    cudaGraphSetConditional(h_in, 0u);
    return;
  }
  if (c->g_init < 0.0) c->g_init = g;
  if (g <= c->target) {
    c->inner_ok = 1;
    cudaGraphSetConditional(h_step, 0u);
    cudaGraphSetConditional(h_in, 0u);
    return;
  }
  c->eta = fmax(eta_min, adaptive ? fmin(0.5, fmax(lin_rtol, 0.1 * c->target / g)) : lin_rtol);
  c->l += 1;
  c->inner_total += 1;
  cudaGraphSetConditional(h_step, 1u);
  cudaGraphSetConditional(h_in, c->l < max_inner ? 1u : 0u);
}

__global__ void ctl_pcg_arm(NewtonCtl* c, double* pscal, int lin_max, cudaGraphConditionalHandle h_pcg) {
  const double rr0 = pscal[3];
  c->tol2 = c->eta * c->eta * rr0;
  pscal[5] = c->tol2;            // the PCG kernels return at once past the target
  c->pcg_it = 0;
  cudaGraphSetConditional(h_pcg, (rr0 > c->tol2 && lin_max > 0) ? 1u : 0u);
}

__global__ void ctl_pcg(NewtonCtl* c, const double* pscal, int chunk, int lin_max,
                        cudaGraphConditionalHandle h_pcg) {
  (void)chunk;
  c->pcg_it = (int)pscal[7];     // iterations that ran (those past the target returned at once)
  const double rr = pscal[3];
  if (!isfinite(rr)) {
    c->abort = 1;
    cudaGraphSetConditional(h_pcg, 0u);
    return;
  }
  const bool breakdown = pscal[6] != 0.0;
  cudaGraphSetConditional(h_pcg, (rr > c->tol2 && c->pcg_it < lin_max && !breakdown) ? 1u : 0u);
}

__global__ void ctl_pcg_done(NewtonCtl* c) { c->lin_total += c->pcg_it; }

// line search (eq. armijo): arm the backtracking loop at a = 1
__global__ void ctl_ls_arm(NewtonCtl* c, cudaGraphConditionalHandle h_ls) {
  c->ls_phi0 = 0.5 * c->gn * c->gn;
  c->ls_alpha = 1.0;
  c->ls_j = 0;
  c->ls_ok = 0;
  cudaGraphSetConditional(h_ls, 1u);
}

// trial point v + a dv with the current a
__global__ void ls_trial(const double* v, const double* dv, const NewtonCtl* c, int64_t n, double* vt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) vt[i] = v[i] + c->ls_alpha * dv[i];
}

// sufficient decrease at the trial point, else a *= beta (at most j_max trials)
__global__ void ctl_ls(NewtonCtl* c, const double* gnorm, double c1, double beta, int j_max,
                       cudaGraphConditionalHandle h_ls) {
  const double gt = *gnorm;
  c->ls_trials += 1;
  c->ls_j += 1;
  if (0.5 * gt * gt <= (1.0 - 2.0 * c1 * c->ls_alpha) * c->ls_phi0) {   // false for a non-finite norm
    c->ls_ok = 1;
    cudaGraphSetConditional(h_ls, 0u);
    return;
  }
  c->ls_alpha *= beta;
  cudaGraphSetConditional(h_ls, c->ls_j < j_max ? 1u : 0u);
}

// accepted: v = trial point; rejected j_max times: keep v and end the inner loop
__global__ void ls_commit(double* v, const double* vt, const NewtonCtl* c, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && c->ls_ok) v[i] = vt[i];
}

__global__ void ctl_ls_done(const NewtonCtl* c, cudaGraphConditionalHandle h_in) {
  if (!c->ls_ok) cudaGraphSetConditional(h_in, 0u);
}

__global__ void ctl_outer(NewtonCtl* c, const double* cnorm, double eps_out, int max_outer,
                          cudaGraphConditionalHandle h_out) {
  c->outer += 1;
  c->cn = *cnorm;
  if (c->abort) {
    cudaGraphSetConditional(h_out, 0u);
    return;
  }
  if (c->inner_ok && c->cn <= eps_out) {
    c->converged = 1;
    cudaGraphSetConditional(h_out, 0u);
    return;
  }
  cudaGraphSetConditional(h_out, c->outer < max_outer ? 1u : 0u);
}

constexpr int kPcgChunk = 8;   // PCG iterations between two device-side checks

// PCG tolerance floor: lin_rtol when the caller sets it, else 1e-10 for the
// float64 element path and 1e-6 for a float32 Hessian (symmetric only to
// rounding; its products carry float32 sums, so tighter solves gain little).
double pcg_rtol_floor(const tl_mesh* m, const tl_params* p) {
  if (p->lin_rtol > 0.0) return p->lin_rtol;
  return m->precision == TL_FP32_ELEM ? 1e-6 : 1e-10;
}

}  // namespace

tl_status launch_force_prec(tl_mesh* m, const double* q_n, const double* v, double h, double* f, bool fp64);

struct NewtonGraph {
  tl_params key = {};
  int precision = -1;
  int64_t tune_gen = -1;
  cudaStream_t cs = nullptr;            // capture stream (the graph is launched on the handle's stream)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double *q_n = nullptr, *v_n = nullptr, *v = nullptr, *f_ext = nullptr, *lam = nullptr, *q_out = nullptr;
  NewtonCtl* ctl = nullptr;
  NewtonCtl* ctl_host = nullptr;        // pinned
};

void newton_graph_destroy(NewtonGraph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  void* ptrs[] = {g->q_n, g->v_n, g->v, g->f_ext, g->lam, g->q_out, g->ctl};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (g->ctl_host) cudaFreeHost(g->ctl_host);
  if (g->cs) cudaStreamDestroy(g->cs);
  delete g;
}

namespace {

cudaError_t capture_handle(cudaStream_t s, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  return cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault);
}

// append a conditional node to the capture of s; its (empty) body is returned
cudaError_t capture_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                cudaGraph_t* body) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Records the whole step into G->graph.  Runs with m->stream = G->cs.
tl_status capture_step(tl_mesh* m, const tl_params* p, NewtonGraph* G) {
  cudaStream_t s = G->cs;
  const int64_t ndof = 3 * m->nn;
  const unsigned nb = (unsigned)((ndof + 255) / 256);
  const size_t vb = (m->precision == TL_FP32_ELEM ? sizeof(float) : sizeof(double));
  const double lin_rtol = pcg_rtol_floor(m, p);
  const int lin_max = p->lin_max_iter > 0 ? p->lin_max_iter : 5000;
  double *g = m->nw_g, *f = m->nw_f, *dv = m->nw_dv, *scal = m->nw_scal;
  void* values = m->nw_values;
  NewtonCtl* c = G->ctl;
  cudaGraphConditionalHandle h_out = 0, h_in = 0, h_step = 0, h_pcg = 0, h_ls = 0;
  cudaGraph_t b_outer = nullptr, b_inner = nullptr, b_step = nullptr, b_pcg = nullptr, b_ls = nullptr,
              tmp = nullptr;
  double* vt = m->nw_vt;
  const int ls_max = p->ls_max_trials > 0 ? p->ls_max_trials : 10;
  const double ls_c1 = p->ls_c1 > 0.0 ? p->ls_c1 : 1e-4, ls_beta = p->ls_beta > 0.0 ? p->ls_beta : 0.5;
  auto end_capture = [&](cudaGraph_t* out) { return cudaStreamEndCapture(s, out); };
  // top level: reference residual at v_n, the outer loop, q = q_n + h v
  TL_CUDA(m, cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  {
    tl_status st = TL_OK;
    cudaError_t e = capture_handle(s, &h_out);
    if (e == cudaSuccess) {
      ctl_reset<<<1, 1, 0, s>>>(c);
      st = launch_force_prec(m, G->q_n, G->v_n, p->h, f, true);
      if (st == TL_OK) st = launch_residual(m, p, G->q_n, G->v_n, G->v_n, f, G->f_ext, G->lam, g, scal);
      if (st == TL_OK) {
        ctl_target<<<1, 1, 0, s>>>(c, scal, p->atol, p->rtol, h_out);
        e = capture_conditional(s, h_out, cudaGraphCondTypeWhile, &b_outer);
        if (e == cudaSuccess) q_from_v<<<nb, 256, 0, s>>>(G->q_n, G->v, p->h, ndof, G->q_out);
      }
    }
    cudaGraph_t top = nullptr;
    cudaError_t e2 = end_capture(&top);
    G->graph = top;
    if (st != TL_OK) return st;
    TL_CUDA(m, e);
    TL_CUDA(m, e2);
  }
  // outer body: inner loop, clamp rows and multiplier update, outer test
  TL_CUDA(m, cudaStreamBeginCaptureToGraph(s, b_outer, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  {
    cudaError_t e = capture_handle(s, &h_in);
    if (e == cudaSuccess) {
      ctl_outer_begin<<<1, 1, 0, s>>>(c, h_in);
      e = capture_conditional(s, h_in, cudaGraphCondTypeWhile, &b_inner);
    }
    if (e == cudaSuccess) {
      const tl_status sc = launch_con_update(m, G->q_n, G->v, p->h, p->rho_alm, 0, &c->inner_ok,
                                             G->lam + 3 * m->nfixed);
      if (sc != TL_OK) e = cudaErrorUnknown;
      clamp_constraint<<<1, 1024, 0, s>>>(m->d_fixed_of_node, m->d_X, G->q_n, G->v, p->h, m->nn, p->rho_alm, 0,
                                           &c->inner_ok, G->lam, scal + 1, m->ncon ? m->d_con_sq : nullptr);
      ctl_outer<<<1, 1, 0, s>>>(c, scal + 1, p->eps_out, p->max_outer, h_out);
    }
    cudaError_t e2 = end_capture(&tmp);
    TL_CUDA(m, e);
    TL_CUDA(m, e2);
  }
  // inner body: residual at v, inner test, conditional Newton step
  TL_CUDA(m, cudaStreamBeginCaptureToGraph(s, b_inner, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  {
    tl_status st = TL_OK;
    cudaError_t e = capture_handle(s, &h_step);
    if (e == cudaSuccess) {
      st = launch_force_prec(m, G->q_n, G->v, p->h, f, true);
      if (st == TL_OK) st = launch_residual(m, p, G->q_n, G->v_n, G->v, f, G->f_ext, G->lam, g, scal);
      if (st == TL_OK) {
        ctl_inner<<<1, 1, 0, s>>>(c, scal, p->max_inner, lin_rtol, p->lin_adaptive, 0.0, h_in,
                                  h_step);
        e = capture_conditional(s, h_step, cudaGraphCondTypeIf, &b_step);
      }
    }
    cudaError_t e2 = end_capture(&tmp);
    if (st != TL_OK) return st;
    TL_CUDA(m, e);
    TL_CUDA(m, e2);
  }
  // Newton step: assemble H (eq. hessian), PCG loop, v += dv
  TL_CUDA(m, cudaStreamBeginCaptureToGraph(s, b_step, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  {
    tl_status st = TL_OK;
    cudaError_t e = capture_handle(s, &h_pcg);
    if (e == cudaSuccess && p->line_search) e = capture_handle(s, &h_ls);
    if (e == cudaSuccess) e = cudaMemsetAsync(values, 0, vb * m->nnz, s);
    if (e == cudaSuccess) {
      st = launch_tangent(m, G->q_n, G->v, p->h, p->h, 1.0, 1.0 / p->h, false, nullptr, values, nullptr);
      if (st == TL_OK) st = launch_add_penalty(m, p->h * p->h * p->rho_alm, values);
      if (st == TL_OK) st = pcg_prepare(m, values, g, dv);
      if (st == TL_OK) {
        ctl_pcg_arm<<<1, 1, 0, s>>>(c, pcg_scalars(m), lin_max, h_pcg);
        e = capture_conditional(s, h_pcg, cudaGraphCondTypeWhile, &b_pcg);
        if (e == cudaSuccess) {
          ctl_pcg_done<<<1, 1, 0, s>>>(c);
          st = pcg_result(m, dv);
          if (st == TL_OK && !p->line_search) axpy_kernel<<<nb, 256, 0, s>>>(G->v, dv, 1.0, ndof);
          if (st == TL_OK && p->line_search) {
            ctl_ls_arm<<<1, 1, 0, s>>>(c, h_ls);
            e = capture_conditional(s, h_ls, cudaGraphCondTypeWhile, &b_ls);
            if (e == cudaSuccess) {
              ls_commit<<<nb, 256, 0, s>>>(G->v, vt, c, ndof);
              ctl_ls_done<<<1, 1, 0, s>>>(c, h_in);
            }
          }
        }
      }
    }
    cudaError_t e2 = end_capture(&tmp);
    if (st != TL_OK) return st;
    TL_CUDA(m, e);
    TL_CUDA(m, e2);
  }
  // line-search body: trial point, its residual and the sufficient-decrease test
  if (p->line_search) {
    TL_CUDA(m, cudaStreamBeginCaptureToGraph(s, b_ls, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    tl_status st = TL_OK;
    ls_trial<<<nb, 256, 0, s>>>(G->v, dv, c, ndof, vt);
    st = launch_force_prec(m, G->q_n, vt, p->h, f, true);
    if (st == TL_OK) st = launch_residual(m, p, G->q_n, G->v_n, vt, f, G->f_ext, G->lam, g, scal);
    if (st == TL_OK) ctl_ls<<<1, 1, 0, s>>>(c, scal, ls_c1, ls_beta, ls_max, h_ls);
    cudaError_t e2 = end_capture(&tmp);
    if (st != TL_OK) return st;
    TL_CUDA(m, e2);
  }
  // PCG body: kPcgChunk iterations and the device-side residual test
  TL_CUDA(m, cudaStreamBeginCaptureToGraph(s, b_pcg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  {
    tl_status st = pcg_iterations(m, values, dv, kPcgChunk);
    if (st == TL_OK) ctl_pcg<<<1, 1, 0, s>>>(c, pcg_scalars(m), kPcgChunk, lin_max, h_pcg);
    cudaError_t e2 = end_capture(&tmp);
    if (st != TL_OK) return st;
    TL_CUDA(m, e2);
  }
  TL_CUDA(m, cudaGraphInstantiate(&G->exec, G->graph, 0));
  return TL_OK;
}

// (Re)build the graph when the parameters or the element precision change.
tl_status ensure_graph(tl_mesh* m, const tl_params* p) {
  const int64_t ndof = 3 * m->nn;
  NewtonGraph* G = m->ngraph;
  if (G && G->exec && G->precision == m->precision && G->tune_gen == m->tune.generation &&
      std::memcmp(&G->key, p, sizeof(tl_params)) == 0)
    return TL_OK;
  if (!G) {
    G = new NewtonGraph();
    m->ngraph = G;
    TL_CUDA(m, cudaStreamCreateWithFlags(&G->cs, cudaStreamNonBlocking));
    TL_CUDA(m, cudaMalloc(&G->q_n, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&G->v_n, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&G->v, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&G->f_ext, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&G->q_out, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&G->lam, sizeof(double) * std::max<int64_t>(1, 3 * m->nfixed + m->ncon)));
    TL_CUDA(m, cudaMalloc(&G->ctl, sizeof(NewtonCtl)));
    TL_CUDA(m, cudaMallocHost(&G->ctl_host, sizeof(NewtonCtl)));
  }
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->graph) cudaGraphDestroy(G->graph);
  G->exec = nullptr;
  G->graph = nullptr;
  // allocations the captured launches need happen before the capture
  TL_TRY(pcg_ensure(m));
  TL_TRY(residual_ensure(m));
  TL_CUDA(m, cudaStreamSynchronize(m->stream));
  cudaStream_t user = m->stream;
  const bool timing = m->timing;
  m->stream = G->cs;
  m->timing = false;
  const tl_status st = capture_step(m, p, G);
  m->stream = user;
  m->timing = timing;
  if (st != TL_OK) {
    if (G->graph) cudaGraphDestroy(G->graph);
    G->graph = nullptr;
    cudaGetLastError();
    return st;
  }
  G->key = *p;
  G->precision = m->precision;
  G->tune_gen = m->tune.generation;
  return TL_OK;
}

}  // namespace

// The step as one graph launch between device copies of the caller's arrays.
tl_status newton_step_graph(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n,
                            const double* v_init, const double* f_ext, double* lambda, double* v_out, double* q_out,
                            tl_newton_stats* stats, std::chrono::steady_clock::time_point t_start) {
  TL_TRY(ensure_graph(m, p));
  NewtonGraph* G = m->ngraph;
  cudaStream_t s = m->stream;
  const size_t vbytes = sizeof(double) * 3 * m->nn;
  const size_t lbytes = sizeof(double) * (3 * m->nfixed + m->ncon);
  TL_CUDA(m, cudaMemcpyAsync(G->q_n, q_n, vbytes, cudaMemcpyDeviceToDevice, s));
  TL_CUDA(m, cudaMemcpyAsync(G->v_n, v_n, vbytes, cudaMemcpyDeviceToDevice, s));
  TL_CUDA(m, cudaMemcpyAsync(G->v, v_init ? v_init : v_n, vbytes, cudaMemcpyDeviceToDevice, s));
  if (f_ext)
    TL_CUDA(m, cudaMemcpyAsync(G->f_ext, f_ext, vbytes, cudaMemcpyDeviceToDevice, s));
  else
    TL_CUDA(m, cudaMemsetAsync(G->f_ext, 0, vbytes, s));
  if (lbytes) TL_CUDA(m, cudaMemcpyAsync(G->lam, lambda, lbytes, cudaMemcpyDeviceToDevice, s));
  TL_CUDA(m, cudaGraphLaunch(G->exec, s));
  TL_CUDA(m, cudaMemcpyAsync(v_out, G->v, vbytes, cudaMemcpyDeviceToDevice, s));
  TL_CUDA(m, cudaMemcpyAsync(q_out, G->q_out, vbytes, cudaMemcpyDeviceToDevice, s));
  if (lbytes) TL_CUDA(m, cudaMemcpyAsync(lambda, G->lam, lbytes, cudaMemcpyDeviceToDevice, s));
  TL_CUDA(m, cudaMemcpyAsync(G->ctl_host, G->ctl, sizeof(NewtonCtl), cudaMemcpyDeviceToHost, s));
  TL_CUDA(m, cudaStreamSynchronize(s));
  const NewtonCtl& c = *G->ctl_host;
  if (stats) {
    stats->inner_iters = c.inner_total;
    stats->outer_iters = c.outer;
    stats->converged = c.converged;
    stats->g_ref = c.g_ref;
    stats->g_norm = c.gn;
    stats->c_norm = c.cn;
    stats->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    stats->ms_assembly = 0.0;   // not split inside the graph
    stats->ms_solver = 0.0;
    stats->lin_iters = c.lin_total;
    stats->ls_trials = c.ls_trials;
    stats->g_init = c.g_init;
  }
  if (c.abort) return fail(m, TL_ERR_NONFINITE, "non-finite residual in the captured Newton step");
  return c.converged ? TL_OK : fail(m, TL_ERR_NOT_CONVERGED, "Newton / ALM iteration caps reached");
}

}  // namespace tl

using namespace tl;

extern "C" tl_status tl_newton_step(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n,
                                    const double* v_init, const double* f_ext, double* lambda, double* v_out,
                                    double* q_out, tl_newton_stats* stats) {
  if (!m || !p || !q_n || !v_n || !v_out || !q_out || !(p->h > 0.0) || p->max_inner < 1 || p->max_outer < 1)
    return TL_ERR_INVALID_ARG;
  if ((m->nfixed > 0 || m->ncon > 0) && !lambda) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  const auto t_start = std::chrono::steady_clock::now();
  const bool use_pcg = p->linear_solver == TL_SOLVER_PCG;
  if (p->use_graph && !use_pcg)
    return fail(m, TL_ERR_UNSUPPORTED, "use_graph needs the PCG inner solver (the direct solver is not captured)");
  if (!use_pcg) {
    tl_status st = solver_setup(m);
    if (st != TL_OK) return st;
  }
  const double lin_rtol = pcg_rtol_floor(m, p);
  const int lin_max = p->lin_max_iter > 0 ? p->lin_max_iter : 5000;
  int lin_total = 0;
  const int64_t ndof = 3 * m->nn;
  const size_t vb = (m->precision == TL_FP32_ELEM ? sizeof(float) : sizeof(double));
  // work buffers: allocated on the first call, owned by the handle
  if (!m->nw_vt) TL_CUDA(m, cudaMalloc(&m->nw_vt, sizeof(double) * ndof));   // line-search trial velocity
  if (!m->nw_g) {
    TL_CUDA(m, cudaMalloc(&m->nw_g, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_f, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_dv, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_scal, sizeof(double) * 4));
    TL_CUDA(m, cudaMalloc(&m->nw_values, vb * m->nnz));
  }
  if (p->use_graph)
    return newton_step_graph(m, p, q_n, v_n, v_init, f_ext, lambda, v_out, q_out, stats, t_start);
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
  const int ls_max = p->ls_max_trials > 0 ? p->ls_max_trials : 10;
  const double ls_c1 = p->ls_c1 > 0.0 ? p->ls_c1 : 1e-4, ls_beta = p->ls_beta > 0.0 ? p->ls_beta : 0.5;
  int inner_total = 0, outer = 0, ls_trials = 0;
  bool converged = false;
  bool g_current = false;     // w.f, w.g and gn already hold the residual at v (an accepted trial)
  double gn = 0.0, cn = 0.0, g_init = -1.0;
  for (outer = 1; outer <= p->max_outer; ++outer) {
    bool inner_ok = false;
    for (int l = 0; l < p->max_inner; ++l) {
      cudaEventRecord(ev[0], s);
      if (!g_current) NTRY(residual(v, &gn));
      g_current = false;
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
        const double eta = std::max(
            0.0, p->lin_adaptive ? std::min(0.5, std::max(lin_rtol, 0.1 * target / gn)) : lin_rtol);
        NTRY(pcg_solve(m, w.values, w.g, w.dv, eta, lin_max, &it));
        lin_total += it;
      } else {
        NTRY(solver_factor_solve(m, w.values, w.g, w.dv));
      }
      bool ls_failed = false;
      if (p->line_search) {
        // eq. armijo: backtrack from a = 1 on phi = ||g||^2 / 2; the trial
        // residual of an accepted step is the next iteration's residual
        const double phi0 = 0.5 * gn * gn;
        double alpha = 1.0, gt = 0.0;
        bool accepted = false;
        for (int j = 0; j < ls_max && !accepted; ++j) {
          axpby_kernel<<<nb, 256, 0, s>>>(v, w.dv, alpha, ndof, m->nw_vt);
          NCUDA(cudaGetLastError());
          ++m->launches;
          ++ls_trials;
          NTRY(residual(m->nw_vt, &gt));
          if (0.5 * gt * gt <= (1.0 - 2.0 * ls_c1 * alpha) * phi0)
            accepted = true;
          else
            alpha *= ls_beta;
        }
        if (accepted) {
          NCUDA(cudaMemcpyAsync(v, m->nw_vt, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
          gn = gt;
          g_current = true;
        } else {
          ls_failed = true;   // Alg. 3: keep v and leave the inner loop
        }
      } else {
        axpy_kernel<<<nb, 256, 0, s>>>(v, w.dv, 1.0, ndof);
        NCUDA(cudaGetLastError());
        ++m->launches;
      }
      cudaEventRecord(ev[2], s);
      cudaEventSynchronize(ev[2]);
      float t1 = 0.f, t2 = 0.f;
      cudaEventElapsedTime(&t1, ev[0], ev[1]);
      cudaEventElapsedTime(&t2, ev[1], ev[2]);
      ms_asm += t1;
      ms_sol += t2;
      ++inner_total;
      if (ls_failed) break;
    }
    g_current = false;        // the multiplier update below changes g
    NTRY(launch_con_update(m, q_n, v, p->h, p->rho_alm, inner_ok ? 1 : 0, nullptr, lambda + 3 * m->nfixed));
    clamp_constraint<<<1, 1024, 0, s>>>(m->d_fixed_of_node, m->d_X, q_n, v, p->h, m->nn, p->rho_alm,
                                         inner_ok ? 1 : 0, nullptr, lambda, w.scal + 1,
                                         m->ncon ? m->d_con_sq : nullptr);
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
    stats->ls_trials = ls_trials;
    stats->g_init = g_init;
  }
  return converged ? TL_OK : fail(m, TL_ERR_NOT_CONVERGED, "Newton / ALM iteration caps reached");
}

// One time step with the AdamW inner solver (Algorithm 2): per inner
// iteration the AdamW update, the internal force at q = q_n + h v (float64
// class) and the gradient g of eq. grad_L with its norm, all on the device; the
// norms go to the host at the check interval (and once for g_0).  After the
// inner loop the velocity is committed (v_n <- v, as printed), lambda += rho c
// and ||c|| is read for the outer test.
extern "C" tl_status tl_adamw_step(tl_mesh* m, const tl_params* p, const tl_adamw_params* a, const double* q_n,
                                   const double* v_n, const double* v_init, const double* f_ext, double* lambda,
                                   double* v_out, double* q_out, tl_adamw_stats* stats) {
  if (!m || !p || !a || !q_n || !v_n || !v_out || !q_out || !(p->h > 0.0) || p->max_outer < 1 ||
      a->max_inner < 1 || a->check_every < 1 || !(a->lr > 0.0) || !(a->beta1 >= 0.0 && a->beta1 < 1.0) ||
      !(a->beta2 >= 0.0 && a->beta2 < 1.0) || !(a->eps > 0.0))
    return TL_ERR_INVALID_ARG;
  if ((m->nfixed > 0 || m->ncon > 0) && !lambda) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  const auto t_start = std::chrono::steady_clock::now();
  const int64_t ndof = 3 * m->nn;
  cudaStream_t s = m->stream;
  const unsigned nb = (unsigned)((ndof + 255) / 256);
  if (!m->nw_g) {
    TL_CUDA(m, cudaMalloc(&m->nw_g, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_f, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_dv, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->nw_scal, sizeof(double) * 4));
  }
  if (!m->aw_m1) {
    TL_CUDA(m, cudaMalloc(&m->aw_m1, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->aw_m2, sizeof(double) * ndof));
    TL_CUDA(m, cudaMalloc(&m->aw_vn, sizeof(double) * ndof));
  }
  TL_TRY(residual_ensure(m));
  double *g = m->nw_g, *f = m->nw_f, *scal = m->nw_scal, *vn = m->aw_vn, *v = v_out;
  TL_CUDA(m, cudaMemcpyAsync(v, v_init ? v_init : v_n, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
  TL_CUDA(m, cudaMemcpyAsync(vn, v_n, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
  auto read2 = [&](double* host) -> tl_status {     // scal[0] = ||g||, scal[2] = ||v||
    TL_CUDA(m, cudaMemcpyAsync(host, scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    TL_CUDA(m, cudaStreamSynchronize(s));
    return TL_OK;
  };
  int total = 0, outer = 0;
  bool converged = false;
  double gn = 0.0, cn = 0.0;
  for (outer = 1; outer <= p->max_outer; ++outer) {
    TL_CUDA(m, cudaMemsetAsync(g, 0, sizeof(double) * ndof, s));
    TL_CUDA(m, cudaMemsetAsync(m->aw_m1, 0, sizeof(double) * ndof, s));
    TL_CUDA(m, cudaMemsetAsync(m->aw_m2, 0, sizeof(double) * ndof, s));
    double g0 = -1.0;
    bool inner_ok = false;
    for (int l = 1; l <= a->max_inner; ++l) {
      const double bc1 = 1.0 - std::pow(a->beta1, (double)l), bc2 = 1.0 - std::pow(a->beta2, (double)l);
      adamw_update<<<nb, 256, 0, s>>>(v, m->aw_m1, m->aw_m2, g, ndof, a->beta1, a->beta2, bc1, bc2, a->lr,
                                      a->weight_decay, a->eps);
      TL_CUDA(m, cudaGetLastError());
      ++m->launches;
      TL_TRY(launch_force_prec(m, q_n, v, p->h, f, true));
      TL_TRY(launch_residual(m, p, q_n, vn, v, f, f_ext, lambda, g, scal));
      ++total;
      const bool check = (l % a->check_every) == 0;
      if (l == 1 || check || l == a->max_inner) {
        if (check) {
          norm_one_block<<<1, 1024, 0, s>>>(v, ndof, scal + 2);
          TL_CUDA(m, cudaGetLastError());
          ++m->launches;
        }
        double hs[3] = {0.0, 0.0, 0.0};
        TL_TRY(read2(hs));
        gn = hs[0];
        if (!std::isfinite(gn)) return fail(m, TL_ERR_NONFINITE, "non-finite AdamW gradient");
        if (l == 1) g0 = gn;
        if (check && (gn <= a->eps_in * (1.0 + hs[2]) || gn <= a->eps_rel * g0)) {
          inner_ok = true;
          break;
        }
      }
    }
    // commit v_n <- v; lambda += rho c(q_n + h v); ||c||
    TL_CUDA(m, cudaMemcpyAsync(vn, v, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
    TL_TRY(launch_con_update(m, q_n, v, p->h, p->rho_alm, 1, nullptr, lambda + 3 * m->nfixed));
    clamp_constraint<<<1, 1024, 0, s>>>(m->d_fixed_of_node, m->d_X, q_n, v, p->h, m->nn, p->rho_alm, 1, nullptr,
                                         lambda, scal + 1, m->ncon ? m->d_con_sq : nullptr);
    TL_CUDA(m, cudaGetLastError());
    ++m->launches;
    TL_CUDA(m, cudaMemcpyAsync(&cn, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    TL_CUDA(m, cudaStreamSynchronize(s));
    if (inner_ok && cn <= p->eps_out) {
      converged = true;
      break;
    }
  }
  if (outer > p->max_outer) outer = p->max_outer;
  q_from_v<<<nb, 256, 0, s>>>(q_n, v, p->h, ndof, q_out);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  TL_CUDA(m, cudaStreamSynchronize(s));
  if (stats) {
    stats->inner_iters = total;
    stats->outer_iters = outer;
    stats->converged = converged ? 1 : 0;
    stats->g_norm = gn;
    stats->c_norm = cn;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  }
  return converged ? TL_OK : fail(m, TL_ERR_NOT_CONVERGED, "AdamW / ALM iteration caps reached");
}
