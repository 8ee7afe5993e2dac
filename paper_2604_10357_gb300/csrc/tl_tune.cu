// Autotuner of the launch shapes (no counterpart in the paper).
//
// The best shape of the two hot launches depends on the mesh (node degrees,
// element order, material mix) and on the element precision, so it is chosen
// by timing, on the handle's own mesh and state, every variant that the
// library compiles:
//   * element pass (fused force + tangent + CSR assembly): persistent grid
//     (SMs x resident CTAs, tiles from a device counter) or one CTA per tile;
//     for the float32 form also the scatter strategy (exchanged 3-entry runs
//     as vector reductions, or one scalar reduction per entry) and the
//     cp.async prefetch of the next tile (or none), and warp specialisation
//     (scatter warps issue a tile's reductions while the compute warps
//     evaluate the next tile) and two CTAs per SM (64 registers, no prefetch);
//     for the fastest exchanged variant also the per-tile aggregation of the
//     node pairs that several elements of a tile share;
//   * PCG product H p: 4, 8 or 16 lanes per node, one neighbour per lane;
//     for the float32 iteration also 8, 16 or 32 lanes per node along the
//     contiguous rows;
//   * residual: 1 or 4 lanes per node, or the double-float mass product;
//   * float32 handles: the float64-class residual force in float64 and in
//     double-float arithmetic (timed and reported only: that choice trades
//     precision, so it stays with the caller).
// Each variant is warmed up once and timed over `reps` launches with CUDA
// events on the handle's stream; the fastest is kept in the handle and used by
// every later call (a captured Newton graph is rebuilt on its next use).
#include <algorithm>
#include <vector>

#include "tl_internal.cuh"

using namespace tl;

namespace {

template <typename F>
tl_status time_reps(tl_mesh* m, int reps, F&& launch, float* ms_out) {
  cudaEvent_t a = nullptr, b = nullptr;
  TL_CUDA(m, cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return fail(m, TL_ERR_CUDA, "event creation");
  }
  tl_status st = launch();                       // warm-up (and first-use setup)
  if (st == TL_OK) {
    cudaEventRecord(a, m->stream);
    for (int r = 0; r < reps && st == TL_OK; ++r) st = launch();
    cudaEventRecord(b, m->stream);
  }
  if (st == TL_OK && cudaEventSynchronize(b) == cudaSuccess) {
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    *ms_out = t / (float)reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

}  // namespace

extern "C" tl_status tl_autotune(tl_mesh* m, const double* q_n, const double* v, double h, int32_t reps,
                                 tl_tune_result* out) {
  if (!m || !q_n || !v || reps < 1) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  if (cudaSetDevice(m->device) != cudaSuccess) return fail(m, TL_ERR_CUDA, "cudaSetDevice");
  const bool fp32 = m->precision == TL_FP32_ELEM;
  const size_t vb = fp32 ? sizeof(float) : sizeof(double);
  void* values = nullptr;
  double* f = nullptr;
  TL_CUDA(m, cudaMalloc(&values, vb * (size_t)m->nnz));
  if (cudaMalloc(&f, sizeof(double) * 3 * m->nn) != cudaSuccess) {
    cudaFree(values);
    return fail(m, TL_ERR_OOM, "autotune buffers");
  }
  const Tune saved = m->tune;
  tl_tune_result r = {};
  tl_status st = TL_OK;
  // element pass: (prefetch, xchg, full grid) variants, and for float32 the
  // warp-specialised and two-CTA kernels; every exchanged float32 variant is
  // timed with and without the per-tile aggregation (the float64 kernels
  // have neither the exchange nor the prefetch)
  const bool agg_ok = fp32 && m->nn < (int64_t(1) << 24) && tile_maps_ensure(m) == TL_OK;
  struct V { int pf, xchg, full, ws, occ2, agg, pair; };
  std::vector<V> variants;
  if (fp32) {
    variants.push_back({1, 1, 0, 1, 0, 0, 0});       // warp-specialised
    variants.push_back({0, 1, 0, 0, 1, 0, 0});       // two CTAs per SM
    if (agg_ok) variants.push_back({0, 1, 0, 0, 1, 1, 0});
    // closed-form pair kernel for SVK segments (with and without the prefetch;
    // Mooney-Rivlin segments take the two-CTA aggregated kernel)
    if (agg_ok) {
      variants.push_back({1, 1, 0, 0, 1, 1, 1});
      variants.push_back({0, 1, 0, 0, 1, 1, 1});
    }
  }
  for (int pf = fp32 ? 1 : 0; pf >= 0; --pf)
    for (int xchg = fp32 ? 1 : 0; xchg >= 0; --xchg)
      for (int full = 0; full <= 1; ++full) {
        variants.push_back({pf, xchg, full, 0, 0, 0, 0});
        if (xchg && agg_ok) variants.push_back({pf, xchg, full, 0, 0, 1, 0});
      }
  float best = 1e30f;
  Tune chosen = saved;
  m->tune.elem_spread = 0;
  chosen.elem_spread = 0;
  for (size_t k = 0; k < variants.size() && st == TL_OK; ++k) {
    const V& vk = variants[k];
    m->tune.elem_prefetch = vk.pf;
    m->tune.elem_xchg = vk.xchg;
    m->tune.elem_full_grid = vk.full;
    m->tune.elem_ws = vk.ws;
    m->tune.elem_occ2 = vk.occ2;
    m->tune.elem_agg = vk.agg;
    m->tune.elem_pair = vk.pair;
    float ms = 0.f;
    st = time_reps(m, reps, [&]() {
      return launch_tangent(m, q_n, v, h, h, 1.0, 1.0 / h, true, f, values, nullptr);
    }, &ms);
    if (st != TL_OK) break;
    if (vk.pair)
      r.ms_pair = r.ms_pair > 0.f ? std::min(r.ms_pair, ms) : ms;
    else if (vk.agg)
      r.ms_agg = r.ms_agg > 0.f ? std::min(r.ms_agg, ms) : ms;
    else if (vk.ws)
      r.ms_ws = ms;
    else if (vk.occ2)
      r.ms_occ2 = ms;
    else
      r.ms_element[4 * (1 - vk.pf) + 2 * (1 - vk.xchg) + vk.full] = ms;
    if (ms < best) {
      best = ms;
      chosen.elem_prefetch = vk.pf;
      chosen.elem_xchg = vk.xchg;
      chosen.elem_full_grid = vk.full;
      chosen.elem_ws = vk.ws;
      chosen.elem_occ2 = vk.occ2;
      chosen.elem_agg = vk.agg;
      chosen.elem_pair = vk.pair;
    }
  }
  // tile order of the fastest element variant: in order or spread
  if (st == TL_OK && !chosen.elem_full_grid && !chosen.elem_ws) {
    m->tune = chosen;
    m->tune.elem_spread = 1;
    float ms = 0.f;
    st = time_reps(m, reps, [&]() {
      return launch_tangent(m, q_n, v, h, h, 1.0, 1.0 / h, true, f, values, nullptr);
    }, &ms);
    if (st == TL_OK) {
      r.ms_spread = ms;
      chosen.elem_spread = ms < best ? 1 : 0;
    }
  }
  m->tune = saved;
  // float64-class residual force of a float32 handle, float64 and
  // double-float: timed and reported, not chosen (the double-float force is
  // a precision trade: 48-bit significands can miss a 1e-8 Newton target
  // under large rotations), so the caller's setting stays
  if (st == TL_OK && fp32 && m->d_geo_df) {
    for (int k = 0; k < 2 && st == TL_OK; ++k) {
      m->tune.force_split = k;
      float ms = 0.f;
      st = time_reps(m, reps, [&]() { return launch_force_prec(m, q_n, v, h, f, true); }, &ms);
      if (st == TL_OK) r.ms_force[k] = ms;
    }
    m->tune.force_split = saved.force_split;
  }
  // PCG product: lanes per node
  if (st == TL_OK) st = pcg_ensure(m);
  m->tune.spmv_row = 0;
  best = 1e30f;
  const int groups[3] = {4, 8, 16};
  for (int k = 0; k < 3 && st == TL_OK; ++k) {
    float ms = 0.f;
    st = time_reps(m, reps, [&]() { return pcg_spmv_only(m, values, groups[k]); }, &ms);
    if (st != TL_OK) break;
    r.ms_spmv[k] = ms;
    if (ms < best) {
      best = ms;
      chosen.spmv_group = groups[k];
      chosen.spmv_row = 0;
    }
  }
  // float32 iteration: the row-contiguous product with 8, 16, 32 lanes per node
  if (st == TL_OK && pcg_float32(m)) {
    const int rgroups[3] = {8, 16, 32};
    m->tune.spmv_row = 1;
    for (int k = 0; k < 3 && st == TL_OK; ++k) {
      float ms = 0.f;
      st = time_reps(m, reps, [&]() { return pcg_spmv_only(m, values, rgroups[k]); }, &ms);
      if (st != TL_OK) break;
      r.ms_spmv_row[k] = ms;
      if (ms < best) {
        best = ms;
        chosen.spmv_group = rgroups[k];
        chosen.spmv_row = 1;
      }
    }
    m->tune.spmv_row = saved.spmv_row;
  }
  // residual: lanes per node (zero force, the handle's current lambda-free state)
  double* g = nullptr;
  if (st == TL_OK && cudaMalloc(&g, sizeof(double) * (3 * m->nn + 1)) != cudaSuccess)
    st = fail(m, TL_ERR_OOM, "autotune buffers");
  if (st == TL_OK) st = residual_ensure(m);
  if (st == TL_OK && cudaMemsetAsync(f, 0, sizeof(double) * 3 * m->nn, m->stream) != cudaSuccess)
    st = fail(m, TL_ERR_CUDA, "memset");
  best = 1e30f;
  const int lanes[2] = {1, 4};
  tl_params prm = {};
  prm.h = h;
  prm.rho_alm = 1e12;
  m->tune.residual_split = 0;
  for (int k = 0; k < 2 && st == TL_OK; ++k) {
    m->tune.residual_lanes = lanes[k];
    float ms = 0.f;
    st = time_reps(m, reps, [&]() {
      return launch_residual(m, &prm, q_n, v, v, f, nullptr, nullptr, g, g + 3 * m->nn);
    }, &ms);
    if (st != TL_OK) break;
    r.ms_residual[k] = ms;
    if (ms < best) {
      best = ms;
      chosen.residual_lanes = lanes[k];
      chosen.residual_split = 0;
    }
  }
  // residual with the double-float mass product, 1 and 4 lanes per node
  if (st == TL_OK && m->d_mass2) {
    m->tune.residual_split = 1;
    for (int k = 0; k < 2 && st == TL_OK; ++k) {
      m->tune.residual_lanes = lanes[k];
      float ms = 0.f;
      st = time_reps(m, reps, [&]() {
        return launch_residual(m, &prm, q_n, v, v, f, nullptr, nullptr, g, g + 3 * m->nn);
      }, &ms);
      if (st != TL_OK) break;
      r.ms_residual_split[k] = ms;
      if (ms < best) {
        best = ms;
        chosen.residual_split = 1;
        chosen.residual_lanes = lanes[k];
      }
    }
    m->tune.residual_split = saved.residual_split;
  }
  cudaStreamSynchronize(m->stream);
  cudaFree(values);
  cudaFree(f);
  if (g) cudaFree(g);
  if (st != TL_OK) {
    m->tune = saved;
    return st;
  }
  chosen.tuned = 1;
  chosen.generation = saved.generation + 1;
  m->tune = chosen;
  r.spmv_group = chosen.spmv_group;
  r.elem_xchg = chosen.elem_xchg;
  r.elem_full_grid = chosen.elem_full_grid;
  r.elem_prefetch = chosen.elem_prefetch;
  r.elem_ws = chosen.elem_ws;
  r.residual_lanes = chosen.residual_lanes;
  r.elem_occ2 = chosen.elem_occ2;
  r.elem_spread = chosen.elem_spread;
  r.pcg_f32 = chosen.pcg_f32;
  r.spmv_row = chosen.spmv_row;
  r.elem_agg = chosen.elem_agg;
  r.residual_split = chosen.residual_split;
  r.force_split = chosen.force_split;
  r.elem_pair = chosen.elem_pair;
  r.elem_fold = chosen.elem_fold;
  if (out) *out = r;
  return TL_OK;
}

extern "C" tl_status tl_tune_get(const tl_mesh* m, tl_tune_result* out) {
  if (!m || !out) return TL_ERR_INVALID_ARG;
  tl_tune_result r = {};
  r.spmv_group = m->tune.spmv_group;
  r.elem_xchg = m->tune.elem_xchg;
  r.elem_full_grid = m->tune.elem_full_grid;
  r.elem_prefetch = m->tune.elem_prefetch;
  r.elem_ws = m->tune.elem_ws;
  r.residual_lanes = m->tune.residual_lanes;
  r.elem_occ2 = m->tune.elem_occ2;
  r.elem_spread = m->tune.elem_spread;
  r.pcg_f32 = m->tune.pcg_f32;
  r.spmv_row = m->tune.spmv_row;
  r.elem_agg = m->tune.elem_agg;
  r.residual_split = m->tune.residual_split;
  r.force_split = m->tune.force_split;
  r.elem_pair = m->tune.elem_pair;
  r.elem_fold = m->tune.elem_fold;
  *out = r;
  return TL_OK;
}

extern "C" tl_status tl_tune_set(tl_mesh* m, const tl_tune_result* in) {
  if (!m || !in) return TL_ERR_INVALID_ARG;
  if (in->spmv_group != 4 && in->spmv_group != 8 && in->spmv_group != 16 && in->spmv_group != 32)
    return TL_ERR_INVALID_ARG;
  if ((in->elem_xchg != 0 && in->elem_xchg != 1) || (in->elem_full_grid != 0 && in->elem_full_grid != 1) ||
      (in->elem_prefetch != 0 && in->elem_prefetch != 1) || (in->elem_ws != 0 && in->elem_ws != 1) ||
      (in->residual_lanes != 1 && in->residual_lanes != 4) || (in->elem_occ2 != 0 && in->elem_occ2 != 1) ||
      (in->elem_spread != 0 && in->elem_spread != 1) || (in->pcg_f32 != 0 && in->pcg_f32 != 1) ||
      (in->spmv_row != 0 && in->spmv_row != 1) || (in->elem_agg != 0 && in->elem_agg != 1) ||
      (in->residual_split != 0 && in->residual_split != 1) || (in->force_split != 0 && in->force_split != 1) ||
      (in->elem_pair != 0 && in->elem_pair != 1) || (in->elem_fold != 0 && in->elem_fold != 1))
    return TL_ERR_INVALID_ARG;
  if ((in->elem_agg || in->elem_pair) && m->precision == TL_FP32_ELEM) TL_TRY(tile_maps_ensure(m));
  m->tune.spmv_group = in->spmv_group;
  m->tune.elem_prefetch = in->elem_prefetch;
  m->tune.elem_ws = in->elem_ws;
  m->tune.residual_lanes = in->residual_lanes;
  m->tune.elem_occ2 = in->elem_occ2;
  m->tune.elem_spread = in->elem_spread;
  m->tune.elem_xchg = in->elem_xchg;
  m->tune.elem_full_grid = in->elem_full_grid;
  m->tune.pcg_f32 = in->pcg_f32;
  m->tune.spmv_row = in->spmv_row;
  m->tune.elem_agg = in->elem_agg;
  m->tune.residual_split = in->residual_split;
  m->tune.force_split = in->force_split;
  m->tune.elem_pair = in->elem_pair;
  m->tune.elem_fold = in->elem_fold;
  m->tune.generation += 1;
  return TL_OK;
}
