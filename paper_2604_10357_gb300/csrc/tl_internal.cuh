// Internal declarations of the T10 Total-Lagrangian GB300 library.
// Paper: arxiv 2604.10357, Sec. 4.1-4.4 (precomputation, fixed sparsity,
// internal force, gradient and Hessian assembly) and Algorithm 3.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "tl.h"

namespace tl {

// Elements processed by one CTA of the element kernels; every material
// segment of the internal element order is padded to a multiple of this.
constexpr int kTile = 32;

// Capacity of a tile's aggregation map (distinct unordered node pairs and
// contributions): 32 elements x 55 upper-triangle blocks.
constexpr int kAggCap = kTile * 55;
// Row stride of a tile's contribution pointers (kAggCap + 1 used): a multiple
// of 8 entries, so every tile's row starts on a 16-byte boundary.
constexpr int kAggCptrStride = kAggCap + 8;

// Tile counters of the persistent element launches (one per launch of a pass).
constexpr int kTileCounters = 256;

// Offset of the upper-triangle block (a, b), a <= b, of element e in the
// exchange buffer of the float32 assembly (9 floats per block, row-major
// [i][k] of K_ab): block rows P and 9 - P of group P hold 11 blocks,
// (P, P..9) then (9-P, 9-P..9); 55 blocks per element.  The tile maps
// (tl_tilemap.cu) and every kernel that fills the buffer share this layout.
__host__ __device__ __forceinline__ int xchg_offset(int e, int a, int b) {
  const int P = a <= 4 ? a : 9 - a;
  const int j = a <= 4 ? b - a : b + 1;
  return e * 495 + P * 99 + j * 9;
}

// Device-side sticky status bits (tl_sync turns them into tl_status).
enum : uint32_t { kFlagInverted = 1u, kFlagNonFinite = 2u, kFlagBadIndex = 4u };

struct MaterialDev {
  int kind;          // tl_material_kind
  int kv;            // Kelvin-Voigt on
  double lam, mu;    // SVK Lame constants
  double C10, C01, kappa;
  double eta, lam_d;
  double rho;
};

// One contiguous run of internal elements sharing a material.
struct Segment {
  int64_t begin, end;     // [begin, end) internal element ids (end - begin = real count)
  int64_t padded_end;     // begin + multiple of kTile
  int mat;                // index into the material table
};

struct Solver;       // sparse direct solver state (tl_solver.cu)
struct PcgWork;      // preconditioned CG state (tl_pcg.cu)
struct NewtonGraph;  // captured Newton step (tl_newton.cu)

// Launch shapes picked per handle by the autotuner (tl_tune.cu).
struct Tune {
  int spmv_group = 4;     // lanes per node in the PCG product H p (4, 8, 16, 32); 8 for float32 handles
  int spmv_row = 0;       // float32 iteration: 1 = row-contiguous product (lanes along the rows); 1 for float32 handles
  int elem_xchg = 1;      // FP32 assembly: 1 = exchanged vector runs, 0 = scalar scatter
  int elem_full_grid = 0; // element kernels: 0 = persistent grid (SMs x occupancy), 1 = one CTA per tile
  int elem_prefetch = 1;  // float32 element kernels: 1 = prefetch the next tile with cp.async
  int elem_ws = 0;        // float32 CSR assembly: 1 = warp-specialised scatter (needs prefetch, persistent grid)
  int residual_lanes = 1; // lanes per node in the residual (1 or 4)
  int residual_split = 1; // residual: 1 = mass product in double-float (float32 pairs, 48-bit significands)
  int force_split = 0;    // float32 handles: 1 = the float64-class residual force in double-float arithmetic
  int elem_occ2 = 1;      // float32 CSR assembly: 1 = two CTAs per SM (64 registers, overlaid exchange buffer)
  int elem_spread = 0;    // element kernels: 1 = tiles in flight spread over the mesh (permuted launch order)
  int pcg_f32 = 1;        // float32 Hessian: 1 = PCG vectors in float32 (dot products float64)
  int elem_agg = 1;       // float32 exchanged assembly: 1 = per-tile aggregation of shared node pairs
  int elem_pair = 1;      // float32 tangent passes: 1 = closed-form pair kernel for SVK (+ KV) segments
  int elem_fold = 1;      // pair kernel: 1 = folded form where c1 + c2 is not small (no cancellation)
  int tuned = 0;
  int64_t generation = 0; // bumped whenever a choice changes (captured graphs are rebuilt)
};

}  // namespace tl

struct tl_mesh {
  int device = 0;
  int num_sms = 1;                // streaming multiprocessors of the device
  cudaStream_t stream = nullptr;
  int precision = TL_FP64;
  int etype = TL_ELEM_T10;        // tl_element_kind
  int nen = 10;                   // nodes (T10) or coefficients (ANCF) per element
  int64_t nn = 0, ne = 0, ne_pad = 0;
  std::vector<tl::MaterialDev> mats;
  std::vector<tl::Segment> segs;
  std::string last_error;

  // internal element order (segments by material, padded)
  int32_t* d_conn = nullptr;      // ne_pad * nen
  int32_t* d_user_of = nullptr;   // ne_pad: user element id, -1 for padding
  double* d_geo64 = nullptr;      // ne_pad * 16: T10 grad L (4x3), V, 0,0,0; ANCF L, W, H, 0...
  double* d_ancf_me = nullptr;    // ANCF: ne_pad * nen(nen+1)/2 exact element mass (upper triangle)
  float* d_geo32 = nullptr;       // same in float32 (TL_FP32_ELEM)
  float* d_geo_df = nullptr;      // same as double-float pairs (TL_FP32_ELEM: float64-class residual force)
  float2* d_uv32 = nullptr;       // TL_FP32_ELEM T10: per DOF {q_n + h v - X, v} in float32, formed once
                                  // per element pass for the pair kernel's gather (3 nn)
  double* d_X = nullptr;          // 3 nn

  // pattern (tl_build_pattern)
  bool have_pattern = false;
  int64_t nnz = 0, nnz_node = 0;
  int32_t* d_node_ptr = nullptr;  // nn + 1
  int32_t* d_node_col = nullptr;  // nnz_node
  int32_t* d_row_ptr = nullptr;   // 3 nn + 1
  int32_t* d_col = nullptr;       // nnz
  uint8_t* d_blk = nullptr;       // ne_pad * nen^2: k of conn[b] in adj(conn[a])
  double* d_mass = nullptr;       // nnz_node consistent mass M_IJ
  double* d_mrow = nullptr;       // nn row sums of M
  int64_t nfixed = 0;
  int32_t* d_fixed_of_node = nullptr;  // nn: j (index in sorted fixed list) or -1
  int32_t* d_fixed_diag = nullptr;     // 3 nfixed: CSR position of (r, r)

  // per-tile aggregation maps of the float32 assembly (tl_tilemap.cu), built on demand
  int4* agg_slot = nullptr;       // ntiles x kAggCap
  uint16_t* agg_cptr = nullptr;   // ntiles x kAggCptrStride
  uint16_t* agg_code = nullptr;   // ntiles x kAggCap
  int32_t* agg_nu = nullptr;      // ntiles

  // general linear constraints c = C q - b (tl_set_constraints), rows after the clamp rows
  int64_t ncon = 0;
  int32_t *d_con_ptr = nullptr, *d_con_col = nullptr;   // C: ncon + 1 row offsets, DOF columns
  double *d_con_val = nullptr, *d_con_b = nullptr;
  int32_t *d_ct_ptr = nullptr, *d_ct_con = nullptr;     // C^T by DOF: 3 nn + 1 offsets, constraint ids
  double* d_ct_val = nullptr;
  double* d_con_w = nullptr;                            // lambda_c + rho c_c(q) of the last residual
  double* d_con_sq = nullptr;                           // ||c_general||^2 of the last multiplier update
  std::vector<int32_t> h_ex_ptr, h_ex_col;              // node pairs coupled by C (pattern fill), host

  // scratch
  uint32_t* d_flags = nullptr;    // sticky device status
  int* d_tile_counters = nullptr; // kTileCounters dynamic tile queues
  double* d_partials = nullptr;   // reduction partials
  double* d_dv = nullptr;         // v - v_n of the last residual (3 nn)
  float2* d_dv2 = nullptr;        // the same as float32 pairs (double-float mass product)
  float2* d_mass2 = nullptr;      // node-level mass as float32 pairs (nnz_node)
  // the same rows in sliced ELL (tl_residual.cu): slices of 32 rows, rows by
  // length within windows of 256; entry k of row lane l of slice s at
  // d_sell_ptr[s] + 32 k + l (padding: own node, zero mass)
  int32_t* d_sell_row = nullptr;  // node of each (slice, lane), -1 past nn (nslices x 32)
  int64_t* d_sell_ptr = nullptr;  // nslices + 1 entry offsets
  int32_t* d_sell_col = nullptr;
  float2* d_sell_m = nullptr;
  int partials_cap = 0;

  tl::Solver* solver = nullptr;
  tl::PcgWork* pcg = nullptr;
  tl::NewtonGraph* ngraph = nullptr;
  tl::Tune tune;
  // Newton work buffers (tl_newton_step), allocated on first use
  double *nw_g = nullptr, *nw_f = nullptr, *nw_dv = nullptr, *nw_scal = nullptr, *nw_vt = nullptr;
  double *aw_m1 = nullptr, *aw_m2 = nullptr, *aw_vn = nullptr;   // AdamW moments, committed velocity
  void* nw_values = nullptr;

  // instrumentation (tl_timing_*)
  bool timing = false;
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_elem, ev_resid;
};

namespace tl {

tl_status fail(tl_mesh* m, tl_status s, const std::string& msg);
tl_status cuda_fail(tl_mesh* m, cudaError_t e, const char* what);

#define TL_CUDA(m, call)                                   \
  do {                                                     \
    cudaError_t _e = (call);                               \
    if (_e != cudaSuccess) return tl::cuda_fail((m), _e, #call); \
  } while (0)

#define TL_TRY(call)                 \
  do {                               \
    tl_status _s = (call);           \
    if (_s != TL_OK) return _s;      \
  } while (0)

// element kernels (tl_element.cu)
tl_status launch_force(tl_mesh* m, const double* q_n, const double* v, double h, double* f);
// force with the element arithmetic forced to float64 when fp64 is set
tl_status launch_force_prec(tl_mesh* m, const double* q_n, const double* v, double h, double* f, bool fp64);

// sparse direct solver (tl_solver.cu) and PCG (tl_pcg.cu)
void solver_destroy(Solver* s);
// per-tile aggregation maps of the float32 assembly (tl_tilemap.cu)
tl_status tile_maps_ensure(tl_mesh* m);
void tile_maps_free(tl_mesh* m);
void pcg_destroy(PcgWork* w);
void newton_graph_destroy(NewtonGraph* g);
tl_status pcg_ensure(tl_mesh* m);
double* pcg_scalars(tl_mesh* m);   // slot 3: r.r of the current PCG iterate
tl_status pcg_prepare(tl_mesh* m, const void* values, const double* g, double* dv);
tl_status pcg_iterations(tl_mesh* m, const void* values, double* dv, int count);
tl_status pcg_result(tl_mesh* m, double* dv);   // dv from the float32 iterate (after the iterations)
bool pcg_float32(const tl_mesh* m);
tl_status pcg_spmv_only(tl_mesh* m, const void* values, int group);   // Ap = H p, for the autotuner
tl_status pcg_solve(tl_mesh* m, const void* values, const double* g, double* dv, double rtol, int max_iter,
                    int* iters_out);
tl_status launch_tangent(tl_mesh* m, const double* q_n, const double* v, double h,
                         double alpha, double beta, double mass_scale, bool do_force,
                         double* f, void* values, void* K_elem);

// ANCF elements (tl_ancf.cu): exact mass, and the element passes
tl_status ancf_build_mass(tl_mesh* m);
tl_status ancf_launch(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                      double mass_scale, bool do_force, bool do_tangent, double* f, void* values, void* K_elem);

// pattern kernels (tl_pattern.cu)
tl_status build_pattern(tl_mesh* m, const int32_t* fixed_nodes, int64_t nfixed);
tl_status expand_slot_map(const tl_mesh* m, int32_t* slot_map, cudaStream_t s);

// residual (tl_residual.cu)
tl_status launch_residual(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n,
                          const double* v, const double* f_int, const double* f_ext,
                          const double* lambda, double* g, double* g_norm);
tl_status launch_add_penalty(tl_mesh* m, double value, void* values);
// general constraints: lambda_c += rho c_c(q_n + h v) when the flag (or
// update) says so, and ||c_general||^2 into m->d_con_sq (no-op without them)
tl_status launch_con_update(tl_mesh* m, const double* q_n, const double* v, double h, double rho,
                            int update, const int32_t* update_flag, double* lambda_general);
tl_status residual_ensure(tl_mesh* m);
tl_status mass_split_build(tl_mesh* m, cudaStream_t s);

// instrumentation helpers (tl_api.cu): a category's event pair is opened
// before and closed after the launches it brackets.
enum TimerCat { kTimeElement = 0, kTimeResidual = 1 };
cudaEvent_t timer_open(tl_mesh* m);
void timer_close(tl_mesh* m, cudaEvent_t start, TimerCat cat);

}  // namespace tl
