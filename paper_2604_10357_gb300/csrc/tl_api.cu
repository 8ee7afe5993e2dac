// C ABI entry points (include/tl.h): handle life cycle, reference-geometry
// precomputation and argument checking.  Every compute step runs in the
// kernels of tl_element.cu, tl_pattern.cu and tl_residual.cu.
//
// Paper: arxiv 2604.10357 Sec. 4.1 (precompute once: reference gradients,
// Jacobians, quadrature weights, mass), Sec. 4.2 (fixed patterns), Sec. 4.3-4.4.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tl_ancf.cuh"
#include "tl_internal.cuh"

namespace tl {

tl_status fail(tl_mesh* m, tl_status s, const std::string& msg) {
  if (m) m->last_error = msg;
  return s;
}

tl_status cuda_fail(tl_mesh* m, cudaError_t e, const char* what) {
  if (m) m->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return TL_ERR_OOM;
  return TL_ERR_CUDA;
}

cudaEvent_t timer_open(tl_mesh* m) {
  if (!m->timing) return nullptr;
  cudaEvent_t ev = nullptr;
  if (!m->ev_pool.empty()) {
    ev = m->ev_pool.back();
    m->ev_pool.pop_back();
  } else if (cudaEventCreate(&ev) != cudaSuccess) {
    return nullptr;
  }
  cudaEventRecord(ev, m->stream);
  return ev;
}

void timer_close(tl_mesh* m, cudaEvent_t start, TimerCat cat) {
  if (!m->timing || !start) return;
  cudaEvent_t ev = nullptr;
  if (!m->ev_pool.empty()) {
    ev = m->ev_pool.back();
    m->ev_pool.pop_back();
  } else if (cudaEventCreate(&ev) != cudaSuccess) {
    m->ev_pool.push_back(start);
    return;
  }
  cudaEventRecord(ev, m->stream);
  (cat == kTimeElement ? m->ev_elem : m->ev_resid).emplace_back(start, ev);
}

namespace {

void free_mesh(tl_mesh* m) {
  if (!m) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(m->device);
  void* ptrs[] = {m->d_conn, m->d_user_of, m->d_geo64, m->d_ancf_me, m->d_geo32, m->d_geo_df, m->d_uv32, m->d_X, m->d_node_ptr, m->d_node_col,
                  m->d_row_ptr, m->d_col, m->d_blk, m->d_mass, m->d_mrow, m->d_fixed_of_node, m->d_fixed_diag,
                  m->d_flags, m->d_tile_counters, m->d_partials, m->d_dv, m->d_dv2, m->d_mass2, m->d_sell_row, m->d_sell_ptr, m->d_sell_col, m->d_sell_m,
                  m->d_con_ptr, m->d_con_col, m->d_con_val, m->d_con_b, m->d_ct_ptr, m->d_ct_con, m->d_ct_val,
                  m->d_con_w, m->d_con_sq, m->nw_g, m->nw_f, m->nw_dv, m->nw_scal, m->nw_vt, m->nw_values,
                  m->aw_m1, m->aw_m2, m->aw_vn};
  solver_destroy(m->solver);
  pcg_destroy(m->pcg);
  tile_maps_free(m);
  newton_graph_destroy(m->ngraph);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
  for (auto& pr : m->ev_elem) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto& pr : m->ev_resid) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  cudaSetDevice(cur);
  delete m;
}

// Reference gradients of the barycentric coordinates of a straight-sided
// tetrahedron: with D = [X1-X0, X2-X0, X3-X0] (columns), grad L_k = row k of
// D^{-1} (k = 1..3), grad L_0 = -(sum), and V = det(D)/6.
bool tet_geometry(const double* X, const int32_t* c, double out[16]) {
  double D[3][3];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) D[d][k] = X[3 * c[k + 1] + d] - X[3 * c[0] + d];
  const double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                     D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                     D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
  if (!(det > 0.0)) return false;
  double inv[3][3];
  inv[0][0] = (D[1][1] * D[2][2] - D[1][2] * D[2][1]) / det;
  inv[0][1] = (D[0][2] * D[2][1] - D[0][1] * D[2][2]) / det;
  inv[0][2] = (D[0][1] * D[1][2] - D[0][2] * D[1][1]) / det;
  inv[1][0] = (D[1][2] * D[2][0] - D[1][0] * D[2][2]) / det;
  inv[1][1] = (D[0][0] * D[2][2] - D[0][2] * D[2][0]) / det;
  inv[1][2] = (D[0][2] * D[1][0] - D[0][0] * D[1][2]) / det;
  inv[2][0] = (D[1][0] * D[2][1] - D[1][1] * D[2][0]) / det;
  inv[2][1] = (D[0][1] * D[2][0] - D[0][0] * D[2][1]) / det;
  inv[2][2] = (D[0][0] * D[1][1] - D[0][1] * D[1][0]) / det;
  for (int d = 0; d < 3; ++d) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
      out[3 * (k + 1) + d] = inv[k][d];
      s += inv[k][d];
    }
    out[d] = -s;
  }
  out[12] = det / 6.0;
  out[13] = out[14] = out[15] = 0.0;
  return true;
}

const int kEdge[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};

// Reason of the last failed tl_mesh_create on this thread (no handle exists).
thread_local std::string g_create_error;

// A fresh handle on the current device.
tl_mesh* new_mesh(void* stream, int32_t precision, int64_t nn, int64_t ne) {
  tl_mesh* m = new (std::nothrow) tl_mesh();
  if (!m) return nullptr;
  cudaGetDevice(&m->device);
  if (cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess ||
      m->num_sms < 1)
    m->num_sms = 1;
  m->stream = (cudaStream_t)stream;
  m->precision = precision;
  if (precision == TL_FP32_ELEM) {     // float32 PCG iteration: the row-contiguous product, 8 lanes per node
    m->tune.spmv_group = 8;
    m->tune.spmv_row = 1;
  }
  m->nn = nn;
  m->ne = ne;
  return m;
}

// Material table: Lame constants of SVK, the Mooney-Rivlin and Kelvin-Voigt
// constants as given; false on an unknown kind.
bool add_materials(tl_mesh* m, const tl_material* mats, int nmat) {
  for (int k = 0; k < nmat; ++k) {
    const tl_material& t = mats[k];
    MaterialDev md{};
    md.kind = t.kind;
    if (t.kind != TL_SVK && t.kind != TL_MOONEY_RIVLIN) return false;
    md.lam = t.E * t.nu / ((1.0 + t.nu) * (1.0 - 2.0 * t.nu));
    md.mu = t.E / (2.0 * (1.0 + t.nu));
    md.C10 = t.C10;
    md.C01 = t.C01;
    md.kappa = t.kappa;
    md.eta = t.eta_d;
    md.lam_d = t.lambda_d;
    md.kv = (t.eta_d != 0.0 || t.lambda_d != 0.0) ? 1 : 0;
    md.rho = t.rho0;
    m->mats.push_back(md);
  }
  return true;
}

// det J0 > 0 at every element quadrature point of an ANCF element, J0 the
// natural-coordinate Jacobian of its reference coefficients.
template <int ET>
bool ancf_jacobians_positive(const double* E0, const int32_t* c, const double dims[3]) {
  for (int q = 0; q < ancf::Traits<ET>::NQP; ++q) {
    double p[3], w;
    ancf::element_point<ET>(q, p, w);
    double J0[3][3] = {}, Ji[3][3];
    for (int a = 0; a < ancf::Traits<ET>::NEN; ++a) {
      double d[3];
      ancf::shape<ET, double>(a, p, dims, nullptr, d);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J0[i][j] += E0[3 * c[a] + i] * d[j];
    }
    if (!(ancf::inv3<double>(J0, Ji) > 0.0)) return false;
  }
  return true;
}

// Internal element order (material segments, each padded to a multiple of
// kTile), then the uploads.  On failure the handle is freed.
tl_status upload_mesh(tl_mesh* m, int nmat, const std::vector<std::vector<int64_t>>& by_mat, const int32_t* conn,
                      int nen, const std::vector<double>& geo_user, const double* X) {
  std::vector<int32_t> h_conn, h_user;
  std::vector<double> h_geo64;
  int64_t pos = 0;
  for (int k = 0; k < nmat; ++k) {
    if (by_mat[k].empty()) continue;
    Segment sg;
    sg.begin = pos;
    sg.end = pos + (int64_t)by_mat[k].size();
    const int64_t padded = ((int64_t)by_mat[k].size() + kTile - 1) / kTile * kTile;
    sg.padded_end = pos + padded;
    sg.mat = k;
    for (int64_t i = 0; i < padded; ++i) {
      if (i < (int64_t)by_mat[k].size()) {
        const int64_t e = by_mat[k][i];
        h_conn.insert(h_conn.end(), conn + nen * e, conn + nen * e + nen);
        h_user.push_back((int32_t)e);
        h_geo64.insert(h_geo64.end(), &geo_user[16 * e], &geo_user[16 * e] + 16);
      } else {
        h_conn.insert(h_conn.end(), nen, 0);
        h_user.push_back(-1);
        h_geo64.insert(h_geo64.end(), 16, 0.0);
      }
    }
    pos += padded;
    m->segs.push_back(sg);
  }
  m->ne_pad = pos;
  const int64_t ne_pad = std::max<int64_t>(pos, 1);
  std::vector<float> h_geo32(h_geo64.begin(), h_geo64.end());
  h_conn.resize((size_t)nen * ne_pad, 0);
  h_user.resize(ne_pad, -1);
  h_geo64.resize(16 * ne_pad, 0.0);
  h_geo32.resize(16 * ne_pad, 0.0f);
  tl_status st = TL_OK;
#define TRYC(call)                        \
  do {                                    \
    cudaError_t _e = (call);              \
    if (_e != cudaSuccess) {              \
      st = cuda_fail(m, _e, #call);       \
      free_mesh(m);                       \
      return st;                          \
    }                                     \
  } while (0)
  TRYC(cudaMalloc(&m->d_conn, sizeof(int32_t) * nen * ne_pad));
  TRYC(cudaMalloc(&m->d_user_of, sizeof(int32_t) * ne_pad));
  TRYC(cudaMalloc(&m->d_geo64, sizeof(double) * 16 * ne_pad));
  TRYC(cudaMalloc(&m->d_geo32, sizeof(float) * 16 * ne_pad));
  TRYC(cudaMalloc(&m->d_X, sizeof(double) * 3 * m->nn));
  TRYC(cudaMalloc(&m->d_flags, sizeof(uint32_t) * 4));
  TRYC(cudaMalloc(&m->d_tile_counters, sizeof(int) * kTileCounters));
  TRYC(cudaMemcpy(m->d_conn, h_conn.data(), sizeof(int32_t) * nen * ne_pad, cudaMemcpyHostToDevice));
  TRYC(cudaMemcpy(m->d_user_of, h_user.data(), sizeof(int32_t) * ne_pad, cudaMemcpyHostToDevice));
  TRYC(cudaMemcpy(m->d_geo64, h_geo64.data(), sizeof(double) * 16 * ne_pad, cudaMemcpyHostToDevice));
  TRYC(cudaMemcpy(m->d_geo32, h_geo32.data(), sizeof(float) * 16 * ne_pad, cudaMemcpyHostToDevice));
  if (m->precision == TL_FP32_ELEM) {
    // double-float copy (hi, lo float pairs) for the float64-class residual force
    std::vector<float> h_geodf(32 * ne_pad);
    for (int64_t i = 0; i < 16 * ne_pad; ++i) {
      const float hi = (float)h_geo64[i];
      h_geodf[2 * i] = hi;
      h_geodf[2 * i + 1] = (float)(h_geo64[i] - (double)hi);
    }
    TRYC(cudaMalloc(&m->d_geo_df, sizeof(float) * 32 * ne_pad));
    TRYC(cudaMemcpy(m->d_geo_df, h_geodf.data(), sizeof(float) * 32 * ne_pad, cudaMemcpyHostToDevice));
    TRYC(cudaMalloc(&m->d_uv32, sizeof(float2) * 3 * std::max<int64_t>(m->nn, 1)));
  }
  TRYC(cudaMemcpy(m->d_X, X, sizeof(double) * 3 * m->nn, cudaMemcpyHostToDevice));
  TRYC(cudaMemset(m->d_flags, 0, sizeof(uint32_t) * 4));
#undef TRYC
  return TL_OK;
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" {

const char* tl_status_string(tl_status s) {
  switch (s) {
    case TL_OK: return "ok";
    case TL_ERR_INVALID_ARG: return "invalid argument";
    case TL_ERR_OOM: return "out of device memory";
    case TL_ERR_CUDA: return "CUDA error";
    case TL_ERR_INVERTED: return "inverted element (det F <= 0)";
    case TL_ERR_NONFINITE: return "non-finite value";
    case TL_ERR_NOT_CONVERGED: return "not converged";
    case TL_ERR_SOLVER: return "sparse solver failure";
    case TL_ERR_TIMEOUT: return "device wait timed out";
    case TL_ERR_OVERFLOW: return "index overflow";
    case TL_ERR_UNSUPPORTED: return "unsupported";
    case TL_ERR_STATE: return "invalid call order";
  }
  return "unknown status";
}

const char* tl_last_error(const tl_mesh* m) { return m ? m->last_error.c_str() : g_create_error.c_str(); }

tl_status tl_mesh_create(const double* X, int64_t nn, const int32_t* conn, int64_t ne, const tl_material* mats,
                         int32_t nmat, const int32_t* mat_of_elem, int32_t precision, void* stream, tl_mesh** out) {
  if (!out) return TL_ERR_INVALID_ARG;
  *out = nullptr;
  if (!X || !conn || !mats || nn <= 0 || ne < 0 || nmat < 1) return TL_ERR_INVALID_ARG;
  if (precision != TL_FP64 && precision != TL_FP32_ELEM) return TL_ERR_INVALID_ARG;
  if (nn >= (int64_t)1 << 29) return TL_ERR_OVERFLOW;      // 9 * 3 nn row bases fit in int32
  g_create_error.clear();
  tl_mesh* m = new_mesh(stream, precision, nn, ne);
  if (!m) return TL_ERR_OOM;
  if (!add_materials(m, mats, nmat)) {
    free_mesh(m);
    return TL_ERR_INVALID_ARG;
  }
  // ---- validate connectivity and geometry; element order by material ------
  std::vector<std::vector<int64_t>> by_mat(nmat);
  std::vector<double> geo_user(16 * (size_t)ne);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* c = conn + 10 * e;
    for (int a = 0; a < 10; ++a)
      if (c[a] < 0 || c[a] >= nn) {
        g_create_error = "element " + std::to_string(e) + " references a node out of range";
        free_mesh(m);
        return TL_ERR_INVALID_ARG;
      }
    if (!tet_geometry(X, c, &geo_user[16 * e])) {
      g_create_error = "element " + std::to_string(e) + " has non-positive volume";
      free_mesh(m);
      return TL_ERR_INVALID_ARG;
    }
    double scale = 0.0;
    for (int d = 0; d < 3; ++d) scale = std::max(scale, std::fabs(X[3 * c[1] + d] - X[3 * c[0] + d]));
    for (int k = 0; k < 6; ++k)
      for (int d = 0; d < 3; ++d) {
        const double mid = 0.5 * (X[3 * c[kEdge[k][0]] + d] + X[3 * c[kEdge[k][1]] + d]);
        if (std::fabs(X[3 * c[4 + k] + d] - mid) > 1e-9 * (scale + std::fabs(mid))) {
          g_create_error = "element " + std::to_string(e) + " is not straight-sided";
          free_mesh(m);
          return TL_ERR_UNSUPPORTED;     // curved T10 elements are not handled
        }
      }
    const int mk = mat_of_elem ? mat_of_elem[e] : 0;
    if (mk < 0 || mk >= nmat) {
      free_mesh(m);
      return TL_ERR_INVALID_ARG;
    }
    by_mat[mk].push_back(e);
  }
  m->nen = 10;
  tl_status us = upload_mesh(m, nmat, by_mat, conn, 10, geo_user, X);
  if (us != TL_OK) return us;
  *out = m;
  return TL_OK;
}

tl_status tl_mesh_create_ancf(int32_t kind, const double* E0, int64_t ncoef, const int32_t* conn, int64_t ne,
                              const double* dims, const tl_material* mats, int32_t nmat,
                              const int32_t* mat_of_elem, int32_t precision, void* stream, tl_mesh** out) {
  if (!out) return TL_ERR_INVALID_ARG;
  *out = nullptr;
  if (!E0 || !conn || !dims || !mats || ncoef <= 0 || ne < 0 || nmat < 1) return TL_ERR_INVALID_ARG;
  if (kind != TL_ELEM_ANCF3243 && kind != TL_ELEM_ANCF3443) return TL_ERR_INVALID_ARG;
  if (precision != TL_FP64 && precision != TL_FP32_ELEM) return TL_ERR_INVALID_ARG;
  if (ncoef >= (int64_t)1 << 29) return TL_ERR_OVERFLOW;
  g_create_error.clear();
  const int nen = kind == TL_ELEM_ANCF3243 ? 8 : 16;
  tl_mesh* m = new_mesh(stream, precision, ncoef, ne);
  if (!m) return TL_ERR_OOM;
  m->etype = kind;
  m->nen = nen;
  if (!add_materials(m, mats, nmat)) {
    free_mesh(m);
    return TL_ERR_INVALID_ARG;
  }
  std::vector<std::vector<int64_t>> by_mat(nmat);
  std::vector<double> geo_user(16 * (size_t)ne, 0.0);
  for (int64_t e = 0; e < ne; ++e) {
    const int32_t* c = conn + (int64_t)nen * e;
    for (int a = 0; a < nen; ++a)
      if (c[a] < 0 || c[a] >= ncoef) {
        g_create_error = "element " + std::to_string(e) + " references a coefficient out of range";
        free_mesh(m);
        return TL_ERR_INVALID_ARG;
      }
    const double* dm = dims + 3 * e;
    if (!(dm[0] > 0.0 && dm[1] > 0.0 && dm[2] > 0.0 && std::isfinite(dm[0] + dm[1] + dm[2]))) {
      g_create_error = "element " + std::to_string(e) + " has non-positive dimensions";
      free_mesh(m);
      return TL_ERR_INVALID_ARG;
    }
    const bool ok = kind == TL_ELEM_ANCF3243 ? ancf_jacobians_positive<ancf::kBeam>(E0, c, dm)
                                             : ancf_jacobians_positive<ancf::kShell>(E0, c, dm);
    if (!ok) {
      g_create_error = "element " + std::to_string(e) + " has a non-positive reference Jacobian";
      free_mesh(m);
      return TL_ERR_INVALID_ARG;
    }
    geo_user[16 * e + 0] = dm[0];
    geo_user[16 * e + 1] = dm[1];
    geo_user[16 * e + 2] = dm[2];
    const int mk = mat_of_elem ? mat_of_elem[e] : 0;
    if (mk < 0 || mk >= nmat) {
      free_mesh(m);
      return TL_ERR_INVALID_ARG;
    }
    by_mat[mk].push_back(e);
  }
  tl_status us = upload_mesh(m, nmat, by_mat, conn, nen, geo_user, E0);
  if (us != TL_OK) return us;
  *out = m;
  return TL_OK;
}

tl_status tl_set_constraints(tl_mesh* m, int64_t ncon, const int32_t* row_ptr, const int32_t* col,
                             const double* val, const double* b) {
  if (!m || ncon < 0 || (ncon > 0 && (!row_ptr || !col || !val || !b))) return TL_ERR_INVALID_ARG;
  if (m->have_pattern) return fail(m, TL_ERR_STATE, "tl_set_constraints must come before tl_build_pattern");
  if (m->ncon > 0) return fail(m, TL_ERR_STATE, "constraints already set");
  if (ncon == 0) return TL_OK;
  const int64_t ndof = 3 * m->nn;
  if (row_ptr[0] != 0) return fail(m, TL_ERR_INVALID_ARG, "constraint row_ptr[0] must be 0");
  for (int64_t r = 0; r < ncon; ++r)
    if (row_ptr[r + 1] < row_ptr[r]) return fail(m, TL_ERR_INVALID_ARG, "constraint row_ptr not ascending");
  const int64_t nnzc = row_ptr[ncon];
  for (int64_t k = 0; k < nnzc; ++k)
    if (col[k] < 0 || col[k] >= ndof) return fail(m, TL_ERR_INVALID_ARG, "constraint column out of range");
  // C^T by DOF (the residual term h C_q^T (lambda + rho c), one DOF per thread)
  std::vector<int32_t> ct_ptr(ndof + 1, 0), ct_con(nnzc);
  std::vector<double> ct_val(nnzc);
  for (int64_t k = 0; k < nnzc; ++k) ++ct_ptr[col[k] + 1];
  for (int64_t i = 0; i < ndof; ++i) ct_ptr[i + 1] += ct_ptr[i];
  {
    std::vector<int32_t> cur(ct_ptr.begin(), ct_ptr.end() - 1);
    for (int64_t r = 0; r < ncon; ++r)
      for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
        const int32_t at = cur[col[k]]++;
        ct_con[at] = (int32_t)r;
        ct_val[at] = val[k];
      }
  }
  // node pairs coupled by a row (the Sec. 4.2 fill), per node
  std::vector<std::vector<int32_t>> ex(m->nn);
  for (int64_t r = 0; r < ncon; ++r) {
    std::vector<int32_t> nodes;
    for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) nodes.push_back(col[k] / 3);
    std::sort(nodes.begin(), nodes.end());
    nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
    for (int32_t I : nodes)
      for (int32_t J : nodes) ex[I].push_back(J);
  }
  m->h_ex_ptr.assign(m->nn + 1, 0);
  m->h_ex_col.clear();
  for (int64_t I = 0; I < m->nn; ++I) {
    std::sort(ex[I].begin(), ex[I].end());
    ex[I].erase(std::unique(ex[I].begin(), ex[I].end()), ex[I].end());
    m->h_ex_col.insert(m->h_ex_col.end(), ex[I].begin(), ex[I].end());
    m->h_ex_ptr[I + 1] = (int32_t)m->h_ex_col.size();
  }
  const size_t nz = (size_t)std::max<int64_t>(nnzc, 1);
  TL_CUDA(m, cudaMalloc(&m->d_con_ptr, sizeof(int32_t) * (ncon + 1)));
  TL_CUDA(m, cudaMalloc(&m->d_con_col, sizeof(int32_t) * nz));
  TL_CUDA(m, cudaMalloc(&m->d_con_val, sizeof(double) * nz));
  TL_CUDA(m, cudaMalloc(&m->d_con_b, sizeof(double) * ncon));
  TL_CUDA(m, cudaMalloc(&m->d_ct_ptr, sizeof(int32_t) * (ndof + 1)));
  TL_CUDA(m, cudaMalloc(&m->d_ct_con, sizeof(int32_t) * nz));
  TL_CUDA(m, cudaMalloc(&m->d_ct_val, sizeof(double) * nz));
  TL_CUDA(m, cudaMalloc(&m->d_con_w, sizeof(double) * ncon));
  TL_CUDA(m, cudaMalloc(&m->d_con_sq, sizeof(double)));
  TL_CUDA(m, cudaMemcpy(m->d_con_ptr, row_ptr, sizeof(int32_t) * (ncon + 1), cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(m->d_con_col, col, sizeof(int32_t) * nnzc, cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(m->d_con_val, val, sizeof(double) * nnzc, cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(m->d_con_b, b, sizeof(double) * ncon, cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(m->d_ct_ptr, ct_ptr.data(), sizeof(int32_t) * (ndof + 1), cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(m->d_ct_con, ct_con.data(), sizeof(int32_t) * nnzc, cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(m->d_ct_val, ct_val.data(), sizeof(double) * nnzc, cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemset(m->d_con_sq, 0, sizeof(double)));
  m->ncon = ncon;
  return TL_OK;
}

tl_status tl_build_pattern(tl_mesh* m, const int32_t* fixed_nodes, int64_t nfixed, int64_t* nnz_out) {
  if (!m || nfixed < 0 || (nfixed > 0 && !fixed_nodes)) return TL_ERR_INVALID_ARG;
  if (m->have_pattern) return fail(m, TL_ERR_STATE, "pattern already built");
  tl_status s = build_pattern(m, fixed_nodes, nfixed);
  if (s != TL_OK) return s;
  // float32 handles: the per-tile aggregation maps of the assembly, built
  // with the pattern so that the default launch shape can use them
  if (m->precision == TL_FP32_ELEM && m->etype == TL_ELEM_T10 && m->nn < (int64_t(1) << 24)) {
    s = tile_maps_ensure(m);
    if (s != TL_OK) return s;
  }
  if (nnz_out) *nnz_out = m->nnz;
  return TL_OK;
}

tl_status tl_get_pattern(const tl_mesh* m, int32_t* row_ptr, int32_t* col, int32_t* slot_map) {
  if (!m) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return TL_ERR_STATE;
  if (row_ptr && cudaMemcpyAsync(row_ptr, m->d_row_ptr, sizeof(int32_t) * (3 * m->nn + 1),
                                 cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess)
    return TL_ERR_CUDA;
  if (col && cudaMemcpyAsync(col, m->d_col, sizeof(int32_t) * m->nnz, cudaMemcpyDeviceToDevice, m->stream) !=
                 cudaSuccess)
    return TL_ERR_CUDA;
  if (slot_map) return expand_slot_map(m, slot_map, m->stream);
  return TL_OK;
}

tl_status tl_eval_force(tl_mesh* m, const double* q_n, const double* v, double h, double* f_int) {
  if (!m || !q_n || !v || !f_int) return TL_ERR_INVALID_ARG;
  return launch_force(m, q_n, v, h, f_int);
}

tl_status tl_eval_tangent(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                          void* K_elem) {
  if (!m || !q_n || !v || !K_elem) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  return launch_tangent(m, q_n, v, h, alpha, beta, 0.0, false, nullptr, nullptr, K_elem);
}

tl_status tl_assemble_hessian(tl_mesh* m, const double* q_n, const double* v, double h, double rho_alm,
                              void* values, double* f_int) {
  if (!m || !q_n || !v || !values || !(h > 0.0)) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  const size_t vb = (m->precision == TL_FP32_ELEM ? sizeof(float) : sizeof(double)) * (size_t)m->nnz;
  TL_CUDA(m, cudaMemsetAsync(values, 0, vb, m->stream));
  tl_status s = launch_tangent(m, q_n, v, h, h, 1.0, 1.0 / h, f_int != nullptr, f_int, values, nullptr);
  if (s != TL_OK) return s;
  return launch_add_penalty(m, h * h * rho_alm, values);
}

tl_status tl_eval_residual(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n, const double* v,
                           const double* f_int, const double* f_ext, const double* lambda, double* g,
                           double* g_norm) {
  if (!m || !p || !q_n || !v_n || !v || !g || !g_norm || !(p->h > 0.0)) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  if (!f_int) {
    tl_status s = launch_force_prec(m, q_n, v, p->h, g, true);   // g <- f_int(q_n + h v, v), float64 class
    if (s != TL_OK) return s;
    f_int = g;
  }
  return launch_residual(m, p, q_n, v_n, v, f_int, f_ext, lambda, g, g_norm);
}

tl_status tl_timing_enable(tl_mesh* m, int32_t on) {
  if (!m) return TL_ERR_INVALID_ARG;
  m->timing = on != 0;
  return TL_OK;
}

tl_status tl_timing_read(tl_mesh* m, tl_timing* out) {
  if (!m || !out) return TL_ERR_INVALID_ARG;
  TL_CUDA(m, cudaStreamSynchronize(m->stream));
  std::memset(out, 0, sizeof(*out));
  auto drain = [&](std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v, double& ms, int64_t& n) {
    for (auto& pr : v) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) ms += t;
      ++n;
      m->ev_pool.push_back(pr.first);
      m->ev_pool.push_back(pr.second);
    }
    v.clear();
  };
  drain(m->ev_elem, out->ms_element, out->n_element);
  drain(m->ev_resid, out->ms_residual, out->n_residual);
  out->launches = m->launches;
  m->launches = 0;
  return TL_OK;
}

tl_status tl_sync(tl_mesh* m) {
  if (!m) return TL_ERR_INVALID_ARG;
  TL_CUDA(m, cudaStreamSynchronize(m->stream));
  uint32_t flags = 0;
  TL_CUDA(m, cudaMemcpy(&flags, m->d_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  TL_CUDA(m, cudaMemset(m->d_flags, 0, sizeof(uint32_t)));
  if (flags & kFlagInverted) return fail(m, TL_ERR_INVERTED, "det F <= 0 at a quadrature point");
  if (flags & kFlagNonFinite) return fail(m, TL_ERR_NONFINITE, "non-finite residual norm");
  if (flags & kFlagBadIndex) return fail(m, TL_ERR_UNSUPPORTED, "index outside the pattern");
  return TL_OK;
}

tl_status tl_mesh_info_get(const tl_mesh* m, tl_mesh_info* out) {
  if (!m || !out) return TL_ERR_INVALID_ARG;
  out->nn = m->nn;
  out->ne = m->ne;
  out->ndof = 3 * m->nn;
  out->nnz = m->nnz;
  out->nnz_node = m->nnz_node;
  out->nfixed = m->nfixed;
  out->precision = m->precision;
  out->nmat = (int32_t)m->mats.size();
  out->ncon = m->ncon;
  out->element_kind = m->etype;
  out->nen = m->nen;
  return TL_OK;
}

void tl_mesh_destroy(tl_mesh* m) { free_mesh(m); }

}  // extern "C"
