// Sparse direct solver for the Newton system H dv = -g (eq.
// newton_linear_system), with the three phases of Sec. 4.6: a symbolic
// analysis once per mesh (fill-reducing ordering + symbolic factorization on
// the fixed pattern), a numeric Cholesky factorization every Newton
// iteration on the same pattern, and triangular solves on the device.
//
// The paper uses cuDSS, which is not available in this toolkit; the vendor
// solver here is cuSOLVER's sparse Cholesky (cusolverSp low-level csrchol).
// Its analysis does not reorder, so a nested-dissection ordering (METIS via
// cusolverSpXcsrmetisndHost) is computed once on the node adjacency and
// lifted to DOFs (3 consecutive DOFs per node); the permuted pattern and a
// gather map from the assembly order are built once on the host, and every
// factorization gathers the assembled values through that map.
#include <cusolverSp.h>
#include <cusolverSp_LOWLEVEL_PREVIEW.h>
#include <cusparse.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "tl_internal.cuh"

namespace tl {

struct Solver {
  cusolverSpHandle_t handle = nullptr;
  cusparseMatDescr_t descr = nullptr;
  csrcholInfo_t info = nullptr;
  int n = 0, nnz = 0;
  bool fp32 = false;
  int32_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  int32_t* d_map = nullptr;     // permuted entry -> assembly-order entry
  int32_t* d_perm = nullptr;    // new DOF -> old DOF
  void* d_vals = nullptr;
  void* d_rhs = nullptr;
  void* d_x = nullptr;
  void* d_buf = nullptr;
  double ms_analysis = 0.0;
};

namespace {

template <typename T>
__global__ void gather_values(const T* __restrict__ src, const int32_t* __restrict__ map, int64_t n, T* dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[map[i]];
}

template <typename T>
__global__ void permute_rhs(const double* __restrict__ g, const int32_t* __restrict__ perm, int n, T* rhs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rhs[i] = T(-g[perm[i]]);
}

template <typename T>
__global__ void unpermute(const T* __restrict__ x, const int32_t* __restrict__ perm, int n, double* dv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dv[perm[i]] = double(x[i]);
}

const char* cusolver_msg(cusolverStatus_t s) {
  switch (s) {
    case CUSOLVER_STATUS_SUCCESS: return "success";
    case CUSOLVER_STATUS_NOT_INITIALIZED: return "not initialized";
    case CUSOLVER_STATUS_ALLOC_FAILED: return "allocation failed";
    case CUSOLVER_STATUS_INVALID_VALUE: return "invalid value";
    case CUSOLVER_STATUS_ARCH_MISMATCH: return "arch mismatch";
    case CUSOLVER_STATUS_EXECUTION_FAILED: return "execution failed";
    case CUSOLVER_STATUS_INTERNAL_ERROR: return "internal error";
    case CUSOLVER_STATUS_MATRIX_TYPE_NOT_SUPPORTED: return "matrix type not supported";
    default: return "error";
  }
}

#define TL_SOLVER(m, call)                                                                   \
  do {                                                                                       \
    cusolverStatus_t _s = (call);                                                            \
    if (_s != CUSOLVER_STATUS_SUCCESS)                                                       \
      return fail((m), TL_ERR_SOLVER, std::string(#call) + ": " + cusolver_msg(_s));         \
  } while (0)

}  // namespace

void solver_destroy(Solver* s) {
  if (!s) return;
  if (s->info) cusolverSpDestroyCsrcholInfo(s->info);
  if (s->descr) cusparseDestroyMatDescr(s->descr);
  if (s->handle) cusolverSpDestroy(s->handle);
  void* ptrs[] = {s->d_rowptr, s->d_col, s->d_map, s->d_perm, s->d_vals, s->d_rhs, s->d_x, s->d_buf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
}

tl_status solver_setup(tl_mesh* m) {
  if (m->solver) return TL_OK;
  if (3 * m->nn > (int64_t)INT32_MAX) return fail(m, TL_ERR_OVERFLOW, "too many DOFs for the solver");
  Solver* s = new Solver();
  m->solver = s;
  s->fp32 = (m->precision == TL_FP32_ELEM);
  s->n = (int)(3 * m->nn);
  s->nnz = (int)m->nnz;
  const int nn = (int)m->nn;
  TL_SOLVER(m, cusolverSpCreate(&s->handle));
  TL_SOLVER(m, cusolverSpSetStream(s->handle, m->stream));
  if (cusparseCreateMatDescr(&s->descr) != CUSPARSE_STATUS_SUCCESS) return fail(m, TL_ERR_SOLVER, "cusparse descr");
  cusparseSetMatType(s->descr, CUSPARSE_MATRIX_TYPE_GENERAL);
  cusparseSetMatIndexBase(s->descr, CUSPARSE_INDEX_BASE_ZERO);

  // ---- ordering: nested dissection of the node graph, lifted to DOFs --------
  std::vector<int32_t> node_ptr(nn + 1), node_col(m->nnz_node), row_ptr(3 * (size_t)nn + 1);
  TL_CUDA(m, cudaMemcpy(node_ptr.data(), m->d_node_ptr, sizeof(int32_t) * (nn + 1), cudaMemcpyDeviceToHost));
  TL_CUDA(m, cudaMemcpy(node_col.data(), m->d_node_col, sizeof(int32_t) * m->nnz_node, cudaMemcpyDeviceToHost));
  TL_CUDA(m, cudaMemcpy(row_ptr.data(), m->d_row_ptr, sizeof(int32_t) * (3 * (size_t)nn + 1), cudaMemcpyDeviceToHost));
  std::vector<int> p(nn);
  cusolverStatus_t ord = cusolverSpXcsrmetisndHost(s->handle, nn, (int)m->nnz_node, s->descr, node_ptr.data(),
                                                   node_col.data(), nullptr, p.data());
  if (ord != CUSOLVER_STATUS_SUCCESS)
    TL_SOLVER(m, cusolverSpXcsrsymrcmHost(s->handle, nn, (int)m->nnz_node, s->descr, node_ptr.data(),
                                          node_col.data(), p.data()));
  std::vector<int> pinv(nn);
  for (int k = 0; k < nn; ++k) pinv[p[k]] = k;

  // ---- permuted pattern and gather map ---------------------------------------
  std::vector<int32_t> brow(3 * (size_t)nn + 1), bcol(s->nnz), bmap(s->nnz), perm(3 * (size_t)nn);
  std::vector<std::pair<int, int>> nbr;
  int64_t pos = 0;
  for (int k = 0; k < nn; ++k) {
    const int I = p[k];
    const int p0 = node_ptr[I], deg = node_ptr[I + 1] - p0;
    nbr.resize(deg);
    for (int t = 0; t < deg; ++t) nbr[t] = {pinv[node_col[p0 + t]], t};
    std::sort(nbr.begin(), nbr.end());
    for (int d = 0; d < 3; ++d) {
      const int64_t r_new = 3 * (int64_t)k + d;
      perm[r_new] = 3 * I + d;
      brow[r_new] = (int32_t)pos;
      const int32_t old_base = row_ptr[3 * (int64_t)I + d];
      for (int t = 0; t < deg; ++t)
        for (int e = 0; e < 3; ++e) {
          bcol[pos] = 3 * nbr[t].first + e;
          bmap[pos] = old_base + 3 * nbr[t].second + e;
          ++pos;
        }
    }
  }
  brow[3 * (size_t)nn] = (int32_t)pos;
  const size_t vb = s->fp32 ? sizeof(float) : sizeof(double);
  TL_CUDA(m, cudaMalloc(&s->d_rowptr, sizeof(int32_t) * brow.size()));
  TL_CUDA(m, cudaMalloc(&s->d_col, sizeof(int32_t) * bcol.size()));
  TL_CUDA(m, cudaMalloc(&s->d_map, sizeof(int32_t) * bmap.size()));
  TL_CUDA(m, cudaMalloc(&s->d_perm, sizeof(int32_t) * perm.size()));
  TL_CUDA(m, cudaMalloc(&s->d_vals, vb * s->nnz));
  TL_CUDA(m, cudaMalloc(&s->d_rhs, vb * s->n));
  TL_CUDA(m, cudaMalloc(&s->d_x, vb * s->n));
  TL_CUDA(m, cudaMemcpy(s->d_rowptr, brow.data(), sizeof(int32_t) * brow.size(), cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(s->d_col, bcol.data(), sizeof(int32_t) * bcol.size(), cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(s->d_map, bmap.data(), sizeof(int32_t) * bmap.size(), cudaMemcpyHostToDevice));
  TL_CUDA(m, cudaMemcpy(s->d_perm, perm.data(), sizeof(int32_t) * perm.size(), cudaMemcpyHostToDevice));

  // ---- symbolic analysis (once) -----------------------------------------------
  TL_SOLVER(m, cusolverSpCreateCsrcholInfo(&s->info));
  TL_SOLVER(m, cusolverSpXcsrcholAnalysis(s->handle, s->n, s->nnz, s->descr, s->d_rowptr, s->d_col, s->info));
  size_t internal = 0, work = 0;
  if (s->fp32)
    TL_SOLVER(m, cusolverSpScsrcholBufferInfo(s->handle, s->n, s->nnz, s->descr, (const float*)s->d_vals,
                                              s->d_rowptr, s->d_col, s->info, &internal, &work));
  else
    TL_SOLVER(m, cusolverSpDcsrcholBufferInfo(s->handle, s->n, s->nnz, s->descr, (const double*)s->d_vals,
                                              s->d_rowptr, s->d_col, s->info, &internal, &work));
  TL_CUDA(m, cudaMalloc(&s->d_buf, std::max<size_t>(work, 16)));
  return TL_OK;
}

// values: assembled H in the CSR order of tl_get_pattern (float or double by
// precision).  g: residual (double).  dv: output Newton direction (double).
tl_status solver_factor_solve(tl_mesh* m, const void* values, const double* g, double* dv) {
  Solver* s = m->solver;
  const unsigned nb_v = (unsigned)((s->nnz + 255) / 256), nb_n = (unsigned)((s->n + 255) / 256);
  if (s->fp32) {
    gather_values<float><<<nb_v, 256, 0, m->stream>>>((const float*)values, s->d_map, s->nnz, (float*)s->d_vals);
    TL_SOLVER(m, cusolverSpScsrcholFactor(s->handle, s->n, s->nnz, s->descr, (const float*)s->d_vals, s->d_rowptr,
                                          s->d_col, s->info, s->d_buf));
    int zp = -1;
    TL_SOLVER(m, cusolverSpScsrcholZeroPivot(s->handle, s->info, 0.0f, &zp));
    if (zp >= 0) return fail(m, TL_ERR_SOLVER, "Newton matrix not positive definite (zero pivot " + std::to_string(zp) + ")");
    permute_rhs<float><<<nb_n, 256, 0, m->stream>>>(g, s->d_perm, s->n, (float*)s->d_rhs);
    TL_SOLVER(m, cusolverSpScsrcholSolve(s->handle, s->n, (const float*)s->d_rhs, (float*)s->d_x, s->info, s->d_buf));
    unpermute<float><<<nb_n, 256, 0, m->stream>>>((const float*)s->d_x, s->d_perm, s->n, dv);
  } else {
    gather_values<double><<<nb_v, 256, 0, m->stream>>>((const double*)values, s->d_map, s->nnz, (double*)s->d_vals);
    TL_SOLVER(m, cusolverSpDcsrcholFactor(s->handle, s->n, s->nnz, s->descr, (const double*)s->d_vals, s->d_rowptr,
                                          s->d_col, s->info, s->d_buf));
    int zp = -1;
    TL_SOLVER(m, cusolverSpDcsrcholZeroPivot(s->handle, s->info, 0.0, &zp));
    if (zp >= 0) return fail(m, TL_ERR_SOLVER, "Newton matrix not positive definite (zero pivot " + std::to_string(zp) + ")");
    permute_rhs<double><<<nb_n, 256, 0, m->stream>>>(g, s->d_perm, s->n, (double*)s->d_rhs);
    TL_SOLVER(m, cusolverSpDcsrcholSolve(s->handle, s->n, (const double*)s->d_rhs, (double*)s->d_x, s->info, s->d_buf));
    unpermute<double><<<nb_n, 256, 0, m->stream>>>((const double*)s->d_x, s->d_perm, s->n, dv);
  }
  TL_CUDA(m, cudaGetLastError());
  m->launches += 3;
  return TL_OK;
}

}  // namespace tl
