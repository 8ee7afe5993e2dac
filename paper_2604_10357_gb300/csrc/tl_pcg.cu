// Preconditioned conjugate gradients for the Newton system H dv = -g on the
// device: an alternative to the direct solver for the inner solve of
// Algorithm 3 (H is symmetric positive definite under the conditions of the
// Sec. 4.4 remark).  Solved to a relative residual the caller chooses, the
// Newton iterates match those of an exact solve to that tolerance, so the
// converged state is the same to the Newton tolerance.
//
// Preconditioner: the inverse of each node's 3x3 diagonal block of H
// (block Jacobi), formed once per factorization call.  One warp per CSR row
// for the product H p (FP64 or FP32 values, FP64 vectors); dot products are
// reduced per block into partials and finished by a one-block kernel that
// also forms alpha / beta on the device; the host reads the residual norm
// every kCheck iterations.
#include <cmath>

#include "tl_internal.cuh"

namespace tl {

struct PcgWork {
  double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *binv = nullptr, *part = nullptr,
         *scal = nullptr;
  int32_t* diag_k = nullptr;   // per node: position of I in its own adjacency
  int nparts = 0;
};

namespace {

constexpr int kBlock = 256;
constexpr int kCheck = 8;

__global__ void node_diag_pos(const int32_t* node_ptr, const int32_t* node_col, int64_t nn, int32_t* diag_k) {
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nn) return;
  int lo = node_ptr[I], hi = node_ptr[I + 1] - 1, k = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = node_col[mid];
    if (v == I) { k = mid - node_ptr[I]; break; }
    if (v < I) lo = mid + 1; else hi = mid - 1;
  }
  diag_k[I] = k;
}

// Inverse of the 3x3 diagonal block of node I (symmetric part used).
template <typename T>
__global__ void block_jacobi(const T* vals, const int32_t* node_ptr, const int32_t* diag_k, int64_t nn,
                             double* binv) {
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const int p0 = node_ptr[I], deg = node_ptr[I + 1] - p0, k = diag_k[I];
  double* o = binv + 9 * I;
  if (k < 0) {                       // node without elements: empty rows
    for (int t = 0; t < 9; ++t) o[t] = 0.0;
    return;
  }
  double a[3][3];
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e) a[d][e] = double(vals[9 * (int64_t)p0 + 3 * deg * d + 3 * k + e]);
  for (int d = 0; d < 3; ++d)
    for (int e = d + 1; e < 3; ++e) a[d][e] = a[e][d] = 0.5 * (a[d][e] + a[e][d]);
  const double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
  const double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
  const double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
  const double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
  const double id = det != 0.0 ? 1.0 / det : 0.0;
  o[0] = c00 * id;
  o[1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
  o[2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
  o[3] = c01 * id;
  o[4] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
  o[5] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
  o[6] = c02 * id;
  o[7] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) * id;
  o[8] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;
}

// Ap = H p (one warp per row) and the partial dot products p . Ap
template <typename T>
__global__ void spmv_dot(const T* __restrict__ vals, const int32_t* __restrict__ col,
                         const int32_t* __restrict__ row_ptr, int64_t n, const double* __restrict__ p,
                         double* __restrict__ Ap, double* part) {
  __shared__ double red[kBlock / 32];
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  double dot = 0.0;
  if (row < n) {
    double acc = 0.0;
    for (int k = row_ptr[row] + lane; k < row_ptr[row + 1]; k += 32) acc += double(vals[k]) * p[col[k]];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      Ap[row] = acc;
      dot = acc * p[row];
    }
  }
  const double t = block_sum(dot, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// finish a partial sum: scal[slot] = sum(part)
__global__ void finish_sum(const double* part, int n, double* scal, int slot) {
  __shared__ double red[32];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
  const double s = block_sum(t, red);
  if (threadIdx.x == 0) scal[slot] = s;
}

// scal layout: 0 rz (current), 1 pAp, 2 rz_new, 3 rr, 4 alpha, 5 beta
// x += alpha p; r -= alpha Ap; z = P r; partials of r.z and r.r
__global__ void update_xr(double* x, double* r, double* z, const double* p, const double* Ap, const double* binv,
                          const double* scal, int64_t nn, double* part_rz, double* part_rr) {
  __shared__ double red[kBlock / 32];
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double alpha = scal[0] / scal[1];
  double rz = 0.0, rr = 0.0;
  if (I < nn) {
    double rv[3];
    for (int d = 0; d < 3; ++d) {
      const int64_t i = 3 * I + d;
      x[i] += alpha * p[i];
      rv[d] = r[i] - alpha * Ap[i];
      r[i] = rv[d];
    }
    const double* B = binv + 9 * I;
    for (int d = 0; d < 3; ++d) {
      const double zd = B[3 * d] * rv[0] + B[3 * d + 1] * rv[1] + B[3 * d + 2] * rv[2];
      z[3 * I + d] = zd;
      rz += rv[d] * zd;
      rr += rv[d] * rv[d];
    }
  }
  const double a = block_sum(rz, red);
  __syncthreads();
  const double b = block_sum(rr, red);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = a;
    part_rr[blockIdx.x] = b;
  }
}

// p = z + beta p with beta = rz_new / rz, then rz <- rz_new
__global__ void update_p(double* p, const double* z, int64_t n, double* scal) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double beta = scal[2] / scal[0];
  if (i < n) p[i] = z[i] + beta * p[i];
}

__global__ void roll_rz(double* scal) { scal[0] = scal[2]; }

// start: x = 0, r = b = -g, z = P r, p = z; partials of r.z and r.r
__global__ void pcg_start(const double* g, double* x, double* r, double* z, double* p, const double* binv,
                          int64_t nn, double* part_rz, double* part_rr) {
  __shared__ double red[kBlock / 32];
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double rz = 0.0, rr = 0.0;
  if (I < nn) {
    double rv[3];
    for (int d = 0; d < 3; ++d) {
      rv[d] = -g[3 * I + d];
      r[3 * I + d] = rv[d];
      x[3 * I + d] = 0.0;
    }
    const double* B = binv + 9 * I;
    for (int d = 0; d < 3; ++d) {
      const double zd = B[3 * d] * rv[0] + B[3 * d + 1] * rv[1] + B[3 * d + 2] * rv[2];
      z[3 * I + d] = zd;
      p[3 * I + d] = zd;
      rz += rv[d] * zd;
      rr += rv[d] * rv[d];
    }
  }
  const double a = block_sum(rz, red);
  __syncthreads();
  const double b = block_sum(rr, red);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = a;
    part_rr[blockIdx.x] = b;
  }
}

}  // namespace

void pcg_destroy(PcgWork* w) {
  if (!w) return;
  void* ptrs[] = {w->r, w->z, w->p, w->Ap, w->binv, w->part, w->scal, w->diag_k};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete w;
}

// Solve H dv = -g to ||r|| <= rtol ||g||.  values in assembly CSR order.
tl_status pcg_solve(tl_mesh* m, const void* values, const double* g, double* dv, double rtol, int max_iter,
                    int* iters_out) {
  cudaStream_t s = m->stream;
  const int64_t nn = m->nn, n = 3 * nn;
  if (!m->pcg) {
    PcgWork* w = new PcgWork();
    m->pcg = w;
    w->nparts = (int)std::max<int64_t>((nn + kBlock - 1) / kBlock, (32 * n + kBlock - 1) / kBlock);
    TL_CUDA(m, cudaMalloc(&w->r, sizeof(double) * n));
    TL_CUDA(m, cudaMalloc(&w->z, sizeof(double) * n));
    TL_CUDA(m, cudaMalloc(&w->p, sizeof(double) * n));
    TL_CUDA(m, cudaMalloc(&w->Ap, sizeof(double) * n));
    TL_CUDA(m, cudaMalloc(&w->binv, sizeof(double) * 9 * nn));
    TL_CUDA(m, cudaMalloc(&w->part, sizeof(double) * 2 * w->nparts));
    TL_CUDA(m, cudaMalloc(&w->scal, sizeof(double) * 8));
    TL_CUDA(m, cudaMalloc(&w->diag_k, sizeof(int32_t) * nn));
    node_diag_pos<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(m->d_node_ptr, m->d_node_col, nn, w->diag_k);
    TL_CUDA(m, cudaGetLastError());
  }
  PcgWork* w = m->pcg;
  const bool fp32 = m->precision == TL_FP32_ELEM;
  const unsigned nbn = (unsigned)((nn + kBlock - 1) / kBlock);
  const unsigned nbr = (unsigned)((32 * n + kBlock - 1) / kBlock);
  const unsigned nbv = (unsigned)((n + kBlock - 1) / kBlock);
  if (fp32)
    block_jacobi<float><<<nbn, kBlock, 0, s>>>((const float*)values, m->d_node_ptr, w->diag_k, nn, w->binv);
  else
    block_jacobi<double><<<nbn, kBlock, 0, s>>>((const double*)values, m->d_node_ptr, w->diag_k, nn, w->binv);
  double* part_rz = w->part;
  double* part_rr = w->part + w->nparts;
  pcg_start<<<nbn, kBlock, 0, s>>>(g, dv, w->r, w->z, w->p, w->binv, nn, part_rz, part_rr);
  finish_sum<<<1, 1024, 0, s>>>(part_rz, nbn, w->scal, 0);
  finish_sum<<<1, 1024, 0, s>>>(part_rr, nbn, w->scal, 3);
  double rr0 = 0.0;
  TL_CUDA(m, cudaMemcpyAsync(&rr0, w->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
  TL_CUDA(m, cudaStreamSynchronize(s));
  const double tol2 = rtol * rtol * rr0;
  int it = 0;
  m->launches += 4;
  while (it < max_iter) {
    for (int k = 0; k < kCheck && it < max_iter; ++k, ++it) {
      if (fp32)
        spmv_dot<float><<<nbr, kBlock, 0, s>>>((const float*)values, m->d_col, m->d_row_ptr, n, w->p, w->Ap, w->part);
      else
        spmv_dot<double><<<nbr, kBlock, 0, s>>>((const double*)values, m->d_col, m->d_row_ptr, n, w->p, w->Ap,
                                                w->part);
      finish_sum<<<1, 1024, 0, s>>>(w->part, nbr, w->scal, 1);
      update_xr<<<nbn, kBlock, 0, s>>>(dv, w->r, w->z, w->p, w->Ap, w->binv, w->scal, nn, part_rz, part_rr);
      finish_sum<<<1, 1024, 0, s>>>(part_rz, nbn, w->scal, 2);
      finish_sum<<<1, 1024, 0, s>>>(part_rr, nbn, w->scal, 3);
      update_p<<<nbv, kBlock, 0, s>>>(w->p, w->z, n, w->scal);
      roll_rz<<<1, 1, 0, s>>>(w->scal);
      m->launches += 7;
    }
    TL_CUDA(m, cudaGetLastError());
    double rr = 0.0;
    TL_CUDA(m, cudaMemcpyAsync(&rr, w->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    TL_CUDA(m, cudaStreamSynchronize(s));
    if (!std::isfinite(rr)) return fail(m, TL_ERR_NONFINITE, "PCG residual not finite");
    if (rr <= tol2) break;
  }
  if (iters_out) *iters_out = it;
  return TL_OK;
}

}  // namespace tl
