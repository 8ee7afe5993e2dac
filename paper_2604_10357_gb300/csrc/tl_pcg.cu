// Preconditioned conjugate gradients for the Newton system H dv = -g on the
// device: an alternative to the direct solver for the inner solve of
// Algorithm 3 (H is symmetric positive definite under the conditions of the
// Sec. 4.4 remark).  Solved to a relative residual the caller chooses, the
// Newton iterates match those of an exact solve to that tolerance, so the
// converged state is the same to the Newton tolerance.
//
// Preconditioner: the inverse of each node's 3x3 diagonal block of H
// (block Jacobi), formed once per factorization call.  The product H p runs
// per node (FP64 or FP32 values, FP64 vectors): the three rows of a node have
// the same columns, so a group of lanes walks the node's neighbour list once,
// reads each neighbour's index and p values once for all three rows (the
// column array of the DOF CSR is not read), and reduces the three sums in
// the group.  Dot products are reduced per block into partials that the last
// block of the same launch sums (three launches per iteration: H p with p.Hp,
// the x / r / z update with r.z and r.r, the p update); alpha and beta are
// formed on the device from alternating r.z slots.  The host reads the
// residual norm every kCheck iterations, or the check runs on the device
// inside the captured Newton graph; the kernels of the iterations after the
// target is reached return at entry, so the check's granularity costs only
// launches.
#include <cmath>
#include <type_traits>

#include "tl_internal.cuh"

namespace tl {

struct PcgWork {
  double *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr, *binv = nullptr, *part = nullptr,
         *scal = nullptr;
  float* p32 = nullptr;        // float32 copy of p (float32 element form)
  // float32 iteration (float32 Hessian): x, r, z, Hp and the Jacobi blocks in float32
  float *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *Ap32 = nullptr, *binv32 = nullptr;
  unsigned* tickets = nullptr; // last-block counters of the two fused reductions
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

// The solve has reached its target (r.r <= slot 5) or broken down (slot 6):
// the remaining iterations of a chunk return at once, so a chunk that
// converges early costs its launches, not its work.  Read at kernel entry by
// every block alike (slot 3 changes only in the last block of update_xr*).
__device__ __forceinline__ bool pcg_done(const double* scal) { return scal[3] <= scal[5] || scal[6] != 0.0; }

// The last block to finish a pass sums the per-block partials in a fixed
// order (deterministic) and writes the total: a ticket counter (zero between
// passes; the last block resets it) replaces a separate one-block launch.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool is_last;
  __threadfence();                       // this block's partials before its ticket
  if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;                        // uniform over the block
}

__device__ __forceinline__ double sum_partials(const double* part, int n, double* red) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += __ldcg(part + i);
  return block_sum(t, red);
}

// Ap = H p with a group of G lanes per node I (rows 3I..3I+2): lane l takes
// the neighbours j = l, l+G, ..., reads node_col once, p[3J..3J+2] once and
// the three 3-entry runs (row 3I+d starts at 9 ptr(I) + 3 deg(I) d), and the
// group reduces the three sums.  Partial dot products p . Ap per block.
// With float32 values (the float32 element form) the products and the lane
// sums are float32 on a float32 copy of p (GB300 runs float64 arithmetic at
// 1/64 of the float32 rate; a float32 H defines the product to ~1e-7 anyway),
// and only the three node sums are widened: Ap and p.Ap stay float64.
template <typename T> struct SpmvAcc { using type = double; };
template <> struct SpmvAcc<float> { using type = float; };

template <typename T, int G>
__global__ void spmv_node(const T* __restrict__ vals, const int32_t* __restrict__ node_ptr,
                          const int32_t* __restrict__ node_col, int64_t nn, const double* __restrict__ p,
                          const float* __restrict__ p32, double* __restrict__ Ap, double* part, double* scal,
                          unsigned* ticket) {
  using A = typename SpmvAcc<T>::type;
  __shared__ double red[kBlock / 32];
  if (pcg_done(scal)) return;
  const int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int l = threadIdx.x & (G - 1);
  A s0 = 0, s1 = 0, s2 = 0;
  double dot = 0.0;
  if (I < nn) {
    const int p0 = node_ptr[I], deg = node_ptr[I + 1] - p0;
    const T* v0 = vals + 9 * (int64_t)p0;
    const T* v1 = v0 + 3 * deg;
    const T* v2 = v1 + 3 * deg;
    for (int j = l; j < deg; j += G) {
      const int J = node_col[p0 + j];
      A x0, x1, x2;
      if constexpr (std::is_same<A, float>::value) {
        x0 = p32[3 * J]; x1 = p32[3 * J + 1]; x2 = p32[3 * J + 2];
      } else {
        x0 = p[3 * (int64_t)J]; x1 = p[3 * (int64_t)J + 1]; x2 = p[3 * (int64_t)J + 2];
      }
      s0 += A(v0[3 * j]) * x0 + A(v0[3 * j + 1]) * x1 + A(v0[3 * j + 2]) * x2;
      s1 += A(v1[3 * j]) * x0 + A(v1[3 * j + 1]) * x1 + A(v1[3 * j + 2]) * x2;
      s2 += A(v2[3 * j]) * x0 + A(v2[3 * j + 1]) * x1 + A(v2[3 * j + 2]) * x2;
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (I < nn && l == 0) {
    const double d0 = s0, d1 = s1, d2 = s2;
    Ap[3 * I] = d0;
    Ap[3 * I + 1] = d1;
    Ap[3 * I + 2] = d2;
    dot = d0 * p[3 * I] + d1 * p[3 * I + 1] + d2 * p[3 * I + 2];
  }
  const double t = block_sum(dot, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (last_block(ticket)) {
    __syncthreads();
    const double tot = sum_partials(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      scal[1] = tot;
      *ticket = 0u;
    }
  }
}

// finish a partial sum: scal[slot] = sum(part)
// No r.r target and no breakdown: the per-iteration kernels run.
__global__ void pcg_clear_target(double* scal) {
  scal[5] = -1.0;
  scal[6] = 0.0;
}

__global__ void finish_sum(const double* part, int n, double* scal, int slot) {
  __shared__ double red[32];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
  const double s = block_sum(t, red);
  if (threadIdx.x == 0) scal[slot] = s;
}

// scal layout: 0 and 2 r.z of alternate iterations (iteration k reads slot
// 2 (k % 2) and writes slot 2 ((k + 1) % 2)), 1 p.Ap, 3 r.r, 5 the r.r target
// (-1: none), 6 breakdown flag, 7 iterations run.
// x += alpha p; r -= alpha Ap; z = P r; r.z and r.r finished by the last block
__global__ void update_xr(double* x, double* r, double* z, const double* p, const double* Ap, const double* binv,
                          double* scal, int64_t nn, double* part_rz, double* part_rr, int parity,
                          unsigned* ticket) {
  __shared__ double red[kBlock / 32];
  if (pcg_done(scal)) return;
  // pAp <= 0: H is not positive definite along p (CG breakdown); stop moving
  // and raise the breakdown slot, which ends the iteration at the next check
  const int rz_old = 2 * parity, rz_new = 2 - 2 * parity;
  const bool ok = scal[1] > 0.0;
  const double alpha = ok ? scal[rz_old] / scal[1] : 0.0;
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) scal[6] = 1.0;
  double rz = 0.0, rr = 0.0;
  // grid-stride over the nodes (a small grid: short launches, few partials)
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nn; I += (int64_t)gridDim.x * blockDim.x) {
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
  if (last_block(ticket)) {
    __syncthreads();
    const double trz = sum_partials(part_rz, gridDim.x, red);
    __syncthreads();
    const double trr = sum_partials(part_rr, gridDim.x, red);
    if (threadIdx.x == 0) {
      scal[rz_new] = trz;
      scal[3] = trr;
      scal[7] += 1.0;                    // iterations run
      *ticket = 0u;
    }
  }
}

// p = z + beta p with beta = (r.z new) / (r.z old)
__global__ void update_p(double* p, float* p32, const double* z, int64_t n, const double* scal, int parity) {
  if (pcg_done(scal)) return;
  const double rz_old = scal[2 * parity], rz_new = scal[2 - 2 * parity];
  const double beta = rz_old != 0.0 ? rz_new / rz_old : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = z[i] + beta * p[i];
    p[i] = v;
    if (p32) p32[i] = float(v);
  }
}

// start: x = 0, r = b = -g, z = P r, p = z; partials of r.z and r.r
__global__ void pcg_start(const double* g, double* x, double* r, double* z, double* p, float* p32,
                          const double* binv, int64_t nn, double* part_rz, double* part_rr, double* scal) {
  __shared__ double red[kBlock / 32];
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I == 0) {
    scal[5] = -1.0;                      // no target until the caller sets one
    scal[6] = 0.0;
    scal[7] = 0.0;
  }
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
      if (p32) p32[3 * I + d] = float(zd);
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

// ---------------------------------------------------------------------------
// Float32 iteration for a float32 Hessian: the vectors x, r, z, p, Hp and the
// Jacobi blocks are float32 (a float32 H defines the Newton direction to
// ~1e-6, the tolerance floor of this solve), halving the vector traffic and
// keeping the arithmetic off GB300's float64 pipe; dot products are summed in
// float64; the input -g and the output dv stay float64.
// ---------------------------------------------------------------------------
__global__ void jacobi_to_f32(const double* binv, int64_t n, float* binv32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) binv32[i] = float(binv[i]);
}

__global__ void pcg_start32(const double* g, float* x, float* r, float* z, float* p, const float* binv,
                            int64_t nn, double* part_rz, double* part_rr, double* scal) {
  __shared__ double red[kBlock / 32];
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I == 0) {
    scal[5] = -1.0;                      // no target until the caller sets one
    scal[6] = 0.0;
    scal[7] = 0.0;
  }
  double rz = 0.0, rr = 0.0;
  if (I < nn) {
    float rv[3];
    for (int d = 0; d < 3; ++d) {
      rv[d] = float(-g[3 * I + d]);
      r[3 * I + d] = rv[d];
      x[3 * I + d] = 0.0f;
    }
    const float* B = binv + 9 * I;
    for (int d = 0; d < 3; ++d) {
      const float zd = B[3 * d] * rv[0] + B[3 * d + 1] * rv[1] + B[3 * d + 2] * rv[2];
      z[3 * I + d] = zd;
      p[3 * I + d] = zd;
      rz += double(rv[d]) * double(zd);
      rr += double(rv[d]) * double(rv[d]);
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

template <int G>
__global__ void spmv_node32(const float* __restrict__ vals, const int32_t* __restrict__ node_ptr,
                            const int32_t* __restrict__ node_col, int64_t nn, const float* __restrict__ p,
                            float* __restrict__ Ap, double* part, double* scal, unsigned* ticket) {
  __shared__ double red[kBlock / 32];
  if (pcg_done(scal)) return;
  const int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
  const int l = threadIdx.x & (G - 1);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  double dot = 0.0;
  if (I < nn) {
    const int p0 = node_ptr[I], deg = node_ptr[I + 1] - p0;
    const float* v0 = vals + 9 * (int64_t)p0;
    const float* v1 = v0 + 3 * deg;
    const float* v2 = v1 + 3 * deg;
    for (int j = l; j < deg; j += G) {
      const int J = node_col[p0 + j];
      const float x0 = p[3 * J], x1 = p[3 * J + 1], x2 = p[3 * J + 2];
      s0 += v0[3 * j] * x0 + v0[3 * j + 1] * x1 + v0[3 * j + 2] * x2;
      s1 += v1[3 * j] * x0 + v1[3 * j + 1] * x1 + v1[3 * j + 2] * x2;
      s2 += v2[3 * j] * x0 + v2[3 * j + 1] * x1 + v2[3 * j + 2] * x2;
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (I < nn && l == 0) {
    Ap[3 * I] = s0;
    Ap[3 * I + 1] = s1;
    Ap[3 * I + 2] = s2;
    dot = double(s0) * double(p[3 * I]) + double(s1) * double(p[3 * I + 1]) + double(s2) * double(p[3 * I + 2]);
  }
  const double t = block_sum(dot, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (last_block(ticket)) {
    __syncthreads();
    const double tot = sum_partials(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      scal[1] = tot;
      *ticket = 0u;
    }
  }
}

// Ap = H p, row-contiguous form (float32 iteration): a group of G lanes per
// node walks the three rows of node I together, lane l taking the positions
// t = l, l+G, ... of each row (neighbour j = t / 3, component k = t % 3), so
// every value load of the group is one contiguous run; the neighbour index
// and p[3J+k] are read once for the three rows.  Grid-stride over the nodes
// with at most `nparts` blocks (the partials of p.Ap).
template <int G>
__global__ void spmv_row32(const float* __restrict__ vals, const int32_t* __restrict__ node_ptr,
                           const int32_t* __restrict__ node_col, int64_t nn, const float* __restrict__ p,
                           float* __restrict__ Ap, double* part, double* scal, unsigned* ticket) {
  static_assert(G >= 4 && G <= 32 && (G & (G - 1)) == 0, "G: power of two in [4, 32]");
  __shared__ double red[kBlock / 32];
  if (pcg_done(scal)) return;
  const int l = threadIdx.x & (G - 1);
  const int64_t groups = (int64_t)gridDim.x * (kBlock / G);
  // the loop bound is tested on the warp's first group, so every lane of a
  // warp runs the same trips and reaches the shuffles together
  const int64_t warp_first = (blockIdx.x * (int64_t)kBlock + (threadIdx.x & ~31)) / G;
  const int sub = (threadIdx.x & 31) / G;
  double dot = 0.0;
  for (int64_t I0 = warp_first; I0 < nn; I0 += groups) {
    const int64_t I = I0 + sub;
    const bool act = I < nn;
    const int p0 = act ? node_ptr[I] : 0, n3 = act ? 3 * (node_ptr[I + 1] - p0) : 0;
    const float* v0 = vals + 9 * (int64_t)p0;
    const float* v1 = v0 + n3;
    const float* v2 = v1 + n3;
    const int32_t* c = node_col + p0;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    int j = l / 3, k = l - 3 * (l / 3);
#pragma unroll 2
    for (int t = l; t < n3; t += G) {
      const float x = p[3 * c[j] + k];
      s0 += v0[t] * x;
      s1 += v1[t] * x;
      s2 += v2[t] * x;
      j += G / 3;
      k += G % 3;
      if (k >= 3) {
        k -= 3;
        ++j;
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (act && l == 0) {
      Ap[3 * I] = s0;
      Ap[3 * I + 1] = s1;
      Ap[3 * I + 2] = s2;
      dot += double(s0) * double(p[3 * I]) + double(s1) * double(p[3 * I + 1]) + double(s2) * double(p[3 * I + 2]);
    }
  }
  const double t = block_sum(dot, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (last_block(ticket)) {
    __syncthreads();
    const double tot = sum_partials(part, gridDim.x, red);
    if (threadIdx.x == 0) {
      scal[1] = tot;
      *ticket = 0u;
    }
  }
}

__global__ void update_xr32(float* x, float* r, float* z, const float* p, const float* Ap, const float* binv,
                            double* scal, int64_t nn, double* part_rz, double* part_rr, int parity,
                            unsigned* ticket) {
  __shared__ double red[kBlock / 32];
  if (pcg_done(scal)) return;
  const int rz_old = 2 * parity, rz_new = 2 - 2 * parity;
  const bool ok = scal[1] > 0.0;
  const float alpha = ok ? float(scal[rz_old] / scal[1]) : 0.0f;
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) scal[6] = 1.0;
  double rz = 0.0, rr = 0.0;
  // grid-stride over the nodes (a small grid: short launches, few partials)
  for (int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; I < nn; I += (int64_t)gridDim.x * blockDim.x) {
    float rv[3];
    for (int d = 0; d < 3; ++d) {
      const int64_t i = 3 * I + d;
      x[i] += alpha * p[i];
      rv[d] = r[i] - alpha * Ap[i];
      r[i] = rv[d];
    }
    const float* B = binv + 9 * I;
    for (int d = 0; d < 3; ++d) {
      const float zd = B[3 * d] * rv[0] + B[3 * d + 1] * rv[1] + B[3 * d + 2] * rv[2];
      z[3 * I + d] = zd;
      rz += double(rv[d]) * double(zd);
      rr += double(rv[d]) * double(rv[d]);
    }
  }
  const double a = block_sum(rz, red);
  __syncthreads();
  const double b = block_sum(rr, red);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = a;
    part_rr[blockIdx.x] = b;
  }
  if (last_block(ticket)) {
    __syncthreads();
    const double trz = sum_partials(part_rz, gridDim.x, red);
    __syncthreads();
    const double trr = sum_partials(part_rr, gridDim.x, red);
    if (threadIdx.x == 0) {
      scal[rz_new] = trz;
      scal[3] = trr;
      scal[7] += 1.0;                    // iterations run
      *ticket = 0u;
    }
  }
}

// p = z + beta p, grid-stride over float4 groups (p and z from cudaMalloc:
// 16-byte aligned) and the scalar tail; a small grid (a few blocks per SM)
// keeps the launch short, which matters most for iterations that return at
// entry.
__global__ void update_p32(float* p, const float* z, int64_t n, const double* scal, int parity) {
  if (pcg_done(scal)) return;
  const double rz_old = scal[2 * parity], rz_new = scal[2 - 2 * parity];
  const float beta = rz_old != 0.0 ? float(rz_new / rz_old) : 0.0f;
  const int64_t n4 = n / 4, stride = (int64_t)gridDim.x * blockDim.x;
  float4* p4 = reinterpret_cast<float4*>(p);
  const float4* z4 = reinterpret_cast<const float4*>(z);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 zv = z4[i];
    float4 pv = p4[i];
    pv.x = zv.x + beta * pv.x;
    pv.y = zv.y + beta * pv.y;
    pv.z = zv.z + beta * pv.z;
    pv.w = zv.w + beta * pv.w;
    p4[i] = pv;
  }
  const int64_t t = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) p[t] = z[t] + beta * p[t];
}

__global__ void widen(const float* x, int64_t n, double* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = double(x[i]);
}

}  // namespace

// The float32 iteration runs for a float32 Hessian unless the autotuner or the
// caller turned it off.
bool pcg_float32(const tl_mesh* m) { return m->precision == TL_FP32_ELEM && m->tune.pcg_f32; }

void pcg_destroy(PcgWork* w) {
  if (!w) return;
  void* ptrs[] = {w->r, w->z, w->p, w->Ap, w->binv, w->part, w->scal, w->diag_k, w->p32, w->tickets,
                  w->x32, w->r32, w->z32, w->Ap32, w->binv32};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete w;
}

// Allocate the PCG work arrays once per handle (no-op afterwards).
tl_status pcg_ensure(tl_mesh* m) {
  if (m->pcg) return TL_OK;
  const int64_t nn = m->nn, n = 3 * nn;
  PcgWork* w = new PcgWork();
  m->pcg = w;
  w->nparts = (int)std::max<int64_t>((nn + kBlock - 1) / kBlock, (32 * nn + kBlock - 1) / kBlock);
  TL_CUDA(m, cudaMalloc(&w->r, sizeof(double) * n));
  TL_CUDA(m, cudaMalloc(&w->z, sizeof(double) * n));
  TL_CUDA(m, cudaMalloc(&w->p, sizeof(double) * n));
  TL_CUDA(m, cudaMalloc(&w->Ap, sizeof(double) * n));
  TL_CUDA(m, cudaMalloc(&w->binv, sizeof(double) * 9 * nn));
  TL_CUDA(m, cudaMalloc(&w->part, sizeof(double) * 2 * w->nparts));
  TL_CUDA(m, cudaMalloc(&w->scal, sizeof(double) * 8));
  TL_CUDA(m, cudaMalloc(&w->diag_k, sizeof(int32_t) * nn));
  TL_CUDA(m, cudaMemsetAsync(w->p, 0, sizeof(double) * n, m->stream));
  TL_CUDA(m, cudaMalloc(&w->tickets, sizeof(unsigned) * 2));
  TL_CUDA(m, cudaMemsetAsync(w->tickets, 0, sizeof(unsigned) * 2, m->stream));
  if (m->precision == TL_FP32_ELEM) {
    TL_CUDA(m, cudaMalloc(&w->p32, sizeof(float) * n));
    TL_CUDA(m, cudaMemsetAsync(w->p32, 0, sizeof(float) * n, m->stream));
    TL_CUDA(m, cudaMalloc(&w->x32, sizeof(float) * n));
    TL_CUDA(m, cudaMalloc(&w->r32, sizeof(float) * n));
    TL_CUDA(m, cudaMalloc(&w->z32, sizeof(float) * n));
    TL_CUDA(m, cudaMalloc(&w->Ap32, sizeof(float) * n));
    TL_CUDA(m, cudaMalloc(&w->binv32, sizeof(float) * 9 * nn));
  }
  node_diag_pos<<<(unsigned)((nn + 255) / 256), 256, 0, m->stream>>>(m->d_node_ptr, m->d_node_col, nn, w->diag_k);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

double* pcg_scalars(tl_mesh* m) { return m->pcg ? m->pcg->scal : nullptr; }

// Block-Jacobi factors of H, x = 0, r = -g, z = P r, p = z, and the scalars
// rz (slot 0) and rr (slot 3); asynchronous.
tl_status pcg_prepare(tl_mesh* m, const void* values, const double* g, double* dv) {
  TL_TRY(pcg_ensure(m));
  PcgWork* w = m->pcg;
  cudaStream_t s = m->stream;
  const int64_t nn = m->nn;
  const unsigned nbn = (unsigned)((nn + kBlock - 1) / kBlock);
  if (m->precision == TL_FP32_ELEM)
    block_jacobi<float><<<nbn, kBlock, 0, s>>>((const float*)values, m->d_node_ptr, w->diag_k, nn, w->binv);
  else
    block_jacobi<double><<<nbn, kBlock, 0, s>>>((const double*)values, m->d_node_ptr, w->diag_k, nn, w->binv);
  double* part_rz = w->part;
  double* part_rr = w->part + w->nparts;
  if (pcg_float32(m)) {
    jacobi_to_f32<<<(unsigned)((9 * nn + kBlock - 1) / kBlock), kBlock, 0, s>>>(w->binv, 9 * nn, w->binv32);
    pcg_start32<<<nbn, kBlock, 0, s>>>(g, w->x32, w->r32, w->z32, w->p32, w->binv32, nn, part_rz, part_rr, w->scal);
    m->launches += 1;
  } else {
    float* p32 = m->precision == TL_FP32_ELEM ? w->p32 : nullptr;
    pcg_start<<<nbn, kBlock, 0, s>>>(g, dv, w->r, w->z, w->p, p32, w->binv, nn, part_rz, part_rr, w->scal);
  }
  finish_sum<<<1, 1024, 0, s>>>(part_rz, nbn, w->scal, 0);
  finish_sum<<<1, 1024, 0, s>>>(part_rr, nbn, w->scal, 3);
  TL_CUDA(m, cudaGetLastError());
  m->launches += 4;
  return TL_OK;
}

template <typename T, int G>
void launch_spmv(tl_mesh* m, const void* values, PcgWork* w, unsigned* nblocks) {
  const int64_t nn = m->nn;
  unsigned nb = (unsigned)((G * nn + kBlock - 1) / kBlock);
  if (std::is_same<T, float>::value && pcg_float32(m) && m->tune.spmv_row) {
    // a grid of at most 8 blocks per SM (one resident wave) and nparts blocks
    nb = (unsigned)std::min(std::min((int64_t)nb, (int64_t)8 * m->num_sms), (int64_t)w->nparts);
    spmv_row32<G><<<nb, kBlock, 0, m->stream>>>((const float*)values, m->d_node_ptr, m->d_node_col, nn, w->p32,
                                                w->Ap32, w->part, w->scal, w->tickets);
  } else if (std::is_same<T, float>::value && pcg_float32(m))
    spmv_node32<G><<<nb, kBlock, 0, m->stream>>>((const float*)values, m->d_node_ptr, m->d_node_col, nn, w->p32,
                                                 w->Ap32, w->part, w->scal, w->tickets);
  else
    spmv_node<T, G><<<nb, kBlock, 0, m->stream>>>((const T*)values, m->d_node_ptr, m->d_node_col, nn, w->p,
                                                  w->p32, w->Ap, w->part, w->scal, w->tickets);
  *nblocks = nb;
}

tl_status pcg_spmv_only(tl_mesh* m, const void* values, int group) {
  TL_TRY(pcg_ensure(m));
  PcgWork* w = m->pcg;
  pcg_clear_target<<<1, 1, 0, m->stream>>>(w->scal);   // the timed product must not return early
  ++m->launches;
  unsigned nbs = 0;
  const bool fp32 = m->precision == TL_FP32_ELEM;
  if (group == 4) fp32 ? launch_spmv<float, 4>(m, values, w, &nbs) : launch_spmv<double, 4>(m, values, w, &nbs);
  else if (group == 16) fp32 ? launch_spmv<float, 16>(m, values, w, &nbs) : launch_spmv<double, 16>(m, values, w, &nbs);
  else if (group == 32) fp32 ? launch_spmv<float, 32>(m, values, w, &nbs) : launch_spmv<double, 32>(m, values, w, &nbs);
  else fp32 ? launch_spmv<float, 8>(m, values, w, &nbs) : launch_spmv<double, 8>(m, values, w, &nbs);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

// `count` PCG iterations (3 launches each); asynchronous, no host reads.
tl_status pcg_iterations(tl_mesh* m, const void* values, double* dv, int count) {
  PcgWork* w = m->pcg;
  cudaStream_t s = m->stream;
  const int64_t nn = m->nn, n = 3 * nn;
  const bool fp32 = m->precision == TL_FP32_ELEM;
  const unsigned nbn = (unsigned)((nn + kBlock - 1) / kBlock);
  const unsigned nbv = (unsigned)((n + kBlock - 1) / kBlock);
  const unsigned nbp = (unsigned)std::min<int64_t>((n / 4 + kBlock - 1) / kBlock + 1, (int64_t)4 * m->num_sms);
  const unsigned nbx = (unsigned)std::min<int64_t>(nbn, (int64_t)2 * m->num_sms);
  const unsigned nbq = (unsigned)std::min<int64_t>(nbv, (int64_t)4 * m->num_sms);
  double* part_rz = w->part;
  double* part_rr = w->part + w->nparts;
  for (int k = 0; k < count; ++k) {
    unsigned nbs = 0;
    const int G = m->tune.spmv_group;
    if (fp32) {
      if (G == 4) launch_spmv<float, 4>(m, values, w, &nbs);
      else if (G == 16) launch_spmv<float, 16>(m, values, w, &nbs);
      else if (G == 32) launch_spmv<float, 32>(m, values, w, &nbs);
      else launch_spmv<float, 8>(m, values, w, &nbs);
    } else {
      if (G == 4) launch_spmv<double, 4>(m, values, w, &nbs);
      else if (G == 16) launch_spmv<double, 16>(m, values, w, &nbs);
      else if (G == 32) launch_spmv<double, 32>(m, values, w, &nbs);
      else launch_spmv<double, 8>(m, values, w, &nbs);
    }
    (void)nbs;
    const int parity = k & 1;            // chunks start at even iterations (count is 8 except the last)
    if (pcg_float32(m)) {
      update_xr32<<<nbx, kBlock, 0, s>>>(w->x32, w->r32, w->z32, w->p32, w->Ap32, w->binv32, w->scal, nn, part_rz,
                                         part_rr, parity, w->tickets + 1);
      update_p32<<<nbp, kBlock, 0, s>>>(w->p32, w->z32, n, w->scal, parity);
    } else {
      update_xr<<<nbx, kBlock, 0, s>>>(dv, w->r, w->z, w->p, w->Ap, w->binv, w->scal, nn, part_rz, part_rr,
                                       parity, w->tickets + 1);
      update_p<<<nbq, kBlock, 0, s>>>(w->p, fp32 ? w->p32 : nullptr, w->z, n, w->scal, parity);
    }
    m->launches += 3;
  }
  TL_CUDA(m, cudaGetLastError());
  return TL_OK;
}

// Solve H dv = -g to ||r|| <= rtol ||g|| (host-driven: the residual norm is
// read every kCheck iterations).  values in assembly CSR order.
tl_status pcg_solve(tl_mesh* m, const void* values, const double* g, double* dv, double rtol, int max_iter,
                    int* iters_out) {
  cudaStream_t s = m->stream;
  TL_TRY(pcg_prepare(m, values, g, dv));
  PcgWork* w = m->pcg;
  double rr0 = 0.0;
  TL_CUDA(m, cudaMemcpyAsync(&rr0, w->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
  TL_CUDA(m, cudaStreamSynchronize(s));
  const double tol2 = rtol * rtol * rr0;
  // the target in slot 5: iterations of a chunk after it is reached return at once
  TL_CUDA(m, cudaMemcpyAsync(w->scal + 5, &tol2, sizeof(double), cudaMemcpyHostToDevice, s));
  int it = 0, run = 0;
  while (it < max_iter && rr0 > tol2) {
    const int k = std::min(kCheck, max_iter - it);
    TL_TRY(pcg_iterations(m, values, dv, k));
    it += k;
    double sc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // slots 3..7
    TL_CUDA(m, cudaMemcpyAsync(sc, w->scal + 3, sizeof(sc), cudaMemcpyDeviceToHost, s));
    TL_CUDA(m, cudaStreamSynchronize(s));
    const double rr = sc[0];
    run = (int)sc[4];
    if (!std::isfinite(rr)) return fail(m, TL_ERR_NONFINITE, "PCG residual not finite");
    if (rr <= tol2 || sc[3] != 0.0) break;
  }
  TL_TRY(pcg_result(m, dv));
  if (iters_out) *iters_out = run;
  return TL_OK;
}

// dv from the float32 iterate (no-op for the float64 iteration, which updates dv in place).
tl_status pcg_result(tl_mesh* m, double* dv) {
  if (!pcg_float32(m)) return TL_OK;
  const int64_t n = 3 * m->nn;
  widen<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, m->stream>>>(m->pcg->x32, n, dv);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

}  // namespace tl
