// Residual of the velocity-level augmented Lagrangian and the clamp-row
// contributions to the Newton matrix.
//
// Paper: arxiv 2604.10357
//   eq. residual / eq. grad_L:  g = M (v - v_n)/h + f_int - f_ext - f_ff
//                                   + h C_q^T (lambda + rho c)
//   Sec. 4.4 (gradient): one thread per coefficient row of M, no atomics;
//   eq. hessian: the h^2 rho C_q^T C_q term (identity rows for clamps).
//
// One thread (or a group of lanes) per node handles its three DOFs (the mass
// CSR row is shared by the three components); ||g||^2 is reduced per block
// into a partials array and summed by a second one-block kernel, so the norm
// is deterministic.
#include <mutex>

#include <cub/device/device_scan.cuh>

#include "tl_internal.cuh"

namespace tl {
namespace {

constexpr int kResBlock = 256;

// General constraints in the residual: g_r += h sum_c C_cr (lambda_c + rho c_c)
// over the constraints c of DOF r (C^T by DOF; w = lambda + rho c, formed
// first).  ptr == nullptr: no general constraints.
struct ConTerm {
  const int32_t* ptr;
  const int32_t* con;
  const double* val;
  const double* w;
};

__device__ __forceinline__ double con_term(const ConTerm& ct, int64_t r) {
  double t = 0.0;
  for (int32_t k = ct.ptr[r]; k < ct.ptr[r + 1]; ++k) t += ct.val[k] * ct.w[ct.con[k]];
  return t;
}

// w_c = lambda_c + rho c_c(q_n + h v), c_c = sum_k C_ck q_k - b_c (one thread per row)
__global__ void con_eval(const int32_t* cptr, const int32_t* ccol, const double* cval, const double* b, int64_t ncon,
                         const double* q_n, const double* v, double h, const double* lambda, double rho, double* w) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncon) return;
  double s = -b[c];
  for (int32_t k = cptr[c]; k < cptr[c + 1]; ++k) {
    const int32_t i = ccol[k];
    s += cval[k] * (q_n[i] + h * v[i]);
  }
  w[c] = (lambda ? lambda[c] : 0.0) + rho * s;
}

// lambda_c += rho c_c when the flag says so; ||c||^2 into *sq (one block)
__global__ void con_update(const int32_t* cptr, const int32_t* ccol, const double* cval, const double* b,
                           int64_t ncon, const double* q_n, const double* v, double h, double rho, int update,
                           const int32_t* update_flag, double* lambda, double* sq) {
  __shared__ double red[32];
  if (update_flag) update = *update_flag;
  double t = 0.0;
  for (int64_t c = threadIdx.x; c < ncon; c += blockDim.x) {
    double s = -b[c];
    for (int32_t k = cptr[c]; k < cptr[c + 1]; ++k) {
      const int32_t i = ccol[k];
      s += cval[k] * (q_n[i] + h * v[i]);
    }
    t += s * s;
    if (update) lambda[c] += rho * s;
  }
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    double u = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (threadIdx.x == 0) *sq = u;
  }
}

// h^2 rho C^T C into the CSR values: one thread per constraint row, every pair
// of its entries, the position of (i, j) by binary search in node I's sorted
// neighbour list (the pattern holds every coupled pair, Sec. 4.2)
template <typename T>
__global__ void con_penalty(const int32_t* cptr, const int32_t* ccol, const double* cval, int64_t ncon,
                            const int32_t* node_ptr, const int32_t* node_col, double value, T* values,
                            uint32_t* flags) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncon) return;
  for (int32_t a = cptr[c]; a < cptr[c + 1]; ++a) {
    const int32_t i = ccol[a], I = i / 3, d = i % 3;
    const int32_t p0 = node_ptr[I], deg = node_ptr[I + 1] - p0;
    for (int32_t bb = cptr[c]; bb < cptr[c + 1]; ++bb) {
      const int32_t j = ccol[bb], J = j / 3, e = j % 3;
      int lo = 0, hi = deg - 1, pos = -1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t x = node_col[p0 + mid];
        if (x == J) {
          pos = mid;
          break;
        }
        if (x < J) lo = mid + 1; else hi = mid - 1;
      }
      if (pos < 0) {
        atomicOr(flags, kFlagBadIndex);
        continue;
      }
      atomicAdd(&values[9 * (int64_t)p0 + 3 * (int64_t)deg * d + 3 * pos + e], T(value * cval[a] * cval[bb]));
    }
  }
}

// Scratch of the allocation-free residual (tl_eval_residual_noalloc): one
// partial sum of ||g||^2 per block of kResBlock nodes.  It lives in the
// library image, so every GPU that loads the library holds these 128 KiB until
// the process exits.  Every call overwrites the entries it uses before reading
// them, so nothing has to be cleared between calls.
constexpr int kNoAllocMaxBlocks = 16384;                    // nn <= 4,194,304
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks];

// LANES lanes per node: lane l sums the mass row entries l, l + LANES, ...
// (rows have ~28 entries), the group combines the three sums and its first
// lane forms the node's three residual components.  A block holds kResBlock
// nodes, so the partial count does not depend on LANES.  dv = v - v_n is read
// precomputed when given (one subtraction per DOF instead of one per mass
// entry: on GB300 the float64 subtractions and multiply-adds bound this
// kernel), else formed inline.
template <int LANES, bool CON>
__global__ void __launch_bounds__(kResBlock * LANES)
    residual_kernel(const int32_t* node_ptr, const int32_t* node_col, const double* mass, const double* mrow,
                    const int32_t* fixed_of_node, const double* X, int64_t nn, double h, double inv_h, double rho,
                    double gx,
                    double gy, double gz, const double* q_n, const double* v_n, const double* v, const double* dv,
                    const double* f_int, const double* f_ext, const double* lambda, double* g,
                    double* partials, ConTerm ct) {
  __shared__ double red[kResBlock * LANES / 32];
  const int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LANES;
  const int l = threadIdx.x & (LANES - 1);
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, sq = 0.0;
  if (I < nn) {
    const int p0 = node_ptr[I], p1 = node_ptr[I + 1];
    if (dv) {
      for (int p = p0 + l; p < p1; p += LANES) {
        const int64_t J = node_col[p];
        const double mij = mass[p];
        acc0 += mij * dv[3 * J];
        acc1 += mij * dv[3 * J + 1];
        acc2 += mij * dv[3 * J + 2];
      }
    } else {
      for (int p = p0 + l; p < p1; p += LANES) {
        const int64_t J = node_col[p];
        const double mij = mass[p];
        acc0 += mij * (v[3 * J] - v_n[3 * J]);
        acc1 += mij * (v[3 * J + 1] - v_n[3 * J + 1]);
        acc2 += mij * (v[3 * J + 2] - v_n[3 * J + 2]);
      }
    }
  }
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) {
    acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
    acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
    acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
  }
  if (I < nn && l == 0) {
    const double acc[3] = {acc0, acc1, acc2};
    const double grav[3] = {gx, gy, gz};
    const int j = fixed_of_node[I];
    const double mr = mrow[I];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int64_t r = 3 * I + d;
      double gd = acc[d] * inv_h + f_int[r] - mr * grav[d];
      if (f_ext) gd -= f_ext[r];
      if (j >= 0) {
        const double c = (q_n[r] + h * v[r]) - X[r];
        gd += h * ((lambda ? lambda[3 * j + d] : 0.0) + rho * c);
      }
      if (CON) gd += h * con_term(ct, r);
      g[r] = gd;
      sq += gd * gd;
    }
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

__global__ void velocity_change(const double* v, const double* v_n, int64_t n, double* dv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dv[i] = v[i] - v_n[i];
}

// ---------------------------------------------------------------------------
// Mass product in double-float arithmetic.  GB300 runs float64 arithmetic at
// 1/64 of the float32 rate, and the float64 multiply-adds of the mass product
// bound the residual kernel above.  Here every float64 operand x is held as
// an unevaluated float32 pair x = x.hi + x.lo (|x.lo| <= ulp(x.hi) / 2, 48
// significant bits), and the row sum of m_IJ dv_J runs in float32 with
// error-free transformations (Dekker's product via FMA, Knuth's two-sum):
//   p = a.hi b.hi exactly as p.hi + p.e (p.e = fma(a.hi, b.hi, -p.hi)),
//   plus the cross terms a.hi b.lo + a.lo b.hi (a.lo b.lo ~ 2^-48 dropped);
//   s = s + p with the rounding error of the high part kept exactly.
// The sum is accurate to a few units of 2^-48 relative to the largest terms
// (float64: 2^-53); it is converted to float64 once per node, and the rest of
// the residual stays float64.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 split_f64(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(__dsub_rn(x, (double)hi)));
}

// The _rn intrinsics are never contracted into FMAs, which the error-free
// transformations rely on.
__device__ __forceinline__ void df_mac(float& s_hi, float& s_lo, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);                      // exact error of the high product
  e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e));        // cross terms
  const float s = __fadd_rn(s_hi, p);                     // two-sum of s_hi and p
  const float bb = __fsub_rn(s, s_hi);
  const float err = __fadd_rn(__fsub_rn(s_hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  s_hi = s;
  s_lo = __fadd_rn(s_lo, __fadd_rn(err, e));
}

__global__ void split_array(const double* x, int64_t n, float2* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = split_f64(x[i]);
}

__global__ void velocity_change_split(const double* v, const double* v_n, int64_t n, float2* dv) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dv[i] = split_f64(v[i] - v_n[i]);
}

// (s_hi, s_lo) += (o_hi, o_lo): two-sum of the high parts, low parts added.
__device__ __forceinline__ void df_combine(float& s_hi, float& s_lo, float o_hi, float o_lo) {
  const float s = __fadd_rn(s_hi, o_hi);
  const float bb = __fsub_rn(s, s_hi);
  const float err = __fadd_rn(__fsub_rn(s_hi, __fsub_rn(s, bb)), __fsub_rn(o_hi, bb));
  s_hi = s;
  s_lo = __fadd_rn(s_lo, __fadd_rn(err, o_lo));
}

// The rest of node I's residual once its mass product acc = (M dv)_I is
// formed: force, gravity, external force, clamp and general-constraint
// terms; g written, its squared norm returned.
template <bool CON>
__device__ __forceinline__ double node_rest(int64_t I, const double (&acc)[3], const double* mrow,
                                            const int32_t* fixed_of_node, const double* X, double h, double inv_h,
                                            double rho, double gx, double gy, double gz, const double* q_n,
                                            const double* v, const double* f_int, const double* f_ext,
                                            const double* lambda, double* g, const ConTerm& ct) {
  const double grav[3] = {gx, gy, gz};
  const int j = fixed_of_node[I];
  const double mr = mrow[I];
  double sq = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t r = 3 * I + d;
    double gd = acc[d] * inv_h + f_int[r] - mr * grav[d];
    if (f_ext) gd -= f_ext[r];
    if (j >= 0) {
      const double c = (q_n[r] + h * v[r]) - X[r];
      gd += h * ((lambda ? lambda[3 * j + d] : 0.0) + rho * c);
    }
    if (CON) gd += h * con_term(ct, r);
    g[r] = gd;
    sq += gd * gd;
  }
  return sq;
}

// The block's sum of sq into partials[blockIdx.x] (every thread calls it).
__device__ __forceinline__ void block_partial(double sq, double* red, double* partials) {
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

// LANES lanes per node: lane l takes the mass-row entries l, l + LANES, ...;
// the lanes' double-float sums are combined by shuffles (two-sums of the high
// parts) and the first lane forms the node's residual.  A block holds
// kResBlock nodes.
template <int LANES, bool CON>
__global__ void __launch_bounds__(kResBlock * LANES)
    residual_split_kernel(const int32_t* node_ptr, const int32_t* node_col, const float2* mass2, const double* mrow,
                          const int32_t* fixed_of_node, const double* X, int64_t nn, double h, double inv_h,
                          double rho, double gx, double gy, double gz, const double* q_n, const double* v,
                          const float2* dv2, const double* f_int, const double* f_ext, const double* lambda,
                          double* g, double* partials, ConTerm ct) {
  __shared__ double red[kResBlock * LANES / 32];
  const int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LANES;
  const int l = threadIdx.x & (LANES - 1);
  double sq = 0.0;
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
  if (I < nn) {
    const int p0 = node_ptr[I], p1 = node_ptr[I + 1];
    for (int p = p0 + l; p < p1; p += LANES) {
      const int64_t J = node_col[p];
      const float2 mij = mass2[p];
      df_mac(h0, l0, mij, dv2[3 * J]);
      df_mac(h1, l1, mij, dv2[3 * J + 1]);
      df_mac(h2, l2, mij, dv2[3 * J + 2]);
    }
  }
#pragma unroll
  for (int o = LANES / 2; o > 0; o >>= 1) {
    const float a0 = __shfl_xor_sync(0xffffffffu, h0, o), b0 = __shfl_xor_sync(0xffffffffu, l0, o);
    const float a1 = __shfl_xor_sync(0xffffffffu, h1, o), b1 = __shfl_xor_sync(0xffffffffu, l1, o);
    const float a2 = __shfl_xor_sync(0xffffffffu, h2, o), b2 = __shfl_xor_sync(0xffffffffu, l2, o);
    df_combine(h0, l0, a0, b0);
    df_combine(h1, l1, a1, b1);
    df_combine(h2, l2, a2, b2);
  }
  if (I < nn && l == 0) {
    const double acc[3] = {(double)h0 + (double)l0, (double)h1 + (double)l1, (double)h2 + (double)l2};
    sq = node_rest<CON>(I, acc, mrow, fixed_of_node, X, h, inv_h, rho, gx, gy, gz, q_n, v, f_int, f_ext, lambda, g,
                        ct);
  }
  block_partial(sq, red, partials);
}

// Sliced ELL copy of the float32-pair mass rows (pattern build, once):
// slices of kSellC = 32 rows, the rows of every window of kSellWin = 256
// rows ordered by length, longest first (a stable sort, so equal lengths keep
// node order), so the 32 rows of a slice have (nearly) one length; entry k
// of the row at lane l of slice s sits at ptr[s] + 32 k + l, padded to the
// slice's longest row with the row's own node and zero mass.  A warp then
// reads entry k of its 32 rows as one contiguous run, where one thread per
// CSR row touched 32 separate rows per load (the row-per-thread kernel was
// bound by L1 wavefronts).
constexpr int kSellC = 32, kSellWin = 256;
// Row entries per round of the residual loop: two, measured on the 960k box
// against one, three, four and eight (0.213 ms per residual pass against
// 0.268, 0.258, 0.263 and 0.266 ms; more loads in flight per warp did not pay
// beyond two).
constexpr int kSellU = 2;
static_assert(kResBlock == kSellWin, "one sorting window per residual block");

__global__ void __launch_bounds__(kSellWin) sell_order(const int32_t* node_ptr, int64_t nn, int32_t* row_of) {
  __shared__ uint32_t key[kSellWin];
  const int64_t w0 = blockIdx.x * (int64_t)kSellWin;
  const int i = threadIdx.x;
  uint32_t k = 0xffffffffu;
  if (w0 + i < nn) {
    const int len = min(node_ptr[w0 + i + 1] - node_ptr[w0 + i], 0xffff);
    k = ((uint32_t)(0xffff - len) << 16) | (uint32_t)i;
  }
  key[i] = k;
  __syncthreads();
  for (int size = 2; size <= kSellWin; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int j = i ^ stride;
      if (j > i) {
        const bool up = (i & size) == 0;
        const uint32_t a = key[i], c = key[j];
        if ((a > c) == up) {
          key[i] = c;
          key[j] = a;
        }
      }
      __syncthreads();
    }
  row_of[w0 + i] = key[i] == 0xffffffffu ? -1 : (int32_t)(w0 + (key[i] & 0xffffu));
}

// cnt[s] = 32 x the longest row of slice s; cnt[nslices] = 0.
__global__ void sell_len(const int32_t* node_ptr, const int32_t* row_of, int64_t nslices, int64_t* cnt) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s > nslices) return;
  int64_t L = 0;
  if (s < nslices)
    for (int r = 0; r < kSellC; ++r) {
      const int32_t I = row_of[s * kSellC + r];
      if (I >= 0) L = max(L, (int64_t)(node_ptr[I + 1] - node_ptr[I]));
    }
  cnt[s] = L * kSellC;
}

__global__ void sell_fill(const int32_t* node_ptr, const int32_t* node_col, const float2* mass2, const int32_t* row_of,
                          const int64_t* ptr, int64_t nslices, int32_t* col, float2* mv) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nslices * kSellC) return;
  const int64_t s = t / kSellC, b = ptr[s], L = (ptr[s + 1] - b) / kSellC;
  const int32_t I = row_of[t];
  int32_t p0 = 0, len = 0;
  if (I >= 0) {
    p0 = node_ptr[I];
    len = node_ptr[I + 1] - p0;
  }
  for (int64_t k = 0; k < L; ++k) {
    const int64_t idx = b + k * kSellC + (t % kSellC);
    const bool real = k < len;
    col[idx] = real ? node_col[p0 + k] : (I >= 0 ? I : 0);
    mv[idx] = real ? mass2[p0 + k] : make_float2(0.0f, 0.0f);
  }
}

// The double-float residual over the sliced ELL rows: thread t -> the row at
// lane t % 32 of slice t / 32 (a block = one sorting window of 256 rows),
// the same arithmetic per entry as residual_split_kernel<1>.
template <bool CON>
__global__ void __launch_bounds__(kResBlock)
    residual_sell_kernel(const int32_t* __restrict__ row_of, const int64_t* __restrict__ ptr,
                         const int32_t* __restrict__ scol, const float2* __restrict__ smass,
                         const double* mrow, const int32_t* fixed_of_node, const double* X, double h, double inv_h,
                         double rho, double gx, double gy, double gz, const double* q_n, const double* v,
                         const float2* __restrict__ dv2, const double* f_int, const double* f_ext,
                         const double* lambda, double* g, double* partials, ConTerm ct) {
  __shared__ double red[kResBlock / 32];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // the grid covers the slices exactly
  const int64_t I = row_of[t];
  double sq = 0.0;
  if (I >= 0) {
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    const int64_t b = ptr[t / kSellC] + (t % kSellC);
    const int L = (int)((ptr[t / kSellC + 1] - ptr[t / kSellC]) / kSellC);   // warp-uniform
    const int32_t* cp = scol + b;
    const float2* mp = smass + b;
    // kSellU entries per round: their columns and masses, then the 3 kSellU
    // gathers of dv, then the arithmetic, so that many loads are in flight
    // (one entry per round left the kernel waiting on each dependent load)
    int k = 0;
    for (; k + kSellU <= L; k += kSellU) {
      int32_t J[kSellU];
      float2 mij[kSellU], d[kSellU][3];
#pragma unroll
      for (int u = 0; u < kSellU; ++u) {
        J[u] = cp[(int64_t)(k + u) * kSellC];
        mij[u] = mp[(int64_t)(k + u) * kSellC];
      }
#pragma unroll
      for (int u = 0; u < kSellU; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[u][c] = dv2[3 * (int64_t)J[u] + c];
#pragma unroll
      for (int u = 0; u < kSellU; ++u) {
        df_mac(h0, l0, mij[u], d[u][0]);
        df_mac(h1, l1, mij[u], d[u][1]);
        df_mac(h2, l2, mij[u], d[u][2]);
      }
    }
    for (; k < L; ++k) {
      const int64_t J = cp[(int64_t)k * kSellC];
      const float2 mij = mp[(int64_t)k * kSellC];
      df_mac(h0, l0, mij, dv2[3 * J]);
      df_mac(h1, l1, mij, dv2[3 * J + 1]);
      df_mac(h2, l2, mij, dv2[3 * J + 2]);
    }
    const double acc[3] = {(double)h0 + (double)l0, (double)h1 + (double)l1, (double)h2 + (double)l2};
    sq = node_rest<CON>(I, acc, mrow, fixed_of_node, X, h, inv_h, rho, gx, gy, gz, q_n, v, f_int, f_ext, lambda, g,
                        ct);
  }
  block_partial(sq, red, partials);
}

__global__ void finish_norm(const double* partials, int n, double* out, uint32_t* flags) {
  __shared__ double red[32];
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += partials[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x < 32) {
    double u = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (threadIdx.x == 0) {
      if (!isfinite(u)) atomicOr(flags, kFlagNonFinite);
      *out = sqrt(u);
    }
  }
}

template <typename T>
__global__ void add_diag(const int32_t* diag, int64_t n, T value, T* values) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) values[diag[t]] += value;
}

}  // namespace

namespace {

// w = lambda + rho c for the general constraint rows (their multipliers follow
// the 3 nfixed clamp multipliers in lambda) and the C^T term of the residual.
tl_status con_prepare(tl_mesh* m, const tl_params* p, const double* q_n, const double* v, const double* lambda,
                      ConTerm* ct) {
  *ct = ConTerm{nullptr, nullptr, nullptr, nullptr};
  if (m->ncon == 0) return TL_OK;
  con_eval<<<(unsigned)((m->ncon + 255) / 256), 256, 0, m->stream>>>(
      m->d_con_ptr, m->d_con_col, m->d_con_val, m->d_con_b, m->ncon, q_n, v, p->h,
      lambda ? lambda + 3 * m->nfixed : nullptr, p->rho_alm, m->d_con_w);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  *ct = ConTerm{m->d_ct_ptr, m->d_ct_con, m->d_ct_val, m->d_con_w};
  return TL_OK;
}

}  // namespace

tl_status launch_con_update(tl_mesh* m, const double* q_n, const double* v, double h, double rho, int update,
                            const int32_t* update_flag, double* lambda_general) {
  if (m->ncon == 0) return TL_OK;
  con_update<<<1, 1024, 0, m->stream>>>(m->d_con_ptr, m->d_con_col, m->d_con_val, m->d_con_b, m->ncon, q_n, v, h,
                                        rho, update, update_flag, lambda_general, m->d_con_sq);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

tl_status mass_sell_build(tl_mesh* m, cudaStream_t s);

// float32 pairs of the node-level mass (double-float mass product); once per
// handle, after the mass is assembled, and their sliced ELL copy.
tl_status mass_split_build(tl_mesh* m, cudaStream_t s) {
  const int64_t n = std::max<int64_t>(m->nnz_node, 1);
  if (!m->d_mass2) TL_CUDA(m, cudaMalloc(&m->d_mass2, sizeof(float2) * n));
  split_array<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->d_mass, n, m->d_mass2);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return mass_sell_build(m, s);
}

// The sliced ELL copy of d_mass2 (pattern build, after mass_split_build).
tl_status mass_sell_build(tl_mesh* m, cudaStream_t s) {
  for (void* p : {(void*)m->d_sell_row, (void*)m->d_sell_ptr, (void*)m->d_sell_col, (void*)m->d_sell_m})
    if (p) cudaFree(p);
  m->d_sell_row = nullptr;
  m->d_sell_ptr = nullptr;
  m->d_sell_col = nullptr;
  m->d_sell_m = nullptr;
  if (m->nn == 0) return TL_OK;
  const int64_t nwin = (m->nn + kSellWin - 1) / kSellWin, nslices = nwin * (kSellWin / kSellC);
  int64_t* d_cnt = nullptr;
  void* d_tmp = nullptr;
  size_t tmp_bytes = 0;
  int64_t total = 0;
  tl_status st = TL_OK;
  auto chk = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == TL_OK) st = cuda_fail(m, e, what);
    return st == TL_OK;
  };
  if (chk(cudaMalloc(&m->d_sell_row, sizeof(int32_t) * nslices * kSellC), "cudaMalloc(sell_row)") &&
      chk(cudaMalloc(&m->d_sell_ptr, sizeof(int64_t) * (nslices + 1)), "cudaMalloc(sell_ptr)") &&
      chk(cudaMalloc(&d_cnt, sizeof(int64_t) * (nslices + 1)), "cudaMalloc(sell counts)")) {
    sell_order<<<(unsigned)nwin, kSellWin, 0, s>>>(m->d_node_ptr, m->nn, m->d_sell_row);
    sell_len<<<(unsigned)((nslices + 1 + 255) / 256), 256, 0, s>>>(m->d_node_ptr, m->d_sell_row, nslices, d_cnt);
    if (chk(cudaGetLastError(), "sell_order / sell_len") &&
        chk(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, d_cnt, m->d_sell_ptr, (int)(nslices + 1), s),
            "cub scan size") &&
        chk(cudaMalloc(&d_tmp, std::max<size_t>(tmp_bytes, 1)), "cudaMalloc(scan scratch)") &&
        chk(cub::DeviceScan::ExclusiveSum(d_tmp, tmp_bytes, d_cnt, m->d_sell_ptr, (int)(nslices + 1), s),
            "cub scan") &&
        chk(cudaMemcpyAsync(&total, m->d_sell_ptr + nslices, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
            "sell total") &&
        chk(cudaStreamSynchronize(s), "sell total sync") &&
        chk(cudaMalloc(&m->d_sell_col, sizeof(int32_t) * std::max<int64_t>(total, 1)), "cudaMalloc(sell_col)") &&
        chk(cudaMalloc(&m->d_sell_m, sizeof(float2) * std::max<int64_t>(total, 1)), "cudaMalloc(sell_m)")) {
      sell_fill<<<(unsigned)((nslices * kSellC + 255) / 256), 256, 0, s>>>(
          m->d_node_ptr, m->d_node_col, m->d_mass2, m->d_sell_row, m->d_sell_ptr, nslices, m->d_sell_col,
          m->d_sell_m);
      chk(cudaGetLastError(), "sell_fill");
      m->launches += 4;
    }
  }
  if (d_cnt) cudaFree(d_cnt);
  if (d_tmp) cudaFree(d_tmp);
  return st;
}

// Norm partials owned by the handle (one per block of kResBlock nodes).
tl_status residual_ensure(tl_mesh* m) {
  if (!m->d_dv) TL_CUDA(m, cudaMalloc(&m->d_dv, sizeof(double) * 3 * m->nn));
  if (!m->d_dv2) TL_CUDA(m, cudaMalloc(&m->d_dv2, sizeof(float2) * 3 * m->nn));
  const int nb = (int)((m->nn + kResBlock - 1) / kResBlock);
  if (nb > m->partials_cap) {
    if (m->d_partials) cudaFree(m->d_partials);
    m->d_partials = nullptr;
    m->partials_cap = 0;
    TL_CUDA(m, cudaMalloc(&m->d_partials, sizeof(double) * nb));
    m->partials_cap = nb;
  }
  return TL_OK;
}

tl_status launch_residual(tl_mesh* m, const tl_params* p, const double* q_n, const double* v_n, const double* v,
                          const double* f_int, const double* f_ext, const double* lambda, double* g,
                          double* g_norm) {
  const int nb = (int)((m->nn + kResBlock - 1) / kResBlock);
  TL_TRY(residual_ensure(m));
  cudaEvent_t t0 = timer_open(m);
  // f_int may alias g: each thread reads its own entries before writing them
  const int64_t n3 = 3 * m->nn;
  ConTerm ct;
  TL_TRY(con_prepare(m, p, q_n, v, lambda, &ct));
  if (m->tune.residual_split && m->d_mass2) {
    velocity_change_split<<<(unsigned)((n3 + 255) / 256), 256, 0, m->stream>>>(v, v_n, n3, m->d_dv2);
    if (m->tune.residual_lanes == 4)
      (ct.ptr ? residual_split_kernel<4, true> : residual_split_kernel<4, false>)<<<nb, kResBlock * 4, 0, m->stream>>>(
          m->d_node_ptr, m->d_node_col, m->d_mass2, m->d_mrow, m->d_fixed_of_node, m->d_X, m->nn, p->h, 1.0 / p->h,
          p->rho_alm, p->gravity[0], p->gravity[1], p->gravity[2], q_n, v, m->d_dv2, f_int, f_ext, lambda, g,
          m->d_partials, ct);
    else if (m->d_sell_m)   // one lane per row, rows in sliced ELL (nb blocks = the slices' windows)
      (ct.ptr ? residual_sell_kernel<true> : residual_sell_kernel<false>)<<<nb, kResBlock, 0, m->stream>>>(
          m->d_sell_row, m->d_sell_ptr, m->d_sell_col, m->d_sell_m, m->d_mrow, m->d_fixed_of_node, m->d_X, p->h,
          1.0 / p->h, p->rho_alm, p->gravity[0], p->gravity[1], p->gravity[2], q_n, v, m->d_dv2, f_int, f_ext,
          lambda, g, m->d_partials, ct);
    else
      (ct.ptr ? residual_split_kernel<1, true> : residual_split_kernel<1, false>)<<<nb, kResBlock, 0, m->stream>>>(
          m->d_node_ptr, m->d_node_col, m->d_mass2, m->d_mrow, m->d_fixed_of_node, m->d_X, m->nn, p->h, 1.0 / p->h,
          p->rho_alm, p->gravity[0], p->gravity[1], p->gravity[2], q_n, v, m->d_dv2, f_int, f_ext, lambda, g,
          m->d_partials, ct);
  } else {
  velocity_change<<<(unsigned)((n3 + 255) / 256), 256, 0, m->stream>>>(v, v_n, n3, m->d_dv);
  if (m->tune.residual_lanes == 4)
    (ct.ptr ? residual_kernel<4, true> : residual_kernel<4, false>)<<<nb, kResBlock * 4, 0, m->stream>>>(
        m->d_node_ptr, m->d_node_col, m->d_mass, m->d_mrow, m->d_fixed_of_node, m->d_X, m->nn, p->h, 1.0 / p->h, p->rho_alm,
        p->gravity[0], p->gravity[1], p->gravity[2], q_n, v_n, v, m->d_dv, f_int, f_ext, lambda, g, m->d_partials, ct);
  else
    (ct.ptr ? residual_kernel<1, true> : residual_kernel<1, false>)<<<nb, kResBlock, 0, m->stream>>>(
        m->d_node_ptr, m->d_node_col, m->d_mass, m->d_mrow, m->d_fixed_of_node, m->d_X, m->nn, p->h, 1.0 / p->h, p->rho_alm,
        p->gravity[0], p->gravity[1], p->gravity[2], q_n, v_n, v, m->d_dv, f_int, f_ext, lambda, g, m->d_partials, ct);
  }
  TL_CUDA(m, cudaGetLastError());
  finish_norm<<<1, 1024, 0, m->stream>>>(m->d_partials, nb, g_norm, m->d_flags);
  TL_CUDA(m, cudaGetLastError());
  m->launches += 3;
  timer_close(m, t0, kTimeResidual);
  return TL_OK;
}

namespace {

// Device address of g_noalloc_partials, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

tl_status noalloc_scratch(tl_mesh* m, int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(m, TL_ERR_UNSUPPORTED, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
    if (e != cudaSuccess || !ptr) return cuda_fail(m, e, "cudaGetSymbolAddress(g_noalloc_partials)");
    g_noalloc_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = g_noalloc_ptr[dev];
  return TL_OK;
}

}  // namespace

tl_status launch_add_penalty(tl_mesh* m, double value, void* values) {
  const int64_t n = 3 * m->nfixed;
  if (n > 0) {
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (m->precision == TL_FP32_ELEM)
      add_diag<float><<<nb, 256, 0, m->stream>>>(m->d_fixed_diag, n, (float)value, (float*)values);
    else
      add_diag<double><<<nb, 256, 0, m->stream>>>(m->d_fixed_diag, n, value, (double*)values);
    TL_CUDA(m, cudaGetLastError());
    ++m->launches;
  }
  if (m->ncon > 0) {    // h^2 rho C^T C of the general rows
    const unsigned nb = (unsigned)((m->ncon + 127) / 128);
    if (m->precision == TL_FP32_ELEM)
      con_penalty<float><<<nb, 128, 0, m->stream>>>(m->d_con_ptr, m->d_con_col, m->d_con_val, m->ncon,
                                                    m->d_node_ptr, m->d_node_col, value, (float*)values,
                                                    m->d_flags);
    else
      con_penalty<double><<<nb, 128, 0, m->stream>>>(m->d_con_ptr, m->d_con_col, m->d_con_val, m->ncon,
                                                     m->d_node_ptr, m->d_node_col, value, (double*)values,
                                                     m->d_flags);
    TL_CUDA(m, cudaGetLastError());
    ++m->launches;
  }
  return TL_OK;
}

}  // namespace tl

extern "C" tl_status tl_eval_residual_noalloc(tl_mesh* m, const tl_params* p, const double* q_n,
                                              const double* v_n, const double* v, const double* f_int,
                                              const double* f_ext, const double* lambda, double* g,
                                              double* g_norm) {
  using namespace tl;
  if (!m || !p || !q_n || !v_n || !v || !f_int || !g || !g_norm || !(p->h > 0.0)) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  const int64_t nb = (m->nn + kResBlock - 1) / kResBlock;
  if (nb > kNoAllocMaxBlocks)
    return fail(m, TL_ERR_UNSUPPORTED,
                "tl_eval_residual_noalloc handles at most 4,194,304 nodes; this mesh has " + std::to_string(m->nn));
  int dev = -1;
  TL_CUDA(m, cudaGetDevice(&dev));
  if (dev != m->device) return fail(m, TL_ERR_INVALID_ARG, "the mesh's device must be current");
  double* partials = nullptr;
  tl_status s = noalloc_scratch(m, dev, &partials);
  if (s != TL_OK) return s;
  ConTerm ct;
  TL_TRY(con_prepare(m, p, q_n, v, lambda, &ct));
  (ct.ptr ? residual_kernel<1, true> : residual_kernel<1, false>)<<<(unsigned)nb, kResBlock, 0, m->stream>>>(
      m->d_node_ptr, m->d_node_col, m->d_mass, m->d_mrow, m->d_fixed_of_node, m->d_X, m->nn, p->h, 1.0 / p->h, p->rho_alm,
      p->gravity[0], p->gravity[1], p->gravity[2], q_n, v_n, v, nullptr, f_int, f_ext, lambda, g, partials, ct);
  TL_CUDA(m, cudaGetLastError());
  finish_norm<<<1, 1024, 0, m->stream>>>(partials, (int)nb, g_norm, m->d_flags);
  TL_CUDA(m, cudaGetLastError());
  m->launches += 2;
  return TL_OK;
}
