// Learned Newton warm start: a per-node MLP 10 -> 64 -> 64 -> 64 -> 3 (tanh
// hidden layers) with bfloat16 weights and activations and float32
// accumulation, its forward and backward passes, the MSE loss gradient and
// the Adam update, all as device kernels.  The paper has no counterpart (it
// starts Newton from v_n, Algorithm 3); the network predicts the start
// v0 = b + s_out r_I MLP(features) on free nodes, where b is the polynomial
// extrapolation of the velocity history (Newton's backward-difference form
// v_n + nabla v_n + nabla^2 v_n + nabla^3 v_n: cubic from v_n .. v_{n-3}, lower
// order when fewer previous velocities are given): a learned correction of
// it.  Inputs: the three backward differences, each over its own scale, the
// nine divided by their norm r_I (the map then does not depend on the
// amplitude of the motion), and the fixed flag.
//
// Layout of the bf16 parameter vector (9219 entries): W1 (64x10), b1 (64),
// W2 (64x64), b2 (64), W3 (64x64), b3 (64), W4 (3x64), b4 (3).
// One thread per sample (node); a block of 128 samples keeps the weights in
// shared memory as float32 and each sample's activation vectors in
// sample-minor shared arrays (conflict-free column access).  Weight gradients
// are reduced over the block's samples in shared memory and added to the
// global gradient once per block.
#include <cuda_bf16.h>

#include <algorithm>

#include "tl_internal.cuh"

namespace tl {
namespace {

constexpr int kS = 128;         // samples per block
constexpr int kLd = kS + 1;     // padded stride of the per-sample columns
constexpr int kNP = 9219;
constexpr int oW1 = 0, oB1 = 640, oW2 = 704, oB2 = 4800, oW3 = 4864, oB3 = 8960, oW4 = 9024, oB4 = 9216;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf_load(const uint16_t* p, int64_t i) {
  return __uint_as_float(((uint32_t)p[i]) << 16);
}
__device__ __forceinline__ uint16_t bf_bits(float x) {
  return (uint16_t)(__float_as_uint(__bfloat162float(__float2bfloat16_rn(x))) >> 16);
}

__device__ void load_weights(const uint16_t* P, float* w) {
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) w[i] = bf_load(P, i);
}

// h_out[j][t] = bf16(tanh(b[j] + sum_k W[j][k] h_in[k][t])), k < K
template <int K>
__device__ __forceinline__ void dense_tanh(const float* W, const float* b, const float* hin, float* hout,
                                           uint16_t* acts, int64_t s, bool valid, int act_off) {
  const int t = threadIdx.x;
  float in[K];
#pragma unroll
  for (int k = 0; k < K; ++k) in[k] = hin[k * kLd + t];
  for (int j = 0; j < 64; ++j) {
    float acc = b[j];
#pragma unroll
    for (int k = 0; k < K; ++k) acc = fmaf(W[j * K + k], in[k], acc);
    const float h = bf(tanhf(acc));
    hout[j * kLd + t] = h;
    if (acts && valid) acts[s * 192 + act_off + j] = bf_bits(h);
  }
}

__global__ void __launch_bounds__(kS) mlp_forward_kernel(const uint16_t* P, const float* feats, int64_t n, float* out,
                                                         uint16_t* acts) {
  extern __shared__ float sm[];
  float* w = sm;                       // kNP (+pad)
  float* A = sm + 9220;                // 64 x kLd
  float* B = A + 64 * kLd;             // 64 x kLd
  load_weights(P, w);
  const int t = threadIdx.x;
  const int64_t s = blockIdx.x * (int64_t)kS + t;
  const bool valid = s < n;
  for (int c = 0; c < 10; ++c) A[c * kLd + t] = valid ? bf(feats[s * 10 + c]) : 0.0f;
  __syncthreads();
  dense_tanh<10>(w + oW1, w + oB1, A, B, acts, s, valid, 0);
  dense_tanh<64>(w + oW2, w + oB2, B, A, acts, s, valid, 64);
  dense_tanh<64>(w + oW3, w + oB3, A, B, acts, s, valid, 128);
  float h3[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) h3[k] = B[k * kLd + t];
  if (!valid) return;
  for (int o = 0; o < 3; ++o) {
    float acc = w[oB4 + o];
#pragma unroll
    for (int k = 0; k < 64; ++k) acc = fmaf(w[oW4 + o * 64 + k], h3[k], acc);
    out[s * 3 + o] = acc;
  }
}

// grads[o] += sum over the block's samples of D[j][t] * H[k][t] for o = j*K + k,
// and of D[j][t] for the biases.
template <int K>
__device__ void block_outer(const float* D, const float* H, int J, float* gW, float* gb) {
  for (int o = threadIdx.x; o < J * K; o += blockDim.x) {
    const int j = o / K, k = o % K;
    float acc = 0.0f;
    for (int t = 0; t < kS; ++t) acc = fmaf(D[j * kLd + t], H[k * kLd + t], acc);
    atomicAdd(&gW[o], acc);
  }
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    float acc = 0.0f;
    for (int t = 0; t < kS; ++t) acc += D[j * kLd + t];
    atomicAdd(&gb[j], acc);
  }
}

// delta_prev[k][t] = (sum_j W[j][k] D[j][t]) * (1 - h[k][t]^2), j < J, k < 64
template <int J>
__device__ void back_delta(const float* W, const float* D, const float* h, float* out) {
  const int t = threadIdx.x;
  float d[J];
#pragma unroll
  for (int j = 0; j < J; ++j) d[j] = D[j * kLd + t];
  for (int k = 0; k < 64; ++k) {
    float acc = 0.0f;
#pragma unroll
    for (int j = 0; j < J; ++j) acc = fmaf(W[j * 64 + k], d[j], acc);
    const float hk = h[k * kLd + t];
    out[k * kLd + t] = acc * (1.0f - hk * hk);
  }
}

__global__ void __launch_bounds__(kS) mlp_backward_kernel(const uint16_t* P, const float* feats, const uint16_t* acts,
                                                          const float* dout, int64_t n, float* grads) {
  extern __shared__ float sm[];
  float* w = sm;
  float* X = sm + 9220;                // 10 x kLd
  float* H1 = X + 10 * kLd;            // 64 x kLd
  float* H2 = H1 + 64 * kLd;
  float* H3 = H2 + 64 * kLd;
  float* D = H3 + 64 * kLd;            // current delta, 64 x kLd
  float* D2 = D + 64 * kLd;            // next delta
  load_weights(P, w);
  const int t = threadIdx.x;
  const int64_t s = blockIdx.x * (int64_t)kS + t;
  const bool valid = s < n;
  for (int c = 0; c < 10; ++c) X[c * kLd + t] = valid ? bf(feats[s * 10 + c]) : 0.0f;
  for (int k = 0; k < 64; ++k) {
    H1[k * kLd + t] = valid ? bf_load(acts, s * 192 + k) : 0.0f;
    H2[k * kLd + t] = valid ? bf_load(acts, s * 192 + 64 + k) : 0.0f;
    H3[k * kLd + t] = valid ? bf_load(acts, s * 192 + 128 + k) : 0.0f;
  }
  for (int o = 0; o < 3; ++o) D[o * kLd + t] = valid ? dout[s * 3 + o] : 0.0f;
  __syncthreads();
  block_outer<64>(D, H3, 3, grads + oW4, grads + oB4);              // layer 4
  back_delta<3>(w + oW4, D, H3, D2);                                 // delta3
  __syncthreads();
  block_outer<64>(D2, H2, 64, grads + oW3, grads + oB3);            // layer 3
  back_delta<64>(w + oW3, D2, H2, D);                                // delta2
  __syncthreads();
  block_outer<64>(D, H1, 64, grads + oW2, grads + oB2);             // layer 2
  back_delta<64>(w + oW2, D, H1, D2);                                // delta1
  __syncthreads();
  block_outer<10>(D2, X, 64, grads + oW1, grads + oB1);             // layer 1
}

__global__ void mse_grad_kernel(const float* out, const float* target, const float* wgt, int64_t n, float* dout,
                                double* loss) {
  __shared__ double red[32];
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double l = 0.0;
  if (s < n) {
    const float ws = wgt[s];
    for (int o = 0; o < 3; ++o) {
      const float d = out[s * 3 + o] - target[s * 3 + o];
      dout[s * 3 + o] = 2.0f * ws * d;
      l += (double)ws * d * d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x < 32) {
    double u = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (threadIdx.x == 0) atomicAdd(loss, u);
  }
}

__global__ void adam_kernel(float* master, uint16_t* P, const float* g, float* m1, float* m2, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.0f - b1) * gi;
  const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  const float th = master[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
  master[i] = th;
  P[i] = bf_bits(th);
}

// Backward differences of the velocity history of DOF r (float64): a
// difference that needs a missing velocity (NULL) is zero.
struct Diffs {
  double d1, d2, d3;
};
__device__ __forceinline__ Diffs history_diffs(const double* v_n, const double* v1, const double* v2,
                                               const double* v3, int64_t r) {
  Diffs d{0.0, 0.0, 0.0};
  if (!v1) return d;
  const double a = v_n[r], b = v1[r];
  d.d1 = a - b;
  if (!v2) return d;
  const double c = v2[r];
  d.d2 = a - 2.0 * b + c;
  if (!v3) return d;
  d.d3 = a - 3.0 * b + 3.0 * c - v3[r];
  return d;
}

// r_I = || (nabla v / s1, nabla^2 v / s2, nabla^3 v / s3) || over the 9
// scaled differences of node I (float64); the inputs are divided by it and
// the correction multiplied by it, so the learned map does not depend on the
// amplitude of the motion.
__device__ __forceinline__ double node_scale(const Diffs (&x)[3], double inv1, double inv2, double inv3) {
  double r2 = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double a = x[d].d1 * inv1, b = x[d].d2 * inv2, c = x[d].d3 * inv3;
    r2 += a * a + b * b + c * c;
  }
  return sqrt(r2);
}

// inputs: (nabla v / s1, nabla^2 v / s2, nabla^3 v / s3) / r_I (float64,
// then float32; zero where r_I = 0), fixed flag
__global__ void features_kernel(const double* v_n, const double* v1, const double* v2, const double* v3,
                                const int32_t* fixed_of_node, int64_t nn, double inv1, double inv2, double inv3,
                                float* feats) {
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nn) return;
  Diffs x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = history_diffs(v_n, v1, v2, v3, 3 * I + d);
  const double r = node_scale(x, inv1, inv2, inv3);
  const double ir = r > 0.0 ? 1.0 / r : 0.0;
  float* f = feats + 10 * I;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    f[d] = float(x[d].d1 * inv1 * ir);
    f[3 + d] = float(x[d].d2 * inv2 * ir);
    f[6 + d] = float(x[d].d3 * inv3 * ir);
  }
  f[9] = fixed_of_node[I] >= 0 ? 1.0f : 0.0f;
}

// v_init = b + s_out r_I out on free nodes (out may be null), 0 on clamped nodes
__global__ void apply_kernel(const float* out, const double* v_n, const double* v1, const double* v2,
                             const double* v3, const int32_t* fixed_of_node, int64_t nn, double inv1, double inv2,
                             double inv3, double s_out, double* v_init) {
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nn) return;
  const bool fixed = fixed_of_node[I] >= 0;
  Diffs x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = history_diffs(v_n, v1, v2, v3, 3 * I + d);
  const double sr = out ? s_out * node_scale(x, inv1, inv2, inv3) : 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t r = 3 * I + d;
    const double base = v_n[r] + x[d].d1 + x[d].d2 + x[d].d3;
    v_init[r] = fixed ? 0.0 : base + (out ? sr * double(out[r]) : 0.0);
  }
}

// target = (v_next - b) / (s_out r_I) on free nodes (float32), 0 on clamped
// nodes and where r_I = 0
__global__ void target_kernel(const double* v_next, const double* v_n, const double* v1, const double* v2,
                              const double* v3, const int32_t* fixed_of_node, int64_t nn, double inv1, double inv2,
                              double inv3, double s_out, float* target) {
  const int64_t I = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (I >= nn) return;
  Diffs x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x[d] = history_diffs(v_n, v1, v2, v3, 3 * I + d);
  const double r = node_scale(x, inv1, inv2, inv3);
  const bool zero = fixed_of_node[I] >= 0 || !(r > 0.0);
  const double inv = zero ? 0.0 : 1.0 / (s_out * r);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t k = 3 * I + d;
    target[k] = zero ? 0.0f : float((v_next[k] - (v_n[k] + x[d].d1 + x[d].d2 + x[d].d3)) * inv);
  }
}

// out[c] += sum_i x[i][c]^2 for c < ncol <= 16: per-thread partial sums over
// a grid-stride range, a block reduction per column, one float64 atomic per
// column and block
constexpr int kSumsqMaxCol = 16;
__global__ void col_sumsq_kernel(const float* x, int64_t n, int ncol, double* out) {
  __shared__ double red[kSumsqMaxCol][8];
  double acc[kSumsqMaxCol];
#pragma unroll
  for (int c = 0; c < kSumsqMaxCol; ++c) acc[c] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < kSumsqMaxCol; ++c)
      if (c < ncol) {
        const double v = x[i * ncol + c];
        acc[c] += v * v;
      }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kSumsqMaxCol; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[c][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < ncol) {
    double v = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[threadIdx.x][k];
    atomicAdd(&out[threadIdx.x], v);
  }
}

constexpr size_t kFwdSmem = sizeof(float) * (9220 + 2 * 64 * kLd);
constexpr size_t kBwdSmem = sizeof(float) * (9220 + 10 * kLd + 5 * 64 * kLd);

tl_status set_smem(const void* k, size_t b) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) == cudaSuccess ? TL_OK
                                                                                                     : TL_ERR_CUDA;
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" {

tl_status tl_mlp_forward(const uint16_t* params, const float* feats, int64_t n, float* out, uint16_t* acts,
                         void* stream) {
  if (!params || !feats || !out || n < 0) return TL_ERR_INVALID_ARG;
  if (n == 0) return TL_OK;
  if (set_smem((const void*)mlp_forward_kernel, kFwdSmem) != TL_OK) return TL_ERR_CUDA;
  mlp_forward_kernel<<<(unsigned)((n + kS - 1) / kS), kS, kFwdSmem, (cudaStream_t)stream>>>(params, feats, n, out,
                                                                                          acts);
  return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}

tl_status tl_mlp_backward(const uint16_t* params, const float* feats, const uint16_t* acts, const float* dout,
                          int64_t n, float* grads, void* stream) {
  if (!params || !feats || !acts || !dout || !grads || n < 0) return TL_ERR_INVALID_ARG;
  if (n == 0) return TL_OK;
  if (set_smem((const void*)mlp_backward_kernel, kBwdSmem) != TL_OK) return TL_ERR_CUDA;
  mlp_backward_kernel<<<(unsigned)((n + kS - 1) / kS), kS, kBwdSmem, (cudaStream_t)stream>>>(params, feats, acts,
                                                                                           dout, n, grads);
  return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}

tl_status tl_mlp_mse_grad(const float* out, const float* target, const float* weight, int64_t n, float* dout,
                          double* loss, void* stream) {
  if (!out || !target || !weight || !dout || !loss || n < 0) return TL_ERR_INVALID_ARG;
  if (n == 0) return TL_OK;
  mse_grad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(out, target, weight, n, dout, loss);
  return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}

tl_status tl_mlp_adam(float* master, uint16_t* params, const float* grads, float* m1, float* m2, int64_t n, float lr,
                      float beta1, float beta2, float eps, int32_t step, void* stream) {
  if (!master || !params || !grads || !m1 || !m2 || n < 0 || step < 1) return TL_ERR_INVALID_ARG;
  const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(master, params, grads, m1, m2, n, lr,
                                                                           beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}

tl_status tl_mlp_features(tl_mesh* m, const double* v_n, const double* v_prev, const double* v_prev2,
                          const double* v_prev3, double s1, double s2, double s3, float* feats) {
  if (!m || !v_n || !feats || !(s1 > 0.0) || !(s2 > 0.0) || !(s3 > 0.0)) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  features_kernel<<<(unsigned)((m->nn + 255) / 256), 256, 0, m->stream>>>(
      v_n, v_prev, v_prev ? v_prev2 : nullptr, v_prev && v_prev2 ? v_prev3 : nullptr, m->d_fixed_of_node, m->nn,
      1.0 / s1, 1.0 / s2, 1.0 / s3, feats);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

tl_status tl_warm_start(tl_mesh* m, const uint16_t* params, const double* v_n, const double* v_prev,
                        const double* v_prev2, const double* v_prev3, double s1, double s2, double s3,
                        double s_out, float* work, double* v_init) {
  if (!m || !v_n || !v_init || (params && !work)) return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  const double* v2 = v_prev ? v_prev2 : nullptr;
  const double* v3 = v2 ? v_prev3 : nullptr;
  float* out = nullptr;
  if (params) {
    float* feats = work;
    out = work + 10 * m->nn;
    tl_status s = tl_mlp_features(m, v_n, v_prev, v2, v3, s1, s2, s3, feats);
    if (s != TL_OK) return s;
    s = tl_mlp_forward(params, feats, m->nn, out, nullptr, m->stream);
    if (s != TL_OK) return fail(m, s, "MLP forward launch failed");
    ++m->launches;
  }
  if (params && !(s1 > 0.0 && s2 > 0.0 && s3 > 0.0)) return TL_ERR_INVALID_ARG;
  apply_kernel<<<(unsigned)((m->nn + 255) / 256), 256, 0, m->stream>>>(
      out, v_n, v_prev, v2, v3, m->d_fixed_of_node, m->nn, params ? 1.0 / s1 : 0.0, params ? 1.0 / s2 : 0.0,
      params ? 1.0 / s3 : 0.0, s_out, v_init);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

tl_status tl_mlp_target(tl_mesh* m, const double* v_next, const double* v_n, const double* v_prev,
                        const double* v_prev2, const double* v_prev3, double s1, double s2, double s3,
                        double s_out, float* target) {
  if (!m || !v_next || !v_n || !target || !(s_out > 0.0) || !(s1 > 0.0) || !(s2 > 0.0) || !(s3 > 0.0))
    return TL_ERR_INVALID_ARG;
  if (!m->have_pattern) return fail(m, TL_ERR_STATE, "tl_build_pattern must come first");
  const double* v2 = v_prev ? v_prev2 : nullptr;
  const double* v3 = v2 ? v_prev3 : nullptr;
  target_kernel<<<(unsigned)((m->nn + 255) / 256), 256, 0, m->stream>>>(v_next, v_n, v_prev, v2, v3,
                                                                       m->d_fixed_of_node, m->nn, 1.0 / s1,
                                                                       1.0 / s2, 1.0 / s3, s_out, target);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

tl_status tl_mlp_col_sumsq(const float* x, int64_t n, int32_t ncol, double* out, void* stream) {
  if (!x || !out || n < 0 || ncol < 1 || ncol > kSumsqMaxCol) return TL_ERR_INVALID_ARG;
  if (n == 0) return TL_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1024);
  col_sumsq_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, n, ncol, out);
  return cudaGetLastError() == cudaSuccess ? TL_OK : TL_ERR_CUDA;
}

}  // extern "C"
