// T10 element kernels: internal force, tangent stiffness and their scatter
// into the fixed-pattern CSR Hessian.  Templates only: the tl_element_*.cu
// files instantiate them (one translation unit per precision and pass, so the
// build compiles them in parallel) and tl_element.cu dispatches.
//
// Paper: arxiv 2604.10357
//   Sec. 4.3  eq. F_assembly, eq. fint_local, eq. fint_global (Stage 1 + 2)
//   Sec. 4.4  eq. tangent_block and the Hessian assembly (eq. hessian)
//
// GB300 design (differs from the paper's two-stage, thread-per-(e,q) /
// thread-per-(e,a) kernels with a stress buffer in global memory):
//   * one fused kernel: a CTA owns kTile = 32 consecutive elements; their
//     connectivity, geometry and slot indices are staged in shared memory and
//     nothing per quadrature point ever goes to global memory;
//   * warps are specialised by role with lanes = elements, so every branch on
//     the role is warp-uniform:
//       qp phase:      warp w -> (quadrature point q = w/3, row i = w%3)
//       tangent phase: warp w -> (row-pair p = w/3, row i = w%3), covering the
//                      block rows a = p and a = 9-p (11 blocks, b >= a), so
//                      the symmetric 30x30 is formed once (55 blocks);
//   * the scatter goes through a per-element slot map (position k of node
//     conn[b] in node conn[a]'s sorted adjacency), so there is no binary
//     search: slot = 9 ptr(I) + 3 deg(I) i + 3 k + j;
//   * TL_FP32_ELEM evaluates the element in float32 from the displacement
//     gradient H (F = I + H, E = (H + H^T + H^T H)/2) and a cancellation-free
//     Mooney-Rivlin stress (deviators of E, J - 1 from the invariants of H).
#pragma once

#include <algorithm>
#include <cstddef>
#include <type_traits>

#include "tl_element_common.cuh"

namespace tl {
namespace elem {

constexpr int E = kTile;          // elements per CTA
constexpr int NWARP = 15;         // 5 qp x 3 rows, and 5 row pairs x 3 rows
constexpr int NT = 32 * NWARP;    // 480 threads

// Warp-specialised variant (float32 CSR assembly): the 15 compute warps plus 5
// scatter warps.  Barrier 1 synchronises the compute warps only; barriers 2
// and 3 hand the exchange buffer between compute and scatter warps.
constexpr int NWS = 5;                 // scatter warps
constexpr int NTW = 32 * (NWARP + NWS);  // 640 threads
enum : int { kBarCompute = 1, kBarFull = 2, kBarEmpty = 3 };

template <bool WS>
__device__ __forceinline__ void bar_compute() {
  if constexpr (WS) asm volatile("bar.sync 1, 480;" ::: "memory");
  else __syncthreads();
}
__device__ __forceinline__ void bar_sync_all(int id) {
  asm volatile("bar.sync %0, 640;" ::"r"(id) : "memory");
}
__device__ __forceinline__ void bar_arrive_all(int id) {
  asm volatile("bar.arrive %0, 640;" ::"r"(id) : "memory");
}

template <typename T>
struct Args {
  const int32_t* conn;
  const T* geo;
  const uint8_t* blk;
  const int32_t* node_ptr;
  const int32_t* user_of;
  const double* q_n;
  const double* v;
  const double* X;
  double h;
  int64_t real_end;    // internal elements >= real_end are padding (per segment)
  MatT<T> mat;
  T alpha, beta;       // tangent = alpha K_t + beta D
  T mass_scale;        // mass term M_e * mass_scale added to the tangent
  double* f;           // force output (atomic add), may be null
  T* values;           // CSR values (atomic add), may be null
  T* K_elem;           // per-element 30x30 output (user order), may be null
  uint32_t* flags;
  int32_t nnz;         // length of values (bounds of the vector reductions)
  int32_t v4_ok;       // values is 16-byte aligned
  int32_t xchg;        // FP32 CSR assembly through the exchange buffer
  int32_t pf_off;      // byte offset of the prefetch buffer in shared memory (-1: none)
  int32_t meta_off;    // byte offset of the second scatter-metadata buffer (warp-specialised kernel)
  int32_t x_alias;     // 1: the exchange buffer overlays the force and tangent arrays (two CTAs per SM)
  int32_t agg;         // 1: per-tile aggregation of shared node pairs (maps below)
  const int4* agg_slot;        // per tile and unordered pair {P, Q}: CSR positions and row strides of
                               // the (P, Q) and (Q, P) blocks (the second -1 when P = Q)
  const uint16_t* agg_cptr;    // per tile: first contribution of each pair
  const uint16_t* agg_code;    // per tile: exchange-buffer block (+ transposed flag) of each contribution
  const int32_t* agg_nu;       // per tile: number of distinct pairs
  const float2* uv;            // pair kernel: per DOF {q_n + h v - X, v} in float32 (pair_prep)
};

// Per-element shared-memory strides padded to odd word counts so that lanes
// (= elements) reading the same offset hit distinct banks.
constexpr int kNStride = 151;    // 5 qp x 30 grad N, + 1
// Tangent rows: 27 entries padded to 28 and 84 per quadrature point, so every
// row starts on a 16-byte boundary (vector shared-memory accesses); the
// per-element stride 420 = 4 (mod 32) keeps eight lanes of a 16-byte access
// on distinct banks.
constexpr int kARow = 28;
constexpr int kAQp = 3 * kARow;           // 84
constexpr int kAStride = 5 * kAQp;        // 420
constexpr int kFStride = 151;    // 5 qp x 30 force entries, + 1
constexpr int kUStride = 31;

// Per-tile scatter metadata: CSR row bases and strides of the 10 nodes and
// the slot blocks of the 32 elements.
struct TileMeta {
  int32_t rbase[10][E];
  int32_t rstr[10][E];
  uint8_t blk[E][100];
};

template <typename T>
struct Smem {
  int32_t node[10][E];
  TileMeta meta;
  T geo[16][E];
  T u[kUStride * E];
  T vel[kUStride * E];
  T n[kNStride * E];
  T fq[kFStride * E];
  T A[kAStride * E];
};

// ---------------------------------------------------------------------------
// Stage the tile: connectivity, row bases, slot indices, geometry and the
// nodal displacement / velocity gathers.
// ---------------------------------------------------------------------------
template <typename T, bool NEED_PATTERN, bool WS = false>
__device__ __forceinline__ void load_tile(const Args<T>& A, Smem<T>& sm, int64_t e0, TileMeta& mt) {
  const int tid = threadIdx.x;
  for (int t = tid; t < E * 10; t += NT) {
    const int e = t / 10, a = t % 10;
    const int node = A.conn[(e0 + e) * 10 + a];
    sm.node[a][e] = node;
    if (NEED_PATTERN && !A.agg) {     // the aggregated scatter reads the tile maps instead
      const int p0 = A.node_ptr[node], p1 = A.node_ptr[node + 1];
      mt.rbase[a][e] = 9 * p0;
      mt.rstr[a][e] = 3 * (p1 - p0);
    }
  }
  if (NEED_PATTERN && !A.agg) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(A.blk + e0 * 100);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&mt.blk[0][0]);
    for (int t = tid; t < E * 25; t += NT) dst[t] = src[t];
  }
  for (int t = tid; t < E * 16; t += NT) {
    const int e = t / 16, c = t % 16;
    sm.geo[c][e] = A.geo[(e0 + e) * 16 + c];
  }
  bar_compute<WS>();
  const double h = A.h;
  for (int t = tid; t < E * 30; t += NT) {
    const int c = t / E, e = t % E;
    const int a = c / 3, d = c % 3;
    const int64_t g = 3 * (int64_t)sm.node[a][e] + d;
    const double vv = A.v[g];
    const double x = A.q_n[g] + h * vv;
    sm.u[c * E + e] = T(x - A.X[g]);
    sm.vel[c * E + e] = T(vv);
  }
  bar_compute<WS>();
}

// ---------------------------------------------------------------------------
// Prefetch of the next tile (float32 kernels).  While a CTA computes tile t it
// copies, with cp.async, the raw data of its next tile into a buffer of its
// own: stage 1 (issued after tile t is staged) the connectivity, geometry and
// slot-block rows; stage 2 (issued once stage 1 has landed, after the qp
// phase) the row-pointer pairs and the nodal q_n, v and X of those nodes.  The
// next tile is then staged from shared memory only.
// ---------------------------------------------------------------------------
template <typename T>
struct Prefetch {
  int32_t conn[E * 10];          // element-major rows, as in global memory
  T geo[E * 16];
  uint8_t blk[E * 100];
  int32_t nptr[2][10][E];        // node_ptr[node], node_ptr[node + 1]
  double qn[30 * E], vv[30 * E], XX[30 * E];   // [c][e], c = 3 a + d
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage 1: the tile's rows of conn (1,280 B), geo (32 x 16 T) and blk
// (3,200 B) are contiguous and 16-byte aligned (tiles start at multiples of
// 32 elements; the arrays come from cudaMalloc).
template <typename T>
__device__ __forceinline__ void prefetch_stage1(const Args<T>& A, Prefetch<T>& P, int64_t e0) {
  const int tid = threadIdx.x;
  const unsigned char* c = reinterpret_cast<const unsigned char*>(A.conn + e0 * 10);
  const unsigned char* g = reinterpret_cast<const unsigned char*>(A.geo + e0 * 16);
  const unsigned char* b = A.blk + e0 * 100;
  constexpr int nc = E * 10 * 4 / 16, ng = E * 16 * (int)sizeof(T) / 16;
  const int nb = A.agg ? 0 : E * 100 / 16;       // slot blocks: not read by the aggregated scatter
  for (int k = tid; k < nc + ng + nb; k += NT) {
    if (k < nc) cp_async16(reinterpret_cast<unsigned char*>(P.conn) + 16 * k, c + 16 * k);
    else if (k < nc + ng) cp_async16(reinterpret_cast<unsigned char*>(P.geo) + 16 * (k - nc), g + 16 * (k - nc));
    else cp_async16(P.blk + 16 * (k - nc - ng), b + 16 * (k - nc - ng));
  }
  cp_async_commit();
}

// Stage 2 (after stage 1 is visible to the block): row pointers and nodal data.
template <typename T>
__device__ __forceinline__ void prefetch_stage2(const Args<T>& A, Prefetch<T>& P) {
  const int tid = threadIdx.x;
  // element index fastest: consecutive threads write consecutive words
  for (int t = tid; t < E * 10; t += NT) {
    const int a = t / E, e = t % E;
    if (A.agg) break;                              // row pointers: only for the per-element scatter
    const int node = P.conn[e * 10 + a];
    cp_async4(&P.nptr[0][a][e], A.node_ptr + node);
    cp_async4(&P.nptr[1][a][e], A.node_ptr + node + 1);
  }
  for (int t = tid; t < E * 30; t += NT) {
    const int c = t / E, e = t % E;
    const int64_t g = 3 * (int64_t)P.conn[e * 10 + c / 3] + c % 3;
    cp_async8(&P.qn[c * E + e], A.q_n + g);
    cp_async8(&P.vv[c * E + e], A.v + g);
    cp_async8(&P.XX[c * E + e], A.X + g);
  }
  cp_async_commit();
}

// Stage the next tile from the prefetch buffer (as load_tile does from global).
template <typename T, bool NEED_PATTERN, bool WS = false>
__device__ __forceinline__ void unpack_tile(const Args<T>& A, Smem<T>& sm, const Prefetch<T>& P, TileMeta& mt) {
  const int tid = threadIdx.x;
  for (int t = tid; t < E * 10; t += NT) {
    const int a = t / E, e = t % E;
    sm.node[a][e] = P.conn[e * 10 + a];
    if (NEED_PATTERN && !A.agg) {
      const int p0 = P.nptr[0][a][e], p1 = P.nptr[1][a][e];
      mt.rbase[a][e] = 9 * p0;
      mt.rstr[a][e] = 3 * (p1 - p0);
    }
  }
  if (NEED_PATTERN && !A.agg) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(P.blk);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&mt.blk[0][0]);
    for (int t = tid; t < E * 25; t += NT) dst[t] = src[t];
  }
  for (int t = tid; t < E * 16; t += NT) {
    const int e = t / 16, c = t % 16;
    sm.geo[c][e] = P.geo[t];
  }
  const double h = A.h;
  for (int t = tid; t < E * 30; t += NT) {
    const int c = t / E, e = t % E;
    const double vv = P.vv[t];
    const double x = P.qn[t] + h * vv;
    sm.u[c * E + e] = T(x - P.XX[t]);
    sm.vel[c * E + e] = T(vv);
  }
  bar_compute<WS>();
}

// Gradients of the 10 shape functions at barycentric point L (straight-sided
// T10): corners (4 L_a - 1) grad L_a, midsides 4 (L_i grad L_j + L_j grad L_i).
template <typename T>
__device__ __forceinline__ void shape_grads(const T (&geo)[16][E], int e, const double Lq[4], T n[10][3]) {
  T gL[4][3];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) gL[c][d] = geo[c * 3 + d][e];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 3; ++d) n[a][d] = (T(4) * T(Lq[a]) - T(1)) * gL[a][d];
#pragma unroll
  for (int m = 4; m < 10; ++m) {
    const int i = edge_i(m), j = edge_j(m);
#pragma unroll
    for (int d = 0; d < 3; ++d) n[m][d] = T(4) * (T(Lq[i]) * gL[j][d] + T(Lq[j]) * gL[i][d]);
  }
}

// Row i of the force and of the scaled tangent at one quadrature point.
template <typename T, int MAT, bool KV, bool WANT_A, int i>
__device__ __forceinline__ void qp_rows(const Args<T>& A, Smem<T>& sm, const QP<T>& s, const T (&n)[10][3],
                                        T wJ, int e, int q) {
  // force row i: f_a,i = wJ sum_J P_iJ n_aJ with P = F S
  T Pi[3];
#pragma unroll
  for (int J = 0; J < 3; ++J) {
    T acc = 0;
#pragma unroll
    for (int M = 0; M < 3; ++M) acc += s.F[i][M] * s.S[M][J];
    Pi[J] = acc * wJ;
  }
#pragma unroll
  for (int a = 0; a < 10; ++a)
    sm.fq[e * kFStride + q * 30 + a * 3 + i] = Pi[0] * n[a][0] + Pi[1] * n[a][1] + Pi[2] * n[a][2];
  if (WANT_A) tangent_row<T, MAT, KV, i>(s, A.mat, A.alpha, A.beta, wJ, &sm.A[e * kAStride + q * kAQp + i * kARow]);
}

// qp phase: warp w -> (q = w / 3, row i = w % 3), lane = element.  The
// kinematics and the constitutive update are shared by the three rows (one
// copy of their code); only the row-specific part is compiled per row.
template <typename T, int MAT, bool KV, bool WANT_A>
__device__ __forceinline__ void qp_phase(const Args<T>& A, Smem<T>& sm, bool& inverted) {
  const int w = threadIdx.x >> 5, e = threadIdx.x & 31;
  const int q = w / 3, i = w % 3;
  double Lq[4];
  qp_bary(q, Lq);
  const T wJ = T(qp_wfrac(q)) * sm.geo[12][e];
  T n[10][3];
  shape_grads(sm.geo, e, Lq, n);
  if (i == 0) {
#pragma unroll
    for (int a = 0; a < 10; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) sm.n[e * kNStride + q * 30 + a * 3 + d] = n[a][d];
  }
  T Hm[3][3], Fd[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Hm[r][c] = 0;
      Fd[r][c] = 0;
    }
#pragma unroll
  for (int a = 0; a < 10; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T ua = sm.u[(a * 3 + r) * E + e];
      T va = T(0);
      if (KV) va = sm.vel[(a * 3 + r) * E + e];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Hm[r][c] += ua * n[a][c];
        if (KV) Fd[r][c] += va * n[a][c];
      }
    }
  QP<T> s;
  constitutive<T, MAT, KV>(Hm, Fd, A.mat, s, inverted);
  switch (i) {     // warp-uniform
    case 0: qp_rows<T, MAT, KV, WANT_A, 0>(A, sm, s, n, wJ, e, q); break;
    case 1: qp_rows<T, MAT, KV, WANT_A, 1>(A, sm, s, n, wJ, e, q); break;
    default: qp_rows<T, MAT, KV, WANT_A, 2>(A, sm, s, n, wJ, e, q); break;
  }
}

// Force phase: warp w handles element DOFs c = w and c = w + 15.
template <typename T>
__device__ __forceinline__ void force_phase(const Args<T>& A, const Smem<T>& sm, int64_t e0) {
  const int w = threadIdx.x >> 5, e = threadIdx.x & 31;
  if (e0 + e >= A.real_end) return;
#pragma unroll
  for (int rep = 0; rep < 2; ++rep) {
    const int c = w + 15 * rep;
    T acc = 0;
#pragma unroll
    for (int q = 0; q < 5; ++q) acc += sm.fq[e * kFStride + q * 30 + c];
    const int a = c / 3, d = c % 3;
    atomicAdd(&A.f[3 * (int64_t)sm.node[a][e] + d], double(acc));
  }
}

// One block row of the element tangent for one element (lane) and component
// i: K_{A0,b}[i][k] for b = A0 .. A0+NB-1, accumulated over the 5 qp, plus the
// mass term, then scattered (the (b, A0) transposed entries too).
template <typename T, int A0, int NB>
__device__ __forceinline__ void tangent_blockrow(const Args<T>& A, const Smem<T>& sm, int64_t e0, int i) {
  const int e = threadIdx.x & 31;
  T acc[NB][3];
#pragma unroll
  for (int j = 0; j < NB; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[j][k] = 0;
#pragma unroll 1
  for (int q = 0; q < 5; ++q) {
    const T* nq = &sm.n[e * kNStride + q * 30];
    const T* Aq = &sm.A[e * kAStride + q * kAQp + i * kARow];
    const T na[3] = {nq[A0 * 3], nq[A0 * 3 + 1], nq[A0 * 3 + 2]};
    T An[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int L = 0; L < 3; ++L)
        An[k][L] = na[0] * Aq[0 * 9 + k * 3 + L] + na[1] * Aq[1 * 9 + k * 3 + L] + na[2] * Aq[2 * 9 + k * 3 + L];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int b = A0 + j;
      const T n0b = nq[b * 3], n1b = nq[b * 3 + 1], n2b = nq[b * 3 + 2];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[j][k] += An[k][0] * n0b + An[k][1] * n1b + An[k][2] * n2b;
    }
  }
  if (e0 + e >= A.real_end) return;
  const T ms = A.mass_scale * A.mat.rho * sm.geo[12][e] * T(1.0 / 420.0);
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    constexpr int a = A0;
    const int b = A0 + j;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k == i) acc[j][k] += ms * T(c_mass420[a][b]);
    if (A.values) {
      const int s_row = sm.meta.rbase[a][e] + sm.meta.rstr[a][e] * i + 3 * sm.meta.blk[e][a * 10 + b];
#pragma unroll
      for (int k = 0; k < 3; ++k) atomic_add_t(&A.values[s_row + k], acc[j][k]);
      if (j > 0) {
        const int kb = 3 * sm.meta.blk[e][b * 10 + a] + i;
#pragma unroll
        for (int k = 0; k < 3; ++k) atomic_add_t(&A.values[sm.meta.rbase[b][e] + sm.meta.rstr[b][e] * k + kb], acc[j][k]);
      }
    }
    if (A.K_elem) {
      const int64_t ue = A.user_of[e0 + e];
      T* Ke = A.K_elem + ue * 900;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        Ke[(3 * a + i) * 30 + 3 * b + k] = acc[j][k];
        if (j > 0) Ke[(3 * b + k) * 30 + 3 * a + i] = acc[j][k];
      }
    }
  }
}

// Accumulate block row A0 (blocks b = A0 .. A0+NB-1, component i) over the 5
// quadrature points and add the mass term; no scatter.
template <typename T, int A0, int NB>
__device__ __forceinline__ void accumulate_blockrow(const Args<T>& A, const Smem<T>& sm, int i, T (&acc)[NB][3]) {
  const int e = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NB; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[j][k] = 0;
#pragma unroll 1
  for (int q = 0; q < 5; ++q) {
    const T* nq = &sm.n[e * kNStride + q * 30];
    const T* Aq = &sm.A[e * kAStride + q * kAQp + i * kARow];
    const T na[3] = {nq[A0 * 3], nq[A0 * 3 + 1], nq[A0 * 3 + 2]};
    T av[27];
#pragma unroll
    for (int c = 0; c < 27; ++c) av[c] = Aq[c];
    T An[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int L = 0; L < 3; ++L)
        An[k][L] = na[0] * av[0 * 9 + k * 3 + L] + na[1] * av[1 * 9 + k * 3 + L] + na[2] * av[2 * 9 + k * 3 + L];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int b = A0 + j;
      const T n0b = nq[b * 3], n1b = nq[b * 3 + 1], n2b = nq[b * 3 + 2];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[j][k] += An[k][0] * n0b + An[k][1] * n1b + An[k][2] * n2b;
    }
  }
  const T ms = A.mass_scale * A.mat.rho * sm.geo[12][e] * T(1.0 / 420.0);
#pragma unroll
  for (int j = 0; j < NB; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k == i) acc[j][k] += ms * T(c_mass420[A0][A0 + j]);
}

// Both block rows of warp group P (a0 = P: b = P..9; a1 = 9 - P: b = 9-P..9)
// in one pass over the quadrature points: the tangent row is read once per
// point for both, and each n_b once (b >= 9 - P serves both rows).  Needs
// ~90 registers: used by the one-CTA-per-SM kernels only.
template <int P>
__device__ __forceinline__ void accumulate_blockrows_merged(const Args<float>& A, const Smem<float>& sm, int i,
                                                           float (&acc0)[10 - P][3], float (&acc1)[P + 1][3]) {
  constexpr int a0 = P, n0 = 10 - P, a1 = 9 - P, n1 = P + 1;
  const int e = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < n0; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc0[j][k] = 0.0f;
#pragma unroll
  for (int j = 0; j < n1; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc1[j][k] = 0.0f;
#pragma unroll 1
  for (int q = 0; q < 5; ++q) {
    const float* nq = &sm.n[e * kNStride + q * 30];
    const float* Aq = &sm.A[e * kAStride + q * kAQp + i * kARow];
    const float na0[3] = {nq[a0 * 3], nq[a0 * 3 + 1], nq[a0 * 3 + 2]};
    const float na1[3] = {nq[a1 * 3], nq[a1 * 3 + 1], nq[a1 * 3 + 2]};
    float av[27];
#pragma unroll
    for (int c = 0; c < 27; ++c) av[c] = Aq[c];
    float An0[3][3], An1[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int L = 0; L < 3; ++L) {
        An0[k][L] = na0[0] * av[k * 3 + L] + na0[1] * av[9 + k * 3 + L] + na0[2] * av[18 + k * 3 + L];
        An1[k][L] = na1[0] * av[k * 3 + L] + na1[1] * av[9 + k * 3 + L] + na1[2] * av[18 + k * 3 + L];
      }
#pragma unroll
    for (int j = 0; j < n0; ++j) {
      const int b = a0 + j;
      const float n0b = nq[b * 3], n1b = nq[b * 3 + 1], n2b = nq[b * 3 + 2];
#pragma unroll
      for (int k = 0; k < 3; ++k) acc0[j][k] += An0[k][0] * n0b + An0[k][1] * n1b + An0[k][2] * n2b;
      if (b >= a1) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          acc1[b - a1][k] += An1[k][0] * n0b + An1[k][1] * n1b + An1[k][2] * n2b;
      }
    }
  }
  const float ms = A.mass_scale * A.mat.rho * sm.geo[12][e] * (1.0f / 420.0f);
#pragma unroll
  for (int j = 0; j < n0; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k == i) acc0[j][k] += ms * c_mass420[a0][a0 + j];
#pragma unroll
  for (int j = 0; j < n1; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k == i) acc1[j][k] += ms * c_mass420[a1][a1 + j];
}

__device__ __forceinline__ void red_v4(float* p, float x, float y, float z, float w) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
__device__ __forceinline__ void red_v2(float* p, float x, float y) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(x), "f"(y) : "memory");
}

// Add the run values[s .. s+2] += (x0, x1, x2).  The run is placed in the
// 16-byte chunk that contains s (zeros in the other lanes) and issued as one
// 16-byte reduction, plus an 8-byte one for the part that spills into the
// next chunk when s is at offset 2 or 3: the instruction sequence does not
// depend on the offset (no divergence), and a lane adds 0 to neighbouring
// entries, which leaves them unchanged.  The last entries of the matrix use
// scalar reductions so no access passes the end of values.
__device__ __forceinline__ void red_run(const Args<float>& A, int s, float x0, float x1, float x2) {
  float* p = A.values;
  const int r = s & 3;
  const int base = s - r;
  if (A.v4_ok && base + 8 <= A.nnz) {
    const float w0 = r == 0 ? x0 : 0.0f;
    const float w1 = r == 0 ? x1 : (r == 1 ? x0 : 0.0f);
    const float w2 = r == 0 ? x2 : (r == 1 ? x1 : (r == 2 ? x0 : 0.0f));
    const float w3 = r == 1 ? x2 : (r == 2 ? x1 : (r == 3 ? x0 : 0.0f));
    const float w4 = r == 2 ? x2 : (r == 3 ? x1 : 0.0f);
    const float w5 = r == 3 ? x2 : 0.0f;
    red_v4(p + base, w0, w1, w2, w3);
    if (r >= 2) red_v2(p + base + 4, w4, w5);
    return;
  }
  atomicAdd(p + s, x0);
  atomicAdd(p + s + 1, x1);
  atomicAdd(p + s + 2, x2);
}

// FP32 assembly of block rows a0 = P and a1 = 9 - P.  The three warps (P, i)
// of one element accumulate the rows i of the same 11 blocks and park them in
// an exchange buffer X (32 elements x 55 blocks x 9 floats, its own shared
// memory after the Smem struct).  After a block-wide barrier each warp issues,
// from X, row i of each of its blocks (a, b) and row i of the transposed block
// (b, a), i.e. column i of (a, b): every write is a contiguous run of three
// CSR entries (row 3I+i, columns 3J..3J+2).  The scatter loop is not unrolled
// (it is bound by the L2 reductions, and unrolled copies of it for every
// block-row pair made the kernel miss in the instruction cache).
template <int P, bool MERGE = false>
__device__ __forceinline__ void tangent_xchg_accumulate(const Args<float>& A, const Smem<float>& sm, float* X,
                                                        int i, bool wait_empty = false, bool block_sync = false) {
  constexpr int a0 = P, n0 = 10 - P, a1 = 9 - P, n1 = P + 1;
  const int e = threadIdx.x & 31;
  float acc0[n0][3], acc1[n1][3];
  if constexpr (MERGE) {
    accumulate_blockrows_merged<P>(A, sm, i, acc0, acc1);
  } else {
    accumulate_blockrow<float, a0, n0>(A, sm, i, acc0);
    accumulate_blockrow<float, a1, n1>(A, sm, i, acc1);
  }
  // warp-specialised kernel: the scatter warps must have finished issuing the
  // previous tile from X (every compute warp takes this branch alike)
  if (wait_empty) bar_sync_all(kBarEmpty);
  // two-CTA variant: X overlays the force and tangent arrays, which every
  // warp must have finished reading (uniform over the block)
  if (block_sync) __syncthreads();
  const int base = e * 495 + P * 99 + i * 3;
#pragma unroll
  for (int j = 0; j < n0; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) X[base + j * 9 + k] = acc0[j][k];
#pragma unroll
  for (int j = 0; j < n1; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) X[base + (n0 + j) * 9 + k] = acc1[j][k];
}

__device__ __forceinline__ void tangent_xchg_scatter(const Args<float>& A, const TileMeta& mt, const float* X,
                                                     int64_t e0, int64_t real_end, int P, int i) {
  const int e = threadIdx.x & 31;
  if (e0 + e >= real_end) return;
  const int n0 = 10 - P;
  const float* xb = X + e * 495 + P * 99;
#pragma unroll 1
  for (int j = 0; j < 11; ++j) {
    const int a = j < n0 ? P : 9 - P;
    const int b = j < n0 ? P + j : 9 - P + (j - n0);
    const float* blkv = xb + j * 9;
    red_run(A, mt.rbase[a][e] + mt.rstr[a][e] * i + 3 * mt.blk[e][a * 10 + b], blkv[3 * i], blkv[3 * i + 1],
            blkv[3 * i + 2]);
    if (b != a)
      red_run(A, mt.rbase[b][e] + mt.rstr[b][e] * i + 3 * mt.blk[e][b * 10 + a], blkv[i], blkv[3 + i],
              blkv[6 + i]);
  }
}

// Sum of the contributions of one unordered pair of the tile map: the 3x3
// block of rows P, columns Q, from upper-triangle blocks of the exchange
// buffer X (as stored, or transposed when the element's block runs from Q to
// P), then one run of three reductions per row of (P, Q) and, for P != Q, per
// row of (Q, P) = (P, Q)^T.
template <typename CodeAt>
__device__ __forceinline__ void agg_pair(const Args<float>& A, const float* X, int4 s, int c0, int c1,
                                         CodeAt code_at) {
  float v[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = 0.0f;
#pragma unroll 1
  for (int c = c0; c < c1; ++c) {
    const int cd = code_at(c);
    const float* xb = X + (cd & 0x7fff);
    const int sd = (cd & 0x8000) ? 1 : 3, sk = (cd & 0x8000) ? 3 : 1;   // row / column strides
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int k = 0; k < 3; ++k) v[3 * d + k] += xb[d * sd + k * sk];
  }
  red_run(A, s.x, v[0], v[1], v[2]);
  red_run(A, s.x + s.y, v[3], v[4], v[5]);
  red_run(A, s.x + 2 * s.y, v[6], v[7], v[8]);
  if (s.z >= 0) {
    red_run(A, s.z, v[0], v[3], v[6]);
    red_run(A, s.z + s.w, v[1], v[4], v[7]);
    red_run(A, s.z + 2 * s.w, v[2], v[5], v[8]);
  }
}

// Aggregated scatter of one tile from the exchange buffer, map in global
// memory: thread -> unordered pair u (consecutive threads, consecutive CSR
// blocks of the rows P).  One sum per CSR block pair and tile instead of one
// reduction per element entry.
__device__ __forceinline__ void tangent_agg_scatter(const Args<float>& A, const float* X, int64_t tile) {
  const int nu = A.agg_nu[tile];
  const int4* slot = A.agg_slot + tile * kAggCap;
  const uint16_t* cptr = A.agg_cptr + tile * kAggCptrStride;
  const uint16_t* code = A.agg_code + tile * kAggCap;
#pragma unroll 1
  for (int u = threadIdx.x; u < nu; u += (int)blockDim.x)
    agg_pair(A, X, slot[u], cptr[u], cptr[u + 1], [&](int c) { return (int)code[c]; });
}

constexpr int kXFloats = 32 * 55 * 9;   // exchange buffer of the FP32 assembly

// Block rows a0 = P (b = P..9) and a1 = 9 - P (b = 9-P..9): 11 blocks, so the
// 15 warps cover the 55 blocks of the symmetric 30x30 exactly once.
template <typename T, int P>
__device__ __forceinline__ void tangent_rows(const Args<T>& A, const Smem<T>& sm, int64_t e0, int i) {
  tangent_blockrow<T, P, 10 - P>(A, sm, e0, i);
  tangent_blockrow<T, 9 - P, P + 1>(A, sm, e0, i);
}

// One tile of 32 elements starting at internal element e0, already staged in
// shared memory.  With a prefetch buffer P the next tile (first element
// e0_next >= 0) is fetched while this one computes.
template <typename T, int MAT, bool KV, bool DO_FORCE, bool DO_TANGENT, bool MERGE = false>
__device__ __forceinline__ void elem_tile(const Args<T>& A, unsigned char* smem_raw, int64_t e0,
                                          Prefetch<T>* P, int64_t e0_next) {
  Smem<T>& sm = *reinterpret_cast<Smem<T>*>(smem_raw);
  if (P && e0_next >= 0) prefetch_stage1(A, *P, e0_next);
  bool inverted = false;
  qp_phase<T, MAT, KV, DO_TANGENT>(A, sm, inverted);
  if (inverted && (e0 + (threadIdx.x & 31)) < A.real_end) atomicOr(A.flags, kFlagInverted);
  if (P) cp_async_wait_all();
  __syncthreads();
  if (P && e0_next >= 0) prefetch_stage2(A, *P);
  if (DO_FORCE) force_phase(A, sm, e0);
  if constexpr (DO_TANGENT) {
    const int w = threadIdx.x >> 5;
    const int p = w / 3, i = w % 3;
    if constexpr (std::is_same<T, float>::value) {
      if (A.xchg) {                    // kernel-argument test: uniform over the block
        const bool alias = A.x_alias != 0;
        float* X = reinterpret_cast<float*>(alias ? smem_raw + offsetof(Smem<float>, fq)
                                                  : smem_raw + sizeof(Smem<float>));
        switch (p) {                   // warp-uniform
          case 0: tangent_xchg_accumulate<0, MERGE>(A, sm, X, i, false, alias); break;
          case 1: tangent_xchg_accumulate<1, MERGE>(A, sm, X, i, false, alias); break;
          case 2: tangent_xchg_accumulate<2, MERGE>(A, sm, X, i, false, alias); break;
          case 3: tangent_xchg_accumulate<3, MERGE>(A, sm, X, i, false, alias); break;
          default: tangent_xchg_accumulate<4, MERGE>(A, sm, X, i, false, alias); break;
        }
        __syncthreads();               // reached by every thread of the block
        if (A.agg)
          tangent_agg_scatter(A, X, e0 / E);
        else
          tangent_xchg_scatter(A, sm.meta, X, e0, A.real_end, p, i);
        return;
      }
    }
    switch (p) {     // warp-uniform
      case 0: tangent_rows<T, 0>(A, sm, e0, i); break;
      case 1: tangent_rows<T, 1>(A, sm, e0, i); break;
      case 2: tangent_rows<T, 2>(A, sm, e0, i); break;
      case 3: tangent_rows<T, 3>(A, sm, e0, i); break;
      default: tangent_rows<T, 4>(A, sm, e0, i); break;
    }
  }
}

// ---------------------------------------------------------------------------
// Force-only pass (the residual's internal force): 5 warps, warp q evaluates
// quadrature point q of the tile's 32 elements (lanes) once and all three
// force rows, so the constitutive update is not repeated per row as in the
// 15-warp kernel, which splits the rows to spread the tangent work.  Small
// shared memory, one CTA per tile, several CTAs per SM.
// ---------------------------------------------------------------------------
constexpr int NTF = 160;

template <typename T>
struct SmemF {
  int32_t node[10][E];
  T geo[16][E];
  T u[kUStride * E];
  T vel[kUStride * E];
  T fq[kFStride * E];
};

template <typename T, int MAT, bool KV>
__device__ __forceinline__ void force_tile(const Args<T>& A, SmemF<T>& sm, int64_t e0) {
  const int tid = threadIdx.x;
  for (int t = tid; t < E * 10; t += NTF) {
    const int e = t / 10, a = t % 10;
    sm.node[a][e] = A.conn[(e0 + e) * 10 + a];
  }
  for (int t = tid; t < E * 16; t += NTF) {
    const int e = t / 16, c = t % 16;
    sm.geo[c][e] = A.geo[(e0 + e) * 16 + c];
  }
  __syncthreads();
  const double h = A.h;
  for (int t = tid; t < E * 30; t += NTF) {
    const int e = t / 30, c = t % 30;
    const int64_t g = 3 * (int64_t)sm.node[c / 3][e] + c % 3;
    const double vv = A.v[g];
    const double x = A.q_n[g] + h * vv;
    double u = x - A.X[g], vr = vv;
    if constexpr (std::is_same<T, dfl>::value) {
      // double-float: displacements and velocities relative to the element's
      // first node, formed in float64 (H = sum_a u_a n_a and Fdot = sum_a v_a n_a
      // are unchanged since sum_a n_a = 0), so the 48-bit significands carry the
      // small within-element differences instead of a large rigid motion
      const int64_t g0 = 3 * (int64_t)sm.node[0][e] + c % 3;
      const double v0 = A.v[g0];
      u -= (A.q_n[g0] + h * v0) - A.X[g0];
      vr -= v0;
    }
    sm.u[c * E + e] = T(u);
    sm.vel[c * E + e] = T(vr);
  }
  __syncthreads();
  const int q = tid >> 5, e = tid & 31;
  double Lq[4];
  qp_bary(q, Lq);
  const T wJ = T(qp_wfrac(q)) * sm.geo[12][e];
  T n[10][3];
  shape_grads(sm.geo, e, Lq, n);
  T Hm[3][3], Fd[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Hm[r][c] = 0;
      Fd[r][c] = 0;
    }
#pragma unroll
  for (int a = 0; a < 10; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const T ua = sm.u[(a * 3 + r) * E + e];
      T va = T(0);
      if (KV) va = sm.vel[(a * 3 + r) * E + e];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Hm[r][c] += ua * n[a][c];
        if (KV) Fd[r][c] += va * n[a][c];
      }
    }
  QP<T> s;
  bool inverted = false;
  constitutive<T, MAT, KV>(Hm, Fd, A.mat, s, inverted);
  if (inverted && e0 + e < A.real_end) atomicOr(A.flags, kFlagInverted);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T Pi[3];
#pragma unroll
    for (int J = 0; J < 3; ++J) {
      T acc = 0;
#pragma unroll
      for (int M = 0; M < 3; ++M) acc += s.F[i][M] * s.S[M][J];
      Pi[J] = acc * wJ;
    }
#pragma unroll
    for (int a = 0; a < 10; ++a)
      sm.fq[e * kFStride + q * 30 + a * 3 + i] = Pi[0] * n[a][0] + Pi[1] * n[a][1] + Pi[2] * n[a][2];
  }
  __syncthreads();
  // sum over the quadrature points and scatter (lanes = elements)
  for (int t = tid; t < E * 30; t += NTF) {
    const int c = t / E, ee = t % E;
    if (e0 + ee >= A.real_end) continue;
    T acc = 0;
#pragma unroll
    for (int qq = 0; qq < 5; ++qq) acc += sm.fq[ee * kFStride + qq * 30 + c];
    atomicAdd(&A.f[3 * (int64_t)sm.node[c / 3][ee] + c % 3], double(acc));
  }
}

// Segment table of one launch: the material segments of the internal element
// order (each a whole number of tiles), walked by one persistent grid.
constexpr int kMaxSeg = 64;

template <typename T>
struct SegEntry {
  int64_t begin;       // first internal element
  int64_t real_end;    // elements >= real_end are padding
  int32_t tile_end;    // cumulative tile count up to and including this segment
  int32_t combo;       // 2 * material kind + Kelvin-Voigt
  MatT<T> mat;
};

template <typename T>
struct SegTable {
  SegEntry<T> s[kMaxSeg];
  int32_t nseg;
  int32_t ntiles;
  int32_t perm_mul;    // tile k of the launch order is tile (k * perm_mul) mod ntiles (1: in order)
};

// Tile of launch-order position k (a bijection when gcd(perm_mul, ntiles) = 1).
template <typename T>
__device__ __forceinline__ int tile_at(const SegTable<T>& S, int k) {
  return S.perm_mul == 1 ? k : (int)(((int64_t)k * S.perm_mul) % S.ntiles);
}

// One tile through the kernel of its (material, Kelvin-Voigt) pair.
template <typename T, int COMBO, bool DO_FORCE, bool DO_TANGENT, bool MERGE = false>
__device__ __forceinline__ void dispatch_tile(const Args<T>& a, unsigned char* smem_raw, int64_t e0, int combo,
                                              Prefetch<T>* P, int64_t e0_next) {
  if constexpr (COMBO < 4) {
    elem_tile<T, COMBO / 2, (COMBO % 2) != 0, DO_FORCE, DO_TANGENT, MERGE>(a, smem_raw, e0, P, e0_next);
  } else {
    switch (combo) {                                 // block-uniform
      case 0: elem_tile<T, TL_SVK, false, DO_FORCE, DO_TANGENT, MERGE>(a, smem_raw, e0, P, e0_next); break;
      case 1: elem_tile<T, TL_SVK, true, DO_FORCE, DO_TANGENT, MERGE>(a, smem_raw, e0, P, e0_next); break;
      case 2: elem_tile<T, TL_MOONEY_RIVLIN, false, DO_FORCE, DO_TANGENT, MERGE>(a, smem_raw, e0, P, e0_next); break;
      default: elem_tile<T, TL_MOONEY_RIVLIN, true, DO_FORCE, DO_TANGENT, MERGE>(a, smem_raw, e0, P, e0_next); break;
    }
  }
}

// Walks the segment table forward (tile indices only grow).
struct SegWalk {
  int sg = 0, t_begin = 0;
  template <typename T>
  __device__ __forceinline__ int64_t e0(const SegTable<T>& S, int t) {
    while (t >= S.s[sg].tile_end) {                  // t < ntiles = tile_end of the last segment
      t_begin = S.s[sg].tile_end;
      ++sg;
    }
    return S.s[sg].begin + (int64_t)(t - t_begin) * E;
  }
};

// One CTA per tile; the tile's segment by a forward walk from the start.
template <typename T, int COMBO>
__global__ void __launch_bounds__(NTF) force_kernel(Args<T> A, SegTable<T> S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemF<T>& sm = *reinterpret_cast<SmemF<T>*>(smem_raw);
  const int t = blockIdx.x;
  if (t >= S.ntiles) return;
  SegWalk w;
  const int64_t e0 = w.e0(S, t);
  Args<T> a = A;
  a.mat = S.s[w.sg].mat;
  a.real_end = S.s[w.sg].real_end;
  if constexpr (COMBO < 4) {
    force_tile<T, COMBO / 2, (COMBO % 2) != 0>(a, sm, e0);
  } else {
    switch (S.s[w.sg].combo) {                       // block-uniform
      case 0: force_tile<T, TL_SVK, false>(a, sm, e0); break;
      case 1: force_tile<T, TL_SVK, true>(a, sm, e0); break;
      case 2: force_tile<T, TL_MOONEY_RIVLIN, false>(a, sm, e0); break;
      default: force_tile<T, TL_MOONEY_RIVLIN, true>(a, sm, e0); break;
    }
  }
}


// Persistent element kernel: CTA b starts with tile b and then takes the next
// unprocessed tile from a device counter (zeroed before the launch), so SMs
// that run faster take more tiles; with counter == nullptr it takes tiles
// b + gridDim.x, b + 2 gridDim.x, ...  Tiles ascend in every CTA, so the
// segment of a tile is found by walking the table forward.  COMBO < 4
// compiles one (material, Kelvin-Voigt) pair, COMBO = 4 all four with a
// block-uniform dispatch per tile (multi-material meshes and batches).  The
// float32 kernels prefetch the next tile (A.pf_off >= 0).  MINB = 2 caps the
// registers at 64 so that two CTAs share an SM (with the exchange buffer
// overlaid on the force and tangent arrays and no prefetch, 105 KB each): the
// latency of one CTA's staging hides behind the other's arithmetic.
template <typename T, int COMBO, bool DO_FORCE, bool DO_TANGENT, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) elem_kernel(Args<T> A, SegTable<T> S, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next;
  Smem<T>& sm = *reinterpret_cast<Smem<T>*>(smem_raw);
  Prefetch<T>* P = A.pf_off >= 0 ? reinterpret_cast<Prefetch<T>*>(smem_raw + A.pf_off) : nullptr;
  // k counts positions of the launch order; tile_at maps them to tiles.  In
  // order (perm_mul = 1) the segment walk only moves forward; with a
  // permutation every tile's segment is walked from the start (<= 64 entries).
  const bool in_order = S.perm_mul == 1;
  SegWalk cur, nxt;
  int k = blockIdx.x;
  if (k >= S.ntiles) return;                         // uniform over the block
  int64_t e0 = cur.e0(S, tile_at(S, k));
  load_tile<T, DO_TANGENT>(A, sm, e0, sm.meta);
  if (threadIdx.x == 0) s_next = counter ? (int)gridDim.x + atomicAdd(counter, 1) : k + (int)gridDim.x;
  __syncthreads();
  while (true) {
    const int k_next = s_next;
    Args<T> a = A;
    a.mat = S.s[cur.sg].mat;
    a.real_end = S.s[cur.sg].real_end;
    nxt = in_order ? cur : SegWalk();
    const int64_t e0_next = (P && k_next < S.ntiles) ? nxt.e0(S, tile_at(S, k_next)) : -1;
    dispatch_tile<T, COMBO, DO_FORCE, DO_TANGENT, (MINB == 1)>(a, smem_raw, e0, S.s[cur.sg].combo, P, e0_next);
    if (P) cp_async_wait_all();
    __syncthreads();                                 // this tile's shared data is consumed
    if (k_next >= S.ntiles) break;
    if (threadIdx.x == 0) s_next = counter ? (int)gridDim.x + atomicAdd(counter, 1) : k_next + (int)gridDim.x;
    k = k_next;
    if (P) {
      cur = nxt;
      e0 = e0_next;
      unpack_tile<T, DO_TANGENT>(A, sm, *P, sm.meta);  // ends with a barrier (also publishes s_next)
    } else {
      if (!in_order) cur = SegWalk();
      e0 = cur.e0(S, tile_at(S, k));
      load_tile<T, DO_TANGENT>(A, sm, e0, sm.meta);    // ends with a barrier (also publishes s_next)
    }
  }
}

// ---------------------------------------------------------------------------
// Warp-specialised float32 CSR assembly: 15 compute warps as above and 5
// scatter warps.  The compute warps stage, evaluate and accumulate tile k and
// park its blocks in X; the scatter warps issue tile k's reductions from X
// while the compute warps already evaluate tile k + 1, so the L2 reduction
// traffic overlaps the arithmetic instead of following it.  Hand-off of X by
// named barriers (every arrive is matched by exactly one sync):
//   compute, tile k >= 1: bar.sync EMPTY (tile k - 1 issued), write X(k),
//                         bar.arrive FULL;  after the last tile n - 1: bar.sync
//                         EMPTY, mark the end, bar.arrive FULL  (n + 1 FULL
//                         arrives, n EMPTY syncs)
//   scatter, k = 0, 1, ...: bar.sync FULL; stop at the end mark; issue tile k;
//                         bar.arrive EMPTY  (n + 1 FULL syncs, n EMPTY arrives)
// The scatter metadata (row bases, strides, slot blocks) of consecutive tiles
// alternate between two buffers, so staging tile k + 1 does not disturb the
// scatter of tile k.
// ---------------------------------------------------------------------------
template <int MAT, bool KV, bool DO_FORCE>
__device__ __forceinline__ void ws_tile(const Args<float>& A, unsigned char* smem_raw, float* X,
                                        Prefetch<float>* P, int64_t e0, int64_t e0_next, bool wait_empty) {
  Smem<float>& sm = *reinterpret_cast<Smem<float>*>(smem_raw);
  if (e0_next >= 0) prefetch_stage1(A, *P, e0_next);
  bool inverted = false;
  qp_phase<float, MAT, KV, true>(A, sm, inverted);
  if (inverted && (e0 + (threadIdx.x & 31)) < A.real_end) atomicOr(A.flags, kFlagInverted);
  cp_async_wait_all();
  bar_compute<true>();
  if (e0_next >= 0) prefetch_stage2(A, *P);
  if (DO_FORCE) force_phase(A, sm, e0);
  const int w = threadIdx.x >> 5;
  const int p = w / 3, i = w % 3;
  switch (p) {                                       // warp-uniform
    case 0: tangent_xchg_accumulate<0>(A, sm, X, i, wait_empty); break;
    case 1: tangent_xchg_accumulate<1>(A, sm, X, i, wait_empty); break;
    case 2: tangent_xchg_accumulate<2>(A, sm, X, i, wait_empty); break;
    case 3: tangent_xchg_accumulate<3>(A, sm, X, i, wait_empty); break;
    default: tangent_xchg_accumulate<4>(A, sm, X, i, wait_empty); break;
  }
}

template <int COMBO, bool DO_FORCE>
__device__ __forceinline__ void ws_dispatch(const Args<float>& a, unsigned char* smem_raw, float* X,
                                            Prefetch<float>* P, int64_t e0, int64_t e0_next, bool wait_empty,
                                            int combo) {
  if constexpr (COMBO < 4) {
    ws_tile<COMBO / 2, (COMBO % 2) != 0, DO_FORCE>(a, smem_raw, X, P, e0, e0_next, wait_empty);
  } else {
    switch (combo) {                                 // block-uniform
      case 0: ws_tile<TL_SVK, false, DO_FORCE>(a, smem_raw, X, P, e0, e0_next, wait_empty); break;
      case 1: ws_tile<TL_SVK, true, DO_FORCE>(a, smem_raw, X, P, e0, e0_next, wait_empty); break;
      case 2: ws_tile<TL_MOONEY_RIVLIN, false, DO_FORCE>(a, smem_raw, X, P, e0, e0_next, wait_empty); break;
      default: ws_tile<TL_MOONEY_RIVLIN, true, DO_FORCE>(a, smem_raw, X, P, e0, e0_next, wait_empty); break;
    }
  }
}

template <int COMBO, bool DO_FORCE>
__global__ void __launch_bounds__(NTW, 1) elem_kernel_ws(Args<float> A, SegTable<float> S, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next;
  __shared__ long long s_e0[2], s_end[2];
  Smem<float>& sm = *reinterpret_cast<Smem<float>*>(smem_raw);
  float* X = reinterpret_cast<float*>(smem_raw + sizeof(Smem<float>));
  Prefetch<float>* P = reinterpret_cast<Prefetch<float>*>(smem_raw + A.pf_off);
  TileMeta* meta1 = reinterpret_cast<TileMeta*>(smem_raw + A.meta_off);
  int t = blockIdx.x;
  if (t >= S.ntiles) return;                         // uniform over the block
  const int warp = threadIdx.x >> 5;
  if (warp >= NWARP) {                               // scatter warps: block-row pair warp - 15
    const int sp = warp - NWARP;
    for (int k = 0;; ++k) {
      bar_sync_all(kBarFull);
      const int par = k & 1;
      const long long e0 = s_e0[par];
      if (e0 < 0) break;
      const TileMeta& mt = par ? *meta1 : sm.meta;
      const long long end = s_end[par];
      for (int i = 0; i < 3; ++i) tangent_xchg_scatter(A, mt, X, e0, end, sp, i);
      bar_arrive_all(kBarEmpty);
    }
    return;
  }
  SegWalk cur, nxt;
  int64_t e0 = cur.e0(S, t);
  load_tile<float, true, true>(A, sm, e0, sm.meta);
  if (threadIdx.x == 0) s_next = counter ? (int)gridDim.x + atomicAdd(counter, 1) : t + (int)gridDim.x;
  bar_compute<true>();
  int k = 0;
  for (;; ++k) {
    const int par = k & 1;
    const int t_next = s_next;
    Args<float> a = A;
    a.mat = S.s[cur.sg].mat;
    a.real_end = S.s[cur.sg].real_end;
    nxt = cur;
    const int64_t e0_next = t_next < S.ntiles ? nxt.e0(S, t_next) : -1;
    ws_dispatch<COMBO, DO_FORCE>(a, smem_raw, X, P, e0, e0_next, k > 0, S.s[cur.sg].combo);
    if (threadIdx.x == 0) {
      s_e0[par] = e0;
      s_end[par] = a.real_end;
    }
    bar_arrive_all(kBarFull);                        // X and the tile's scatter data are ready
    cp_async_wait_all();
    bar_compute<true>();                             // the next tile's prefetch has landed
    if (t_next >= S.ntiles) break;
    if (threadIdx.x == 0) s_next = counter ? (int)gridDim.x + atomicAdd(counter, 1) : t_next + (int)gridDim.x;
    t = t_next;
    cur = nxt;
    e0 = e0_next;
    unpack_tile<float, true, true>(A, sm, *P, par ? sm.meta : *meta1);   // ends with a compute barrier
  }
  bar_sync_all(kBarEmpty);                           // the last tile has been issued
  if (threadIdx.x == 0) s_e0[(k + 1) & 1] = -1;
  bar_arrive_all(kBarFull);
}

// The closed-form pair kernel of SVK (+ KV) segments, float32 element form
// (tl_element_pair.cu): one persistent launch over the segments of S.
tl_status pair_launch(tl_mesh* m, const Args<float>& A, const SegTable<float>& S, bool kv, bool do_force,
                      int* counter);
tl_status pair_prep(tl_mesh* m, const double* q_n, const double* v, double h);

template <typename T, bool DO_FORCE, bool DO_TANGENT>
tl_status launch_all(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                     double mass_scale, double* f, void* values, void* K_elem) {
  // the force-only variant does not need the tangent array (last member);
  // the FP32 CSR assembly adds its exchange buffer after the struct
  const bool xchg = std::is_same<T, float>::value && DO_TANGENT && values && !K_elem && m->tune.elem_xchg;
  size_t smem = DO_TANGENT ? sizeof(Smem<T>) + (xchg ? sizeof(float) * kXFloats : 0)
                           : offsetof(Smem<T>, A);
  // the warp-specialised float32 assembly keeps a second scatter-metadata
  // buffer; the float32 kernels prefetch the next tile into a buffer after
  // the rest
  const bool ws = xchg && m->tune.elem_prefetch && m->tune.elem_ws && !m->tune.elem_full_grid;
  int meta_off = -1, pf_off = -1;
  if (ws) {
    smem = (smem + 15) / 16 * 16;
    meta_off = (int)smem;
    smem += sizeof(TileMeta);
  }
  if (std::is_same<T, float>::value && m->tune.elem_prefetch) {
    smem = (smem + 15) / 16 * 16;
    pf_off = (int)smem;
    smem += sizeof(Prefetch<T>);
  }
  Args<T> A;
  A.conn = m->d_conn;
  A.geo = std::is_same<T, float>::value ? reinterpret_cast<const T*>(m->d_geo32)
          : std::is_same<T, dfl>::value   ? reinterpret_cast<const T*>(m->d_geo_df)
                                          : reinterpret_cast<const T*>(m->d_geo64);
  A.blk = m->d_blk;
  A.node_ptr = m->d_node_ptr;
  A.user_of = m->d_user_of;
  A.q_n = q_n;
  A.v = v;
  A.X = m->d_X;
  A.h = h;
  A.real_end = 0;
  A.mat = MatT<T>{};
  A.alpha = T(alpha);
  A.beta = T(beta);
  A.mass_scale = T(mass_scale);
  A.f = f;
  A.values = reinterpret_cast<T*>(values);
  A.K_elem = reinterpret_cast<T*>(K_elem);
  A.flags = m->d_flags;
  A.nnz = (int32_t)m->nnz;
  A.v4_ok = ((reinterpret_cast<uintptr_t>(values) & 15u) == 0) ? 1 : 0;
  A.xchg = xchg ? 1 : 0;
  A.pf_off = pf_off;
  A.meta_off = meta_off;
  A.x_alias = 0;
  // per-tile aggregation: exchanged float32 assembly without warp
  // specialisation, once the maps exist (built by the autotuner or tl_tune_set)
  A.agg = (xchg && !ws && m->tune.elem_agg && m->agg_nu) ? 1 : 0;
  A.agg_slot = m->agg_slot;
  A.agg_cptr = m->agg_cptr;
  A.agg_code = m->agg_code;
  A.agg_nu = m->agg_nu;
  A.uv = nullptr;
  // float32 tangent passes: SVK segments go to the closed-form pair kernel
  // (CSR values through the tile maps, or K_elem), in launches of their own
  const bool pair_mode = std::is_same<T, float>::value && DO_TANGENT && m->tune.elem_pair &&
                         ((K_elem && !values) || (values && !K_elem && m->tune.elem_agg && m->agg_nu));
  cudaEvent_t t0 = timer_open(m);
  if constexpr (std::is_same<T, float>::value) {
    if (pair_mode) {
      // the pair kernel gathers float32 {u, v} per DOF, formed here once per pass
      // instead of once per element that shares the node
      bool any_svk = false;
      for (const Segment& sg : m->segs) any_svk = any_svk || (m->mats[sg.mat].kind == TL_SVK && sg.padded_end > sg.begin);
      if (any_svk) {
        if (!m->d_uv32) return fail(m, TL_ERR_INVALID_ARG, "pair kernel without its float32 nodal buffer");
        TL_TRY(pair_prep(m, q_n, v, h));
        A.uv = m->d_uv32;
      }
    }
  }
  // Segments in groups of at most kMaxSeg, one persistent launch per group.
  // The float32 kernels include an all-materials variant; the float64 ones
  // (heavier, compiled per material) take one launch per run of segments of
  // the same (material, Kelvin-Voigt) pair.
  constexpr bool kMixed = std::is_same<T, float>::value;
  int nlaunch = 0;
  // pair mode: the SVK segments of all bodies first (pair kernel), then the
  // Mooney-Rivlin ones (generic kernel), each in as few launches as possible
  for (int pass = 0; pass < (pair_mode ? 2 : 1); ++pass) {
  size_t k = 0;
  while (k < m->segs.size()) {
    SegTable<T> S;
    S.nseg = 0;
    S.ntiles = 0;
    S.perm_mul = 1;
    int combo0 = -1;
    bool mixed = false;
    for (; k < m->segs.size() && S.nseg < kMaxSeg; ++k) {
      const Segment& sg = m->segs[k];
      const int64_t nt = (sg.padded_end - sg.begin) / E;
      if (nt == 0) continue;
      const MaterialDev& md = m->mats[sg.mat];
      const int combo = 2 * (md.kind == TL_SVK ? 0 : 1) + (md.kv ? 1 : 0);
      if (pair_mode && (combo < 2) != (pass == 0)) continue;   // the other pass's kind
      if (!kMixed && combo0 >= 0 && combo != combo0) break;   // next launch starts here
      SegEntry<T>& se = S.s[S.nseg++];
      se.begin = sg.begin;
      se.real_end = sg.end;
      S.ntiles += (int32_t)nt;
      se.tile_end = S.ntiles;
      se.combo = combo;
      se.mat = to_matT<T>(md);
      if (combo0 < 0) combo0 = combo;
      mixed = mixed || combo != combo0;
    }
    if (S.ntiles == 0) continue;
    if constexpr (DO_FORCE && !DO_TANGENT) {
      void (*fkern)(Args<T>, SegTable<T>) = nullptr;
      switch (mixed ? 4 : combo0) {
        case 0: fkern = force_kernel<T, 0>; break;
        case 1: fkern = force_kernel<T, 1>; break;
        case 2: fkern = force_kernel<T, 2>; break;
        case 3: fkern = force_kernel<T, 3>; break;
        default:
          if constexpr (kMixed) fkern = force_kernel<T, 4>;
          break;
      }
      if (!fkern) return fail(m, TL_ERR_UNSUPPORTED, "force kernel selection");
      const size_t fsmem = sizeof(SmemF<T>);
      TL_CUDA(m, cudaFuncSetAttribute(fkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));
      fkern<<<(unsigned)S.ntiles, NTF, fsmem, m->stream>>>(A, S);
      TL_CUDA(m, cudaGetLastError());
      ++m->launches;
      continue;
    } else {   // the 15-warp kernels (not instantiated for force-only passes)
    if constexpr (std::is_same<T, float>::value) {
      if (pair_mode && combo0 < 2) {
        bool kv = false;
        for (int j = 0; j < S.nseg; ++j) kv = kv || S.s[j].combo == 1;
        int* counter = nlaunch < kTileCounters ? m->d_tile_counters + nlaunch : nullptr;
        ++nlaunch;
        TL_TRY(pair_launch(m, A, S, kv, DO_FORCE, counter));
        continue;
      }
    }
    void (*kern)(Args<T>, SegTable<T>, int*) = nullptr;
    int threads = NT;
    if constexpr (std::is_same<T, float>::value && DO_TANGENT) {
      if (ws) {
        threads = NTW;
        switch (mixed ? 4 : combo0) {
          case 0: kern = elem_kernel_ws<0, DO_FORCE>; break;
          case 1: kern = elem_kernel_ws<1, DO_FORCE>; break;
          case 2: kern = elem_kernel_ws<2, DO_FORCE>; break;
          case 3: kern = elem_kernel_ws<3, DO_FORCE>; break;
          default: kern = elem_kernel_ws<4, DO_FORCE>; break;
        }
      }
    }
    // two CTAs per SM (registers capped at 64; the exchange buffer overlays
    // the force and tangent arrays; no prefetch buffer): one material kind only
    Args<T> Al = A;
    size_t smem_l = smem;
    if constexpr (std::is_same<T, float>::value && DO_TANGENT) {
      if (!kern && xchg && m->tune.elem_occ2 && !mixed) {
        Al.x_alias = 1;
        Al.pf_off = -1;
        Al.meta_off = -1;
        smem_l = sizeof(Smem<T>);
        switch (combo0) {
          case 0: kern = elem_kernel<T, 0, DO_FORCE, DO_TANGENT, 2>; break;
          case 1: kern = elem_kernel<T, 1, DO_FORCE, DO_TANGENT, 2>; break;
          case 2: kern = elem_kernel<T, 2, DO_FORCE, DO_TANGENT, 2>; break;
          default: kern = elem_kernel<T, 3, DO_FORCE, DO_TANGENT, 2>; break;
        }
      }
    }
    if (!kern) switch (mixed ? 4 : combo0) {
      case 0: kern = elem_kernel<T, 0, DO_FORCE, DO_TANGENT>; break;
      case 1: kern = elem_kernel<T, 1, DO_FORCE, DO_TANGENT>; break;
      case 2: kern = elem_kernel<T, 2, DO_FORCE, DO_TANGENT>; break;
      case 3: kern = elem_kernel<T, 3, DO_FORCE, DO_TANGENT>; break;
      default:
        if constexpr (kMixed) kern = elem_kernel<T, 4, DO_FORCE, DO_TANGENT>;
        break;
    }
    if (!kern) return fail(m, TL_ERR_UNSUPPORTED, "element kernel selection");
    TL_CUDA(m, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_l));
    int occ = 1;
    TL_CUDA(m, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem_l));
    const bool full = m->tune.elem_full_grid != 0;
    const int grid = full ? S.ntiles : (int)std::min<int64_t>(S.ntiles, (int64_t)m->num_sms * std::max(occ, 1));
    // spread: tiles in flight at the same time lie ~ntiles/grid apart, so their
    // reductions go to distant CSR rows (the warp-specialised kernel keeps order)
    if (m->tune.elem_spread && !full && threads == NT && S.ntiles > 2 * grid) {
      int mul = (S.ntiles + grid - 1) / grid;
      auto gcd = [](int a, int b) { while (b) { const int r = a % b; a = b; b = r; } return a; };
      while (gcd(mul, S.ntiles) != 1) ++mul;
      S.perm_mul = mul;
    }
    int* counter = nullptr;
    if (!full && nlaunch < kTileCounters) {
      counter = m->d_tile_counters + nlaunch;
      TL_CUDA(m, cudaMemsetAsync(counter, 0, sizeof(int), m->stream));
    }
    ++nlaunch;
    kern<<<(unsigned)grid, (unsigned)threads, smem_l, m->stream>>>(Al, S, counter);
    TL_CUDA(m, cudaGetLastError());
    ++m->launches;
    }
  }
  }
  timer_close(m, t0, kTimeElement);
  return TL_OK;
}

}  // namespace elem
}  // namespace tl
