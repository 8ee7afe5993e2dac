// Closed-form pair kernel of the float32 element form for St. Venant-Kirchhoff
// (+ Kelvin-Voigt): internal force, the 30x30 tangent h K_t + D + M/h and
// its aggregated scatter into the fixed-pattern CSR Hessian.
//
// Paper: arxiv 2604.10357
//   Sec. 4.3  eq. F_assembly, eq. fint_local (the force)
//   Sec. 4.4  eq. tangent_block: [K_ab]_ik = sum_q A_iJkL n_aJ n_bL wJ0
//
// For SVK (+ KV) the contraction of eq. tangent_block with the shape-function
// gradients has a closed form per node pair (a, b) and quadrature point:
//   [K_ab]_ik = wJ0 [ c1 g_a,i g_b,k + c2 (g_b,i g_a,k + (n_a.n_b) B_ik)
//                     + alpha delta_ik n_a.S n_b ]
// with g_a = F n_a, B = F F^T, S = S_el + S_v, c1 = alpha lambda + beta
// lambda_d and c2 = alpha mu + beta eta (alpha K_t + beta D, the Newton
// matrix h K_t + D with the viscous geometric term in K_t).  Each block costs
// 36 multiply-adds per point from vectors held in registers, instead of the
// 27-entry tangent row the generic kernel contracts with n_a and n_b from
// shared memory for every block row.
//
// Folded form (FOLD): c1 and c2 are constant over the element, so with
// P_ab = sum_q wJ0 g_a g_b^T the two rank-one terms are c1 P_ab + c2 P_ab^T,
// and the B and identity terms M_ab (symmetric) satisfy
// c1 M + c2 M^T = (c1 + c2) M.  The kernel therefore accumulates
//   Q_ab = sum_q [ wJ0 g_a g_b^T + (n_a.n_b) Bh' + (n_a.t') I ],
//   Bh' = c2 wJ0 B / (c1 + c2),  t' = alpha wJ0 S n_b / (c1 + c2),
// and forms K_ab = c1 Q_ab + c2 Q_ab^T once per tile: 27 instructions per
// block and point instead of 36, with the same 9 accumulators.  The host
// takes it only where c1 + c2 is not small against c1 and c2 (no
// cancellation); otherwise the unfolded form runs.
//
// Layout: a CTA of 192 threads, lanes = the 32 elements of a tile; warps 0-4
// compute, warp 5 helps to stage and scatter.
//   phase A, warp q: the kinematics and the constitutive update at point q;
//            it stores n_a (10 x float4), F, wJ0 S, c2 wJ0 B and wJ0 per
//            (element, point) in shared memory;
//   phase C, warp t: the 11 blocks of one round of a 5-team round robin over
//            node pairs {2t, 2t+1}: its own pair (3 blocks) and the 4 blocks
//            against each of the pairs t+1 and t+2 (mod 5), so the 5 warps
//            form the 55 blocks of the symmetric 30x30 exactly once with 11
//            blocks each; the accumulators stay in registers over the 5
//            points, and the force of nodes 2t, 2t+1 falls out of the same
//            vectors (f_a = sum_q F (wJ0 S n_a));
//   then the blocks go to the exchange buffer (the layout of the tile maps)
//   and the tile's distinct node pairs are reduced into the CSR values once
//   per tile (tangent_agg_scatter), or written to K_elem.
// The next tile's connectivity and geometry and the current tile's map are
// copied into shared memory with cp.async while the tile computes.  The nodal
// inputs are float32 {u = q_n + h v - X, v} per DOF, formed once per pass
// (pair_prep), so the kernel itself runs no float64 arithmetic, only a few
// conversions (a point's barycentric coordinates, and its nodal forces for
// the float64 force vector).
#include "tl_element_impl.cuh"

namespace tl {
namespace elem {
namespace {

constexpr int NTP = 192;          // threads per CTA (warps 0-4 compute; any further warps stage and scatter)
static_assert(NTP % 32 == 0 && NTP >= 160, "five compute warps");

// Wait until at most N of this thread's most recent cp.async groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// Per-element strides (floats) of the point data, chosen so that the eight
// lanes of a 16-byte shared-memory phase fall on distinct bank quads:
// 124 = 28 (mod 32), 204 = 12 (mod 32).
constexpr int kQd = 24;           // F (9), wJ0 S (6), c2 wJ0 B (6), wJ0, pad
constexpr int kQStride = 5 * kQd + 4;
constexpr int kNv = 40;           // 10 nodes x float4 (n_a, 0)
constexpr int kNvStride = 5 * kNv + 4;

// u and vel stay outside the exchange buffer, so the next tile's nodal data
// can be stored while other warps still scatter this tile.
struct SmemP {
  int32_t node[10][E];
  float geo[16][E];
  float u[30 * E];
  float vel[30 * E];
  union {
    struct {
      float qd[E * kQStride];
      float nv[E * kNvStride];
    } a;
    float X[kXFloats];            // exchange buffer, after the point data is consumed
  } r;
};

// The tile's aggregation map (tl_tilemap.cu), copied into shared memory with
// cp.async while the tile computes, so the scatter reads no global memory
// but the CSR values.
struct MapP {
  int4 slot[kAggCap];
  uint16_t cptr[kAggCptrStride];
  uint16_t code[kAggCap];
};

// Prefetch of the next tile: its connectivity, geometry and map size.
struct PrefP {
  int32_t conn[E * 10];
  float geo[E * 16];
  int32_t nu;
  int32_t pad[3];
};

// Nodal data of the 30 element DOFs of a tile, one thread's share: {u, v}
// of DOF (c, e) for t = threadIdx.x + j NTP, c = t / 32, e = t % 32, from the
// float32 array that pair_prep forms once per pass; the node of (c, e) is
// conn_rows[e][c / 3] (element-major rows).  The loads of the next tile are
// issued before the current tile's scatter and consumed after it, so their
// latency hides behind the reductions.
constexpr int kNodalIt = E * 30 / NTP;
static_assert(E * 30 % NTP == 0 && NTP % E == 0, "nodal gather");
struct NodalRegs {
  float2 uv[kNodalIt];
};

__device__ __forceinline__ void nodal_load(const Args<float>& A, const int32_t* conn_rows, NodalRegs& r) {
#pragma unroll
  for (int j = 0; j < kNodalIt; ++j) {
    const int c = (int)(threadIdx.x >> 5) + j * (NTP / E), e = threadIdx.x & 31;
    const int64_t g = 3 * (int64_t)conn_rows[e * 10 + c / 3] + c % 3;
    r.uv[j] = A.uv[g];
  }
}

template <bool KV>
__device__ __forceinline__ void nodal_store(SmemP& sm, const NodalRegs& r) {
#pragma unroll
  for (int j = 0; j < kNodalIt; ++j) {
    const int t = threadIdx.x + j * NTP;
    sm.u[t] = r.uv[j].x;
    if (KV) sm.vel[t] = r.uv[j].y;
  }
}

// Per DOF: u = q_n + h v - X formed in float64, then rounded to float32, and
// v rounded to float32 (the pair kernel's nodal inputs).
__global__ void uv32_kernel(const double* __restrict__ q_n, const double* __restrict__ v,
                            const double* __restrict__ X, double h, int64_t n, float2* __restrict__ uv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = v[i];
    uv[i] = make_float2(float(q_n[i] + h * vi - X[i]), float(vi));
  }
}

// First tile of a CTA, from global memory.
template <bool KV>
__device__ __forceinline__ void load_tile_p(const Args<float>& A, SmemP& sm, int64_t e0) {
  const int tid = threadIdx.x;
  for (int t = tid; t < E * 10; t += NTP) {
    const int e = t / 10, a = t % 10;
    sm.node[a][e] = A.conn[(e0 + e) * 10 + a];
  }
  for (int t = tid; t < E * 16; t += NTP) {
    const int e = t / 16, c = t % 16;
    sm.geo[c][e] = A.geo[(e0 + e) * 16 + c];
  }
  NodalRegs r;
  nodal_load(A, A.conn + e0 * 10, r);
  nodal_store<KV>(sm, r);
  __syncthreads();
}

// Prefetch of tile e0: its conn rows (1,280 B) and geometry (2,048 B),
// contiguous and 16-byte aligned (tiles start at multiples of 32 elements of
// arrays from cudaMalloc), and its map size.
__device__ __forceinline__ void pf_stage1(const Args<float>& A, PrefP& P, int64_t e0) {
  const unsigned char* c = reinterpret_cast<const unsigned char*>(A.conn + e0 * 10);
  const unsigned char* g = reinterpret_cast<const unsigned char*>(A.geo + e0 * 16);
  constexpr int nc = E * 10 * 4 / 16, ng = E * 16 * 4 / 16;
  for (int k = threadIdx.x; k < nc + ng; k += NTP) {
    if (k < nc) cp_async16(reinterpret_cast<unsigned char*>(P.conn) + 16 * k, c + 16 * k);
    else cp_async16(reinterpret_cast<unsigned char*>(P.geo) + 16 * (k - nc), g + 16 * (k - nc));
  }
  if (A.values && threadIdx.x == NTP - 1) cp_async4(&P.nu, A.agg_nu + e0 / E);
  cp_async_commit();
}

// The map of tile `tile` with nu (<= kAggCap) distinct pairs: slot[0, nu),
// cptr[0, nu] and the kAggCap contribution codes, in 16-byte pieces (every
// row starts on a 16-byte boundary; the last piece of cptr may carry unused
// entries of the same row).
__device__ __forceinline__ void map_copy(const Args<float>& A, MapP& M, int64_t tile, int nu) {
  const unsigned char* s = reinterpret_cast<const unsigned char*>(A.agg_slot + tile * kAggCap);
  const unsigned char* c = reinterpret_cast<const unsigned char*>(A.agg_cptr + tile * kAggCptrStride);
  const unsigned char* d = reinterpret_cast<const unsigned char*>(A.agg_code + tile * kAggCap);
  const int ns = nu, nc = (nu + 8) / 8;
  constexpr int nd = kAggCap * 2 / 16;
  static_assert(kAggCap * 2 % 16 == 0 && kAggCptrStride % 8 == 0, "map rows of whole 16-byte pieces");
  for (int k = threadIdx.x; k < ns + nc + nd; k += NTP) {
    if (k < ns) cp_async16(reinterpret_cast<unsigned char*>(M.slot) + 16 * k, s + 16 * k);
    else if (k < ns + nc) cp_async16(reinterpret_cast<unsigned char*>(M.cptr) + 16 * (k - ns), c + 16 * (k - ns));
    else cp_async16(reinterpret_cast<unsigned char*>(M.code) + 16 * (k - ns - nc), d + 16 * (k - ns - nc));
  }
  cp_async_commit();
}

// Next tile from the prefetch buffer and the nodal data loaded ahead.
template <bool KV>
__device__ __forceinline__ void unpack_p(const Args<float>& A, SmemP& sm, const PrefP& P, const NodalRegs& r) {
  const int tid = threadIdx.x;
  for (int t = tid; t < E * 10; t += NTP) {
    const int a = t / E, e = t % E;
    sm.node[a][e] = P.conn[e * 10 + a];
  }
  for (int t = tid; t < E * 16; t += NTP) {
    const int e = t / 16, c = t % 16;
    sm.geo[c][e] = P.geo[t];
  }
  nodal_store<KV>(sm, r);
  __syncthreads();
}

// values[s .. s+2] += (x0, x1, x2) as two reductions: an 8-byte one on the
// even-aligned pair and a 4-byte one on the other entry.  values comes from
// cudaMalloc (8-byte aligned) and the run lies inside it.
__device__ __forceinline__ void red3(float* values, int s, float x0, float x1, float x2) {
  const bool odd = (s & 1) != 0;          // selects, not branches: lanes of a warp differ
  float* p = values + s;
  red_v2(p + (odd ? 1 : 0), odd ? x1 : x0, odd ? x2 : x1);
  atomicAdd(p + (odd ? 0 : 2), odd ? x0 : x2);
}

// Aggregated scatter from the exchange buffer with the tile's map in shared
// memory: thread -> unordered node pair u (consecutive threads, consecutive
// CSR blocks), its block of rows P summed once over the contributing element
// blocks (as stored, or transposed), then reduced into both (P, Q) and, for
// P != Q, (Q, P) = (P, Q)^T.
__device__ __forceinline__ void map_scatter(const Args<float>& A, const float* X, const MapP& M, int nu) {
  float* vals = A.values;
#pragma unroll 1
  for (int u = threadIdx.x; u < nu; u += NTP) {
    const int4 s = M.slot[u];
    const int c0 = M.cptr[u], c1 = M.cptr[u + 1];
    float v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = 0.0f;
#pragma unroll 2
    for (int c = c0; c < c1; ++c) {
      const int cd = M.code[c];
      const float* xb = X + (cd & 0x7fff);
      const bool tr = (cd & 0x8000) != 0;   // the block runs from Q to P: add its transpose
      float x[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) x[k] = xb[k];
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int k = 0; k < 3; ++k) v[3 * d + k] += (d == k || !tr) ? x[3 * d + k] : x[3 * k + d];
    }
    red3(vals, s.x, v[0], v[1], v[2]);
    red3(vals, s.x + s.y, v[3], v[4], v[5]);
    red3(vals, s.x + 2 * s.y, v[6], v[7], v[8]);
    if (s.z >= 0) {
      red3(vals, s.z, v[0], v[3], v[6]);
      red3(vals, s.z + s.w, v[1], v[4], v[7]);
      red3(vals, s.z + 2 * s.w, v[2], v[5], v[8]);
    }
  }
}

// Phase A, warp q, lane e: shape gradients, F = I + H, the SVK (+ KV)
// stress, and the per-point data of phase C.
// bscale: the factor of wJ0 B stored for phase C (c2, or c2 / (c1 + c2) folded).
template <bool KV>
__device__ __forceinline__ void phase_a(const MatT<float>& mat, float bscale, SmemP& sm, bool& inverted) {
  const int q = threadIdx.x >> 5, e = threadIdx.x & 31;
  double Lq[4];
  qp_bary(q, Lq);
  const float wJ = float(qp_wfrac(q)) * sm.geo[12][e];
  float n[10][3];
  shape_grads(sm.geo, e, Lq, n);
  float4* nq = reinterpret_cast<float4*>(&sm.r.a.nv[e * kNvStride + q * kNv]);
#pragma unroll
  for (int a = 0; a < 10; ++a) nq[a] = make_float4(n[a][0], n[a][1], n[a][2], 0.0f);
  float Hm[3][3], Fd[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Hm[r][c] = 0.0f;
      Fd[r][c] = 0.0f;
    }
#pragma unroll
  for (int a = 0; a < 10; ++a)
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float ua = sm.u[(a * 3 + r) * E + e];
      float va = 0.0f;
      if (KV) va = sm.vel[(a * 3 + r) * E + e];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Hm[r][c] += ua * n[a][c];
        if (KV) Fd[r][c] += va * n[a][c];
      }
    }
  QP<float> s;
  constitutive<float, TL_SVK, KV>(Hm, Fd, mat, s, inverted);
  const float c2w = bscale * wJ;
  float4* qd = reinterpret_cast<float4*>(&sm.r.a.qd[e * kQStride + q * kQd]);
  qd[0] = make_float4(s.F[0][0], s.F[0][1], s.F[0][2], s.F[1][0]);
  qd[1] = make_float4(s.F[1][1], s.F[1][2], s.F[2][0], s.F[2][1]);
  qd[2] = make_float4(s.F[2][2], wJ * s.S[0][0], wJ * s.S[0][1], wJ * s.S[0][2]);
  qd[3] = make_float4(wJ * s.S[1][1], wJ * s.S[1][2], wJ * s.S[2][2], c2w * s.B[0][0]);
  qd[4] = make_float4(c2w * s.B[0][1], c2w * s.B[0][2], c2w * s.B[1][1], c2w * s.B[1][2]);
  qd[5] = make_float4(c2w * s.B[2][2], wJ, 0.0f, 0.0f);
}

// Row-major index of the symmetric 3x3 stored as (00, 01, 02, 11, 12, 22).
__device__ __forceinline__ constexpr int sym6(int i, int k) {
  return i <= k ? (i == 0 ? k : (i == 1 ? 2 + k : 5)) : (k == 0 ? i : (k == 1 ? 2 + i : 5));
}

// Vectors of node a at one point: its gradient n, g = F n, u = c1 wJ0 g,
// w = c2 wJ0 g, t = alpha wJ0 S n (and wJ0 S n for the force); folded:
// u = wJ0 g, t = alpha wJ0 S n / (c1 + c2), no w.
struct NodeA {
  float n[3], g[3], u[3], w[3], t[3];
};

__device__ __forceinline__ void mat3_vec(const float (&F)[3][3], const float (&x)[3], float (&y)[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = F[i][0] * x[0] + F[i][1] * x[1] + F[i][2] * x[2];
}

__device__ __forceinline__ void sym_vec(const float (&S)[6], const float (&x)[3], float (&y)[3]) {
  y[0] = S[0] * x[0] + S[1] * x[1] + S[2] * x[2];
  y[1] = S[1] * x[0] + S[3] * x[1] + S[4] * x[2];
  y[2] = S[2] * x[0] + S[4] * x[1] + S[5] * x[2];
}

template <bool DO_FORCE, bool FOLD>
__device__ __forceinline__ void node_a(const float4& nv, const float (&F)[3][3], const float (&Sw)[6], float c1w,
                                       float c2w, float alpha, NodeA& a, float (&f)[3]) {
  a.n[0] = nv.x;
  a.n[1] = nv.y;
  a.n[2] = nv.z;
  mat3_vec(F, a.n, a.g);
  float s[3];
  sym_vec(Sw, a.n, s);
  if (DO_FORCE) {
    float fs[3];
    mat3_vec(F, s, fs);
#pragma unroll
    for (int i = 0; i < 3; ++i) f[i] += fs[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    a.u[i] = c1w * a.g[i];
    if (!FOLD) a.w[i] = c2w * a.g[i];
    a.t[i] = alpha * s[i];
  }
}

// K_ab += u_a g_b^T + g_b w_a^T + (n_a.n_b) Bh + (t_a.n_b) I  (one point);
// folded: Q_ab += u_a g_b^T + (n_a.n_b) Bh' + (t'_a.n_b) I.
template <bool FOLD>
__device__ __forceinline__ void pair_acc(float (&K)[9], const NodeA& a, const float (&gb)[3], const float (&nb)[3],
                                         const float (&Bh)[6]) {
  const float nn = a.n[0] * nb[0] + a.n[1] * nb[1] + a.n[2] * nb[2];
  const float ns = a.t[0] * nb[0] + a.t[1] * nb[1] + a.t[2] * nb[2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float x = fmaf(a.u[i], gb[k], K[3 * i + k]);
      if (!FOLD) x = fmaf(a.w[k], gb[i], x);
      x = fmaf(nn, Bh[sym6(i, k)], x);
      if (i == k) x += ns;
      K[3 * i + k] = x;
    }
}

// Block (a, b) of element e into the exchange buffer (transposed when a > b).
__device__ __forceinline__ void put_block(float* X, int e, int a, int b, const float (&K)[9]) {
  if (a <= b) {
    float* p = X + xchg_offset(e, a, b);
#pragma unroll
    for (int c = 0; c < 9; ++c) p[c] = K[c];
  } else {
    float* p = X + xchg_offset(e, b, a);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) p[3 * k + i] = K[3 * i + k];
  }
}

__device__ __forceinline__ void put_kelem(float* Ke, int a, int b, const float (&K)[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Ke[(3 * a + i) * 30 + 3 * b + k] = K[3 * i + k];
      if (a != b) Ke[(3 * b + k) * 30 + 3 * a + i] = K[3 * i + k];
    }
}

template <bool KV, bool DO_FORCE, bool FOLD>
__device__ __forceinline__ void pair_tile(const Args<float>& A, SmemP& sm, int64_t e0, const MatT<float>& mat,
                                          int64_t real_end, MapP* M, int nu, bool wait_pf) {
  const float beta = A.beta;
  const float c1 = A.alpha * mat.lam + (KV ? beta * mat.lam_d : 0.0f);
  const float c2 = A.alpha * mat.mu + (KV ? beta * mat.eta : 0.0f);
  const float inv_s = FOLD ? 1.0f / (c1 + c2) : 1.0f;     // the host checked c1 + c2 for FOLD
  const float alpha = FOLD ? A.alpha * inv_s : A.alpha;    // t' (folded) or t
  bool inverted = false;
  const int w = threadIdx.x >> 5, e = threadIdx.x & 31;
  if (w < 5) phase_a<KV>(mat, FOLD ? c2 * inv_s : c2, sm, inverted);
  if (inverted && e0 + e < real_end) atomicOr(A.flags, kFlagInverted);
  // the next tile's prefetch (committed before the map) has landed; the map
  // may still be in flight
  if (wait_pf) {
    if (M) cp_async_wait_group<1>();
    else cp_async_wait_all();
  }
  __syncthreads();
  // phase C: warp w -> round w of the round robin over the node pairs
  const int a0 = 2 * w, a1 = a0 + 1;
  const int w1 = w + 1 < 5 ? w + 1 : w - 4, w2 = w + 2 < 5 ? w + 2 : w - 3;
  const int cn[4] = {2 * w1, 2 * w1 + 1, 2 * w2, 2 * w2 + 1};
  float K[11][9];
#pragma unroll
  for (int j = 0; j < 11; ++j)
#pragma unroll
    for (int c = 0; c < 9; ++c) K[j][c] = 0.0f;
  float f0[3] = {0.0f, 0.0f, 0.0f}, f1[3] = {0.0f, 0.0f, 0.0f};
  const bool compute = w < 5;
#pragma unroll 1
  for (int q = 0; q < (compute ? 5 : 0); ++q) {
    const float4* qd = reinterpret_cast<const float4*>(&sm.r.a.qd[e * kQStride + q * kQd]);
    const float4 d0 = qd[0], d1 = qd[1], d2 = qd[2], d3 = qd[3], d4 = qd[4], d5 = qd[5];
    const float F[3][3] = {{d0.x, d0.y, d0.z}, {d0.w, d1.x, d1.y}, {d1.z, d1.w, d2.x}};
    const float Sw[6] = {d2.y, d2.z, d2.w, d3.x, d3.y, d3.z};
    const float Bh[6] = {d3.w, d4.x, d4.y, d4.z, d4.w, d5.x};
    const float wJ = d5.y;
    const float c1w = FOLD ? wJ : c1 * wJ, c2w = c2 * wJ;
    const float4* nq = reinterpret_cast<const float4*>(&sm.r.a.nv[e * kNvStride + q * kNv]);
    NodeA A0, A1;
    node_a<DO_FORCE, FOLD>(nq[a0], F, Sw, c1w, c2w, alpha, A0, f0);
    node_a<DO_FORCE, FOLD>(nq[a1], F, Sw, c1w, c2w, alpha, A1, f1);
    pair_acc<FOLD>(K[0], A0, A0.g, A0.n, Bh);
    pair_acc<FOLD>(K[1], A0, A1.g, A1.n, Bh);
    pair_acc<FOLD>(K[2], A1, A1.g, A1.n, Bh);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 v = nq[cn[j]];
      const float nb[3] = {v.x, v.y, v.z};
      float gb[3];
      mat3_vec(F, nb, gb);
      pair_acc<FOLD>(K[3 + 2 * j], A0, gb, nb, Bh);
      pair_acc<FOLD>(K[4 + 2 * j], A1, gb, nb, Bh);
    }
  }
  const bool real = compute && e0 + e < real_end;
  if (DO_FORCE && real) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      atomicAdd(&A.f[3 * (int64_t)sm.node[a0][e] + d], double(f0[d]));
      atomicAdd(&A.f[3 * (int64_t)sm.node[a1][e] + d], double(f1[d]));
    }
  }
  if (FOLD) {   // K_ab = c1 Q_ab + c2 Q_ab^T
#pragma unroll
    for (int j = 0; j < 11; ++j) {
      float* Q = K[j];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = i + 1; k < 3; ++k) {
          const float qik = Q[3 * i + k], qki = Q[3 * k + i];
          Q[3 * i + k] = fmaf(c1, qik, c2 * qki);
          Q[3 * k + i] = fmaf(c1, qki, c2 * qik);
        }
      Q[0] *= c1 + c2;
      Q[4] *= c1 + c2;
      Q[8] *= c1 + c2;
    }
  }
  // the mass term M_e * mass_scale on the diagonal of every block
  const int ra[11] = {a0, a0, a1, a0, a1, a0, a1, a0, a1, a0, a1};
  const int rb[11] = {a0, a1, a1, cn[0], cn[0], cn[1], cn[1], cn[2], cn[2], cn[3], cn[3]};
  const float ms = A.mass_scale * mat.rho * sm.geo[12][e] * (1.0f / 420.0f);
#pragma unroll
  for (int j = 0; j < 11 && compute; ++j) {
    const float mj = ms * c_mass420[ra[j]][rb[j]];
    K[j][0] += mj;
    K[j][4] += mj;
    K[j][8] += mj;
  }
  if (A.K_elem) {
    if (real) {
      float* Ke = A.K_elem + (int64_t)A.user_of[e0 + e] * 900;
#pragma unroll
      for (int j = 0; j < 11; ++j) put_kelem(Ke, ra[j], rb[j], K[j]);
    }
  }
  if (A.values) {
    __syncthreads();                   // the point data (aliased by X) is consumed
    if (compute) {
#pragma unroll
      for (int j = 0; j < 11; ++j) put_block(sm.r.X, e, ra[j], rb[j], K[j]);
    }
    cp_async_wait_all();               // the map has landed
    __syncthreads();
  }
}

template <bool KV, bool DO_FORCE, bool FOLD>
__global__ void __launch_bounds__(NTP, 2) pair_kernel(Args<float> A, SegTable<float> S, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_next;
  SmemP& sm = *reinterpret_cast<SmemP*>(smem_raw);
  // CSR values: the map buffer and the prefetch buffer follow (A.pf_off);
  // K_elem output: neither
  MapP* M = A.values ? reinterpret_cast<MapP*>(smem_raw + sizeof(SmemP)) : nullptr;
  PrefP* P = A.pf_off >= 0 ? reinterpret_cast<PrefP*>(smem_raw + A.pf_off) : nullptr;
  SegWalk cur, nxt;
  int k = blockIdx.x;
  if (k >= S.ntiles) return;                         // uniform over the block
  int64_t e0 = cur.e0(S, k);
  int nu = M ? A.agg_nu[e0 / E] : 0;
  load_tile_p<KV>(A, sm, e0);
  if (threadIdx.x == 0) s_next = counter ? (int)gridDim.x + atomicAdd(counter, 1) : k + (int)gridDim.x;
  __syncthreads();
  while (true) {
    const int k_next = s_next;
    const MatT<float> mat = S.s[cur.sg].mat;
    const int64_t real_end = S.s[cur.sg].real_end;
    nxt = cur;
    const int64_t e0_next = (P && k_next < S.ntiles) ? nxt.e0(S, k_next) : -1;
    if (e0_next >= 0) pf_stage1(A, *P, e0_next);     // committed first ...
    if (M) map_copy(A, *M, e0 / E, nu);              // ... then this tile's map
    pair_tile<KV, DO_FORCE, FOLD>(A, sm, e0, mat, real_end, M, nu, e0_next >= 0);
    // the next tile's nodal loads (its conn rows have landed) in flight
    // during this tile's scatter
    NodalRegs nr;
    if (e0_next >= 0) nodal_load(A, P->conn, nr);
    if (M) map_scatter(A, sm.r.X, *M, nu);
    cp_async_wait_all();
    // with CSR values, the barrier after the exchange-buffer writes already
    // put phase C's reads of node / geo before the unpack below, which writes
    // nothing the scatter reads (u and vel lie outside the exchange buffer);
    // the K_elem path has no such barrier
    if (!M) __syncthreads();
    if (k_next >= S.ntiles) break;
    if (threadIdx.x == 0) s_next = counter ? (int)gridDim.x + atomicAdd(counter, 1) : k_next + (int)gridDim.x;
    k = k_next;
    if (P) {
      cur = nxt;
      e0 = e0_next;
      nu = M ? P->nu : 0;
      unpack_p<KV>(A, sm, *P, nr);                   // ends with a barrier (also publishes s_next)
    } else {
      e0 = cur.e0(S, k);
      nu = M ? A.agg_nu[e0 / E] : 0;
      load_tile_p<KV>(A, sm, e0);                    // ends with a barrier (also publishes s_next)
    }
  }
}

}  // namespace
}  // namespace elem
}  // namespace tl

namespace tl {
namespace elem {

// The float32 {u, v} of every DOF for the pair kernel (m->d_uv32).
tl_status pair_prep(tl_mesh* m, const double* q_n, const double* v, double h) {
  const int64_t n = 3 * m->nn;
  if (n == 0) return TL_OK;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, (int64_t)m->num_sms * 32);
  uv32_kernel<<<(unsigned)blocks, threads, 0, m->stream>>>(q_n, v, m->d_X, h, n, m->d_uv32);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

// One persistent launch of the pair kernel over the SVK segments of S.
tl_status pair_launch(tl_mesh* m, const Args<float>& A0, const SegTable<float>& S, bool kv, bool do_force,
                      int* counter) {
  Args<float> A = A0;
  size_t smem = sizeof(SmemP);
  if (A.values) smem += sizeof(MapP);
  A.pf_off = -1;
  if (m->tune.elem_prefetch) {
    smem = (smem + 15) / 16 * 16;
    A.pf_off = (int)smem;
    smem += sizeof(PrefP);
  }
  // folded form where c1 + c2 is at least a quarter of max(|c1|, |c2|) for
  // every segment of the launch (at most two bits lost to cancellation)
  bool fold = true;
  for (int j = 0; j < S.nseg; ++j) {
    const MatT<float>& mt = S.s[j].mat;
    const double c1 = A.alpha * (double)mt.lam + (kv ? A.beta * (double)mt.lam_d : 0.0);
    const double c2 = A.alpha * (double)mt.mu + (kv ? A.beta * (double)mt.eta : 0.0);
    const double sum = c1 + c2;
    fold = fold && sum != 0.0 && std::fabs(sum) >= 0.25 * std::max(std::fabs(c1), std::fabs(c2));
  }
  if (m->tune.elem_fold == 0) fold = false;
  using Kern = void (*)(Args<float>, SegTable<float>, int*);
  const Kern table[2][2][2] = {
      {{pair_kernel<false, false, false>, pair_kernel<false, false, true>},
       {pair_kernel<false, true, false>, pair_kernel<false, true, true>}},
      {{pair_kernel<true, false, false>, pair_kernel<true, false, true>},
       {pair_kernel<true, true, false>, pair_kernel<true, true, true>}}};
  Kern kern = table[kv ? 1 : 0][do_force ? 1 : 0][fold ? 1 : 0];
  TL_CUDA(m, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 1;
  TL_CUDA(m, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NTP, smem));
  const bool full = m->tune.elem_full_grid != 0;
  const int grid = full ? S.ntiles : (int)std::min<int64_t>(S.ntiles, (int64_t)m->num_sms * std::max(occ, 1));
  if (full) counter = nullptr;
  if (counter) TL_CUDA(m, cudaMemsetAsync(counter, 0, sizeof(int), m->stream));
  kern<<<(unsigned)grid, NTP, smem, m->stream>>>(A, S, counter);
  TL_CUDA(m, cudaGetLastError());
  ++m->launches;
  return TL_OK;
}

}  // namespace elem
}  // namespace tl
