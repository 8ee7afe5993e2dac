// Element kernel of the ANCF3243 beam and ANCF3443 shell elements: internal
// force, tangent and its CSR assembly, in float64 or in the float32 element
// form, instantiated per element kind and arithmetic type in tl_ancf_*.cu.
//
// Paper: arxiv 2604.10357 Sec. 4.3 (Stage 1: P at every (element, quadrature
// point), 12 points per beam and 48 per shell element; Stage 2: f_a = sum_q
// P grad S_a w J0, eq. fint_local) and Sec. 4.4 (eq. tangent_block, 24 x 24
// and 48 x 48 element tangents, scattered into the fixed CSR pattern).
//
// One CTA holds EPB elements.  Staging: per coefficient, the displacement
// u = q_n + h v - e0 and the velocity (formed in float64) and the reference
// coefficient e0, positions taken relative to the element's first position
// (the Jacobian depends only on differences of positions; this keeps float32
// exact to its precision on a 100 km beam).  Phase 1: a thread per (element, point)
// computes J0 from the reference coefficients, grad_X S_a = J0^{-T} dS_a,
// F, the stresses, and keeps per point n_a = grad_X S_a, g_a = F n_a,
// s_a = S n_a, F, B = F F^T, w J0 (and the tangent rows for Mooney-Rivlin)
// in shared memory; nothing of Stage 1 goes to global memory.  Force: a
// thread per (element, a) sums w J0 F s_a over the points.  Tangent: a
// thread per (element, block pair a <= b) sums the 3 x 3 block over the
// points, adds the exact element mass on its diagonal, and writes the block
// and its transpose through the slot map (the Hessian is symmetric).
#pragma once

#include <type_traits>

#include "tl_ancf.cuh"
#include "tl_element_common.cuh"

namespace tl {
namespace ancf {

template <typename T>
struct Args {
  const int32_t* conn;      // ne_pad x NEN coefficient ids
  const double* geo;        // ne_pad x 16: L, W, H
  const uint8_t* blk;       // ne_pad x NEN^2 slot blocks
  const int32_t* node_ptr;
  const int32_t* user_of;
  const double* me;         // ne_pad x NP exact element mass (upper triangle)
  const double *q_n, *v, *X;
  double h, mass_scale;
  T alpha, beta;
  double* f;
  T* values;
  T* K_elem;
  uint32_t* flags;
  int64_t begin, end;       // this segment's element range
  MatT<T> mat;
};

template <int ET>
struct Cfg {
  static constexpr int NEN = Traits<ET>::NEN, NQP = Traits<ET>::NQP, NP = NEN * (NEN + 1) / 2;
  static constexpr int EPB = ET == kBeam ? 8 : 1;           // elements per CTA
  static constexpr int NT = ET == kBeam ? 288 : 160;        // >= EPB * NP pair threads
};

// Resident CTAs per SM the register budget is capped for.  float64: 1 beam /
// 2 shell CTAs.  The float32 form needs fewer registers; its St. Venant-
// Kirchhoff kernels were measured at 2 to 7 CTAs (500,000-element beam,
// 200 x 200 shell): the beam 1.64 / 1.33 / 1.26 / 1.23 ms at 2 / 3 / 4 / 5
// CTAs (5: 4 bytes of spills, 160 with Kelvin-Voigt, which keeps 4), the
// shell 1.14 / 1.08 / 1.10 ms at 3 / 6 / 7 (no spills at 6); the Mooney-Rivlin
// kernels spill at those caps and keep 2 / 3.
template <typename T, int ET, int MAT, bool KV>
constexpr int min_blocks() {
  return std::is_same<T, float>::value
             ? (ET == kBeam ? (MAT == TL_SVK ? (KV ? 4 : 5) : 2) : (MAT == TL_SVK ? 6 : 3))
             : (ET == kBeam ? 1 : 2);
}

// Per-point record in shared memory (elements of type T).  WG (float64 SVK
// tangents): the weighted vectors wJ0 c1 g_a and wJ0 c2 g_a and the scalars
// wJ0 c2, wJ0 alpha are kept too, so that the pair loop runs no multiplies
// outside its multiply-adds (float64 operations are GB300's scarce resource;
// the float32 form keeps the smaller record: its pair loop is bound by
// shared-memory loads, not arithmetic).
template <int ET, bool TAN, bool MR, bool WG>
struct Rec {
  static constexpr int NEN = Traits<ET>::NEN;
  static constexpr int oN = 0;
  static constexpr int oG = 3 * NEN;                        // tangent only
  static constexpr int oS = TAN ? 6 * NEN : 3 * NEN;
  static constexpr int oF = oS + 3 * NEN;
  static constexpr int oB = oF + 9;                         // tangent only
  static constexpr int oW = TAN ? oB + 9 : oF + 9;
  static constexpr int oX = oW + 1;                         // WG: wJ0 c2, wJ0 alpha
  static constexpr int oH1 = oX + (WG ? 2 : 0);             // WG: wJ0 c1 g_a
  static constexpr int oH2 = oH1 + (WG ? 3 * NEN : 0);      // WG: wJ0 c2 g_a
  static constexpr int oA = oH2 + (WG ? 3 * NEN : 0);       // Mooney-Rivlin tangent rows
  static constexpr int R = oA + (TAN && MR ? 81 : 0);
};

template <typename T, bool TAN, bool MR>
__host__ __device__ constexpr bool weighted_g() {
  return std::is_same<T, double>::value && TAN && !MR;
}

// Dynamic shared memory: the per-point records, then the staged coefficients
// (u, v, e0 per coefficient: 9 values) and the element dimensions (4).
template <typename T, int ET, bool TAN, bool MR>
constexpr size_t smem_bytes() {
  return sizeof(T) * ((size_t)Rec<ET, TAN, MR, weighted_g<T, TAN, MR>()>::R * Cfg<ET>::NQP +
                      9 * Cfg<ET>::NEN + 4) * Cfg<ET>::EPB;
}

template <typename T, int ET, int MAT, bool KV, bool DO_FORCE, bool DO_TANGENT>
__global__ void __launch_bounds__(Cfg<ET>::NT, min_blocks<T, ET, MAT, KV>()) elem_kernel(Args<T> A) {
  constexpr int NEN = Cfg<ET>::NEN, NQP = Cfg<ET>::NQP, NP = Cfg<ET>::NP, EPB = Cfg<ET>::EPB, NT = Cfg<ET>::NT;
  constexpr bool MR = MAT == TL_MOONEY_RIVLIN;
  constexpr bool WG = weighted_g<T, DO_TANGENT, MR>();
  using RC = Rec<ET, DO_TANGENT, MR, WG>;
  const T c1 = A.alpha * A.mat.lam + (KV ? A.beta * A.mat.lam_d : T(0));
  const T c2 = A.alpha * A.mat.mu + (KV ? A.beta * A.mat.eta : T(0));
  extern __shared__ unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  T* stg = sm + (size_t)RC::R * NQP * EPB;                  // [el][a][u 3, v 3, e0 3]
  T* sdim = stg + 9 * NEN * EPB;                            // [el][L, W, H, -]
  __shared__ int32_t s_conn[EPB][NEN];
  const int64_t ebase = A.begin + (int64_t)blockIdx.x * EPB;
  for (int t = threadIdx.x; t < EPB * NEN; t += NT) {
    const int64_t e = ebase + t / NEN;
    s_conn[t / NEN][t % NEN] = e < A.end ? A.conn[e * NEN + t % NEN] : 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < EPB * NEN * 3; t += NT) {
    const int el = t / (NEN * 3), a = (t / 3) % NEN, i = t % 3;
    if (ebase + el >= A.end) continue;
    const int c = s_conn[el][a];
    const double vi = A.v[3 * c + i], x0 = A.X[3 * c + i];
    T* st = stg + (el * NEN + a) * 9;
    st[i] = T((A.q_n[3 * c + i] + A.h * vi) - x0);
    st[3 + i] = T(vi);
    // positions relative to the element's first position coefficient
    st[6 + i] = T((a & 3) == 0 ? x0 - A.X[3 * s_conn[el][0] + i] : x0);
  }
  for (int t = threadIdx.x; t < EPB * 3; t += NT) {
    const int64_t e = ebase + t / 3;
    if (e < A.end) sdim[4 * (t / 3) + t % 3] = T(A.geo[e * 16 + t % 3]);
  }
  __syncthreads();

  // ---- phase 1: kinematics and stresses at every (element, point) --------
  bool inverted = false;
  for (int t = threadIdx.x; t < EPB * NQP; t += NT) {
    const int el = t / NQP, q = t % NQP;
    const int64_t e = ebase + el;
    if (e >= A.end) continue;
    T* rec = sm + (size_t)(el * NQP + q) * RC::R;
    const T* st = stg + el * NEN * 9;
    const T dims[3] = {sdim[4 * el], sdim[4 * el + 1], sdim[4 * el + 2]};
    T p[3], wq;
    element_point<ET, T>(q, p, wq);
    T J0[3][3] = {};
    for (int a = 0; a < NEN; ++a) {
      T d[3];
      shape<ET, T>(a, p, dims, nullptr, d);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T x0 = st[a * 9 + 6 + i];
#pragma unroll
        for (int j = 0; j < 3; ++j) J0[i][j] += x0 * d[j];
      }
    }
    T Ji[3][3];
    const T det = inv3<T>(J0, Ji);
    if (!(det > T(0))) inverted = true;
    T Hm[3][3] = {}, Fd[3][3] = {};
    for (int a = 0; a < NEN; ++a) {
      T d[3], n[3];
      shape<ET, T>(a, p, dims, nullptr, d);
#pragma unroll
      for (int J = 0; J < 3; ++J) n[J] = d[0] * Ji[0][J] + d[1] * Ji[1][J] + d[2] * Ji[2][J];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T ui = st[a * 9 + i], vi = st[a * 9 + 3 + i];
#pragma unroll
        for (int J = 0; J < 3; ++J) {
          Hm[i][J] += ui * n[J];
          if (KV) Fd[i][J] += vi * n[J];
        }
      }
#pragma unroll
      for (int J = 0; J < 3; ++J) rec[RC::oN + 3 * a + J] = n[J];
    }
    QP<T> s;
    constitutive<T, MAT, KV>(Hm, Fd, A.mat, s, inverted);
    const T wJ = wq * det;
    for (int a = 0; a < NEN; ++a) {
      const T n0 = rec[RC::oN + 3 * a], n1 = rec[RC::oN + 3 * a + 1], n2 = rec[RC::oN + 3 * a + 2];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        rec[RC::oS + 3 * a + i] = s.S[i][0] * n0 + s.S[i][1] * n1 + s.S[i][2] * n2;
        if (DO_TANGENT) {
          const T gi = s.F[i][0] * n0 + s.F[i][1] * n1 + s.F[i][2] * n2;
          rec[RC::oG + 3 * a + i] = gi;
          if (WG) {
            rec[RC::oH1 + 3 * a + i] = (wJ * c1) * gi;
            rec[RC::oH2 + 3 * a + i] = (wJ * c2) * gi;
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        rec[RC::oF + 3 * i + j] = s.F[i][j];
        if (DO_TANGENT) rec[RC::oB + 3 * i + j] = s.B[i][j];
      }
    rec[RC::oW] = wJ;
    if (WG) {
      rec[RC::oX] = wJ * c2;
      rec[RC::oX + 1] = wJ * A.alpha;
    }
    if constexpr (DO_TANGENT && MR) {
      tangent_row<T, MAT, KV, 0>(s, A.mat, A.alpha, A.beta, wJ, rec + RC::oA);
      tangent_row<T, MAT, KV, 1>(s, A.mat, A.alpha, A.beta, wJ, rec + RC::oA + 27);
      tangent_row<T, MAT, KV, 2>(s, A.mat, A.alpha, A.beta, wJ, rec + RC::oA + 54);
    }
  }
  if (inverted) atomicOr(A.flags, kFlagInverted);
  __syncthreads();

  // ---- force: f_a = sum_q w J0 F (S n_a) ----------------------------------
  if (DO_FORCE) {
    for (int t = threadIdx.x; t < EPB * NEN; t += NT) {
      const int el = t / NEN, a = t % NEN;
      if (ebase + el >= A.end) continue;
      T fa[3] = {T(0), T(0), T(0)};
      for (int q = 0; q < NQP; ++q) {
        const T* rec = sm + (size_t)(el * NQP + q) * RC::R;
        const T wJ = rec[RC::oW];
        const T s0 = rec[RC::oS + 3 * a], s1 = rec[RC::oS + 3 * a + 1], s2 = rec[RC::oS + 3 * a + 2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          fa[i] += wJ * (rec[RC::oF + 3 * i] * s0 + rec[RC::oF + 3 * i + 1] * s1 + rec[RC::oF + 3 * i + 2] * s2);
      }
      const int c = s_conn[el][a];
#pragma unroll
      for (int i = 0; i < 3; ++i) atomicAdd(&A.f[3 * c + i], (double)fa[i]);
    }
  }

  // ---- tangent blocks (a <= b) ---------------------------------------------
  if (DO_TANGENT) {
    for (int t = threadIdx.x; t < EPB * NP; t += NT) {
      const int el = t / NP, pr = t % NP;
      const int64_t e = ebase + el;
      if (e >= A.end) continue;
      int a, b;
      pair_of(pr, NEN, a, b);
      T K[3][3] = {};
      for (int q = 0; q < NQP; ++q) {
        const T* rec = sm + (size_t)(el * NQP + q) * RC::R;
        const T* na = rec + RC::oN + 3 * a;
        const T* nb = rec + RC::oN + 3 * b;
        if constexpr (WG) {
          // the same block from the weighted vectors: (wJ c1 g_a)_i g_b,k + (wJ c2 g_b)_i g_a,k + ...
          const T* ga = rec + RC::oG + 3 * a;
          const T* gb = rec + RC::oG + 3 * b;
          const T* h1a = rec + RC::oH1 + 3 * a;
          const T* h2b = rec + RC::oH2 + 3 * b;
          const T* sb = rec + RC::oS + 3 * b;
          const T nn = na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2];
          const T sn = na[0] * sb[0] + na[1] * sb[1] + na[2] * sb[2];
          const T w2n = rec[RC::oX] * nn, w3 = rec[RC::oX + 1] * sn;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const T hai = h1a[i], hbi = h2b[i];
#pragma unroll
            for (int k = 0; k < 3; ++k)
              K[i][k] += hai * gb[k] + hbi * ga[k] + w2n * rec[RC::oB + 3 * i + k];
            K[i][i] += w3;
          }
        } else if constexpr (!MR) {
          // [K_ab]_ik = wJ [c1 g_a,i g_b,k + c2 (g_b,i g_a,k + (n_a.n_b) B_ik) + alpha d_ik n_a.S n_b]
          const T wJ = rec[RC::oW];
          const T* ga = rec + RC::oG + 3 * a;
          const T* gb = rec + RC::oG + 3 * b;
          const T* sb = rec + RC::oS + 3 * b;
          const T nn = na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2];
          const T sn = na[0] * sb[0] + na[1] * sb[1] + na[2] * sb[2];
          const T w1 = wJ * c1, w2 = wJ * c2, w2n = w2 * nn, w3 = wJ * A.alpha * sn;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const T gai = ga[i], gbi = gb[i];
#pragma unroll
            for (int k = 0; k < 3; ++k)
              K[i][k] += w1 * gai * gb[k] + w2 * gbi * ga[k] + w2n * rec[RC::oB + 3 * i + k];
            K[i][i] += w3;
          }
        } else {
          // [K_ab]_ik = sum_J n_a,J sum_L A^_iJkL n_b,L (rows already scaled by wJ, alpha, beta)
          const T* Ar = rec + RC::oA;
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J = 0; J < 3; ++J) {
              const T* r = Ar + i * 27 + J * 9;
#pragma unroll
              for (int k = 0; k < 3; ++k)
                K[i][k] += na[J] * (r[k * 3] * nb[0] + r[k * 3 + 1] * nb[1] + r[k * 3 + 2] * nb[2]);
            }
        }
      }
      if (A.mass_scale != 0.0) {
        const T ms = T(A.mass_scale * A.me[e * NP + pr]);
        K[0][0] += ms;
        K[1][1] += ms;
        K[2][2] += ms;
      }
      if (A.values) {
        const int I = s_conn[el][a], Jn = s_conn[el][b];
        const uint8_t* bk = A.blk + e * (NEN * NEN);
        const int pI = A.node_ptr[I], dI = A.node_ptr[I + 1] - pI;
        const int kab = bk[a * NEN + b];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) atomicAdd(&A.values[9 * pI + 3 * dI * i + 3 * kab + k], K[i][k]);
        if (a != b) {
          const int pJ = A.node_ptr[Jn], dJ = A.node_ptr[Jn + 1] - pJ;
          const int kba = bk[b * NEN + a];
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i) atomicAdd(&A.values[9 * pJ + 3 * dJ * k + 3 * kba + i], K[i][k]);
        }
      }
      if (A.K_elem) {
        constexpr int ND = 3 * NEN;
        T* Ke = A.K_elem + (int64_t)A.user_of[e] * ND * ND;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            Ke[(3 * a + i) * ND + 3 * b + k] = K[i][k];
            if (a != b) Ke[(3 * b + k) * ND + 3 * a + i] = K[i][k];
          }
      }
    }
  }
}

// One launch per material segment; dispatch on (material kind, Kelvin-Voigt,
// pass).  T = float instantiates the tangent passes only (the float32 element
// form; its forces for the residual come from the float64 kernels).
template <typename T, int ET>
tl_status launch_kind(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                      double mass_scale, bool do_force, bool do_tangent, double* f, T* values, T* K_elem) {
  Args<T> A;
  A.conn = m->d_conn;
  A.geo = m->d_geo64;
  A.blk = m->d_blk;
  A.node_ptr = m->d_node_ptr;
  A.user_of = m->d_user_of;
  A.me = m->d_ancf_me;
  A.q_n = q_n;
  A.v = v;
  A.X = m->d_X;
  A.h = h;
  A.alpha = T(alpha);
  A.beta = T(beta);
  A.mass_scale = mass_scale;
  A.f = f;
  A.values = values;
  A.K_elem = K_elem;
  A.flags = m->d_flags;
  constexpr bool kF64 = std::is_same<T, double>::value;
  for (const Segment& sg : m->segs) {
    const int64_t cnt = sg.end - sg.begin;
    if (cnt == 0) continue;
    const MaterialDev& md = m->mats[sg.mat];
    A.begin = sg.begin;
    A.end = sg.end;
    A.mat = to_matT<T>(md);
    const int combo = 2 * (md.kind == TL_SVK ? 0 : 1) + (md.kv ? 1 : 0);
    const int pass = (do_force ? 1 : 0) + (do_tangent ? 2 : 0);
    void (*kern)(Args<T>) = nullptr;
    size_t smem = 0;
#define TL_ANCF_CASE(MATK, KVK, FO, TA)                                             \
  kern = elem_kernel<T, ET, MATK, KVK, FO, TA>;                                      \
  smem = smem_bytes<T, ET, TA, MATK == TL_MOONEY_RIVLIN>();
    if constexpr (kF64) {
      switch (combo * 4 + pass) {
        case 0 * 4 + 1: TL_ANCF_CASE(TL_SVK, false, true, false) break;
        case 1 * 4 + 1: TL_ANCF_CASE(TL_SVK, true, true, false) break;
        case 2 * 4 + 1: TL_ANCF_CASE(TL_MOONEY_RIVLIN, false, true, false) break;
        case 3 * 4 + 1: TL_ANCF_CASE(TL_MOONEY_RIVLIN, true, true, false) break;
        default: break;
      }
    }
    switch (combo * 4 + pass) {
      case 0 * 4 + 2: TL_ANCF_CASE(TL_SVK, false, false, true) break;
      case 0 * 4 + 3: TL_ANCF_CASE(TL_SVK, false, true, true) break;
      case 1 * 4 + 2: TL_ANCF_CASE(TL_SVK, true, false, true) break;
      case 1 * 4 + 3: TL_ANCF_CASE(TL_SVK, true, true, true) break;
      case 2 * 4 + 2: TL_ANCF_CASE(TL_MOONEY_RIVLIN, false, false, true) break;
      case 2 * 4 + 3: TL_ANCF_CASE(TL_MOONEY_RIVLIN, false, true, true) break;
      case 3 * 4 + 2: TL_ANCF_CASE(TL_MOONEY_RIVLIN, true, false, true) break;
      case 3 * 4 + 3: TL_ANCF_CASE(TL_MOONEY_RIVLIN, true, true, true) break;
      default: break;
    }
#undef TL_ANCF_CASE
    if (!kern) return pass == 0 ? TL_OK : fail(m, TL_ERR_UNSUPPORTED, "ANCF element pass selection");
    TL_CUDA(m, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t nblk = (cnt + Cfg<ET>::EPB - 1) / Cfg<ET>::EPB;
    kern<<<(unsigned)nblk, Cfg<ET>::NT, smem, m->stream>>>(A);
    TL_CUDA(m, cudaGetLastError());
    ++m->launches;
  }
  return TL_OK;
}

}  // namespace ancf
}  // namespace tl
