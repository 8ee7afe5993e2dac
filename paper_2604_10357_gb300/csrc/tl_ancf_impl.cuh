// Element kernel of the ANCF3243 beam and ANCF3443 shell elements (float64):
// internal force, tangent and its CSR assembly, instantiated per element
// kind in tl_ancf_beam.cu and tl_ancf_shell.cu.
//
// Paper: arxiv 2604.10357 Sec. 4.3 (Stage 1: P at every (element, quadrature
// point), 12 points per beam and 48 per shell element; Stage 2: f_a = sum_q
// P grad S_a w J0, eq. fint_local) and Sec. 4.4 (eq. tangent_block, 24 x 24
// and 48 x 48 element tangents, scattered into the fixed CSR pattern).
//
// One CTA holds EPB elements.  Phase 1: a thread per (element, point)
// computes J0 from the reference coefficients, grad_X S_a = J0^{-T} dS_a,
// F, the stresses, and keeps per point n_a = grad_X S_a, g_a = F n_a,
// s_a = S n_a, F, B = F F^T, w J0 (and the tangent rows for Mooney-Rivlin)
// in shared memory; nothing of Stage 1 goes to global memory.  Force: a
// thread per (element, a) sums w J0 F s_a over the points.  Tangent: a
// thread per (element, block pair a <= b) sums the 3 x 3 block over the
// points, adds the exact element mass on its diagonal, and writes the block
// and its transpose through the slot map (the Hessian is symmetric).
#pragma once

#include "tl_ancf.cuh"
#include "tl_element_common.cuh"

namespace tl {
namespace ancf {

struct Args {
  const int32_t* conn;      // ne_pad x NEN coefficient ids
  const double* geo;        // ne_pad x 16: L, W, H
  const uint8_t* blk;       // ne_pad x NEN^2 slot blocks
  const int32_t* node_ptr;
  const int32_t* user_of;
  const double* me;         // ne_pad x NP exact element mass (upper triangle)
  const double *q_n, *v, *X;
  double h, alpha, beta, mass_scale;
  double* f;
  double* values;
  double* K_elem;
  uint32_t* flags;
  int64_t begin, end;       // this segment's element range
  MatT<double> mat;
};

template <int ET>
struct Cfg {
  static constexpr int NEN = Traits<ET>::NEN, NQP = Traits<ET>::NQP, NP = NEN * (NEN + 1) / 2;
  static constexpr int EPB = ET == kBeam ? 8 : 1;           // elements per CTA
  static constexpr int NT = ET == kBeam ? 288 : 160;        // >= EPB * NP pair threads
  static constexpr int MINB = ET == kBeam ? 1 : 2;          // resident CTAs per SM the registers allow
};

// Per-point record in shared memory (doubles).
template <int ET, bool TAN, bool MR>
struct Rec {
  static constexpr int NEN = Traits<ET>::NEN;
  static constexpr int oN = 0;
  static constexpr int oG = 3 * NEN;                        // tangent only
  static constexpr int oS = TAN ? 6 * NEN : 3 * NEN;
  static constexpr int oF = oS + 3 * NEN;
  static constexpr int oB = oF + 9;                         // tangent only
  static constexpr int oW = TAN ? oB + 9 : oF + 9;
  static constexpr int oA = oW + 1;                         // Mooney-Rivlin tangent rows
  static constexpr int R = oA + (TAN && MR ? 81 : 0);
};

template <int ET, bool TAN, bool MR>
constexpr size_t smem_bytes() {
  return sizeof(double) * (size_t)Rec<ET, TAN, MR>::R * Cfg<ET>::NQP * Cfg<ET>::EPB;
}

template <int ET, int MAT, bool KV, bool DO_FORCE, bool DO_TANGENT>
__global__ void __launch_bounds__(Cfg<ET>::NT, Cfg<ET>::MINB) elem_kernel(Args A) {
  constexpr int NEN = Cfg<ET>::NEN, NQP = Cfg<ET>::NQP, NP = Cfg<ET>::NP, EPB = Cfg<ET>::EPB, NT = Cfg<ET>::NT;
  constexpr bool MR = MAT == TL_MOONEY_RIVLIN;
  using RC = Rec<ET, DO_TANGENT, MR>;
  extern __shared__ double sm[];
  __shared__ int32_t s_conn[EPB][NEN];
  const int64_t ebase = A.begin + (int64_t)blockIdx.x * EPB;
  for (int t = threadIdx.x; t < EPB * NEN; t += NT) {
    const int64_t e = ebase + t / NEN;
    s_conn[t / NEN][t % NEN] = e < A.end ? A.conn[e * NEN + t % NEN] : 0;
  }
  __syncthreads();

  // ---- phase 1: kinematics and stresses at every (element, point) --------
  bool inverted = false;
  for (int t = threadIdx.x; t < EPB * NQP; t += NT) {
    const int el = t / NQP, q = t % NQP;
    const int64_t e = ebase + el;
    if (e >= A.end) continue;
    double* rec = sm + (size_t)(el * NQP + q) * RC::R;
    const double dims[3] = {A.geo[e * 16 + 0], A.geo[e * 16 + 1], A.geo[e * 16 + 2]};
    double p[3], w;
    element_point<ET>(q, p, w);
    double J0[3][3] = {};
    for (int a = 0; a < NEN; ++a) {
      double d[3];
      shape<ET>(a, p, dims, nullptr, d);
      const int c = s_conn[el][a];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double x0 = A.X[3 * c + i];
#pragma unroll
        for (int j = 0; j < 3; ++j) J0[i][j] += x0 * d[j];
      }
    }
    double Ji[3][3];
    const double det = inv3(J0, Ji);
    if (!(det > 0.0)) inverted = true;
    double Hm[3][3] = {}, Fd[3][3] = {};
    for (int a = 0; a < NEN; ++a) {
      double d[3], n[3];
      shape<ET>(a, p, dims, nullptr, d);
#pragma unroll
      for (int J = 0; J < 3; ++J) n[J] = d[0] * Ji[0][J] + d[1] * Ji[1][J] + d[2] * Ji[2][J];
      const int c = s_conn[el][a];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double vi = A.v[3 * c + i];
        const double ui = (A.q_n[3 * c + i] + A.h * vi) - A.X[3 * c + i];
#pragma unroll
        for (int J = 0; J < 3; ++J) {
          Hm[i][J] += ui * n[J];
          Fd[i][J] += vi * n[J];
        }
      }
#pragma unroll
      for (int J = 0; J < 3; ++J) rec[RC::oN + 3 * a + J] = n[J];
    }
    QP<double> s;
    constitutive<double, MAT, KV>(Hm, Fd, A.mat, s, inverted);
    for (int a = 0; a < NEN; ++a) {
      const double n0 = rec[RC::oN + 3 * a], n1 = rec[RC::oN + 3 * a + 1], n2 = rec[RC::oN + 3 * a + 2];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        rec[RC::oS + 3 * a + i] = s.S[i][0] * n0 + s.S[i][1] * n1 + s.S[i][2] * n2;
        if (DO_TANGENT) rec[RC::oG + 3 * a + i] = s.F[i][0] * n0 + s.F[i][1] * n1 + s.F[i][2] * n2;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        rec[RC::oF + 3 * i + j] = s.F[i][j];
        if (DO_TANGENT) rec[RC::oB + 3 * i + j] = s.B[i][j];
      }
    const double wJ = w * det;
    rec[RC::oW] = wJ;
    if constexpr (DO_TANGENT && MR) {
      tangent_row<double, MAT, KV, 0>(s, A.mat, A.alpha, A.beta, wJ, rec + RC::oA);
      tangent_row<double, MAT, KV, 1>(s, A.mat, A.alpha, A.beta, wJ, rec + RC::oA + 27);
      tangent_row<double, MAT, KV, 2>(s, A.mat, A.alpha, A.beta, wJ, rec + RC::oA + 54);
    }
  }
  if (inverted) atomicOr(A.flags, kFlagInverted);
  __syncthreads();

  // ---- force: f_a = sum_q w J0 F (S n_a) ----------------------------------
  if (DO_FORCE) {
    for (int t = threadIdx.x; t < EPB * NEN; t += NT) {
      const int el = t / NEN, a = t % NEN;
      if (ebase + el >= A.end) continue;
      double fa[3] = {0.0, 0.0, 0.0};
      for (int q = 0; q < NQP; ++q) {
        const double* rec = sm + (size_t)(el * NQP + q) * RC::R;
        const double wJ = rec[RC::oW];
        const double s0 = rec[RC::oS + 3 * a], s1 = rec[RC::oS + 3 * a + 1], s2 = rec[RC::oS + 3 * a + 2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          fa[i] += wJ * (rec[RC::oF + 3 * i] * s0 + rec[RC::oF + 3 * i + 1] * s1 + rec[RC::oF + 3 * i + 2] * s2);
      }
      const int c = s_conn[el][a];
#pragma unroll
      for (int i = 0; i < 3; ++i) atomicAdd(&A.f[3 * c + i], fa[i]);
    }
  }

  // ---- tangent blocks (a <= b) ---------------------------------------------
  if (DO_TANGENT) {
    const double c1 = A.alpha * A.mat.lam + (KV ? A.beta * A.mat.lam_d : 0.0);
    const double c2 = A.alpha * A.mat.mu + (KV ? A.beta * A.mat.eta : 0.0);
    for (int t = threadIdx.x; t < EPB * NP; t += NT) {
      const int el = t / NP, pr = t % NP;
      const int64_t e = ebase + el;
      if (e >= A.end) continue;
      int a, b;
      pair_of(pr, NEN, a, b);
      double K[3][3] = {};
      for (int q = 0; q < NQP; ++q) {
        const double* rec = sm + (size_t)(el * NQP + q) * RC::R;
        const double* na = rec + RC::oN + 3 * a;
        const double* nb = rec + RC::oN + 3 * b;
        if constexpr (!MR) {
          // [K_ab]_ik = wJ [c1 g_a,i g_b,k + c2 (g_b,i g_a,k + (n_a.n_b) B_ik) + alpha d_ik n_a.S n_b]
          const double wJ = rec[RC::oW];
          const double* ga = rec + RC::oG + 3 * a;
          const double* gb = rec + RC::oG + 3 * b;
          const double* sb = rec + RC::oS + 3 * b;
          const double nn = na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2];
          const double sn = na[0] * sb[0] + na[1] * sb[1] + na[2] * sb[2];
          const double w1 = wJ * c1, w2 = wJ * c2, w2n = w2 * nn, w3 = wJ * A.alpha * sn;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const double gai = ga[i], gbi = gb[i];
#pragma unroll
            for (int k = 0; k < 3; ++k)
              K[i][k] += w1 * gai * gb[k] + w2 * gbi * ga[k] + w2n * rec[RC::oB + 3 * i + k];
            K[i][i] += w3;
          }
        } else {
          // [K_ab]_ik = sum_J n_a,J sum_L A^_iJkL n_b,L (rows already scaled by wJ, alpha, beta)
          const double* Ar = rec + RC::oA;
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int J = 0; J < 3; ++J) {
              const double* r = Ar + i * 27 + J * 9;
#pragma unroll
              for (int k = 0; k < 3; ++k)
                K[i][k] += na[J] * (r[k * 3] * nb[0] + r[k * 3 + 1] * nb[1] + r[k * 3 + 2] * nb[2]);
            }
        }
      }
      if (A.mass_scale != 0.0) {
        const double ms = A.mass_scale * A.me[e * NP + pr];
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
        double* Ke = A.K_elem + (int64_t)A.user_of[e] * ND * ND;
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
// pass).
template <int ET>
tl_status launch_kind(tl_mesh* m, const double* q_n, const double* v, double h, double alpha, double beta,
                      double mass_scale, bool do_force, bool do_tangent, double* f, double* values,
                      double* K_elem) {
  Args A;
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
  A.alpha = alpha;
  A.beta = beta;
  A.mass_scale = mass_scale;
  A.f = f;
  A.values = values;
  A.K_elem = K_elem;
  A.flags = m->d_flags;
  for (const Segment& sg : m->segs) {
    const int64_t cnt = sg.end - sg.begin;
    if (cnt == 0) continue;
    const MaterialDev& md = m->mats[sg.mat];
    A.begin = sg.begin;
    A.end = sg.end;
    A.mat = to_matT<double>(md);
    const int combo = 2 * (md.kind == TL_SVK ? 0 : 1) + (md.kv ? 1 : 0);
    const int pass = (do_force ? 1 : 0) + (do_tangent ? 2 : 0);
    void (*kern)(Args) = nullptr;
    size_t smem = 0;
#define TL_ANCF_CASE(MATK, KVK, FO, TA)                                             \
  kern = elem_kernel<ET, MATK, KVK, FO, TA>;                                         \
  smem = smem_bytes<ET, TA, MATK == TL_MOONEY_RIVLIN>();
    switch (combo * 4 + pass) {
      case 0 * 4 + 1: TL_ANCF_CASE(TL_SVK, false, true, false) break;
      case 0 * 4 + 2: TL_ANCF_CASE(TL_SVK, false, false, true) break;
      case 0 * 4 + 3: TL_ANCF_CASE(TL_SVK, false, true, true) break;
      case 1 * 4 + 1: TL_ANCF_CASE(TL_SVK, true, true, false) break;
      case 1 * 4 + 2: TL_ANCF_CASE(TL_SVK, true, false, true) break;
      case 1 * 4 + 3: TL_ANCF_CASE(TL_SVK, true, true, true) break;
      case 2 * 4 + 1: TL_ANCF_CASE(TL_MOONEY_RIVLIN, false, true, false) break;
      case 2 * 4 + 2: TL_ANCF_CASE(TL_MOONEY_RIVLIN, false, false, true) break;
      case 2 * 4 + 3: TL_ANCF_CASE(TL_MOONEY_RIVLIN, false, true, true) break;
      case 3 * 4 + 1: TL_ANCF_CASE(TL_MOONEY_RIVLIN, true, true, false) break;
      case 3 * 4 + 2: TL_ANCF_CASE(TL_MOONEY_RIVLIN, true, false, true) break;
      case 3 * 4 + 3: TL_ANCF_CASE(TL_MOONEY_RIVLIN, true, true, true) break;
      default: return TL_OK;   // nothing requested
    }
#undef TL_ANCF_CASE
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
