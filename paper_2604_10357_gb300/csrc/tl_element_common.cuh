// Quadrature-point arithmetic of the element kernels (tl_element.cu): shape
// gradients, constitutive laws and their tangents.
//
// Paper: arxiv 2604.10357 Sec. 4.3 (eq. F_assembly, P = P_el + P_vis, T10 with
// the 5-point Keast rule) and Sec. 4.4 (the material tangent A_{iJkL} entering
// eq. tangent_block).  Constitutive forms: SVK, compressible Mooney-Rivlin and
// Kelvin-Voigt as stated in include/tl.h.
#pragma once

#include "tl_dfloat.cuh"
#include "tl_internal.cuh"

namespace tl {
namespace {

// Keast 5-point rule: barycentric coordinates and weights (fraction of V).
__device__ __forceinline__ void qp_bary(int q, double L[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) L[k] = (q == 0) ? 0.25 : (k == q - 1 ? 0.5 : 1.0 / 6.0);
}
__device__ __forceinline__ double qp_wfrac(int q) { return q == 0 ? -0.8 : 0.45; }

// Exact consistent mass of a straight-sided T10 in units of rho V / 420.
__constant__ float c_mass420[10][10] = {
    {6, 1, 1, 1, -4, -6, -4, -4, -6, -6},     {1, 6, 1, 1, -4, -4, -6, -6, -4, -6},
    {1, 1, 6, 1, -6, -4, -4, -6, -6, -4},     {1, 1, 1, 6, -6, -6, -6, -4, -4, -4},
    {-4, -4, -6, -6, 32, 16, 16, 16, 16, 8},  {-6, -4, -4, -6, 16, 32, 16, 8, 16, 16},
    {-4, -6, -4, -6, 16, 16, 32, 16, 8, 16},  {-4, -6, -6, -4, 16, 8, 16, 32, 16, 16},
    {-6, -4, -6, -4, 16, 16, 8, 16, 32, 16},  {-6, -6, -4, -4, 8, 16, 16, 16, 16, 32}};

// midside node m (4..9) lies on corners (ei[m-4], ej[m-4])
__device__ __forceinline__ int edge_i(int m) { return (m == 4 || m == 6 || m == 7) ? 0 : (m == 5 || m == 8) ? 1 : 2; }
__device__ __forceinline__ int edge_j(int m) { return (m == 4) ? 1 : (m == 5 || m == 6) ? 2 : 3; }

template <typename T>
struct MatT {
  T lam, mu, C10, C01, kappa, eta, lam_d, rho;
};

template <typename T>
__device__ __forceinline__ T rcbrt_t(T x);
template <>
__device__ __forceinline__ float rcbrt_t<float>(float x) { return rcbrtf(x); }
template <>
__device__ __forceinline__ double rcbrt_t<double>(double x) { return rcbrt(x); }
template <>
__device__ __forceinline__ dfl rcbrt_t<dfl>(dfl x) {      // float64 reciprocal cube root, once per qp
  return dfl(rcbrt((double)x));
}

// ---------------------------------------------------------------------------
// Constitutive update at one quadrature point.
// In:  Hm = displacement gradient, Fd = velocity gradient (if KV).
// Out: F, total second Piola-Kirchhoff stress S (elastic + viscous),
//      and everything the tangent rows need.
// ---------------------------------------------------------------------------
template <typename T>
struct QP {
  T F[3][3];
  T S[3][3];       // S_el + S_v
  T Sv[3][3];      // viscous part
  T G[3][3];       // F^{-T} (MR)
  T Q[3][3];       // I1 F - F C (MR)
  T B[3][3];       // F F^T
  T C[3][3];
  T J, I1, I2;
};

template <typename T>
__device__ __forceinline__ void sym3_inverse(const T C[3][3], T detC, T Ci[3][3]) {
  const T inv = T(1) / detC;
  Ci[0][0] = (C[1][1] * C[2][2] - C[1][2] * C[2][1]) * inv;
  Ci[0][1] = (C[0][2] * C[2][1] - C[0][1] * C[2][2]) * inv;
  Ci[0][2] = (C[0][1] * C[1][2] - C[0][2] * C[1][1]) * inv;
  Ci[1][1] = (C[0][0] * C[2][2] - C[0][2] * C[2][0]) * inv;
  Ci[1][2] = (C[0][2] * C[1][0] - C[0][0] * C[1][2]) * inv;
  Ci[2][2] = (C[0][0] * C[1][1] - C[0][1] * C[1][0]) * inv;
  Ci[1][0] = Ci[0][1];
  Ci[2][0] = Ci[0][2];
  Ci[2][1] = Ci[1][2];
}

template <typename T, int MAT, bool KV>
__device__ __forceinline__ void constitutive(const T Hm[3][3], const T Fd[3][3], const MatT<T>& mp,
                                             QP<T>& s, bool& inverted) {
  // F = I + H;  E = (H + H^T + H^T H)/2
  T Em[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      s.F[i][j] = Hm[i][j] + (i == j ? T(1) : T(0));
      T hh = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) hh += Hm[k][i] * Hm[k][j];
      Em[i][j] = T(0.5) * (Hm[i][j] + Hm[j][i] + hh);
    }
  // J - 1 from the invariants of H: det(I+H) = 1 + trH + (tr^2 H - tr H^2)/2 + det H
  const T trH = Hm[0][0] + Hm[1][1] + Hm[2][2];
  T trH2 = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) trH2 += Hm[i][k] * Hm[k][i];
  const T detH = Hm[0][0] * (Hm[1][1] * Hm[2][2] - Hm[1][2] * Hm[2][1]) -
                 Hm[0][1] * (Hm[1][0] * Hm[2][2] - Hm[1][2] * Hm[2][0]) +
                 Hm[0][2] * (Hm[1][0] * Hm[2][1] - Hm[1][1] * Hm[2][0]);
  const T Jm1 = trH + T(0.5) * (trH * trH - trH2) + detH;
  s.J = T(1) + Jm1;
  if (!(s.J > T(0))) inverted = true;
  const T trE = Em[0][0] + Em[1][1] + Em[2][2];

  if (MAT == TL_SVK) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) s.S[i][j] = T(2) * mp.mu * Em[i][j] + (i == j ? mp.lam * trE : T(0));
  } else {
    // C = I + 2E; S = C^{-1} [4a dev E + 2b((2 + 4 trE) dev E - 4 dev(E^2))] + kappa (J-1) J C^{-1}
    // with a = C10 J^{-2/3}, b = C01 J^{-4/3}.
    T Cm[3][3], Ci[3][3], dE[3][3], dE2[3][3];
    T E2[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        Cm[i][j] = T(2) * Em[i][j] + (i == j ? T(1) : T(0));
        T acc = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) acc += Em[i][k] * Em[k][j];
        E2[i][j] = acc;
      }
    const T trE2 = E2[0][0] + E2[1][1] + E2[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        dE[i][j] = Em[i][j] - (i == j ? trE / T(3) : T(0));
        dE2[i][j] = E2[i][j] - (i == j ? trE2 / T(3) : T(0));
      }
    const T J = s.J;
    sym3_inverse(Cm, J * J, Ci);
    const T r = rcbrt_t<T>(J);
    const T a = mp.C10 * r * r;
    const T b = mp.C01 * r * r * r * r;
    T Mm[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Mm[i][j] = T(4) * a * dE[i][j] + T(2) * b * ((T(2) + T(4) * trE) * dE[i][j] - T(4) * dE2[i][j]);
    const T vol = mp.kappa * Jm1 * J;
    T Sx[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T acc = vol * Ci[i][j];
#pragma unroll
        for (int k = 0; k < 3; ++k) acc += Ci[i][k] * Mm[k][j];
        Sx[i][j] = acc;
      }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) s.S[i][j] = T(0.5) * (Sx[i][j] + Sx[j][i]);
    // tangent ingredients
    s.I1 = T(3) + T(2) * trE;
    // I2 = (I1^2 - tr C^2)/2 ; tr C^2 = 3 + 4 trE + 4 tr E^2
    s.I2 = T(0.5) * (s.I1 * s.I1 - (T(3) + T(4) * trE + T(4) * trE2));
    const T Ji = T(1) / J;
    // G = F^{-T} = cof(F) / J
    const T(&F)[3][3] = s.F;
    s.G[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) * Ji;
    s.G[0][1] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) * Ji;
    s.G[0][2] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) * Ji;
    s.G[1][0] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * Ji;
    s.G[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * Ji;
    s.G[1][2] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * Ji;
    s.G[2][0] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * Ji;
    s.G[2][1] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * Ji;
    s.G[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * Ji;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) s.C[i][j] = Cm[i][j];
    // Q = F (I1 I - C)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T acc = s.I1 * F[i][j];
#pragma unroll
        for (int k = 0; k < 3; ++k) acc -= F[i][k] * Cm[k][j];
        s.Q[i][j] = acc;
      }
  }
  // B = F F^T (SVK and MR tangents, Kelvin-Voigt tangent)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) acc += s.F[i][k] * s.F[j][k];
      s.B[i][j] = acc;
    }
  if (KV) {
    // Edot = sym(F^T Fdot) = sym(Fdot + H^T Fdot); S_v = lam_d tr(Edot) I + 2 eta Edot
    T Ed[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T a1 = Fd[i][j], a2 = Fd[j][i];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          a1 += Hm[k][i] * Fd[k][j];
          a2 += Hm[k][j] * Fd[k][i];
        }
        Ed[i][j] = T(0.5) * (a1 + a2);
      }
    const T trEd = Ed[0][0] + Ed[1][1] + Ed[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        s.Sv[i][j] = T(2) * mp.eta * Ed[i][j] + (i == j ? mp.lam_d * trEd : T(0));
        s.S[i][j] += s.Sv[i][j];
      }
  }
}

// Tangent entry A^_{iJkL} for fixed row i (27 values at [J*9 + k*3 + L]),
// scaled by wJ0:  alpha * A_t + beta * A_vis.
template <typename T, int MAT, bool KV, int i>
__device__ __forceinline__ void tangent_row(const QP<T>& s, const MatT<T>& mp, T alpha, T beta, T wJ, T* out) {
  if (MAT == TL_SVK) {
    // A_t = d_ik S_JL + lam F_iJ F_kL + mu (B_ik d_JL + F_iL F_kJ)
    // A_v = lam_d F_iJ F_kL + eta (B_ik d_JL + F_iL F_kJ)
    const T cFF = wJ * (alpha * mp.lam + (KV ? beta * mp.lam_d : T(0)));
    const T cB = wJ * (alpha * mp.mu + (KV ? beta * mp.eta : T(0)));
    const T cS = wJ * alpha;
#pragma unroll
    for (int J = 0; J < 3; ++J)
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int L = 0; L < 3; ++L) {
          T v = cFF * s.F[i][J] * s.F[k][L] + cB * (s.F[i][L] * s.F[k][J] + (J == L ? s.B[i][k] : T(0)));
          if (i == k) v += cS * s.S[J][L];
          out[J * 9 + k * 3 + L] = v;
        }
  } else {
    // Mooney-Rivlin tangent (d_ik X_JL + cB B_ik d_JL + rank-one and swap terms)
    const T r = rcbrt_t<T>(s.J);
    const T a = mp.C10 * r * r;
    const T b = mp.C01 * r * r * r * r;
    const T J = s.J;
    const T cdd = T(2) * a + T(2) * b * s.I1;
    const T cC = -T(2) * b;
    const T cB = -T(2) * b;
    const T cFF = T(4) * b;
    const T cFFs = -T(2) * b;
    const T cFG = -(T(4) / T(3)) * a;
    const T cQG = -(T(8) / T(3)) * b;
    const T cGG = (T(4) / T(9)) * a * s.I1 + (T(16) / T(9)) * b * s.I2 + mp.kappa * (T(2) * J * J - J);
    const T cGGs = (T(2) / T(3)) * a * s.I1 + (T(4) / T(3)) * b * s.I2 - mp.kappa * (J * J - J);
    const T wa = wJ * alpha;
    const T wb = wJ * beta;
#pragma unroll
    for (int Jx = 0; Jx < 3; ++Jx)
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int L = 0; L < 3; ++L) {
          const T FiJ = s.F[i][Jx], FkL = s.F[k][L], FiL = s.F[i][L], FkJ = s.F[k][Jx];
          const T GiJ = s.G[i][Jx], GkL = s.G[k][L], GiL = s.G[i][L], GkJ = s.G[k][Jx];
          T vA = cFF * FiJ * FkL + cFFs * FiL * FkJ + cFG * (FiJ * GkL + GiJ * FkL) +
                 cQG * (s.Q[i][Jx] * GkL + GiJ * s.Q[k][L]) + cGG * GiJ * GkL + cGGs * GiL * GkJ;
          if (Jx == L) vA += cB * s.B[i][k];
          if (i == k) {
            vA += cC * s.C[Jx][L] + (Jx == L ? cdd : T(0));
            if (KV) vA += s.Sv[Jx][L];      // geometric term of the viscous stress
          }
          T v = wa * vA;
          if (KV) v += wb * (mp.lam_d * FiJ * FkL + mp.eta * (FiL * FkJ + (Jx == L ? s.B[i][k] : T(0))));
          out[Jx * 9 + k * 3 + L] = v;
        }
  }
}

template <typename T>
__device__ __forceinline__ void atomic_add_t(T* p, T v);
template <>
__device__ __forceinline__ void atomic_add_t<float>(float* p, float v) { atomicAdd(p, v); }
template <>
__device__ __forceinline__ void atomic_add_t<double>(double* p, double v) { atomicAdd(p, v); }

template <typename T>
MatT<T> to_matT(const MaterialDev& md) {
  MatT<T> m;
  m.lam = T(md.lam);
  m.mu = T(md.mu);
  m.C10 = T(md.C10);
  m.C01 = T(md.C01);
  m.kappa = T(md.kappa);
  m.eta = T(md.eta);
  m.lam_d = T(md.lam_d);
  m.rho = T(md.rho);
  return m;
}

}  // namespace
}  // namespace tl
