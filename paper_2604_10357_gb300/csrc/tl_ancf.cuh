// ANCF3243 beam and ANCF3443 shell elements: closed-form shape functions,
// their natural-coordinate derivatives and the Gauss-Legendre rules, shared
// by the host-side validation (tl_api.cu) and the kernels (tl_ancf.cu).
//
// Paper: arxiv 2604.10357 Sec. 4.3 (8 shape functions per beam element and 16
// per shell element, four coefficient vectors r, r_x, r_y, r_z per physical
// node; 3 x 2 x 2 and 4 x 4 x 3 Gauss-Legendre rules) and Sec. 2 (q holds
// positions and position gradients).
//
// Beam (length L, width W, height H; xi along the axis, x = L (1 + xi)/2,
// y = W eta / 2, z = H zeta / 2): the cubic Hermite polynomials of the end
// positions and axial slopes, plus y r_y + z r_z interpolated linearly along
// the axis.  Shell (L x W x H; x = L (1 + xi)/2, y = W (1 + eta)/2,
// z = H zeta / 2; corners (-1,-1), (1,-1), (1,1), (-1,1)): the 12-term
// incomplete bicubic rectangle functions of r, r_x, r_y at the corners, plus
// z times the bilinear corner functions for r_z.  Coefficient a = 4 c + k
// (c: node / corner, k: r, r_x, r_y, r_z).
#pragma once

#include <cmath>

namespace tl {
namespace ancf {

enum : int { kBeam = 0, kShell = 1 };

template <int ET>
struct Traits;
template <>
struct Traits<kBeam> {
  static constexpr int NEN = 8, NQP = 12, NMQ = 16;   // shape functions, element / mass points
};
template <>
struct Traits<kShell> {
  static constexpr int NEN = 16, NQP = 48, NMQ = 32;
};

// n-point Gauss-Legendre abscissa / weight on [-1, 1], i = 0..n-1 (n = 2, 3, 4),
// evaluated in T (float: single-precision square roots, no float64 work).
template <typename T>
__host__ __device__ inline void gauss(int n, int i, T& x, T& w) {
  if (n == 2) {
    x = (i == 0 ? T(-1) : T(1)) / sqrt(T(3));
    w = T(1);
  } else if (n == 3) {
    x = i == 1 ? T(0) : (i == 0 ? T(-1) : T(1)) * sqrt(T(0.6));
    w = i == 1 ? T(8) / T(9) : T(5) / T(9);
  } else {   // 4 points: +-sqrt(3/7 -+ 2/7 sqrt(6/5)), weights (18 +- sqrt 30)/36
    const T r = T(2) / T(7) * sqrt(T(1.2));
    const bool inner = (i == 1 || i == 2);
    x = (i < 2 ? T(-1) : T(1)) * sqrt(T(3) / T(7) + (inner ? -r : r));
    w = (T(18) + (inner ? T(1) : T(-1)) * sqrt(T(30))) / T(36);
  }
}

// Point q of the element rule (xi slowest, zeta fastest) and its weight.
template <int ET, typename T>
__host__ __device__ inline void element_point(int q, T p[3], T& w) {
  T w0, w1, w2;
  if (ET == kBeam) {            // 3 x 2 x 2
    gauss<T>(3, q / 4, p[0], w0);
    gauss<T>(2, (q / 2) % 2, p[1], w1);
    gauss<T>(2, q % 2, p[2], w2);
  } else {                      // 4 x 4 x 3
    gauss<T>(4, q / 12, p[0], w0);
    gauss<T>(4, (q / 3) % 4, p[1], w1);
    gauss<T>(3, q % 3, p[2], w2);
  }
  w = w0 * w1 * w2;
}

// Point q of the mass rule (exact for S_a S_b of a rectangular element).
template <int ET>
__host__ __device__ inline void mass_point(int q, double p[3], double& w) {
  double w0, w1, w2;
  if (ET == kBeam) {            // 4 x 2 x 2
    gauss<double>(4, q / 4, p[0], w0);
    gauss<double>(2, (q / 2) % 2, p[1], w1);
    gauss<double>(2, q % 2, p[2], w2);
  } else {                      // 4 x 4 x 2
    gauss<double>(4, q / 8, p[0], w0);
    gauss<double>(4, (q / 2) % 4, p[1], w1);
    gauss<double>(2, q % 2, p[2], w2);
  }
  w = w0 * w1 * w2;
}

// Shape function a: value S (optional) and d/d(xi, eta, zeta) at p; dims = L, W, H
// (T = double, or float for the float32 element form).
template <int ET, typename T>
__host__ __device__ inline void shape(int a, const T p[3], const T dims[3], T* S, T d[3]) {
  const T xi = p[0], eta = p[1], zeta = p[2];
  const T L = dims[0], W = dims[1], H = dims[2];
  if (ET == kBeam) {
    const int node = a >> 2, k = a & 3;
    const T sg = node ? T(1.0) : -T(1.0);          // end at xi = -1 (node 0) or +1 (node 1)
    const T lin = T(0.5) * (T(1.0) + sg * xi);     // linear end function
    switch (k) {
      case 0:   // (2 -+ 3 xi +- xi^3) / 4
        if (S) *S = T(0.25) * (T(2.0) + sg * (T(3.0) * xi - xi * xi * xi));
        d[0] = T(0.75) * sg * (T(1.0) - xi * xi);
        d[1] = d[2] = T(0.0);
        break;
      case 1:   // L (1 + sg xi)^2 (sg xi - 1) sg / 8
      {
        const T a1 = T(1.0) + sg * xi;
        if (S) *S = T(0.125) * L * sg * a1 * a1 * (sg * xi - T(1.0));
        d[0] = T(0.125) * L * a1 * (T(3.0) * sg * xi - T(1.0));
        d[1] = d[2] = T(0.0);
        break;
      }
      case 2:   // y lin
        if (S) *S = T(0.5) * W * eta * lin;
        d[0] = T(0.25) * W * eta * sg;
        d[1] = T(0.5) * W * lin;
        d[2] = T(0.0);
        break;
      default:  // z lin
        if (S) *S = T(0.5) * H * zeta * lin;
        d[0] = T(0.25) * H * zeta * sg;
        d[1] = T(0.0);
        d[2] = T(0.5) * H * lin;
        break;
    }
  } else {
    const int c = a >> 2, k = a & 3;
    const T xc = (c == 1 || c == 2) ? T(1.0) : -T(1.0);
    const T yc = (c >= 2) ? T(1.0) : -T(1.0);
    const T A = T(1.0) + xc * xi, B = T(1.0) + yc * eta;
    switch (k) {
      case 0: {  // A B (2 + xc xi + yc eta - xi^2 - eta^2) / 8
        const T g = T(2.0) + xc * xi + yc * eta - xi * xi - eta * eta;
        if (S) *S = T(0.125) * A * B * g;
        d[0] = T(0.125) * B * (xc * g + A * (xc - T(2.0) * xi));
        d[1] = T(0.125) * A * (yc * g + B * (yc - T(2.0) * eta));
        d[2] = T(0.0);
        break;
      }
      case 1:    // (L/16) xc A^2 (xc xi - 1) B
        if (S) *S = L / T(16.0) * xc * A * A * (xc * xi - T(1.0)) * B;
        d[0] = L / T(16.0) * A * B * (T(3.0) * xc * xi - T(1.0));
        d[1] = L / T(16.0) * xc * A * A * (xc * xi - T(1.0)) * yc;
        d[2] = T(0.0);
        break;
      case 2:    // (W/16) yc B^2 (yc eta - 1) A
        if (S) *S = W / T(16.0) * yc * B * B * (yc * eta - T(1.0)) * A;
        d[0] = W / T(16.0) * yc * B * B * (yc * eta - T(1.0)) * xc;
        d[1] = W / T(16.0) * A * B * (T(3.0) * yc * eta - T(1.0));
        d[2] = T(0.0);
        break;
      default:   // (H/8) zeta A B
        if (S) *S = T(0.125) * H * zeta * A * B;
        d[0] = T(0.125) * H * zeta * xc * B;
        d[1] = T(0.125) * H * zeta * yc * A;
        d[2] = T(0.125) * H * A * B;
        break;
    }
  }
}

// det of a 3 x 3 matrix and its inverse (returns det).
template <typename T>
__host__ __device__ inline T inv3(const T J[3][3], T Ji[3][3]) {
  const T c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const T c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const T c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const T det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  const T r = T(1.0) / det;
  Ji[0][0] = c00 * r;
  Ji[1][0] = c01 * r;
  Ji[2][0] = c02 * r;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * r;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * r;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * r;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * r;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * r;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * r;
  return det;
}

// Upper-triangle block pair pr -> (a, b), a <= b, row-major over a.
__host__ __device__ inline void pair_of(int pr, int nen, int& a, int& b) {
  a = 0;
  int row = nen;
  while (pr >= row) {
    pr -= row;
    ++a;
    --row;
  }
  b = a + pr;
}

}  // namespace ancf
}  // namespace tl
