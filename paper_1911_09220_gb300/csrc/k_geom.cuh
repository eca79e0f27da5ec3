// Element geometry for the setup-type kernels (Sec. 3.1): the trilinear map
// of the 8 vertices, or the order-k nodal map of a curved mesh. Both give
// J[r][c] = d x_r / d xhat_c and x at the tensor Gauss point (q1, q2, q3).
#pragma once

#include <stdint.h>

// Trilinear map on [0,1]^3 from the 8 vertex coordinates (local order
// (0,0,0) (1,0,0) (1,1,0) (0,1,0), then z = 1).
struct Hex8Geo {
  const double* coords;
  const int32_t* hex;
  const double* qpts;  // Gauss points on [0,1]
  double X[8][3];
  __device__ static int cx(int v) { return (v == 1 || v == 2 || v == 5 || v == 6); }
  __device__ static int cy(int v) { return (v == 2 || v == 3 || v == 6 || v == 7); }
  __device__ static int cz(int v) { return v >= 4; }
  __device__ void load(int64_t e) {
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int32_t g = hex[8 * e + v];
#pragma unroll
      for (int d = 0; d < 3; ++d) X[v][d] = coords[3 * (int64_t)g + d];
    }
  }
  __device__ void map_ref(double a, double b, double c, double x[3]) const {
    x[0] = x[1] = x[2] = 0.0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const double N = (cx(v) ? a : 1.0 - a) * (cy(v) ? b : 1.0 - b) * (cz(v) ? c : 1.0 - c);
#pragma unroll
      for (int d = 0; d < 3; ++d) x[d] += N * X[v][d];
    }
  }
  __device__ void jacobian_ref(double a, double b, double c, double J[3][3]) const {
#pragma unroll
    for (int r = 0; r < 3; ++r) J[r][0] = J[r][1] = J[r][2] = 0.0;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const double fa = cx(v) ? a : 1.0 - a, da = cx(v) ? 1.0 : -1.0;
      const double fb = cy(v) ? b : 1.0 - b, db = cy(v) ? 1.0 : -1.0;
      const double fc = cz(v) ? c : 1.0 - c, dc = cz(v) ? 1.0 : -1.0;
      const double g0 = da * fb * fc, g1 = fa * db * fc, g2 = fa * fb * dc;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        J[r][0] += X[v][r] * g0;
        J[r][1] += X[v][r] * g1;
        J[r][2] += X[v][r] * g2;
      }
    }
  }
  __device__ void jacobian(int q1, int q2, int q3, double J[3][3]) const {
    jacobian_ref(qpts[q1], qpts[q2], qpts[q3], J);
  }
  __device__ void map(int q1, int q2, int q3, double x[3]) const { map_ref(qpts[q1], qpts[q2], qpts[q3], x); }
};

// Order-k nodal map: x(xhat) = sum_i X_i w_i(xhat) with the (k+1)^3 GLL
// Lagrange functions w_i (lexicographic, first index fastest) and element
// e's nodal coordinates X [(k+1)^3][3]. gB, gG [Q][k+1]: the 1D functions
// and derivatives at the Gauss points.
struct NodalGeo {
  const double* nodes;  // [ne][(k+1)^3][3]
  const double* gB;
  const double* gG;
  int K;                // k + 1
  const double* Xe;
  __device__ void load(int64_t e) { Xe = nodes + e * (int64_t)K * K * K * 3; }
  __device__ void jacobian(int q1, int q2, int q3, double J[3][3]) const {
#pragma unroll
    for (int r = 0; r < 3; ++r) J[r][0] = J[r][1] = J[r][2] = 0.0;
    for (int i3 = 0; i3 < K; ++i3) {
      const double b3 = gB[q3 * K + i3], g3 = gG[q3 * K + i3];
      for (int i2 = 0; i2 < K; ++i2) {
        const double b2 = gB[q2 * K + i2], g2 = gG[q2 * K + i2];
        for (int i1 = 0; i1 < K; ++i1) {
          const double b1 = gB[q1 * K + i1], g1 = gG[q1 * K + i1];
          const double w0 = g1 * b2 * b3, w1 = b1 * g2 * b3, w2 = b1 * b2 * g3;
          const double* x = Xe + 3 * ((i3 * K + i2) * K + i1);
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            J[r][0] += x[r] * w0;
            J[r][1] += x[r] * w1;
            J[r][2] += x[r] * w2;
          }
        }
      }
    }
  }
  __device__ void map(int q1, int q2, int q3, double xo[3]) const {
    xo[0] = xo[1] = xo[2] = 0.0;
    for (int i3 = 0; i3 < K; ++i3)
      for (int i2 = 0; i2 < K; ++i2) {
        const double b23 = gB[q2 * K + i2] * gB[q3 * K + i3];
        for (int i1 = 0; i1 < K; ++i1) {
          const double w = gB[q1 * K + i1] * b23;
          const double* x = Xe + 3 * ((i3 * K + i2) * K + i1);
#pragma unroll
          for (int r = 0; r < 3; ++r) xo[r] += x[r] * w;
        }
      }
  }
};

__device__ inline double det3(const double J[3][3]) {
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}
