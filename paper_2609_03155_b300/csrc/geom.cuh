// Trilinear element map and 3 x 3 inverse, shared by the quadrature kernels.
#pragma once

namespace dpg {

// Trilinear map of the corner coordinates X (8 x 3) at reference point xi.
__device__ __forceinline__ void geom(const double* X, const double xi[3], double J[3][3], double x[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = 0.0;
    J[a][0] = J[a][1] = J[a][2] = 0.0;
  }
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    double f0 = (v & 1) ? xi[0] : 1.0 - xi[0], d0 = (v & 1) ? 1.0 : -1.0;
    double f1 = (v & 2) ? xi[1] : 1.0 - xi[1], d1 = (v & 2) ? 1.0 : -1.0;
    double f2 = (v & 4) ? xi[2] : 1.0 - xi[2], d2 = (v & 4) ? 1.0 : -1.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double Xa = X[3 * v + a];
      x[a] += f0 * f1 * f2 * Xa;
      J[a][0] += d0 * f1 * f2 * Xa;
      J[a][1] += f0 * d1 * f2 * Xa;
      J[a][2] += f0 * f1 * d2 * Xa;
    }
  }
}

__device__ __forceinline__ double inv3(const double J[3][3], double Ji[3][3]) {
  double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  double id = 1.0 / det;
  Ji[0][0] = c00 * id;
  Ji[1][0] = c01 * id;
  Ji[2][0] = c02 * id;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  return det;
}

}  // namespace dpg
