// Geometry of an affine tetrahedron shared by the element kernels.
#pragma once

namespace tam {

// Gradients of the barycentric coordinates and the volume of a tet.
__device__ __forceinline__ bool tet_geometry(const double* __restrict__ X, const int* v, double g[4][3], double& vol) {
  double x0 = X[3 * v[0]], y0 = X[3 * v[0] + 1], z0 = X[3 * v[0] + 2];
  double a[3][3];  // rows: edge vectors x_k - x_0
  for (int k = 0; k < 3; ++k) {
    a[k][0] = X[3 * v[k + 1]] - x0;
    a[k][1] = X[3 * v[k + 1] + 1] - y0;
    a[k][2] = X[3 * v[k + 1] + 2] - z0;
  }
  // cofactors: grad l_{k+1} = (row k of inverse of the matrix with columns a_k)
  double c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
  double c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
  double c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
  double det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
  vol = det / 6.0;
  if (!(vol > 0.0) || !isfinite(vol)) return false;
  double id = 1.0 / det;
  // grad l1 = (a1 x a2)/det, grad l2 = (a2 x a0)/det, grad l3 = (a0 x a1)/det
  g[1][0] = c00 * id; g[1][1] = c01 * id; g[1][2] = c02 * id;
  g[2][0] = (a[2][1] * a[0][2] - a[2][2] * a[0][1]) * id;
  g[2][1] = (a[2][2] * a[0][0] - a[2][0] * a[0][2]) * id;
  g[2][2] = (a[2][0] * a[0][1] - a[2][1] * a[0][0]) * id;
  g[3][0] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
  g[3][1] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
  g[3][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
  for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
  return true;
}

}  // namespace tam
