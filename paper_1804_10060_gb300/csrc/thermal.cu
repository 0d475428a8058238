// The thermal half of the model (paper Sec. 3): the heat equation
//   rho c_v dT/dt - div(kappa grad T) = 0,  kappa grad T . n = beta (T - T_bc) on Gamma_N^T,
// discretised by the theta-method (Eq. wf_thermal) on P1/P2 tetrahedra and
// solved by Newton's method on the full linearisation (Sec. 3 "Solution
// strategy"), each Newton step by CG preconditioned with the scalar
// smoothed-aggregation AMG of this library (constant near-nullspace), and the
// adaptive time step of Eq. dt_spec.
//
// With c_v(T) = c0 + c1 T and kappa(T) = k0 + k1 T (affine per material) the
// theta-weighted coefficients are those of T_theta = (1 - theta) T_m + theta T:
//   F_i = int rho c_v(T_theta) (T - T_m)/dt phi_i + int kappa(T_theta) grad T_theta . grad phi_i
//         - int_Gamma beta (T_theta - T_bc) phi_i
//   J_ij = dF_i/dT_j = int rho (c1 theta (T - T_m)/dt + c_v(T_theta)/dt) phi_j phi_i
//         + theta int (k1 phi_j grad T_theta . grad phi_i + kappa(T_theta) grad phi_j . grad phi_i)
//         - theta int_Gamma beta phi_j phi_i
// The steady problem drops the mass terms and takes theta = 1.
//
// Integration: the mass terms use the reference tensors int phi_a phi_b phi_c
// and int phi_a phi_b, the conduction terms quadrature at every point, the
// Robin terms the face mass matrix -- all exact for the polynomial degrees
// involved, from Gauss-Jacobi product (Stroud conical) rules generated here
// on the host.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "handles.cuh"
#include "tet.cuh"

namespace tam {
namespace {

// ---------------------------------------------------------------------------
// Quadrature: Gauss-Jacobi rules on [0, 1] with weight (1 - x)^alpha, by the
// eigenvalues of the Jacobi matrix (bisection on Sturm counts) and the
// weights w_i = 1 / sum_k p_k(x_i)^2 of the orthonormal polynomials.
// ---------------------------------------------------------------------------
void gauss_jacobi01(int n, int alpha, std::vector<double>& x, std::vector<double>& w) {
  // recurrence of the monic Jacobi polynomials P^(alpha, 0) on [-1, 1]
  std::vector<double> a(n), b(n, 0.0);
  const double al = alpha;
  for (int k = 0; k < n; ++k) {
    const double s = 2.0 * k + al;
    a[k] = (k == 0 && alpha == 0) ? 0.0 : -al * al / (s * (s + 2.0));
    if (k > 0) b[k] = 4.0 * k * k * (k + al) * (k + al) / (s * s * (s + 1.0) * (s - 1.0));
  }
  const double mu0 = std::pow(2.0, al + 1.0) / (al + 1.0);
  auto count_below = [&](double t) {  // eigenvalues of the Jacobi matrix below t
    int c = 0;
    double q = 1.0;
    for (int k = 0; k < n; ++k) {
      q = a[k] - t - (k > 0 ? b[k] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++c;
    }
    return c;
  };
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double lo = -1.0, hi = 1.0;  // the nodes lie inside (-1, 1)
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (count_below(mid) > i) hi = mid; else lo = mid;
    }
    const double t = 0.5 * (lo + hi);
    // orthonormal polynomials at t
    double pm = 0.0, p = 1.0 / std::sqrt(mu0), sum = p * p;
    for (int k = 0; k + 1 < n; ++k) {
      const double pn = ((t - a[k]) * p - (k > 0 ? std::sqrt(b[k]) * pm : 0.0)) / std::sqrt(b[k + 1]);
      pm = p;
      p = pn;
      sum += p * p;
    }
    x[i] = 0.5 * (1.0 + t);                       // to [0, 1]
    w[i] = (1.0 / sum) / std::pow(2.0, al + 1.0);  // weight (1 - x)^alpha dx on [0, 1]
  }
}

// Points (barycentric l0..l3) and weights (summing to 1, i.e. divided by the
// reference volume 1/6) of the conical product rule with n points per axis:
// exact for polynomials of degree 2n - 1 on the tetrahedron.
void tet_rule(int n, std::vector<double>& pts, std::vector<double>& wts) {
  std::vector<double> x1, w1, x2, w2, x3, w3;
  gauss_jacobi01(n, 0, x1, w1);
  gauss_jacobi01(n, 1, x2, w2);
  gauss_jacobi01(n, 2, x3, w3);
  pts.clear();
  wts.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        const double z = x3[k], y = x2[j] * (1.0 - z), xx = x1[i] * (1.0 - x2[j]) * (1.0 - z);
        pts.insert(pts.end(), {1.0 - xx - y - z, xx, y, z});
        wts.push_back(6.0 * w1[i] * w2[j] * w3[k]);
      }
}

// The same on a triangle (barycentric m0..m2, weights summing to 1).
void tri_rule(int n, std::vector<double>& pts, std::vector<double>& wts) {
  std::vector<double> x1, w1, x2, w2;
  gauss_jacobi01(n, 0, x1, w1);
  gauss_jacobi01(n, 1, x2, w2);
  pts.clear();
  wts.clear();
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double y = x2[j], xx = x1[i] * (1.0 - y);
      pts.insert(pts.end(), {1.0 - xx - y, xx, y});
      wts.push_back(2.0 * w1[i] * w2[j]);
    }
}

// Lagrange basis functions on the reference cell / face, barycentric input.
constexpr int EDGE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
constexpr int FEDGE[3][2] = {{0, 1}, {1, 2}, {2, 0}};

double cell_phi(int deg, int a, const double* l) {
  if (deg == 1) return l[a];
  if (a < 4) return l[a] * (2.0 * l[a] - 1.0);
  return 4.0 * l[EDGE[a - 4][0]] * l[EDGE[a - 4][1]];
}

double face_phi(int deg, int a, const double* m) {
  if (deg == 1) return m[a];
  if (a < 3) return m[a] * (2.0 * m[a] - 1.0);
  return 4.0 * m[FEDGE[a - 3][0]] * m[FEDGE[a - 3][1]];
}

// ---------------------------------------------------------------------------
// Constant tables (filled once per device by thermal_tables()):
//   d_T3p2[a][b][c] = int phi_a phi_b phi_c / |K| (P2), d_M2p2 = int phi_a phi_b / |K|,
//   the same for P1, the face mass matrices int psi_a psi_b / |F|, and the P2
//   conduction rule (11 points: barycentrics and weights / |K|) with the P2
//   basis values there.  The P2 tables the kernel indexes per lane live in
//   global memory (read through L1): constant memory serialises a warp's
//   accesses to different addresses.
// ---------------------------------------------------------------------------
constexpr int NQ2 = 11;
__device__ double d_T3p2[10][10][10];
__device__ double d_M2p2[10][10];
__constant__ double c_T3p1[4][4][4];
__constant__ double c_M2p1[4][4];
__constant__ double c_F2p2[6][6];
__constant__ double c_F2p1[3][3];
__device__ double d_qc[NQ2][5];  // l0..l3, weight (sum 1)

// Keast's 11-point rule on the tetrahedron: exact for every polynomial of
// degree <= 4 (one negative weight); barycentrics and weights normalised to
// sum 1.  Degree 4 is what the P2 conduction integrands reach (kappa(T_theta)
// grad phi_i . grad phi_j: 2 + 1 + 1; k1 phi_j grad T_theta . grad phi_i: the same).
void keast11(std::vector<double>& p, std::vector<double>& w) {
  p.clear();
  w.clear();
  auto add = [&](const double (&l)[4], double wt) {
    p.insert(p.end(), l, l + 4);
    w.push_back(wt);
  };
  add({0.25, 0.25, 0.25, 0.25}, -6.0 * 74.0 / 5625.0);
  for (int k = 0; k < 4; ++k) {
    double l[4] = {1.0 / 14.0, 1.0 / 14.0, 1.0 / 14.0, 1.0 / 14.0};
    l[k] = 11.0 / 14.0;
    add(l, 6.0 * 343.0 / 45000.0);
  }
  const double a = (1.0 + std::sqrt(5.0 / 14.0)) / 4.0, b = (1.0 - std::sqrt(5.0 / 14.0)) / 4.0;
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j) {
      double l[4] = {b, b, b, b};
      l[i] = l[j] = a;
      add(l, 6.0 * 56.0 / 2250.0);
    }
}

std::mutex g_tab_mutex;
bool g_tab_ready[64] = {};
void thermal_point_values();

void thermal_tables() {
  int dev = 0;
  TAM_CUDA(cudaGetDevice(&dev));
  TAM_CHECK(dev >= 0 && dev < 64, TAM_ERR_UNSUPPORTED, "thermal: device id too large");
  std::lock_guard<std::mutex> lock(g_tab_mutex);
  if (g_tab_ready[dev]) return;
  std::vector<double> p, w;
  tet_rule(4, p, w);  // degree 7 >= 6 (three P2 functions)
  double T3[10][10][10] = {}, M2[10][10] = {}, T3a[4][4][4] = {}, M2a[4][4] = {};
  for (size_t q = 0; q < w.size(); ++q) {
    const double* l = &p[4 * q];
    double f2[10], f1[4];
    for (int a = 0; a < 10; ++a) f2[a] = cell_phi(2, a, l);
    for (int a = 0; a < 4; ++a) f1[a] = cell_phi(1, a, l);
    for (int a = 0; a < 10; ++a)
      for (int b = 0; b < 10; ++b) {
        M2[a][b] += w[q] * f2[a] * f2[b];
        for (int c = 0; c < 10; ++c) T3[a][b][c] += w[q] * f2[a] * f2[b] * f2[c];
      }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        M2a[a][b] += w[q] * f1[a] * f1[b];
        for (int c = 0; c < 4; ++c) T3a[a][b][c] += w[q] * f1[a] * f1[b] * f1[c];
      }
  }
  std::vector<double> fp, fw;
  tri_rule(3, fp, fw);  // degree 5 >= 4
  double F2[6][6] = {}, F1[3][3] = {};
  for (size_t q = 0; q < fw.size(); ++q) {
    const double* m = &fp[3 * q];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) F2[a][b] += fw[q] * face_phi(2, a, m) * face_phi(2, b, m);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) F1[a][b] += fw[q] * face_phi(1, a, m) * face_phi(1, b, m);
  }
  keast11(p, w);  // degree 4 (kappa(T_theta) grad phi . grad phi on P2)
  double qc[NQ2][5];
  for (int q = 0; q < NQ2; ++q) {
    for (int k = 0; k < 4; ++k) qc[q][k] = p[4 * q + k];
    qc[q][4] = w[q];
  }
  TAM_CUDA(cudaMemcpyToSymbol(d_T3p2, T3, sizeof(T3)));
  TAM_CUDA(cudaMemcpyToSymbol(d_M2p2, M2, sizeof(M2)));
  TAM_CUDA(cudaMemcpyToSymbol(c_T3p1, T3a, sizeof(T3a)));
  TAM_CUDA(cudaMemcpyToSymbol(c_M2p1, M2a, sizeof(M2a)));
  TAM_CUDA(cudaMemcpyToSymbol(c_F2p2, F2, sizeof(F2)));
  TAM_CUDA(cudaMemcpyToSymbol(c_F2p1, F1, sizeof(F1)));
  TAM_CUDA(cudaMemcpyToSymbol(d_qc, qc, sizeof(qc)));
  thermal_point_values();
  g_tab_ready[dev] = true;
}

// P2 basis values at the conduction points (cell-independent)
__device__ double d_phic[NQ2][10];

void thermal_point_values() {
  std::vector<double> p, w;
  keast11(p, w);
  double ph[NQ2][10];
  for (int q = 0; q < NQ2; ++q)
    for (int a = 0; a < 10; ++a) ph[q][a] = cell_phi(2, a, &p[4 * q]);
  TAM_CUDA(cudaMemcpyToSymbol(d_phic, ph, sizeof(ph)));
}

// ---------------------------------------------------------------------------
// Element kernels: residual F and Jacobian J of Eq. wf_thermal, scattered
// with FP64 atomics into F and J's block-CSR (1x1 blocks) pattern; rows and
// columns of Dirichlet nodes are left out (set by thermal_dirichlet_kernel).
// ---------------------------------------------------------------------------
struct ThArgs {
  const double* X;            // coords [n, 3]
  const int* cells;           // [n_cells, npc]
  const int* mat;             // [n_cells]
  const double* props;        // [n_mat, 5]: rho, c0, c1, k0, k1
  const double* T;            // iterate of T_{m+1}
  const double* T_old;        // T_m, NULL: steady
  double dt, theta;
  const int* rp;
  const int* ci;
  double* J;                  // values [nnz]
  double* F;                  // [n]
  const unsigned char* dmask;
  int n_cells;
  int* bad;                   // degenerate cell flag
};

__device__ __forceinline__ void scatter_J(const ThArgs& A, int ni, int nj, double v) {
  if (A.dmask[ni] || A.dmask[nj]) return;
  const int slot = bsearch_i32(A.ci, A.rp[ni], A.rp[ni + 1], nj);
  if (slot >= 0) atomicAdd(&A.J[slot], v);
}

// P1: thread per cell, closed forms (constant gradients, kappa(T_theta) linear).
__global__ void thermal_p1_kernel(ThArgs A) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n_cells) return;
  int v[4];
  for (int a = 0; a < 4; ++a) v[a] = A.cells[(size_t)c * 4 + a];
  double g[4][3], vol;
  if (!tet_geometry(A.X, v, g, vol)) {
    atomicExch(A.bad, 1);
    return;
  }
  const double* pr = A.props + 5 * A.mat[c];
  const double rho = pr[0], c0 = pr[1], c1 = pr[2], k0 = pr[3], k1 = pr[4];
  const bool steady = A.T_old == nullptr;
  const double th = steady ? 1.0 : A.theta;
  double Tt[4], dT[4], tm = 0.0;
  for (int a = 0; a < 4; ++a) {
    const double t = A.T[v[a]];
    Tt[a] = steady ? t : (1.0 - th) * A.T_old[v[a]] + th * t;
    dT[a] = steady ? 0.0 : (t - A.T_old[v[a]]) / A.dt;
    tm += 0.25 * Tt[a];
  }
  double gT[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) gT[d] += Tt[a] * g[a][d];
  const double kbar = k0 + k1 * tm;  // mean of kappa(T_theta) over the cell
  double gi[4];
  for (int i = 0; i < 4; ++i) gi[i] = gT[0] * g[i][0] + gT[1] * g[i][1] + gT[2] * g[i][2];
  for (int i = 0; i < 4; ++i) {
    double f = vol * kbar * gi[i];
    if (!steady) {
      double m = 0.0;
      for (int b = 0; b < 4; ++b) {
        double cb = c0 * c_M2p1[b][i];
        for (int a = 0; a < 4; ++a) cb += c1 * Tt[a] * c_T3p1[a][b][i];
        m += dT[b] * cb;
      }
      f += rho * vol * m;
    }
    if (!A.dmask[v[i]]) atomicAdd(&A.F[v[i]], f);
    for (int j = 0; j < 4; ++j) {
      const double gg = g[j][0] * g[i][0] + g[j][1] * g[i][1] + g[j][2] * g[i][2];
      double jv = th * vol * (0.25 * k1 * gi[i] + kbar * gg);
      if (!steady) {
        double m = 0.0, cm = c0 * c_M2p1[j][i];
        for (int b = 0; b < 4; ++b) {
          m += c1 * th * dT[b] * c_T3p1[j][b][i];
          cm += c1 * Tt[b] * c_T3p1[b][j][i];
        }
        jv += rho * vol * (m + cm / A.dt);
      }
      scatter_J(A, v[i], v[j], jv);
    }
  }
}

// P2: a warp per cell.  The lanes first evaluate, at the 11 conduction points,
// the basis gradients, grad T_theta and kappa(T_theta) (into shared memory),
// then grad T_theta . grad phi_i per point, the symmetric conduction sums
// once per pair i <= j, and finally the 100 Jacobian and 10 residual entries
// (FP64 is GB300's slow pipe: the symmetric part and the mass sums are not
// recomputed per entry).
constexpr int P2T_WARPS = 4;

__global__ void __launch_bounds__(P2T_WARPS * 32) thermal_p2_kernel(ThArgs A) {
  __shared__ double sg[P2T_WARPS][NQ2][10][3];
  __shared__ double sq[P2T_WARPS][NQ2][5];   // kappa w vol, k1 w vol, grad T_theta
  __shared__ double st[P2T_WARPS][2][10];    // T_theta, (T - T_old)/dt
  __shared__ double stg[P2T_WARPS][NQ2][10]; // grad T_theta . grad phi_i per point
  __shared__ double ssym[P2T_WARPS][55];     // symmetric conduction part, pairs i <= j
  __shared__ double sw[P2T_WARPS][10];       // mass weights
  __shared__ int sv[P2T_WARPS][10];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * P2T_WARPS + wid;
  if (c >= A.n_cells) return;  // warp-uniform
  if (lane < 10) sv[wid][lane] = A.cells[(size_t)c * 10 + lane];
  __syncwarp();
  double g[4][3], vol;
  if (!tet_geometry(A.X, sv[wid], g, vol)) {
    if (lane == 0) atomicExch(A.bad, 1);
    return;
  }
  const double* pr = A.props + 5 * A.mat[c];
  const double rho = pr[0], c0 = pr[1], c1 = pr[2], k0 = pr[3], k1 = pr[4];
  const bool steady = A.T_old == nullptr;
  const double th = steady ? 1.0 : A.theta;
  if (lane < 10) {
    const int n = sv[wid][lane];
    const double t = A.T[n];
    st[wid][0][lane] = steady ? t : (1.0 - th) * A.T_old[n] + th * t;
    st[wid][1][lane] = steady ? 0.0 : (t - A.T_old[n]) / A.dt;
  }
  __syncwarp();
  if (lane < NQ2) {
    const int q = lane;
    const double* l = d_qc[q];
    double tq = 0.0, gt[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 10; ++a) {
      double gr[3];
      if (a < 4) {
        const double s = 4.0 * l[a] - 1.0;
        for (int d = 0; d < 3; ++d) gr[d] = s * g[a][d];
      } else {
        const int e = a - 4;  // edges 01, 02, 03, 12, 13, 23
        const int p0 = e < 3 ? 0 : (e < 5 ? 1 : 2), p1 = e < 3 ? e + 1 : (e == 3 ? 2 : 3);
        for (int d = 0; d < 3; ++d) gr[d] = 4.0 * (l[p1] * g[p0][d] + l[p0] * g[p1][d]);
      }
      const double ta = st[wid][0][a];
      tq += ta * __ldg(&d_phic[q][a]);
      for (int d = 0; d < 3; ++d) {
        sg[wid][q][a][d] = gr[d];
        gt[d] += ta * gr[d];
      }
    }
    const double wv = l[4] * vol;
    sq[wid][q][0] = (k0 + k1 * tq) * wv;
    sq[wid][q][1] = k1 * wv;
    for (int d = 0; d < 3; ++d) sq[wid][q][2 + d] = gt[d];
  }
  __syncwarp();
  // per point and basis function: tg[q][i] = grad T_theta . grad phi_i
  for (int e = lane; e < NQ2 * 10; e += 32) {
    const int q = e / 10, i = e - q * 10;
    const double* gi = sg[wid][q][i];
    const double* sp = sq[wid][q];
    stg[wid][q][i] = sp[2] * gi[0] + sp[3] * gi[1] + sp[4] * gi[2];
  }
  // mass weights: (T3 is symmetric in its three indices) the mass part of
  // J_ij is rho vol (c0 M_ij / dt + sum_b T3_ijb w_b), w_b = c1 (theta dT_b/dt + T_theta,b / dt)
  if (!steady && lane < 10) sw[wid][lane] = c1 * (th * st[wid][1][lane] + st[wid][0][lane] / A.dt);
  __syncwarp();
  // the symmetric conduction part, sum_q kappa w vol grad phi_i . grad phi_j, once per pair i <= j
  for (int e = lane; e < 55; e += 32) {
    int i = 0, r = e;
    while (r >= 10 - i) {
      r -= 10 - i;
      ++i;
    }
    const int j = i + r;
    double acc = 0.0;
    for (int q = 0; q < NQ2; ++q) {
      const double* gi = sg[wid][q][i];
      const double* gj = sg[wid][q][j];
      acc += sq[wid][q][0] * (gj[0] * gi[0] + gj[1] * gi[1] + gj[2] * gi[2]);
    }
    ssym[wid][e] = acc;
  }
  __syncwarp();
  for (int e = lane; e < 110; e += 32) {
    if (e < 100) {
      const int i = e / 10, j = e % 10;
      const int lo = i < j ? i : j, hi = i < j ? j : i;
      double acc = ssym[wid][lo * 10 - lo * (lo - 1) / 2 + (hi - lo)];
      for (int q = 0; q < NQ2; ++q) acc += sq[wid][q][1] * __ldg(&d_phic[q][j]) * stg[wid][q][i];
      acc *= th;
      if (!steady) {
        double m = c0 * __ldg(&d_M2p2[i][j]) / A.dt;
        for (int b2 = 0; b2 < 10; ++b2) m += sw[wid][b2] * __ldg(&d_T3p2[i][j][b2]);
        acc += rho * vol * m;
      }
      scatter_J(A, sv[wid][i], sv[wid][j], acc);
    } else {
      const int i = e - 100;
      double f = 0.0;
      for (int q = 0; q < NQ2; ++q) f += sq[wid][q][0] * stg[wid][q][i];
      if (!steady) {
        double m = 0.0;
        for (int b2 = 0; b2 < 10; ++b2) {
          double cb = c0 * __ldg(&d_M2p2[b2][i]);
          for (int a2 = 0; a2 < 10; ++a2) cb += c1 * st[wid][0][a2] * __ldg(&d_T3p2[a2][b2][i]);
          m += st[wid][1][b2] * cb;
        }
        f += rho * vol * m;
      }
      if (!A.dmask[sv[wid][i]]) atomicAdd(&A.F[sv[wid][i]], f);
    }
  }
}

// Robin faces, thread per face: F_i -= beta |F| sum_a (T_theta - T_bc)_a M_ai,
// J_ij -= theta beta |F| M_ij, M the face mass matrix / |F|.
template <int NF>
__global__ void thermal_face_kernel(ThArgs A, int n_faces, const int* __restrict__ faces,
                                    const double* __restrict__ beta, const double* __restrict__ Tbc) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_faces) return;
  int v[NF];
  for (int a = 0; a < NF; ++a) v[a] = faces[(size_t)f * NF + a];
  double e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = A.X[3 * (size_t)v[1] + d] - A.X[3 * (size_t)v[0] + d];
    e2[d] = A.X[3 * (size_t)v[2] + d] - A.X[3 * (size_t)v[0] + d];
  }
  const double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2],
               cz = e1[0] * e2[1] - e1[1] * e2[0];
  const double bw = beta[f] * 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  const bool steady = A.T_old == nullptr;
  const double th = steady ? 1.0 : A.theta;
  double d[NF];
  for (int a = 0; a < NF; ++a) {
    const double t = A.T[v[a]];
    d[a] = (steady ? t : (1.0 - th) * A.T_old[v[a]] + th * t) - Tbc[v[a]];
  }
  for (int i = 0; i < NF; ++i) {
    double s = 0.0;
    for (int a = 0; a < NF; ++a) s += d[a] * (NF == 3 ? c_F2p1[a][i] : c_F2p2[a][i]);
    if (!A.dmask[v[i]]) atomicAdd(&A.F[v[i]], -bw * s);
    for (int j = 0; j < NF; ++j) scatter_J(A, v[i], v[j], -th * bw * (NF == 3 ? c_F2p1[i][j] : c_F2p2[i][j]));
  }
}

// Dirichlet rows of the Newton system: J row = identity, F = 0.
__global__ void thermal_dirichlet_kernel(int n, const unsigned char* __restrict__ dmask, const int* __restrict__ rp,
                                         const int* __restrict__ ci, double* __restrict__ J, double* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !dmask[i]) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) J[p] = ci[p] == i ? 1.0 : 0.0;
  F[i] = 0.0;
}

// T_i = T_D,i on Dirichlet nodes
__global__ void thermal_impose_kernel(int n, const unsigned char* __restrict__ dmask, const double* __restrict__ Td,
                                      double* __restrict__ T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && dmask[i]) T[i] = Td[i];
}

// out[0] = sum F^2 (grid reduction)
__global__ void norm2_kernel(const double* __restrict__ F, long long n, GridReduce gr, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc[0] += F[i] * F[i];
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) *out = tot[0];
}

// T -= delta
__global__ void newton_update_kernel(double* __restrict__ T, const double* __restrict__ delta, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    T[i] -= delta[i];
}

// out = max |a - b| (non-negative doubles compare like their bit patterns)
__global__ void max_change_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n,
                                  unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i] - b[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

}  // namespace
}  // namespace tam

// ---------------------------------------------------------------------------
// The thermal problem handle and Newton's method
// ---------------------------------------------------------------------------
struct tam_thermal_s {
  int n_nodes = 0, n_cells = 0, npc = 0, n_mat = 0, n_faces = 0, nf = 0;
  const double* X = nullptr;   // caller-owned device arrays
  const int* cells = nullptr;
  const int* mat = nullptr;
  const int* faces = nullptr;
  tam::DBuf<double> props;     // [n_mat * 5]
  tam_matrix_s* J = nullptr;   // Newton Jacobian (1x1 blocks), with J->dmask
  tam::DBuf<double> F, delta, red, out;
  tam::DBuf<unsigned int> ticket;
  tam::DBuf<unsigned long long> mx;
  tam_amg_s* H = nullptr;      // AMG hierarchy of an earlier Jacobian (reused while it serves)
  amg_params prm{};
  int setups = 0;
  ~tam_thermal_s() {
    delete H;
    delete J;
  }
};

namespace tam {
namespace {

// F and J at the iterate T (T_old == NULL: steady)
void thermal_assemble(tam_thermal_s* th, const double* T, const double* T_old, double dt, double theta,
                      const double* beta, const double* Tbc, cudaStream_t s) {
  TAM_CHECK(T && (th->n_faces == 0 || (beta && Tbc)), TAM_ERR_INVALID_ARG,
            "thermal: T, and beta / T_bc for the Robin faces, are required");
  TAM_CHECK(!T_old || (dt > 0.0 && theta > 0.0 && theta <= 1.0), TAM_ERR_INVALID_ARG,
            "thermal: a transient step needs dt > 0 and 0 < theta <= 1");
  thermal_tables();
  Bsr& A = th->J->A;
  const int n = th->n_nodes;
  A.vals.zero();
  th->F.zero();
  DBuf<int> bad(1, s);
  bad.zero();
  ThArgs a{th->X, th->cells, th->mat, th->props.p, T, T_old, dt, theta, A.row_ptr.p, A.col_idx.p, A.vals.p,
           th->F.p, th->J->dmask.p, th->n_cells, bad.p};
  if (th->n_cells > 0) {
    if (th->npc == 4)
      thermal_p1_kernel<<<grid_for(th->n_cells, 128), 128, 0, s>>>(a);
    else
      thermal_p2_kernel<<<grid_for(th->n_cells, P2T_WARPS), P2T_WARPS * 32, 0, s>>>(a);
    TAM_LAUNCH_CHECK();
  }
  if (th->n_faces > 0) {
    if (th->nf == 3)
      thermal_face_kernel<3><<<grid_for(th->n_faces, 128), 128, 0, s>>>(a, th->n_faces, th->faces, beta, Tbc);
    else
      thermal_face_kernel<6><<<grid_for(th->n_faces, 128), 128, 0, s>>>(a, th->n_faces, th->faces, beta, Tbc);
    TAM_LAUNCH_CHECK();
  }
  thermal_dirichlet_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, th->J->dmask.p, A.row_ptr.p, A.col_idx.p, A.vals.p,
                                                           th->F.p);
  TAM_LAUNCH_CHECK();
  TAM_CHECK(read_back_int(bad.p, s) == 0, TAM_ERR_DEGENERATE_CELL, "thermal: a cell has non-positive volume");
  // the SpMV copy and the exponent range of the new values
  sell_refresh_values(A, th->J->S, s);
  operator_exponent_range(A, &th->J->vmax_exp, &th->J->finite, s);
  th->J->df_ok = th->J->finite && std::abs(th->J->vmax_exp) <= kDfExpLimit && th->J->S.vals_df.p;
}

double thermal_norm(tam_thermal_s* th, cudaStream_t s) {
  const long long n = th->n_nodes;
  norm2_kernel<<<stride_grid(n, 256, 4), 256, 0, s>>>(th->F.p, n, GridReduce{th->red.p, th->ticket.p}, th->out.p);
  TAM_LAUNCH_CHECK();
  return std::sqrt(read_back_double(th->out.p, s));
}

}  // namespace
}  // namespace tam

using namespace tam;

extern "C" {

int tam_thermal_create(int n_nodes, const double* coords, int n_cells, int nodes_per_cell, const int* cells,
                       const int* cell_material, int n_mat, const double* thermal_props_host, int n_faces,
                       const int* faces, const unsigned char* dirichlet_mask, const amg_params* params,
                       tam_thermal* out, void* stream) {
  try {
    set_last_error("");
    TAM_CHECK(out, TAM_ERR_INVALID_ARG, "tam_thermal_create: out is NULL");
    *out = nullptr;
    TAM_CHECK(n_nodes > 0 && n_cells >= 0 && n_mat > 0 && n_faces >= 0 && (nodes_per_cell == 4 || nodes_per_cell == 10),
              TAM_ERR_INVALID_ARG, "tam_thermal_create: bad sizes");
    TAM_CHECK(coords && (cells || !n_cells) && (cell_material || !n_cells) && thermal_props_host && (faces || !n_faces),
              TAM_ERR_INVALID_ARG, "tam_thermal_create: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    validate_mesh(n_nodes, n_cells, nodes_per_cell, cells, cell_material, n_mat, "tam_thermal_create", s);
    auto th = new tam_thermal_s();
    try {
      th->n_nodes = n_nodes;
      th->n_cells = n_cells;
      th->npc = nodes_per_cell;
      th->n_mat = n_mat;
      th->n_faces = n_faces;
      th->nf = nodes_per_cell == 4 ? 3 : 6;
      th->X = coords;
      th->cells = cells;
      th->mat = cell_material;
      th->faces = faces;
      if (n_faces > 0) validate_mesh(n_nodes, n_faces, th->nf, faces, nullptr, 1, "tam_thermal_create (faces)", s);
      th->props = DBuf<double>((size_t)n_mat * 5, s);
      TAM_CUDA(cudaMemcpyAsync(th->props.p, thermal_props_host, sizeof(double) * 5 * n_mat, cudaMemcpyHostToDevice, s));
      if (params) th->prm = *params; else amg_params_default(&th->prm);
      th->J = new tam_matrix_s();
      th->J->n_nodes = n_nodes;
      th->J->dmask = DBuf<unsigned char>((size_t)n_nodes, s);
      if (dirichlet_mask)
        TAM_CUDA(cudaMemcpyAsync(th->J->dmask.p, dirichlet_mask, n_nodes, cudaMemcpyDeviceToDevice, s));
      else
        th->J->dmask.zero();
      Bsr& A = th->J->A;
      A.br = A.bc = 1;
      DBuf<int> inc_ptr, inc, flag(2, s);
      flag.zero();
      build_node_pattern(n_nodes, n_cells, nodes_per_cell, cells, th->J->dmask.p, A, inc_ptr, inc, flag.p, s);
      A.vals = DBuf<double>((size_t)std::max(1LL, A.nnzb), s);
      A.vals.zero();
      bsr_to_sell(A, th->J->S, s, true);
      th->F = DBuf<double>((size_t)n_nodes, s);
      th->delta = DBuf<double>((size_t)n_nodes, s);
      th->red = DBuf<double>((size_t)sm_count() * 4, s);
      th->out = DBuf<double>(2, s);
      th->ticket = DBuf<unsigned int>(1, s);
      th->ticket.zero();
      th->mx = DBuf<unsigned long long>(1, s);
      TAM_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      delete th;
      throw;
    }
    *out = th;
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return TAM_ERR_INTERNAL;
  }
}

int tam_thermal_destroy(tam_thermal th) {
  try {
    delete th;
    return TAM_OK;
  } catch (...) {
    return TAM_ERR_INTERNAL;
  }
}

int tam_thermal_residual(tam_thermal th, const double* T, const double* T_old, double dt, double theta,
                         const double* beta, const double* T_bc, double* F_out, void* stream) {
  try {
    set_last_error("");
    TAM_CHECK(th && T && F_out, TAM_ERR_INVALID_ARG, "tam_thermal_residual: NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    thermal_assemble(th, T, T_old, dt, theta, beta, T_bc, s);
    TAM_CUDA(cudaMemcpyAsync(F_out, th->F.p, sizeof(double) * th->n_nodes, cudaMemcpyDeviceToDevice, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int tam_thermal_export_jacobian(tam_thermal th, int* row_ptr, int* col_idx, double* vals, long long* nnz_host,
                                void* stream) {
  try {
    set_last_error("");
    TAM_CHECK(th, TAM_ERR_INVALID_ARG, "tam_thermal_export_jacobian: NULL handle");
    const Bsr& A = th->J->A;
    if (nnz_host) *nnz_host = A.nnzb;
    if (!row_ptr) return TAM_OK;
    TAM_CHECK(col_idx && vals, TAM_ERR_INVALID_ARG, "tam_thermal_export_jacobian: NULL array");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    TAM_CUDA(cudaMemcpyAsync(row_ptr, A.row_ptr.p, sizeof(int) * ((size_t)A.n_rows + 1), cudaMemcpyDeviceToDevice, s));
    TAM_CUDA(cudaMemcpyAsync(col_idx, A.col_idx.p, sizeof(int) * (size_t)A.nnzb, cudaMemcpyDeviceToDevice, s));
    TAM_CUDA(cudaMemcpyAsync(vals, A.vals.p, sizeof(double) * (size_t)A.nnzb, cudaMemcpyDeviceToDevice, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int tam_thermal_newton(tam_thermal th, double* T, const double* T_old, double dt, double theta, const double* beta,
                       const double* T_bc, const double* T_dirichlet, double rtol, int max_newton, double lin_rtol,
                       int lin_max_iter, int reuse, int* newton_iters, int* linear_iters, int* setups,
                       double* rel_resid, void* stream) {
  NvtxRange nvtx("tam: thermal Newton");
  try {
    set_last_error("");
    TAM_CHECK(th && T && rtol >= 0.0 && max_newton >= 0 && lin_rtol > 0.0 && lin_max_iter > 0,
              TAM_ERR_INVALID_ARG, "tam_thermal_newton: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int n = th->n_nodes;
    if (T_dirichlet) {
      thermal_impose_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, th->J->dmask.p, T_dirichlet, T);
      TAM_LAUNCH_CHECK();
    }
    const int setups0 = th->setups;
    int it = 0, lin_total = 0, status = TAM_OK;
    double f0 = 0.0, fn = 0.0;
    for (;; ++it) {
      thermal_assemble(th, T, T_old, dt, theta, beta, T_bc, s);
      fn = thermal_norm(th, s);
      if (it == 0) f0 = fn;
      if (!std::isfinite(fn)) { status = TAM_ERR_NAN; break; }
      if (fn <= rtol * f0 || fn == 0.0) break;
      if (it == max_newton) { status = TAM_ERR_NOT_CONVERGED; break; }
      // solve J delta = F: a hierarchy of an earlier Jacobian while it serves
      // (reuse != 0), a new one when there is none, when asked, when the range
      // of J's values moved out of the double-float range, or when the reused
      // one fails to reach the tolerance
      bool fresh = false;
      if (th->H && (!reuse || (th->H->levels[0].Aop.df && !th->J->df_ok))) {
        delete th->H;
        th->H = nullptr;
      }
      if (!th->H) {
        th->H = amg_build(th->J, th->X, th->prm, s);
        ++th->setups;
        fresh = true;
      } else {
        amg_refresh_finest(th->H, s);
      }
      int li = 0, st = TAM_OK;
      for (int attempt = 0; attempt < 2; ++attempt) {
        th->delta.zero();
        double rel = 0.0;
        st = pcg_solve(th->H, th->F.p, th->delta.p, lin_rtol, 0.0, lin_max_iter, &li, &rel, s);
        lin_total += li;
        if (st == TAM_OK || fresh) break;
        delete th->H;  // the reused hierarchy no longer serves: rebuild once
        th->H = amg_build(th->J, th->X, th->prm, s);
        ++th->setups;
        fresh = true;
      }
      if (st != TAM_OK && st != TAM_ERR_NOT_CONVERGED) { status = st; break; }
      newton_update_kernel<<<stride_grid(n, 256, 8), 256, 0, s>>>(T, th->delta.p, n);
      TAM_LAUNCH_CHECK();
    }
    TAM_CUDA(cudaStreamSynchronize(s));
    if (newton_iters) *newton_iters = it;
    if (linear_iters) *linear_iters = lin_total;
    if (setups) *setups = th->setups - setups0;
    if (rel_resid) *rel_resid = f0 > 0.0 ? fn / f0 : 0.0;
    if (status != TAM_OK) set_last_error("tam_thermal_newton: Newton did not converge (status per code)");
    return status;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int tam_thermal_max_change(const double* a, const double* b, long long n, double* max_host, void* stream) {
  try {
    set_last_error("");
    TAM_CHECK(a && b && max_host && n >= 0, TAM_ERR_INVALID_ARG, "tam_thermal_max_change: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DBuf<unsigned long long> mx(1, s);
    mx.zero();
    if (n > 0) {
      max_change_kernel<<<stride_grid(n, 256, 8), 256, 0, s>>>(a, b, n, mx.p);
      TAM_LAUNCH_CHECK();
    }
    unsigned long long bits = 0;
    TAM_CUDA(cudaMemcpyAsync(&bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    double m;
    std::memcpy(&m, &bits, sizeof(m));
    *max_host = m;
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

int tam_thermal_next_dt(double dt, double max_change, double dT_max, double eps, double* dt_next_host,
                        int* accepted_host) {
  try {
    set_last_error("");
    TAM_CHECK(dt > 0.0 && max_change >= 0.0 && dT_max > 0.0 && eps > 0.0 && eps <= 1.0 && dt_next_host &&
                  accepted_host,
              TAM_ERR_INVALID_ARG, "tam_thermal_next_dt: bad argument");
    if (max_change > dT_max) {  // repeat the step with half the time step
      *accepted_host = 0;
      *dt_next_host = 0.5 * dt;
    } else {
      *accepted_host = 1;
      *dt_next_host = max_change > 0.0 ? eps * dT_max / max_change * dt : 2.0 * dt;
    }
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

}  // extern "C"
