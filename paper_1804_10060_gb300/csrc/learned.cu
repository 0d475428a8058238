// Node features for the learned initial guess and the guarded guess itself.
//
// Features per node (8, FP32): x, y, z, T, grad T (3), distance to the
// clamped boundary.  grad T at a node is the volume-weighted mean over its
// cells of the gradient of the temperature interpolant at the cell centroid
// (P1: the constant gradient; P2: sum over edges of T_edge (g_a + g_b), the
// exact centroid value of the quadratic interpolant).  The distance field is
// supplied by the caller (it is geometry, not solver output).
#include <cmath>

#include "handles.cuh"
#include "tet.cuh"

struct tam_mlp_s;

namespace tam {

void mlp_forward_device(tam_mlp_s* M, long long n, const float* X, float* Y, int bf16, cudaStream_t s);
int mlp_n_in(tam_mlp_s* M);
int mlp_n_out(tam_mlp_s* M);

namespace {

__constant__ int c_p2e[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

__global__ void grad_t_kernel(const double* __restrict__ X, const int* __restrict__ cells, int npc, int n_cells,
                              const double* __restrict__ T, double* __restrict__ gsum, double* __restrict__ wsum) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  int v[10];
  for (int a = 0; a < npc; ++a) v[a] = cells[(size_t)c * npc + a];
  double g[4][3], vol;
  if (!tet_geometry(X, v, g, vol)) return;
  double gt[3] = {0, 0, 0};
  if (npc == 4) {
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) gt[d] += T[v[a]] * g[a][d];
  } else {
    for (int e = 0; e < 6; ++e) {
      const double te = T[v[4 + e]];
      for (int d = 0; d < 3; ++d) gt[d] += te * (g[c_p2e[e][0]][d] + g[c_p2e[e][1]][d]);
    }
  }
  for (int a = 0; a < npc; ++a) {
    for (int d = 0; d < 3; ++d) atomicAdd(&gsum[3 * (size_t)v[a] + d], vol * gt[d]);
    atomicAdd(&wsum[v[a]], vol);
  }
}

__global__ void features_kernel(int n, const double* __restrict__ X, const double* __restrict__ T,
                                const double* __restrict__ gsum, const double* __restrict__ wsum,
                                const double* __restrict__ dist, float* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w = wsum[i] > 0.0 ? 1.0 / wsum[i] : 0.0;
  float* f = F + (size_t)i * 8;
  f[0] = (float)X[3 * (size_t)i];
  f[1] = (float)X[3 * (size_t)i + 1];
  f[2] = (float)X[3 * (size_t)i + 2];
  f[3] = T ? (float)T[i] : 0.f;
  f[4] = (float)(gsum[3 * (size_t)i] * w);
  f[5] = (float)(gsum[3 * (size_t)i + 1] * w);
  f[6] = (float)(gsum[3 * (size_t)i + 2] * w);
  f[7] = dist ? (float)dist[i] : 0.f;
}

// x (FP64) from the network output; Dirichlet rows take the prescribed value
__global__ void guess_to_x_kernel(int n, const float* __restrict__ Y, const unsigned char* __restrict__ dmask,
                                  const double* __restrict__ rhs, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < 3; ++d) {
    const size_t k = 3 * (size_t)i + d;
    x[k] = dmask[i] ? rhs[k] : (double)Y[k];
  }
}

__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, long long n, GridReduce gr,
                           double* __restrict__ out) {
  __shared__ double sh[32];
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc[0] += a[i] * b[i];
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) *out = tot[0];
}

}  // namespace
}  // namespace tam

using namespace tam;

extern "C" int tam_node_features(int n_nodes, const double* coords, int n_cells, int nodes_per_cell, const int* cells,
                                 const double* T, const double* dist, float* features, void* stream) {
  try {
    set_last_error("");
    TAM_CHECK(n_nodes > 0 && n_cells >= 0 && (nodes_per_cell == 4 || nodes_per_cell == 10) && coords &&
                  (cells || n_cells == 0) && features,
              TAM_ERR_INVALID_ARG, "tam_node_features: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DBuf<double> gsum((size_t)n_nodes * 3, s), wsum((size_t)n_nodes, s);
    gsum.zero();
    wsum.zero();
    if (T && n_cells > 0) {
      grad_t_kernel<<<grid_for(n_cells, 128), 128, 0, s>>>(coords, cells, nodes_per_cell, n_cells, T, gsum.p, wsum.p);
      TAM_LAUNCH_CHECK();
    }
    features_kernel<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, coords, T, gsum.p, wsum.p, dist, features);
    TAM_LAUNCH_CHECK();
    TAM_CUDA(cudaStreamSynchronize(s));
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}

// The network's output is first smoothed by smooth_degree Chebyshev-Jacobi
// steps on K x = rhs (over [0.1, 1.1] lambda_max(D^-1 K)): a node-wise
// network leaves a small but rough error, which K amplifies, and a point
// smoother removes exactly those components.  The guess is then kept only if
// it lowers the preconditioned residual energy <r, M r> (r = rhs - K x,
// M = one AMG V-cycle) below that of the zero guess <rhs, M rhs> -- the
// quantity CG's error is measured in up to the preconditioner.
extern "C" int tam_learned_guess(tam_mlp_s* M, tam_amg H, const float* features, const double* rhs, int bf16,
                                 int smooth_degree, double* x, int* used_host, double* energy_ratio_host,
                                 void* stream) {
  NvtxRange nvtx("tam: learned initial guess");
  try {
    set_last_error("");
    TAM_CHECK(M && H && features && rhs && x, TAM_ERR_INVALID_ARG, "tam_learned_guess: NULL argument");
    TAM_CHECK(mlp_n_in(M) == 8 && mlp_n_out(M) == 3, TAM_ERR_INVALID_ARG,
              "tam_learned_guess: the network must map 8 node features to 3 displacements");
    TAM_CHECK(smooth_degree >= 0 && smooth_degree <= 64, TAM_ERR_INVALID_ARG,
              "tam_learned_guess: smooth_degree must be 0..64");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    tam_matrix_s* K = H->K;
    TAM_CHECK(K->A.br == 3, TAM_ERR_INVALID_ARG, "tam_learned_guess: needs an elastic (3x3-block) hierarchy");
    const int n = K->n_nodes;
    const long long N = 3LL * n;
    DBuf<float> Y((size_t)N, s);
    mlp_forward_device(M, n, features, Y.p, bf16, s);
    guess_to_x_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, Y.p, K->dmask.p, rhs, x);
    TAM_LAUNCH_CHECK();
    if (smooth_degree > 0) smooth_fine(H, rhs, x, smooth_degree, 0.1, 1.1, s);
    const unsigned g = stride_grid(N, 256, 8);
    DBuf<double> r((size_t)N, s), z((size_t)N, s), part(g, s), out(2, s);
    DBuf<unsigned int> ticket(1, s);
    ticket.zero();
    GridReduce gr{part.p, ticket.p};
    sell_spmv<3, 3>(K->S, x, EpiResidual<3>{rhs, r.p, n, nullptr}, s, K->df_ok);
    vcycle_apply(H, r.p, z.p, nullptr, s);
    dot_kernel<<<g, 256, 0, s>>>(r.p, z.p, N, gr, out.p);
    TAM_LAUNCH_CHECK();
    vcycle_apply(H, rhs, z.p, nullptr, s);
    dot_kernel<<<g, 256, 0, s>>>(rhs, z.p, N, gr, out.p + 1);
    TAM_LAUNCH_CHECK();
    double e[2];
    TAM_CUDA(cudaMemcpyAsync(e, out.p, sizeof(e), cudaMemcpyDeviceToHost, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    const double ratio = e[1] > 0 ? e[0] / e[1] : e[0];
    const bool use = std::isfinite(ratio) && ratio < 1.0;
    if (!use) TAM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)N, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    if (used_host) *used_host = use ? 1 : 0;
    if (energy_ratio_host) *energy_ratio_host = ratio;
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  }
}
