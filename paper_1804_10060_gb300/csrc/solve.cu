// AMG V-cycle and preconditioned CG (paper Sec. 2.1: CG with a preconditioner
// that bounds the condition number independently of h; Sec. 5.1: smoothed
// aggregation with Chebyshev smoothing).
//
// V-cycle on level l (A_l, D_l, Chebyshev on D^-1 A over [lo, hi] lambda):
//   x  = Cheb(A, b, x = 0)           pre-smoothing, `degree` steps
//   t  = b - A x                     residual
//   b' = R t,  x' = V-cycle(l+1, b') restriction + coarse correction
//   x += P x'                        prolongation
//   x  = Cheb(A, b, x)               post-smoothing (same polynomial)
// and the coarsest level applies its dense inverse.  Each Chebyshev step is
// ONE fused SpMV kernel: res = D^-1 (b - A x), d = c_d d + c_r res, x' = x + d.
//
// PCG keeps every scalar on the device; kernels after a stop (convergence,
// breakdown, NaN, iteration cap) return at entry, so a fixed-length CUDA
// graph of one iteration can be replayed without host round trips.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <functional>
#include <type_traits>
#include <vector>

#include "handles.cuh"

namespace tam {
namespace {

constexpr int TPB = 256;

__global__ void cheb_first_zero_kernel(const double* __restrict__ b, const double* __restrict__ dinv,
                                       const double* __restrict__ consts, double* __restrict__ d,
                                       double* __restrict__ x, long long N, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const double cr = consts[3];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double di = cr * dinv[i] * b[i];
    d[i] = di;
    x[i] = di;
  }
}

// One Chebyshev step fused into the SpMV of x.
template <int BR>
struct EpiCheb {
  const double* b;
  const double* x;     // current iterate (own rows)
  const double* dinv;
  const double* coef;  // (c_d, c_r) of this step
  double* d;
  double* xn;          // next iterate (other buffer)
  int n_rows;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const double (&acc)[BR], double*) const {
    if (row >= n_rows) return;
    const double cd = coef[0], cr = coef[1];
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      size_t i = (size_t)row * BR + r;
      double res = dinv[i] * (b[i] - acc[r]);
      double di = cd != 0.0 ? cd * d[i] + cr * res : cr * res;
      d[i] = di;
      xn[i] = x[i] + di;
    }
  }
};

// y = Ainv b (dense), warp per row
__global__ void dense_gemv_kernel(const double* __restrict__ A, const double* __restrict__ b, double* __restrict__ y,
                                  int N, const int* __restrict__ stop) {
  if (stop && *stop) return;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= N) return;
  const double* a = A + (size_t)row * N;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) s = fma(a[j], b[j], s);
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}

// ---------------------------------------------------------------------------
// PCG kernels
// ---------------------------------------------------------------------------
// 2^e for |e| <= 1000, built from its bits (exact)
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// The power of two the solve divides b and x by: b's RMS entry moves to about
// 2^half_exp, half K's largest entry exponent, so that the solution-like
// vectors (about b / |K|) sit near 2^-half_exp and every vector the
// double-float SpMVs split stays far inside FP32's exponent range.  Scaling by
// a power of two is exact, so in range the iterates are the unscaled ones
// times 2^-e bit for bit.
__device__ __forceinline__ int centering_exp(double bb, long long N, int half_exp) {
  if (!(bb > 0.0) || !isfinite(bb) || N <= 0) return 0;
  const int e = ilogb(sqrt(bb / (double)N)) - half_exp;
  return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}

__global__ void pcg_start_kernel(const double* __restrict__ b, long long N, GridReduce gr, PcgScalars* sc,
                                 double rtol, double atol, int max_iter, int half_exp) {
  __shared__ double sh[32];
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    acc[0] += b[i] * b[i];
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) {
    const int e = centering_exp(tot[0], N, half_exp);
    const double inv = pow2(-e);
    sc->scale_exp = e;
    sc->bb = tot[0] * inv * inv;
    double t = fmax(rtol * sqrt(tot[0]), atol) * inv;
    sc->tol2 = t * t;
    sc->iter = 0;
    sc->max_iter = max_iter;
    sc->stop = 0;
    sc->status = TAM_OK;
    sc->rho = sc->alpha = sc->beta = 0.0;
    sc->rr = 0.0;
    sc->loops = 0;
  }
}

// dst = src 2^(dir * scale_exp) (dst may be src): into and out of the solve's scaling
__global__ void pcg_scale_kernel(const double* __restrict__ src, double* __restrict__ dst, long long N,
                                 const PcgScalars* __restrict__ sc, int dir) {
  const int e = sc->scale_exp;
  if (e == 0 && src == dst) return;
  const double f = pow2(dir * e);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] * f;
}

// r = b - K x and ||r||^2 -> stop if already converged
template <int BR>
struct EpiInitResidual {
  const double* b;
  double* r;
  int n_rows;
  GridReduce gr;
  PcgScalars* sc;
  double* hist;  // residual history (||r_k||^2 in the solve's scaling), entry 0
  __device__ bool skip() const { return false; }
  __device__ void operator()(int row, const double (&acc)[BR], double* sh) const {
    double s[1] = {0.0};
    if (row < n_rows)
#pragma unroll
      for (int k = 0; k < BR; ++k) {
        size_t i = (size_t)row * BR + k;
        double v = b[i] - acc[k];
        r[i] = v;
        s[0] += v * v;
      }
    double tot[1];
    if (grid_reduce<1>(gr, s, tot, sh) && threadIdx.x == 0) {
      sc->rr = tot[0];
      hist[0] = tot[0];
      if (!isfinite(tot[0])) { sc->status = TAM_ERR_NAN; sc->stop = 1; }
      else if (tot[0] <= sc->tol2) sc->stop = 1;
      else if (sc->max_iter <= 0) { sc->status = TAM_ERR_NOT_CONVERGED; sc->stop = 1; }
    }
  }
};

// rho = r . z (> 0 for an SPD preconditioner);  first call also sets p = z
__global__ void pcg_rz_kernel(const double* __restrict__ r, const double* __restrict__ z, double* __restrict__ p,
                              long long N, GridReduce gr, PcgScalars* sc, int first) {
  __shared__ double sh[32];
  if (sc->stop) return;
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    acc[0] += r[i] * z[i];
    if (first) p[i] = z[i];
  }
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) {
    const double rz = tot[0];
    if (!isfinite(rz)) { sc->status = TAM_ERR_NAN; sc->stop = 1; return; }
    if (!(rz > 0.0)) { sc->status = TAM_ERR_INDEFINITE_PRECOND; sc->stop = 1; return; }
    if (!first) sc->beta = rz / sc->rho;
    sc->rho = rz;
  }
}

// q = K p and p . q -> alpha
template <int BR>
struct EpiPq {
  const double* p;
  double* q;
  int n_rows;
  GridReduce gr;
  PcgScalars* sc;
  __device__ bool skip() const { return sc->stop; }
  __device__ void operator()(int row, const double (&acc)[BR], double* sh) const {
    double s[1] = {0.0};
    if (row < n_rows)
#pragma unroll
      for (int k = 0; k < BR; ++k) {
        size_t i = (size_t)row * BR + k;
        q[i] = acc[k];
        s[0] += p[i] * acc[k];
      }
    double tot[1];
    if (grid_reduce<1>(gr, s, tot, sh) && threadIdx.x == 0) {
      const double pq = tot[0];
      if (!isfinite(pq)) { sc->status = TAM_ERR_NAN; sc->stop = 1; }
      else if (!(pq > 0.0)) { sc->status = TAM_ERR_BREAKDOWN; sc->stop = 1; }
      else sc->alpha = sc->rho / pq;
    }
  }
};

// x += alpha p; r -= alpha q; ||r||^2; convergence / cap
__global__ void pcg_update_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                                  const double* __restrict__ q, long long N, GridReduce gr, PcgScalars* sc,
                                  double* __restrict__ hist, int hist_cap) {
  __shared__ double sh[32];
  if (sc->stop) return;
  const double a = sc->alpha;
  double acc[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    x[i] += a * p[i];
    double ri = r[i] - a * q[i];
    r[i] = ri;
    acc[0] += ri * ri;
  }
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) {
    sc->rr = tot[0];
    sc->iter += 1;
    if (sc->iter < hist_cap) hist[sc->iter] = tot[0];
    if (!isfinite(tot[0])) { sc->status = TAM_ERR_NAN; sc->stop = 1; }
    else if (tot[0] <= sc->tol2) sc->stop = 1;
    else if (sc->iter >= sc->max_iter) { sc->status = TAM_ERR_NOT_CONVERGED; sc->stop = 1; }
  }
}

__global__ void pcg_direction_kernel(const double* __restrict__ z, double* __restrict__ p, long long N,
                                     const PcgScalars* sc) {
  if (sc->stop) return;
  const double beta = sc->beta;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// final ||b - K x||^2
template <int BR>
struct EpiResNorm {
  const double* b;
  int n_rows;
  GridReduce gr;
  double* out;
  __device__ bool skip() const { return false; }
  __device__ void operator()(int row, const double (&acc)[BR], double* sh) const {
    double s[1] = {0.0};
    if (row < n_rows)
#pragma unroll
      for (int k = 0; k < BR; ++k) {
        double v = b[(size_t)row * BR + k] - acc[k];
        s[0] += v * v;
      }
    double tot[1];
    if (grid_reduce<1>(gr, s, tot, sh) && threadIdx.x == 0) *out = tot[0];
  }
};

unsigned vec_grid(long long N) { return stride_grid(N, TPB, 8); }

// The last node of a loop body: continue while *stop == 0 and the failsafe
// count stays below *limit + add.
__global__ void loop_control_kernel(cudaGraphConditionalHandle h, const int* __restrict__ stop, int* __restrict__ count,
                                    const int* __restrict__ limit, int add) {
  const int c = ++*count;
  cudaGraphSetConditional(h, (*stop == 0 && c < *limit + add) ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Dispatch on block shapes (3x3, 6x6 for A; 3x6, 6x3, 6x6, 3x3 for P and R)
// ---------------------------------------------------------------------------
void cheb_step(const Level& L, const double* b, const double* x, double* d, double* xn, int step, const int* stop,
               cudaStream_t s) {
  const double* coef = L.consts.p + 2 + 2 * step;
  if (L.bs == 3)
    spop_apply<3, 3>(L.Aop, x, EpiCheb<3>{b, x, L.dinv.p, coef, d, xn, L.n_rows, stop}, s);
  else if (L.bs == 6)
    spop_apply<6, 6>(L.Aop, x, EpiCheb<6>{b, x, L.dinv.p, coef, d, xn, L.n_rows, stop}, s);
  else
    spop_apply<1, 1>(L.Aop, x, EpiCheb<1>{b, x, L.dinv.p, coef, d, xn, L.n_rows, stop}, s);
}

void residual(const Level& L, const double* b, const double* x, double* t, const int* stop, cudaStream_t s) {
  if (L.bs == 3)
    spop_apply<3, 3>(L.Aop, x, EpiResidual<3>{b, t, L.n_rows, stop}, s);
  else if (L.bs == 6)
    spop_apply<6, 6>(L.Aop, x, EpiResidual<6>{b, t, L.n_rows, stop}, s);
  else
    spop_apply<1, 1>(L.Aop, x, EpiResidual<1>{b, t, L.n_rows, stop}, s);
}

void restrict_to(const Level& L, const double* t, double* bc, const int* stop, cudaStream_t s) {
  // R: rows = coarse nodes (kdim), cols = fine nodes (bs)
  const int nr = L.R.n_rows;
  if (L.kdim == 6 && L.bs == 3) spop_apply<6, 3>(L.Rop, t, EpiStore<6>{bc, nr, stop}, s);
  else if (L.kdim == 6 && L.bs == 6) spop_apply<6, 6>(L.Rop, t, EpiStore<6>{bc, nr, stop}, s);
  else if (L.kdim == 1) spop_apply<1, 1>(L.Rop, t, EpiStore<1>{bc, nr, stop}, s);
  else spop_apply<3, 3>(L.Rop, t, EpiStore<3>{bc, nr, stop}, s);
}

void prolong_add(const Level& L, const double* xc, double* x, const int* stop, cudaStream_t s) {
  const int nr = L.P.n_rows;
  if (L.kdim == 6 && L.bs == 3) spop_apply<3, 6>(L.Pop, xc, EpiAdd<3>{x, nr, stop}, s);
  else if (L.kdim == 6 && L.bs == 6) spop_apply<6, 6>(L.Pop, xc, EpiAdd<6>{x, nr, stop}, s);
  else if (L.kdim == 1) spop_apply<1, 1>(L.Pop, xc, EpiAdd<1>{x, nr, stop}, s);
  else spop_apply<3, 3>(L.Pop, xc, EpiAdd<3>{x, nr, stop}, s);
}

// Chebyshev coefficients (c_d, c_r) for `degree` steps on the absolute
// interval [l0, l1], laid out like Level::consts from index 2 (same
// three-term recurrence as the level smoothers).
std::vector<double> cheb_coefficients(double l0, double l1, int degree) {
  std::vector<double> c(2 + 2 * (size_t)degree, 0.0);
  const double theta = 0.5 * (l1 + l0), delta = 0.5 * (l1 - l0), sigma = theta / delta;
  double rho = 1.0 / sigma;
  c[3] = 1.0 / theta;
  for (int i = 1; i < degree; ++i) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c[2 + 2 * i] = rn * rho;
    c[3 + 2 * i] = 2.0 * rn / delta;
    rho = rn;
  }
  return c;
}

// V-cycle on level l with rhs b; the result lands in *out (level 0: caller's z)
void vcycle_level(tam_amg_s* H, int l, const double* b, double* out, const int* stop, cudaStream_t s) {
  Level& L = H->levels[l];
  const long long N = (long long)L.n_rows * L.bs;
  if (l == (int)H->levels.size() - 1) {
    dense_gemv_kernel<<<grid_for((long long)H->n_coarse * 32, TPB), TPB, 0, s>>>(H->coarse_inv.p, b, out,
                                                                                  H->n_coarse, stop);
    TAM_LAUNCH_CHECK();
    return;
  }
  const int deg = L.deg;
  double* xa = L.xa.p;
  double* xb = L.xb.p;
  // pre-smoothing from zero
  cheb_first_zero_kernel<<<vec_grid(N), TPB, 0, s>>>(b, L.dinv.p, L.consts.p, L.d.p, xa, N, stop);
  TAM_LAUNCH_CHECK();
  for (int k = 1; k < deg; ++k) {
    cheb_step(L, b, xa, L.d.p, xb, k, stop, s);
    std::swap(xa, xb);
  }
  residual(L, b, xa, L.t.p, stop, s);
  Level& C = H->levels[l + 1];
  restrict_to(L, L.t.p, C.b.p, stop, s);
  double* xc = C.y.p;
  vcycle_level(H, l + 1, C.b.p, xc, stop, s);
  prolong_add(L, xc, xa, stop, s);
  // post-smoothing from x
  for (int k = 0; k < deg; ++k) {
    double* dst = (k == deg - 1) ? out : xb;
    cheb_step(L, b, xa, L.d.p, dst, k, stop, s);
    xb = xa;
    xa = dst;
  }
}

// z = M^-1 r with the hierarchy's V-cycle precision
void precondition(tam_amg_s* H, const double* r, double* z, const int* stop, cudaStream_t s) {
  if (H->prm.level_precision > 0) vcycle_apply_low(H, r, z, stop, s);
  else vcycle_level(H, 0, r, z, stop, s);
}

// f(std::integral_constant<int, BR>) for K's block size (3: elasticity, 1: a scalar problem)
template <class F>
void by_block(int br, F&& f) {
  if (br == 1) f(std::integral_constant<int, 1>());
  else f(std::integral_constant<int, 3>());
}

void spmv_outer_pq(tam_amg_s* H, cudaStream_t s) {
  GridReduce gr{H->partials.p, H->ticket.p};
  by_block(H->K->A.br, [&](auto B) {
    constexpr int BR = decltype(B)::value;
    sell_spmv<BR, BR>(H->K->S, H->p.p, EpiPq<BR>{H->p.p, H->q.p, H->K->n_nodes, gr, H->sc.p}, s,
                      H->levels[0].Aop.df, /*acc=*/true);
  });
}

void enqueue_iteration(tam_amg_s* H, double* x, cudaStream_t s) {
  const long long N = (long long)H->K->n_nodes * H->K->A.br;
  GridReduce gr{H->partials.p, H->ticket.p};
  const int* stop = &H->sc.p->stop;
  spmv_outer_pq(H, s);
  pcg_update_kernel<<<vec_grid(N), TPB, 0, s>>>(x, H->r.p, H->p.p, H->q.p, N, gr, H->sc.p, H->hist.p,
                                                (int)H->hist.n);
  TAM_LAUNCH_CHECK();
  precondition(H, H->r.p, H->z.p, stop, s);
  pcg_rz_kernel<<<vec_grid(N), TPB, 0, s>>>(H->r.p, H->z.p, H->p.p, N, gr, H->sc.p, 0);
  TAM_LAUNCH_CHECK();
  pcg_direction_kernel<<<vec_grid(N), TPB, 0, s>>>(H->z.p, H->p.p, N, H->sc.p);
  TAM_LAUNCH_CHECK();
}

}  // namespace

cudaGraphExec_t build_loop_graph(const std::function<void(cudaStream_t)>& enqueue, const int* stop, int* count,
                                 const int* limit, int limit_add, long long* body_kernels) {
  cudaGraph_t g = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool capturing = false;
  try {
    TAM_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    TAM_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    TAM_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    TAM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    TAM_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    capturing = true;
    captured_and_reset();
    g_capturing = true;
    enqueue(cs);
    loop_control_kernel<<<1, 1, 0, cs>>>(h, stop, count, limit, limit_add);
    TAM_LAUNCH_CHECK();
    g_capturing = false;
    *body_kernels = captured_and_reset();
    cudaGraph_t out = nullptr;
    capturing = false;
    TAM_CUDA(cudaStreamEndCapture(cs, &out));
    TAM_CUDA(cudaGraphInstantiate(&exec, g, 0));
  } catch (...) {
    g_capturing = false;
    captured_and_reset();
    if (capturing) {
      cudaGraph_t partial = nullptr;
      cudaStreamEndCapture(cs, &partial);
    }
    cudaGetLastError();
    if (cs) cudaStreamDestroy(cs);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaStreamDestroy(cs);
  cudaGraphDestroy(g);
  return exec;
}

void spmv_K(tam_matrix_s* K, const double* x, double* y, cudaStream_t s) {
  by_block(K->A.br, [&](auto B) {
    constexpr int BR = decltype(B)::value;
    sell_spmv<BR, BR>(K->S, x, EpiStore<BR>{y, K->n_nodes, nullptr}, s, K->df_ok, /*acc=*/true);
  });
}

double residual_norm_K(tam_matrix_s* K, const double* b, const double* x, cudaStream_t s) {
  const unsigned grid = sell_grid(K->S);
  DBuf<double> partials(grid, s), out(1, s);
  DBuf<unsigned int> ticket(1, s);
  ticket.zero();
  GridReduce gr{partials.p, ticket.p};
  by_block(K->A.br, [&](auto B) {
    constexpr int BR = decltype(B)::value;
    sell_spmv<BR, BR>(K->S, x, EpiResNorm<BR>{b, K->n_nodes, gr, out.p}, s, /*df=*/false);
  });
  return std::sqrt(read_back_double(out.p, s));
}

void vcycle_apply(tam_amg_s* H, const double* r, double* z, const int* stop, cudaStream_t s) {
  precondition(H, r, z, stop, s);
}

int pcg_solve(tam_amg_s* H, const double* b, double* x, double rtol, double atol, int max_iter, int* iters,
              double* rel, cudaStream_t s) {
  NvtxRange nvtx("tam: AMG-PCG solve");
  TAM_CHECK(b && x && rtol >= 0.0 && atol >= 0.0 && max_iter >= 0, TAM_ERR_INVALID_ARG, "amg_pcg_solve: bad argument");
  const long long N = (long long)H->K->n_nodes * H->K->A.br;
  GridReduce gr{H->partials.p, H->ticket.p};
  PcgScalars* sc = H->sc.p;
  if (!H->bs.p) H->bs = DBuf<double>((size_t)N, s);
  if (!H->xs.p) H->xs = DBuf<double>((size_t)N, s);
  // residual history: ||r_k||^2 for k = 0 .. iterations (its pointer and size
  // are captured in the iteration graph: a longer one rebuilds the graph)
  if ((long long)H->hist.n < (long long)max_iter + 1) {
    H->hist = DBuf<double>((size_t)std::max(max_iter + 1, 1024), s);
    if (H->iter_exec) {
      cudaGraphExecDestroy(H->iter_exec);
      H->iter_exec = nullptr;
    }
  }
  // the solve runs on its own copies b 2^-e and x 2^-e (e from ||b|| and K's
  // range, see centering_exp), so the iteration graph never depends on the
  // caller's buffers
  double* const xu = x;
  pcg_start_kernel<<<vec_grid(N), TPB, 0, s>>>(b, N, gr, sc, rtol, atol, max_iter, H->K->vmax_exp / 2);
  TAM_LAUNCH_CHECK();
  pcg_scale_kernel<<<vec_grid(N), TPB, 0, s>>>(b, H->bs.p, N, sc, -1);
  TAM_LAUNCH_CHECK();
  pcg_scale_kernel<<<vec_grid(N), TPB, 0, s>>>(xu, H->xs.p, N, sc, -1);
  TAM_LAUNCH_CHECK();
  b = H->bs.p;
  x = H->xs.p;
  by_block(H->K->A.br, [&](auto B) {
    constexpr int BR = decltype(B)::value;
    sell_spmv<BR, BR>(H->K->S, x, EpiInitResidual<BR>{b, H->r.p, H->K->n_nodes, gr, sc, H->hist.p}, s,
                      H->levels[0].Aop.df,
                      /*acc=*/true);
  });
  precondition(H, H->r.p, H->z.p, &sc->stop, s);
  pcg_rz_kernel<<<vec_grid(N), TPB, 0, s>>>(H->r.p, H->z.p, H->p.p, N, gr, sc, 1);
  TAM_LAUNCH_CHECK();
  // the iterations as one graph: a device-side WHILE loop over one iteration,
  // built on the first solve with this hierarchy, one launch per solve
  // (TAM_PCG_HOST_LOOP=1 in the environment: the same iterations as plain
  // launches from a host loop that reads the stop flag after each -- for
  // profilers that do not trace kernels inside conditional graph nodes)
  static const bool host_loop = [] {
    const char* e = std::getenv("TAM_PCG_HOST_LOOP");
    return e && std::atoi(e) != 0;
  }();
  if (host_loop) {
    for (int k = 0; k < max_iter + 2; ++k) {
      enqueue_iteration(H, x, s);
      if (read_back_int(&sc->stop, s)) break;
    }
  } else {
    if (!H->iter_exec)
      H->iter_exec = build_loop_graph([&](cudaStream_t cs) { enqueue_iteration(H, x, cs); }, &sc->stop,
                                      &sc->loops, &sc->max_iter, 2, &H->graph_kernels);
    TAM_CUDA(cudaGraphLaunch(H->iter_exec, s));
  }
  // final true residual, always a plain FP64 product; then x back to the caller's scale
  DBuf<double> rn(1, s);
  by_block(H->K->A.br, [&](auto B) {
    constexpr int BR = decltype(B)::value;
    sell_spmv<BR, BR>(H->K->S, x, EpiResNorm<BR>{b, H->K->n_nodes, gr, rn.p}, s, /*df=*/false);
  });
  pcg_scale_kernel<<<vec_grid(N), TPB, 0, s>>>(x, xu, N, sc, +1);
  TAM_LAUNCH_CHECK();
  PcgScalars host;
  TAM_CUDA(cudaMemcpyAsync(&host, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
  double rr = read_back_double(rn.p, s);  // synchronises the stream
  count_graph_launch(H->graph_kernels * host.loops);
  H->hist_len = std::min<long long>((long long)host.iter + 1, (long long)H->hist.n);
  H->hist_scale_exp = host.scale_exp;
  if (iters) *iters = host.iter;
  double nb = std::sqrt(host.bb);
  if (rel) *rel = nb > 0 ? std::sqrt(rr) / nb : std::sqrt(rr);
  int status = host.status;
  if (status == TAM_OK && !host.stop) status = TAM_ERR_NOT_CONVERGED;
  return status;
}

// x <- `degree` Chebyshev-Jacobi steps on the finest system K x = b starting
// from x, over [lo, hi] * lambda_max(D^-1 K): removes the rough error
// components of an initial guess (those the point smoother acts on) at the
// cost of `degree` SpMVs with K.
void smooth_fine(tam_amg_s* H, const double* b, double* x, int degree, double lo, double hi, cudaStream_t s) {
  TAM_CHECK(degree >= 1 && degree <= 64 && hi > lo && lo > 0, TAM_ERR_INVALID_ARG, "smooth_fine: bad degree or interval");
  Level& L = H->levels[0];
  const long long N = (long long)L.n_rows * L.bs;
  if (H->smooth_deg != degree || H->smooth_lo != lo || H->smooth_hi != hi) {
    // coefficients kept on the device for repeated calls with the same polynomial
    const std::vector<double> c = cheb_coefficients(lo * L.lambda_host, hi * L.lambda_host, degree);
    H->smooth_coef = DBuf<double>(c.size(), s);
    TAM_CUDA(cudaMemcpyAsync(H->smooth_coef.p, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice, s));
    TAM_CUDA(cudaStreamSynchronize(s));  // c is a host temporary
    H->smooth_deg = degree;
    H->smooth_lo = lo;
    H->smooth_hi = hi;
  }
  const double* coef = H->smooth_coef.p;
  double* cur = x;
  double* nxt = L.xb.p;
  for (int k = 0; k < degree; ++k) {
    by_block(L.bs, [&](auto B) {
      constexpr int BR = decltype(B)::value;
      spop_apply<BR, BR>(L.Aop, cur, EpiCheb<BR>{b, cur, L.dinv.p, coef + 2 + 2 * k, L.d.p, nxt, L.n_rows, nullptr},
                         s);
    });
    std::swap(cur, nxt);
  }
  if (cur != x) TAM_CUDA(cudaMemcpyAsync(x, cur, sizeof(double) * (size_t)N, cudaMemcpyDeviceToDevice, s));
}

}  // namespace tam
