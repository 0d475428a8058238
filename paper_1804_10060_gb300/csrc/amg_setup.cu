// Smoothed-aggregation AMG setup (paper Sec. 2.1 "Multigrid preconditioned
// iterative solvers" and Sec. 5.1 "Solver configuration").
//
// Per level: point-Jacobi diagonal, Lanczos estimate of lambda_max(D^-1 A)
// (the paper stresses that Chebyshev smoothing needs an adequate estimate),
// strength graph, aggregation by a distance-2 maximal independent set,
// tentative prolongator by modified Gram-Schmidt of the near-nullspace (the
// six rigid-body modes on the finest level), prolongator smoothing
// P = (I - 4/(3 lambda) D^-1 A) P_tent, R = P^T and the Galerkin product
// A_c = R A P.  The coarsest operator is inverted densely (Gauss-Jordan).
// The Lanczos estimate of a level runs on a second stream, concurrently with
// the level's aggregation and tentative prolongator (only the smoothing of
// the prolongator needs lambda_max).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "handles.cuh"

namespace cg = cooperative_groups;

namespace tam {
namespace {

constexpr int TPB = 256;

// ---------------------------------------------------------------------------
// Diagonal, rigid-body modes
// ---------------------------------------------------------------------------
__global__ void point_dinv_kernel(const int* __restrict__ rp, const int* __restrict__ ci,
                                  const double* __restrict__ v, int n, int bs, double* __restrict__ dinv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int slot = bsearch_i32(ci, rp[i], rp[i + 1], i);
  for (int r = 0; r < bs; ++r) {
    double d = slot >= 0 ? v[(size_t)slot * bs * bs + r * bs + r] : 0.0;
    dinv[(size_t)i * bs + r] = d != 0.0 ? 1.0 / d : 0.0;
  }
}

__global__ void centroid_kernel(const double* __restrict__ X, int n, GridReduce gr, double* __restrict__ out) {
  __shared__ double sh[32];
  double v[3] = {0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) v[d] += X[3 * (size_t)i + d];
  double tot[3];
  if (grid_reduce<3>(gr, v, tot, sh) && threadIdx.x == 0)
    for (int d = 0; d < 3; ++d) out[d] = tot[d] / n;
}

// B[(3i + r) * k + col]: translations, then rotations about x, y, z through c.
__global__ void rigid_modes_kernel(const double* __restrict__ X, const unsigned char* __restrict__ dmask, int n,
                                   const double* __restrict__ c, int k, double* __restrict__ B) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double m[3][6] = {};
  if (!dmask[i]) {
    double dx = X[3 * (size_t)i] - c[0], dy = X[3 * (size_t)i + 1] - c[1], dz = X[3 * (size_t)i + 2] - c[2];
    m[0][0] = m[1][1] = m[2][2] = 1.0;
    m[1][3] = -dz; m[2][3] = dy;
    m[0][4] = dz;  m[2][4] = -dx;
    m[0][5] = -dy; m[1][5] = dx;
  }
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < k; ++q) B[(3 * (size_t)i + r) * k + q] = m[r][q];
}

// The near-nullspace of a scalar diffusion operator: the constant (zero on
// Dirichlet nodes).
__global__ void constant_mode_kernel(const unsigned char* __restrict__ dmask, int n, double* __restrict__ B) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) B[i] = dmask[i] ? 0.0 : 1.0;
}

// ---------------------------------------------------------------------------
// Lanczos estimate of lambda_max(D^-1 A) on S = D^-1/2 A D^-1/2
// ---------------------------------------------------------------------------
struct LanczosWork {
  double* v;      // current Lanczos vector
  double* vp;     // previous
  double* u;      // s .* v (SpMV input)
  double* w;      // work
  const double* s;  // D^-1/2
  double* ab;     // alpha[0..k), beta[k..2k)
  int* m;         // number of completed steps (breakdown stops early)
  long long N;
};

__global__ void lanczos_init_kernel(const double* __restrict__ dinv, long long N, int level, double* __restrict__ s,
                                    double* __restrict__ v, GridReduce gr, double* __restrict__ norm2) {
  __shared__ double sh[32];
  double acc[1] = {0.0};
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    double di = dinv[k];
    double sk = di > 0.0 ? sqrt(di) : 0.0;
    s[k] = sk;
    uint64_t z = splitmix64(((uint64_t)(level + 1) << 40) | (uint64_t)k);
    double vk = sk > 0.0 ? (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5 : 0.0;
    v[k] = vk;
    acc[0] += vk * vk;
  }
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) *norm2 = tot[0];
}

__global__ void lanczos_normalize_kernel(long long N, double* __restrict__ v, const double* __restrict__ s,
                                         double* __restrict__ u, double* __restrict__ vp, const double* __restrict__ norm2) {
  double inv = 1.0 / sqrt(*norm2);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    double vk = v[k] * inv;
    v[k] = vk;
    u[k] = s[k] * vk;
    vp[k] = 0.0;
  }
}

// SpMV epilogue: w = s .* (A u), alpha_j = w . v
template <int BR>
struct EpiLanczos {
  double* w;
  const double* s;
  const double* v;
  int n_rows;
  GridReduce gr;
  double* alpha_out;
  const int* done;
  __device__ bool skip() const { return *done; }
  __device__ void operator()(int row, const double (&acc)[BR], double* sh) const {
    double dot[1] = {0.0};
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        size_t i = (size_t)row * BR + r;
        double wi = s[i] * acc[r];
        w[i] = wi;
        dot[0] += wi * v[i];
      }
    double tot[1];
    if (grid_reduce<1>(gr, dot, tot, sh) && threadIdx.x == 0) *alpha_out = tot[0];
  }
};

__global__ void lanczos_orth_kernel(LanczosWork L, int j, GridReduce gr, const int* __restrict__ done) {
  __shared__ double sh[32];
  if (*done) return;
  const double a = L.ab[j];
  const int K = 0;  // unused
  (void)K;
  const double bprev = j > 0 ? L.ab[64 + j - 1] : 0.0;
  double acc[1] = {0.0};
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < L.N; k += (long long)gridDim.x * blockDim.x) {
    double wk = L.w[k] - a * L.v[k] - bprev * L.vp[k];
    L.w[k] = wk;
    acc[0] += wk * wk;
  }
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) L.ab[64 + j] = sqrt(tot[0]);
}

__global__ void lanczos_advance_kernel(LanczosWork L, int j, int* __restrict__ done) {
  if (*done) return;
  const double a = L.ab[j], b = L.ab[64 + j];
  if (!(b > 1e-14 * fabs(a))) {
    // breakdown: the Krylov space is invariant; keep the j+1 steps done so far
    if (blockIdx.x == 0 && threadIdx.x == 0) { *L.m = j + 1; }
    return;
  }
  const double inv = 1.0 / b;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < L.N; k += (long long)gridDim.x * blockDim.x) {
    double vn = L.w[k] * inv;
    L.vp[k] = L.v[k];
    L.v[k] = vn;
    L.u[k] = L.s[k] * vn;
  }
}

__global__ void lanczos_mark_done_kernel(const LanczosWork L, int j, int* __restrict__ done) {
  // runs after advance: if breakdown was recorded at step j, stop the remaining steps
  if (*L.m == j + 1) *done = 1;
}

// Largest eigenvalue of the symmetric tridiagonal (alpha, beta) of order m by
// bisection with Sturm sequence counts; then Chebyshev/omega constants.
__global__ void tridiag_lmax_kernel(const double* __restrict__ ab, const int* __restrict__ m_ptr, int kmax,
                                    double cheb_lo, double cheb_hi, int degree, double* __restrict__ consts) {
  int m = *m_ptr;
  if (m <= 0 || m > kmax) m = kmax;
  const double* a = ab;
  const double* b = ab + 64;
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i < m - 1 ? fabs(b[i]) : 0.0);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  // count of eigenvalues < x
  auto count_below = [&](double x) {
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      q = a[i] - x - (i > 0 ? bb / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++c;
    }
    return c;
  };
  // multisection by one warp: the lanes test 32 interior points of [lo, hi]
  // (x is above the largest Ritz value iff all m eigenvalues lie below it, a
  // condition monotone in x), and the interval shrinks 33-fold per round
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < 60 && hi - lo > 1e-15 * fmax(fabs(hi), fabs(lo)); ++it) {
    const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const unsigned above = __ballot_sync(0xffffffffu, count_below(x) >= m);
    const int first = above ? __ffs(above) - 1 : 32;  // lowest lane whose point is above
    const double xl = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
    const double xh = __shfl_sync(0xffffffffu, x, first < 32 ? first : 31);
    const double nlo = first > 0 ? xl : lo, nhi = first < 32 ? xh : hi;
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return;
  const double lam = 0.5 * (lo + hi);
  consts[0] = lam;
  consts[1] = 4.0 / (3.0 * lam);
  const double l0 = cheb_lo * lam, l1 = cheb_hi * lam;
  const double theta = 0.5 * (l1 + l0), delta = 0.5 * (l1 - l0), sigma = theta / delta;
  double rho = 1.0 / sigma;
  consts[2] = 0.0;
  consts[3] = 1.0 / theta;
  for (int i = 1; i < degree; ++i) {
    double rn = 1.0 / (2.0 * sigma - rho);
    consts[2 + 2 * i] = rn * rho;
    consts[3 + 2 * i] = 2.0 * rn / delta;
    rho = rn;
  }
}

// ---------------------------------------------------------------------------
// Strength graph and aggregation
// ---------------------------------------------------------------------------
// Frobenius norm of every block (one thread per block: consecutive threads
// read consecutive blocks), then each row's diagonal norm.
__global__ void block_norms_kernel(const double* __restrict__ v, long long nnzb, int bb, double* __restrict__ nrm) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnzb; p += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = 0; e < bb; ++e) {
      double x = v[(size_t)p * bb + e];
      s += x * x;
    }
    nrm[p] = sqrt(s);
  }
}

__global__ void diag_norms_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ nrm,
                                  int n, double* __restrict__ dnrm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double dn = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) dn = nrm[p];
  dnrm[i] = dn;
}

__global__ void strength_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ nrm,
                                const double* __restrict__ dnrm, int n, double theta, unsigned char* __restrict__ strong,
                                unsigned char* __restrict__ isolated) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cnt = 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    bool st = (j != i) && nrm[p] > 0.0 && nrm[p] >= theta * sqrt(dnrm[i] * dnrm[j]);
    strong[p] = st;
    cnt += st;
  }
  isolated[i] = cnt == 0;
}

__device__ __forceinline__ unsigned long long prio30(int level, int i) {
  return splitmix64(((uint64_t)(unsigned)level << 32) | (uint64_t)(unsigned)i) >> 34;
}

enum : unsigned char { ST_UND = 0, ST_ROOT = 1, ST_OUT = 2 };

__device__ __forceinline__ unsigned long long mis_tuple(unsigned char st, int level, int i) {
  if (st == ST_OUT) return 0ull;
  unsigned long long s = st == ST_ROOT ? 2ull : 1ull;
  return (s << 62) | (prio30(level, i) << 32) | (unsigned)i;
}

__global__ void mis_init_kernel(const unsigned char* __restrict__ isolated, int n, unsigned char* __restrict__ state) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) state[i] = isolated[i] ? ST_OUT : ST_UND;
}

// A round whose predecessor left no node undecided (prev_und, null for the
// first round) does nothing, so the host can launch several rounds per check.
// tup[i] = mis_tuple(state[i], level, i), kept current by mis_round2_kernel
// (so the rounds read each neighbour's tuple instead of rehashing its id)
__global__ void mis_tuple_init_kernel(const unsigned char* __restrict__ state, int n, int level,
                                      unsigned long long* __restrict__ tup) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tup[i] = mis_tuple(state[i], level, i);
}

__global__ void mis_round1_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const unsigned char* __restrict__ strong,
                                  const unsigned long long* __restrict__ tup, int n, unsigned long long* __restrict__ m1,
                                  const int* __restrict__ prev_und) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (prev_und && *prev_und == 0)) return;
  unsigned long long m = tup[i];
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (strong[p]) {
      const unsigned long long t = tup[ci[p]];
      m = t > m ? t : m;
    }
  m1[i] = m;
}

__global__ void mis_round2_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const unsigned char* __restrict__ strong,
                                  unsigned char* __restrict__ state, const unsigned long long* __restrict__ m1, int n,
                                  int level, int distance, const int* __restrict__ prev_und,
                                  int* __restrict__ undecided, unsigned long long* __restrict__ tup) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || (prev_und && *prev_und == 0)) return;
  if (state[i] != ST_UND) return;
  unsigned long long m = m1[i];  // max over the closed 1-neighbourhood
  if (distance == 2)
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (strong[p]) {
        unsigned long long t = m1[ci[p]];
        m = t > m ? t : m;
      }
  const unsigned long long mine = tup[i];  // mis_tuple(ST_UND, level, i)
  if (m == mine) {
    state[i] = ST_ROOT;
    tup[i] = mis_tuple(ST_ROOT, level, i);
  } else if ((m >> 62) == 2ull) {
    state[i] = ST_OUT;
    tup[i] = 0ull;
  } else {
    atomicAdd(undecided, 1);
  }
}

__global__ void root_flag_kernel(const unsigned char* __restrict__ state, const unsigned char* __restrict__ isolated, int n,
                                 int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (state[i] == ST_ROOT && !isolated[i]) ? 1 : 0;
}

// phase 2: roots keep their id; others join the adjacent root of largest key
__global__ void agg_phase2_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const unsigned char* __restrict__ strong,
                                  const unsigned char* __restrict__ state, const unsigned char* __restrict__ isolated,
                                  const int* __restrict__ root_id, int n, int level, int* __restrict__ agg2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (isolated[i]) { agg2[i] = -1; return; }
  if (state[i] == ST_ROOT) { agg2[i] = root_id[i]; return; }
  unsigned long long best = 0;
  int bj = -1;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    if (strong[p] && state[j] == ST_ROOT) {
      unsigned long long key = (prio30(level, j) << 32) | (unsigned)j;
      if (bj < 0 || key > best) { best = key; bj = j; }
    }
  }
  agg2[i] = bj >= 0 ? root_id[bj] : -1;
}

// phase 3: left-over nodes join the aggregate of the attached neighbour of largest key
__global__ void agg_phase3_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const unsigned char* __restrict__ strong,
                                  const unsigned char* __restrict__ isolated, const int* __restrict__ agg2, int n, int level,
                                  int* __restrict__ agg3, int* __restrict__ fail) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int a = agg2[i];
  if (a < 0 && !isolated[i]) {
    unsigned long long best = 0;
    int bj = -1;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      int j = ci[p];
      if (strong[p] && agg2[j] >= 0) {
        unsigned long long key = (prio30(level, j) << 32) | (unsigned)j;
        if (bj < 0 || key > best) { best = key; bj = j; }
      }
    }
    if (bj >= 0) a = agg2[bj];
    else atomicExch(fail, 1);
  }
  agg3[i] = a;
}

// ---------------------------------------------------------------------------
// Tentative prolongator
// ---------------------------------------------------------------------------
__global__ void has_agg_kernel(const int* __restrict__ agg, int n, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cnt[i] = agg[i] >= 0 ? 1 : 0;
}

__global__ void ptent_pattern_kernel(const int* __restrict__ agg, const int* __restrict__ rp, int n, int* __restrict__ ci,
                                     const double* __restrict__ B, int bs, int k, double* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || agg[i] < 0) return;
  int p = rp[i];
  ci[p] = agg[i];
  for (int r = 0; r < bs; ++r)
    for (int q = 0; q < k; ++q) v[(size_t)p * bs * k + r * k + q] = B[((size_t)i * bs + r) * k + q];
}

__global__ void agg_count_kernel(const int* __restrict__ agg, int n, int* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) atomicAdd(&cnt[agg[i]], 1);
}

__global__ void agg_fill_kernel(const int* __restrict__ agg, int n, const int* __restrict__ ap, int* __restrict__ cursor,
                                int* __restrict__ mem) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) mem[ap[agg[i]] + atomicAdd(&cursor[agg[i]], 1)] = i;
}

// warp per aggregate: members sorted by rank (node ids are unique)
__global__ void agg_sort_kernel(const int* __restrict__ ap, int n_agg, const int* __restrict__ mem, int* __restrict__ out) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n_agg) return;
  int s = ap[w], e = ap[w + 1];
  for (int p = s + lane; p < e; p += 32) {
    int key = mem[p], rank = 0;
    for (int q = s; q < e; ++q) rank += mem[q] < key;
    out[s + rank] = key;
  }
}

// warp per aggregate: modified Gram-Schmidt on the P_tent blocks (rows:
// member nodes in increasing id, bs rows each; columns: k modes).  An
// aggregate of at most QR_CAP rows is copied into the warp's shared-memory
// tile once, orthonormalised there and written back (the global path walks
// the node map for every access of every pass); larger ones work in place.
// Both paths do the same operations in the same order.
constexpr int QR_WARPS = 4, QR_CAP = 192;

template <class F>
__device__ __forceinline__ void mgs_columns(int rows, int k, int lane, double droptol, double (&R)[6][6],
                                            const F& elem) {
  for (int c = 0; c < k; ++c) {
    double nn = 0.0;
    for (int r = lane; r < rows; r += 32) { double x = elem(r, c); nn += x * x; }
    const double norm0 = sqrt(warp_sum(nn));
    for (int j = 0; j < c; ++j) {
      double d = 0.0;
      for (int r = lane; r < rows; r += 32) d += elem(r, j) * elem(r, c);
      d = warp_sum(d);
      R[j][c] = d;
      for (int r = lane; r < rows; r += 32) elem(r, c) -= d * elem(r, j);
      __syncwarp();
    }
    double n2 = 0.0;
    for (int r = lane; r < rows; r += 32) { double x = elem(r, c); n2 += x * x; }
    const double nv = sqrt(warp_sum(n2));
    const bool keep = norm0 > 0.0 && nv > droptol * norm0;
    R[c][c] = keep ? nv : 0.0;
    const double inv = keep ? 1.0 / nv : 0.0;
    for (int r = lane; r < rows; r += 32) elem(r, c) *= inv;
    __syncwarp();
  }
}

__global__ void __launch_bounds__(QR_WARPS * 32)
ptent_qr_kernel(const int* __restrict__ ap, const int* __restrict__ mem, int n_agg, const int* __restrict__ prp,
                double* __restrict__ pv, int bs, int k, double droptol, double* __restrict__ Bc) {
  __shared__ double tile[QR_WARPS][QR_CAP * 6];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * QR_WARPS + wid;
  if (w >= n_agg) return;  // warp-uniform; no block-wide barrier below
  const int s = ap[w], e = ap[w + 1];
  const int rows = (e - s) * bs;
  double R[6][6];
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) R[a][b] = 0.0;
  auto gaddr = [&](int row, int col) -> double* {
    const int node = mem[s + row / bs];
    return pv + (size_t)prp[node] * bs * k + (row % bs) * k + col;
  };
  if (rows <= QR_CAP) {
    double* t = tile[wid];
    for (int r = lane; r < rows; r += 32) {
      const double* src = gaddr(r, 0);  // the row's k values are contiguous
      for (int c = 0; c < k; ++c) t[r * k + c] = src[c];
    }
    __syncwarp();
    mgs_columns(rows, k, lane, droptol, R, [&](int r, int c) -> double& { return t[r * k + c]; });
    for (int r = lane; r < rows; r += 32) {
      double* dst = gaddr(r, 0);
      for (int c = 0; c < k; ++c) dst[c] = t[r * k + c];
    }
  } else {
    mgs_columns(rows, k, lane, droptol, R, [&](int r, int c) -> double& { return *gaddr(r, c); });
  }
  if (lane == 0)
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) Bc[((size_t)w * k + a) * k + b] = R[a][b];
}

// P = (I - omega D^-1 A) P_tent, in place on the values of A*P_tent
// One warp per row: a row's blocks are contiguous, so the lanes stride its
// bs * k values (coalesced) instead of one thread walking them.
template <int BS, int KD>
__global__ void smooth_prolongator_kernel(const int* __restrict__ rp, const int* __restrict__ ci, double* __restrict__ v,
                                          int n, const double* __restrict__ dinv,
                                          const double* __restrict__ consts, const int* __restrict__ agg,
                                          const int* __restrict__ ptrp, const double* __restrict__ ptv) {
  constexpr int bs = BS, k = KD;  // constants: the index divisions below become multiplications
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  const double omega = consts[1];
  const int a = agg[i], bk = bs * k, p0 = rp[i];
  const int len = (rp[i + 1] - p0) * bk;
  const double* __restrict__ pt = a >= 0 ? ptv + (size_t)ptrp[i] * bk : nullptr;  // P_tent's block of row i
  double* __restrict__ vr = v + (size_t)p0 * bk;
  for (int rel = lane; rel < len; rel += 32) {
    const int p = p0 + rel / bk, e = rel % bk, r = e / k;
    const double sc = -omega * dinv[(size_t)i * bs + r];
    double val = sc * vr[rel];
    if (ci[p] == a) val += pt[e];
    vr[rel] = val;
  }
}

// ---------------------------------------------------------------------------
// Coarsest level: dense Gauss-Jordan inverse (SPD, no pivoting)
// ---------------------------------------------------------------------------
__global__ void bsr_to_dense_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                                    int n, int bs, double* __restrict__ D, int N) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    for (int r = 0; r < bs; ++r)
      for (int c = 0; c < bs; ++c) D[(size_t)(i * bs + r) * N + j * bs + c] = v[(size_t)p * bs * bs + r * bs + c];
  }
}

__global__ void dense_inactive_kernel(double* __restrict__ D, int N, unsigned char* __restrict__ inactive) {
  int i = blockIdx.x;
  __shared__ int nz;
  if (threadIdx.x == 0) nz = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x)
    if (D[(size_t)i * N + j] != 0.0) nz = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    inactive[i] = nz ? 0 : 1;
    if (!nz) D[(size_t)i * N + i] = 1.0;
  }
}

// In-place Gauss-Jordan inversion of an SPD matrix (no pivoting needed),
// blocked by panels K = [k0, k0 + b) of GJB columns.  With A = [A_KK A_KJ;
// A_IK A_IJ], eliminating K gives [A_KK^-1, A_KK^-1 A_KJ; -A_IK A_KK^-1,
// A_IJ - A_IK A_KK^-1 A_KJ], the state the unblocked method reaches after b
// pivots (D_kj /= p, D_ik = -D_ik / p, D_kk = 1 / p).  Per panel:
//   1. block 0 inverts D_KK in shared memory by unblocked Gauss-Jordan (its
//      pivots are the unblocked method's: positive for an SPD matrix);
//   2. the new row panel D_KK^-1 D_KJ goes to rpan (GJB x N, a thread per
//      element) and the column panel D_IK is saved (cpan, N x GJB);
//   3. D_IJ -= cpan rpan, D_IK = -cpan D_KK^-1, and rpan is copied to D_KJ.
// Three grid-wide barriers per panel instead of two per pivot (the barriers,
// not the N^3 multiply-adds, dominated: 624 of them on a 312-DOF level).
constexpr int GJB = 32;

__global__ void __launch_bounds__(256) gj_coop_kernel(double* __restrict__ D, int N, double* __restrict__ cpan,
                                                      double* __restrict__ rpan, int* __restrict__ bad) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sd[GJB][GJB + 1];  // the diagonal block (step 1), then its inverse (steps 2-3)
  __shared__ double ck[GJB];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int k0 = 0; k0 < N; k0 += GJB) {
    const int b = min(GJB, N - k0);
    if (blockIdx.x == 0) {  // 1.
      for (int e = threadIdx.x; e < b * b; e += blockDim.x) sd[e / b][e % b] = D[(size_t)(k0 + e / b) * N + k0 + e % b];
      __syncthreads();
      for (int k = 0; k < b; ++k) {
        const double p = sd[k][k];
        if (threadIdx.x == 0 && !(p > 0.0)) *bad = 1;
        const double inv = 1.0 / p;
        if (threadIdx.x < b) ck[threadIdx.x] = sd[threadIdx.x][k];
        __syncthreads();
        if (threadIdx.x < b && threadIdx.x != k) sd[k][threadIdx.x] *= inv;
        __syncthreads();
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
          const int i = e / b, j = e % b;
          if (i == k) {
            if (j == k) sd[k][k] = inv;
            continue;
          }
          if (j == k) sd[i][k] = -ck[i] * inv;
          else sd[i][j] -= ck[i] * sd[k][j];
        }
        __syncthreads();
      }
      for (int e = threadIdx.x; e < b * b; e += blockDim.x) D[(size_t)(k0 + e / b) * N + k0 + e % b] = sd[e / b][e % b];
    }
    grid.sync();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) sd[e / b][e % b] = D[(size_t)(k0 + e / b) * N + k0 + e % b];
    __syncthreads();
    // 2. new row panel (a thread per element, columns outside K) and the
    // saved column panel
    for (int e = tid; e < b * (N - b); e += nth) {
      const int r = e / (N - b), jj = e % (N - b), j = jj < k0 ? jj : jj + b;
      double v = 0.0;
      for (int t = 0; t < b; ++t) v = fma(sd[r][t], D[(size_t)(k0 + t) * N + j], v);
      rpan[(size_t)r * N + j] = v;
    }
    for (int e = tid; e < (N - b) * b; e += nth) {
      const int ii = e / b, c = e % b, i = ii < k0 ? ii : ii + b;
      cpan[(size_t)i * GJB + c] = D[(size_t)i * N + k0 + c];
    }
    grid.sync();
    // 3. the rest and the column panel (a thread per element of the rows outside K)
    for (int e = tid; e < (N - b) * N; e += nth) {
      const int ii = e / N, j = e % N, i = ii < k0 ? ii : ii + b;
      const double* __restrict__ ci = cpan + (size_t)i * GJB;
      double v = 0.0;
      if (j >= k0 && j < k0 + b) {
        for (int t = 0; t < b; ++t) v = fma(ci[t], sd[t][j - k0], v);
        D[(size_t)i * N + j] = -v;
      } else {
        for (int t = 0; t < b; ++t) v = fma(ci[t], rpan[(size_t)t * N + j], v);
        D[(size_t)i * N + j] -= v;
      }
    }
    for (int e = tid; e < b * (N - b); e += nth) {
      const int r = e / (N - b), jj = e % (N - b), j = jj < k0 ? jj : jj + b;
      D[(size_t)(k0 + r) * N + j] = rpan[(size_t)r * N + j];
    }
    grid.sync();
  }
}

__global__ void dense_zero_inactive_kernel(double* __restrict__ D, int N, const unsigned char* __restrict__ inactive) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (j >= N) return;
  if (inactive[i] || inactive[j]) D[(size_t)i * N + j] = 0.0;
}

}  // namespace

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------
// SpMV layout of a coarse-level operator (see SpOp): SELL-32 for many short
// rows, the interleaved store for 2-8 lanes per row, whole warps per row over
// an 8-lane interleaved store for the few long rows of the coarsest levels,
// else lanes per row over the block-CSR arrays.  Double-float values where
// use_df says so, and for the whole-warp rows unless FP64 is asked for: with
// one or two blocks per thread those kernels are bound by the FP64 pipe (the
// multiply-adds and the closing reduction), not by memory.
static void plan_spop(SpOp& op, Bsr& A, Sell& S, LprStore& store, int spmv_fp64, cudaStream_t s) {
  bool df = use_df(A, spmv_fp64);
  op = SpOp{&A, &S, choose_lpr(A), df};
  if (op.lpr == 0) {
    bsr_to_sell(A, S, s, df);
    return;
  }
  op.tpr = rows_tpr(A.n_rows, A.nnzb, op.lpr);
  if (A.br == 6 && A.bc == 6 && (op.tpr || op.lpr != 8)) {
    // 6x6 blocks in few long rows or in short rows (all but the many medium
    // rows that take the 8-lane store): block-row lanes over the
    // block-CSR arrays, double-float unless FP64 is forced (the FP64 pipe
    // would bound it, as on the whole-warp rows below)
    op.tpr = 0;
    op.brw = blockrow_wpr(A.n_rows, A.nnzb, A.br);
    if (spmv_fp64 != 1) op.df = df = true;
    if (df) build_df_values(A, s);
    return;
  }
  if (op.tpr && spmv_fp64 != 1) op.df = df = true;
  const int store_lpr = op.tpr ? ROWS_LPR : (lpr_store_pays(op.lpr) ? op.lpr : 0);
  if (store_lpr) {
    build_lpr_store(A, store_lpr, df, store, s);
    op.L = &store;
  } else if (df) {
    build_df_values(A, s);
  }
}

// Runs on its own stream s (beside the level's aggregation) with its own
// grid-reduce scratch gr; writes lambda_max and the Chebyshev constants to
// L.consts, which the caller allocated before the fork.
static void lanczos_lambda(tam_amg_s* H, Level& L, int level, cudaStream_t s, GridReduce gr) {
  const long long N = (long long)L.n_rows * L.bs;
  const int k = std::min(std::max(H->prm.eig_iters, 1), 64);
  DBuf<double> v(N, s), vp(N, s), u(N, s), w(N, s), sv(N, s), ab(128, s), nrm(1, s);
  DBuf<int> mdone(2, s);
  ab.zero();
  TAM_CUDA(cudaMemsetAsync(mdone.p, 0, 2 * sizeof(int), s));
  const unsigned g = std::min<unsigned>(grid_for(N, TPB), (unsigned)H->max_grid);
  lanczos_init_kernel<<<g, TPB, 0, s>>>(L.dinv.p, N, level, sv.p, v.p, gr, nrm.p);
  TAM_LAUNCH_CHECK();
  lanczos_normalize_kernel<<<g, TPB, 0, s>>>(N, v.p, sv.p, u.p, vp.p, nrm.p);
  TAM_LAUNCH_CHECK();
  LanczosWork LW{v.p, vp.p, u.p, w.p, sv.p, ab.p, mdone.p, N};
  int* done = mdone.p + 1;
  TAM_CUDA(cudaMemcpyAsync(mdone.p, &k, sizeof(int), cudaMemcpyHostToDevice, s));
  for (int j = 0; j < k; ++j) {
    if (L.bs == 3) {
      EpiLanczos<3> epi{w.p, sv.p, v.p, L.n_rows, gr, ab.p + j, done};
      spop_apply<3, 3>(L.Aop, u.p, epi, s);
    } else if (L.bs == 6) {
      EpiLanczos<6> epi{w.p, sv.p, v.p, L.n_rows, gr, ab.p + j, done};
      spop_apply<6, 6>(L.Aop, u.p, epi, s);
    } else {
      EpiLanczos<1> epi{w.p, sv.p, v.p, L.n_rows, gr, ab.p + j, done};
      spop_apply<1, 1>(L.Aop, u.p, epi, s);
    }
    lanczos_orth_kernel<<<g, TPB, 0, s>>>(LW, j, gr, done);
    TAM_LAUNCH_CHECK();
    if (j + 1 < k) {
      lanczos_advance_kernel<<<g, TPB, 0, s>>>(LW, j, done);
      TAM_LAUNCH_CHECK();
      lanczos_mark_done_kernel<<<1, 1, 0, s>>>(LW, j, done);
      TAM_LAUNCH_CHECK();
    }
  }
  tridiag_lmax_kernel<<<1, 32, 0, s>>>(ab.p, mdone.p, k, H->prm.cheb_lo, H->prm.cheb_hi, std::max(L.deg, 1),
                                       L.consts.p);
  TAM_LAUNCH_CHECK();
}

// A second stream for work that overlaps the main one: a level's Lanczos
// estimate runs beside its aggregation, tentative prolongator and A P_tent,
// which do not need lambda_max; the main stream waits for it only before the
// prolongator smoothing.  The destructor drains the stream, so buffers the
// side work uses must be declared before this object.
struct SideStream {
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork_ev = nullptr, done_ev = nullptr;
  bool pending = false;
  SideStream() {
    cudaError_t e = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      release();
      TAM_CUDA(e);
    }
  }
  SideStream(const SideStream&) = delete;
  SideStream& operator=(const SideStream&) = delete;
  void fork(cudaStream_t s) {
    TAM_CUDA(cudaEventRecord(fork_ev, s));
    TAM_CUDA(cudaStreamWaitEvent(s2, fork_ev, 0));
  }
  void done() {
    TAM_CUDA(cudaEventRecord(done_ev, s2));
    pending = true;
  }
  void join(cudaStream_t s) {
    if (!pending) return;
    TAM_CUDA(cudaStreamWaitEvent(s, done_ev, 0));
    pending = false;
  }
  void release() {
    if (s2) {
      cudaStreamSynchronize(s2);
      cudaStreamDestroy(s2);
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (done_ev) cudaEventDestroy(done_ev);
    s2 = nullptr;
    fork_ev = done_ev = nullptr;
  }
  ~SideStream() { release(); }
};

static int aggregate(Level& L, int level, double theta, int distance, cudaStream_t s) {
  const Bsr& A = *L.A;
  const int n = A.n_rows;
  DBuf<double> nrm((size_t)A.nnzb, s), dnrm(n, s);
  DBuf<unsigned char> strong((size_t)A.nnzb, s), isolated(n, s), state(n, s);
  block_norms_kernel<<<stride_grid(A.nnzb, TPB, 16), TPB, 0, s>>>(A.vals.p, A.nnzb,
                                                                                          (int)A.block_elems(), nrm.p);
  TAM_LAUNCH_CHECK();
  diag_norms_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, nrm.p, n, dnrm.p);
  TAM_LAUNCH_CHECK();
  strength_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, nrm.p, dnrm.p, n, theta, strong.p,
                                                   isolated.p);
  TAM_LAUNCH_CHECK();
  mis_init_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(isolated.p, n, state.p);
  TAM_LAUNCH_CHECK();
  DBuf<unsigned long long> m1(n, s), tup(n, s);
  mis_tuple_init_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(state.p, n, level, tup.p);
  TAM_LAUNCH_CHECK();
  // und[it]: nodes still undecided after round it; rounds launched 8 at a
  // time between host checks (a round after one that left none is a no-op)
  constexpr int kMaxRounds = 1024, kBatch = 8;
  DBuf<int> und(kMaxRounds, s);
  und.zero();
  for (int it = 0;; ++it) {
    const int* prev = it > 0 ? und.p + it - 1 : nullptr;
    mis_round1_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, strong.p, tup.p, n, m1.p, prev);
    TAM_LAUNCH_CHECK();
    mis_round2_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, strong.p, state.p, m1.p, n, level,
                                                       distance, prev, und.p + it, tup.p);
    TAM_LAUNCH_CHECK();
    if ((it + 1) % kBatch == 0 || it + 1 == kMaxRounds) {
      if (read_back_int(und.p + it, s) == 0) break;
      TAM_CHECK(it + 1 < kMaxRounds, TAM_ERR_INTERNAL, "amg_setup: MIS-2 did not terminate");
    }
  }
  DBuf<int> root_id((size_t)n + 1, s);
  root_flag_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(state.p, isolated.p, n, root_id.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i32(root_id.p, root_id.p, n, s);
  DBuf<int> agg2(n, s), fail(1, s);
  fail.zero();
  agg_phase2_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, strong.p, state.p, isolated.p, root_id.p,
                                                     n, level, agg2.p);
  TAM_LAUNCH_CHECK();
  L.agg = DBuf<int>(n, s);
  agg_phase3_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, strong.p, isolated.p, agg2.p, n, level,
                                                     L.agg.p, fail.p);
  TAM_LAUNCH_CHECK();
  int n_agg = 0, failed = 0;
  read_back_int2(root_id.p + n, fail.p, &n_agg, &failed, s);
  TAM_CHECK(failed == 0, TAM_ERR_INTERNAL, "amg_setup: aggregation left a node unassigned");
  return n_agg;
}

// P_tent and the coarse near-nullspace Bc [n_agg*k, k]
static void tentative(Level& L, const double* B, double droptol, DBuf<double>& Bc, cudaStream_t s) {
  const int n = L.n_rows, bs = L.bs, k = L.kdim, na = L.n_agg;
  Bsr& Pt = L.Pt;
  Pt.n_rows = n;
  Pt.n_cols = na;
  Pt.br = bs;
  Pt.bc = k;
  Pt.row_ptr = DBuf<int>((size_t)n + 1, s);
  has_agg_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(L.agg.p, n, Pt.row_ptr.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i32(Pt.row_ptr.p, Pt.row_ptr.p, n, s);
  Pt.nnzb = read_back_int(Pt.row_ptr.p + n, s);
  Pt.col_idx = DBuf<int>((size_t)Pt.nnzb, s);
  Pt.vals = DBuf<double>((size_t)Pt.nnzb * bs * k, s);
  ptent_pattern_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(L.agg.p, Pt.row_ptr.p, n, Pt.col_idx.p, B, bs, k, Pt.vals.p);
  TAM_LAUNCH_CHECK();
  DBuf<int> ap((size_t)na + 1, s), cursor(na, s), mem((size_t)std::max<long long>(Pt.nnzb, 1), s),
      sorted((size_t)std::max<long long>(Pt.nnzb, 1), s);
  ap.zero();
  cursor.zero();
  agg_count_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(L.agg.p, n, ap.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i32(ap.p, ap.p, na, s);
  agg_fill_kernel<<<grid_for(n, TPB), TPB, 0, s>>>(L.agg.p, n, ap.p, cursor.p, mem.p);
  TAM_LAUNCH_CHECK();
  agg_sort_kernel<<<grid_for((long long)na * 32, TPB), TPB, 0, s>>>(ap.p, na, mem.p, sorted.p);
  TAM_LAUNCH_CHECK();
  Bc = DBuf<double>((size_t)na * k * k, s);
  ptent_qr_kernel<<<grid_for(na, QR_WARPS), QR_WARPS * 32, 0, s>>>(ap.p, sorted.p, na, Pt.row_ptr.p, Pt.vals.p, bs,
                                                                   k, 1e-10, Bc.p);
  TAM_LAUNCH_CHECK();
  (void)droptol;
}

static void coarse_inverse(tam_amg_s* H, const Level& L, cudaStream_t s) {
  const int N = L.n_rows * L.bs;
  TAM_CHECK(N <= 12000, TAM_ERR_UNSUPPORTED, "amg_setup: coarsest level too large for the dense solve");
  H->n_coarse = N;
  H->coarse_inv = DBuf<double>((size_t)N * N, s);
  H->coarse_inv.zero();
  const Bsr& A = *L.A;
  bsr_to_dense_kernel<<<grid_for(L.n_rows, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, A.vals.p, L.n_rows, L.bs,
                                                              H->coarse_inv.p, N);
  TAM_LAUNCH_CHECK();
  DBuf<unsigned char> inactive(N, s);
  dense_inactive_kernel<<<N, 128, 0, s>>>(H->coarse_inv.p, N, inactive.p);
  TAM_LAUNCH_CHECK();
  DBuf<double> colk((size_t)N * GJB, s), rowk((size_t)N * GJB, s);
  DBuf<int> bad(1, s);
  bad.zero();
  dim3 ug(grid_for(N, TPB), N);
  // all panels in one cooperative launch (grid-wide barriers between the
  // three steps of a panel) instead of 3N / GJB kernel launches
  int dev = 0, n_sm = 0, per_sm = 0;
  TAM_CUDA(cudaGetDevice(&dev));
  TAM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  TAM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gj_coop_kernel, TPB, 0));
  TAM_CHECK(per_sm >= 1, TAM_ERR_INTERNAL, "amg_setup: Gauss-Jordan kernel cannot be resident");
  double* dp = H->coarse_inv.p;
  double* cp = colk.p;
  double* rp = rowk.p;
  int* bp = bad.p;
  int n_arg = N;
  void* args[] = {&dp, &n_arg, &cp, &rp, &bp};
  TAM_CUDA(cudaLaunchCooperativeKernel((const void*)gj_coop_kernel, dim3(n_sm), dim3(TPB), args, 0, s));
  TAM_LAUNCH_CHECK();
  dense_zero_inactive_kernel<<<ug, TPB, 0, s>>>(H->coarse_inv.p, N, inactive.p);
  TAM_LAUNCH_CHECK();
  TAM_CHECK(read_back_int(bad.p, s) == 0, TAM_ERR_INTERNAL, "amg_setup: coarsest operator is not positive definite");
}

static void alloc_level_vectors(Level& L, cudaStream_t s) {
  size_t N = (size_t)L.n_rows * L.bs;
  L.b = DBuf<double>(N, s);
  L.xa = DBuf<double>(N, s);
  L.xb = DBuf<double>(N, s);
  L.d = DBuf<double>(N, s);
  L.t = DBuf<double>(N, s);
  L.y = DBuf<double>(N, s);
}

// Setup phase timing with CUDA events (no extra synchronisation): the time
// between mark(p) and the next mark is charged to phase p.
struct PhaseTimer {
  std::vector<std::pair<int, cudaEvent_t>> marks;
  bool open = false;  // an NVTX range of the current phase is pushed
  void mark(int phase, cudaStream_t s) {
    static const char* const names[8] = {"tam setup: lambda_max",  "tam setup: aggregation",
                                         "tam setup: tentative",   "tam setup: smoothing",
                                         "tam setup: transpose",   "tam setup: galerkin",
                                         "tam setup: layout",      "tam setup: coarse inverse"};
    if (open) nvtxRangePop();
    open = phase >= 0 && phase < 8;
    if (open) nvtxRangePushA(names[phase]);
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    marks.emplace_back(phase, e);
  }
  void finish(double* ms) {
    for (size_t i = 0; i + 1 < marks.size(); ++i) {
      float t = 0.f;
      if (marks[i].first >= 0 && cudaEventElapsedTime(&t, marks[i].second, marks[i + 1].second) == cudaSuccess)
        ms[marks[i].first] += t;
    }
  }
  ~PhaseTimer() {
    if (open) nvtxRangePop();
    for (auto& m : marks) cudaEventDestroy(m.second);
  }
};

// The parameters the setup runs with: the double-float products (SpMV and
// setup) need K's entries within 2^-kDfExpLimit..2^kDfExpLimit (FP32's
// exponent range, with room for the products), so outside it the automatic
// choices fall back to FP64 and the requests that need FP32 arithmetic are
// refused with the range in the message.
static amg_params effective_params(const tam_matrix_s* K, const amg_params& in) {
  amg_params p = in;
  // BF16 finest values weaken the smoother on P2 matrices enough to double the
  // iterations (measured on the P2 disc: 169 vs 77); such a request keeps FP32
  if (p.level_precision == 2 && K->nodes_per_cell == 10) p.level_precision = 1;
  TAM_CHECK(K->finite, TAM_ERR_INVALID_ARG, "amg_setup: K has an inf or NaN entry");
  TAM_CHECK(K->A.br == 3 || p.level_precision == 0, TAM_ERR_UNSUPPORTED,
            "amg_setup: the FP32 V-cycle (level_precision 1/2) is built for 3x3-block (elastic) operators only");
  if (K->df_ok) return p;
  const std::string why = "largest |K| entry is 2^" + std::to_string(K->vmax_exp) + "; FP32 arithmetic needs 2^-" +
                          std::to_string(kDfExpLimit) + "..2^" + std::to_string(kDfExpLimit);
  TAM_CHECK(p.spmv_fp64 != 2, TAM_ERR_INVALID_ARG, "amg_setup: spmv_fp64 = 2 (double-float SpMVs): " + why);
  TAM_CHECK(p.level_precision == 0, TAM_ERR_INVALID_ARG, "amg_setup: level_precision 1/2 (FP32 V-cycle): " + why);
  if (p.spmv_fp64 == 0) p.spmv_fp64 = 1;
  p.setup_fp64 = 1;
  return p;
}

tam_amg_s* amg_build(tam_matrix_s* K, const double* coords, const amg_params& prm_in, cudaStream_t s) {
  NvtxRange nvtx("tam: AMG setup");
  const amg_params prm = effective_params(K, prm_in);
  TAM_CHECK(prm.level_precision >= 0 && prm.level_precision <= 2, TAM_ERR_INVALID_ARG,
            "amg_setup: level_precision must be 0 (FP64), 1 (FP32) or 2 (FP32, BF16 finest values)");
  TAM_CHECK(prm.smoother_degree >= 1 && prm.smoother_degree <= 8 && prm.eig_iters >= 1 && prm.eig_iters <= 64 &&
                prm.max_levels >= 1 && prm.max_levels <= 20 && prm.coarse_max_dofs >= 1 && prm.coarse_min_dofs >= 0 && prm.aggressive_levels >= 0 &&
                prm.small_level_dofs >= 0 && prm.small_level_degree >= 1 && prm.small_level_degree <= 32 &&
                prm.cheb_hi > prm.cheb_lo && prm.cheb_lo > 0 && prm.strength_theta >= 0 &&
                prm.strength_theta_scale >= 0 && (prm.setup_fp64 == 0 || prm.setup_fp64 == 1) &&
                prm.spmv_fp64 >= 0 && prm.spmv_fp64 <= 2,
            TAM_ERR_INVALID_ARG, "amg_setup: parameter out of range");
  auto H = new tam_amg_s();
  PhaseTimer T;
  try {
    H->K = K;
    H->prm = prm;
    const int n0 = K->n_nodes;
    H->max_grid = 8 * 1024;
    {
      unsigned g0 = sell_grid(K->S);
      H->max_grid = std::max<int>(65536, (int)g0);  // covers every reducing SpMV launch of the hierarchy
    }
    H->partials = DBuf<double>((size_t)H->max_grid * 4, s);
    H->ticket = DBuf<unsigned int>(1, s);
    H->ticket.zero();
    GridReduce gr{H->partials.p, H->ticket.p};
    // near-nullspace: the rigid-body modes of elasticity (3x3 blocks), the
    // constant for a scalar operator (1x1 blocks: the heat equation)
    const bool scalar = K->A.br == 1;
    const int k = scalar ? 1 : (prm.use_rotations ? 6 : 3);
    // near-nullspace of the finest level
    DBuf<double> cen(3, s);
    centroid_kernel<<<std::min<unsigned>(grid_for(n0, TPB), 1024), TPB, 0, s>>>(coords, n0, gr, cen.p);
    TAM_LAUNCH_CHECK();
    DBuf<double> B((size_t)n0 * 3 * k, s);
    if (scalar)
      constant_mode_kernel<<<grid_for(n0, TPB), TPB, 0, s>>>(K->dmask.p, n0, B.p);
    else
      rigid_modes_kernel<<<grid_for(n0, TPB), TPB, 0, s>>>(coords, K->dmask.p, n0, cen.p, k, B.p);
    TAM_LAUNCH_CHECK();
    H->levels.reserve(prm.max_levels);  // references into `levels` stay valid while it grows
    H->levels.emplace_back();
    H->levels[0].A = &K->A;
    H->levels[0].AS = &K->S;
    {
      // K's split copies exist for its SELL form and, when its own operator
      // runs on the block-CSR arrays, for those (see fem_assemble_elasticity)
      const bool df0 = use_df(K->A, prm.spmv_fp64);
      Level& L0 = H->levels[0];
      L0.Aop = SpOp{&K->A, &K->S, choose_lpr(K->A), df0};
      if (lpr_store_pays(L0.Aop.lpr)) {
        build_lpr_store(K->A, L0.Aop.lpr, df0, L0.AL, s);
        L0.Aop.L = &L0.AL;
      }
    }
    // the Lanczos estimates' own grid-reduce scratch (they run on the side
    // stream, concurrently with reductions on s), then the side stream itself
    DBuf<double> lz_partials((size_t)H->max_grid * 4, s);
    DBuf<unsigned int> lz_ticket(1, s);
    lz_ticket.zero();
    SideStream side;
    for (int lev = 0;; ++lev) {
      Level& L = H->levels[lev];
      L.n_rows = L.A->n_rows;
      L.bs = L.A->br;
      L.kdim = k;
      L.deg = (long long)L.n_rows * L.bs <= prm.small_level_dofs ? prm.small_level_degree : prm.smoother_degree;
      L.dinv = DBuf<double>((size_t)L.n_rows * L.bs, s);
      T.mark(0, s);
      point_dinv_kernel<<<grid_for(L.n_rows, TPB), TPB, 0, s>>>(L.A->row_ptr.p, L.A->col_idx.p, L.A->vals.p, L.n_rows,
                                                                L.bs, L.dinv.p);
      TAM_LAUNCH_CHECK();
      L.consts = DBuf<double>(2 + 2 * (size_t)std::max(L.deg, 1), s);
      side.fork(s);
      lanczos_lambda(H, L, lev, side.s2, GridReduce{lz_partials.p, lz_ticket.p});
      side.done();
      alloc_level_vectors(L, s);
      const bool last = (long long)L.n_rows * L.bs <= prm.coarse_max_dofs || lev == prm.max_levels - 1;
      if (!last) {
        T.mark(1, s);
        // distance-2 (aggressive) roots on the first aggressive_levels levels,
        // distance-1 below; an aggressive aggregation that would leave too
        // small a coarse grid is redone with distance-1 roots
        const bool aggressive = lev < prm.aggressive_levels;
        const double theta = prm.strength_theta * std::pow(prm.strength_theta_scale, (double)lev);
        L.n_agg = aggregate(L, lev, theta, aggressive ? 2 : 1, s);
        if (aggressive && prm.coarse_min_dofs > 0 && (long long)L.n_agg * k < prm.coarse_min_dofs)
          L.n_agg = aggregate(L, lev, theta, 1, s);
      }
      if (last || L.n_agg == 0 || L.n_agg >= L.n_rows) {
        L.n_agg = 0;
        L.agg.reset();
        T.mark(0, s);
        side.join(s);  // before the cooperative launch of the coarse inverse
        T.mark(7, s);
        coarse_inverse(H, L, s);
        break;
      }
      DBuf<double> Bc;
      T.mark(2, s);
      tentative(L, B.p, 1e-10, Bc, s);
      // P = (I - omega D^-1 A) P_tent, computed on the pattern of A P_tent
      T.mark(3, s);
      const SpgemmArith arith = prm.setup_fp64 ? SpgemmArith::kFp64 : SpgemmArith::kDoubleFloat;
      // double-float: A is split once for both of its products, and A P stays
      // split (its only use is R (A P))
      DBuf<float2> As;
      if (arith == SpgemmArith::kDoubleFloat) As = split_values(*L.A, s);
      SpgemmSplit spA;
      spA.x = As.p;
      if (!bsr_spgemm_tentative(*L.A, L.Pt, L.agg.p, L.P, s, arith, As.p)) bsr_spgemm(*L.A, L.Pt, L.P, s, arith, spA);
      T.mark(0, s);  // waiting for lambda_max counts as its phase
      side.join(s);
      T.mark(3, s);
      {
        const unsigned g = grid_for((long long)L.n_rows * 32, TPB);
        auto launch = [&](auto kern) {
          kern<<<g, TPB, 0, s>>>(L.P.row_ptr.p, L.P.col_idx.p, L.P.vals.p, L.n_rows, L.dinv.p, L.consts.p, L.agg.p,
                                 L.Pt.row_ptr.p, L.Pt.vals.p);
        };
        if (L.bs == 3 && k == 6) launch(smooth_prolongator_kernel<3, 6>);
        else if (L.bs == 6 && k == 6) launch(smooth_prolongator_kernel<6, 6>);
        else if (L.bs == 1 && k == 1) launch(smooth_prolongator_kernel<1, 1>);
        else if (L.bs == 3 && k == 3) launch(smooth_prolongator_kernel<3, 3>);
        else throw Error(TAM_ERR_UNSUPPORTED, "amg_setup: prolongator block shape not instantiated");
        TAM_LAUNCH_CHECK();
      }
      T.mark(4, s);
      bsr_transpose(L.P, L.R, s);
      {
        Bsr AP;
        DBuf<float2> APs;
        T.mark(5, s);
        SpgemmSplit spAP;
        spAP.x = As.p;
        if (arith == SpgemmArith::kDoubleFloat) spAP.c = &APs;
        bsr_spgemm(*L.A, L.P, AP, s, arith, spAP);
        H->levels.emplace_back();
        Level& C = H->levels[lev + 1];
        SpgemmSplit spR;
        spR.y = APs.p;
        spR.symmetric = true;  // R = P^T and A symmetric
        bsr_spgemm(L.R, AP, C.A_own, s, arith, spR);
        C.A = &C.A_own;
        C.AS = &C.AS_own;
        plan_spop(C.Aop, C.A_own, C.AS_own, C.AL, prm.spmv_fp64, s);
      }
      T.mark(6, s);
      plan_spop(L.Pop, L.P, L.PS, L.PL, prm.spmv_fp64, s);
      plan_spop(L.Rop, L.R, L.RS, L.RL, prm.spmv_fp64, s);
      B = std::move(Bc);
    }
    H->r = DBuf<double>((size_t)n0 * 3, s);
    H->z = DBuf<double>((size_t)n0 * 3, s);
    H->p = DBuf<double>((size_t)n0 * 3, s);
    H->q = DBuf<double>((size_t)n0 * 3, s);
    H->sc = DBuf<PcgScalars>(1, s);
    if (prm.level_precision > 0) {
      T.mark(6, s);
      build_low_precision(H, s);
    }
    T.mark(-1, s);
    side.join(s);
    TAM_CUDA(cudaStreamSynchronize(s));
    T.finish(H->setup_ms);
    for (Level& L : H->levels) {
      L.lambda_host = read_back_double(L.consts.p, s);
      TAM_CHECK(std::isfinite(L.lambda_host) && L.lambda_host > 0.0, TAM_ERR_INTERNAL,
                "amg_setup: lambda_max estimate is not positive");
    }
  } catch (...) {
    delete H;
    throw;
  }
  return H;
}

// After K's values changed in place (same pattern): the finest level's
// diagonal, its lanes-per-row store or split copy, so that a hierarchy built
// on earlier values can keep preconditioning the new K (its coarse levels and
// the lambda_max estimate stay as they were).  The captured PCG iteration is
// dropped, since the store's buffers are new.
void amg_refresh_finest(tam_amg_s* H, cudaStream_t s) {
  Level& L = H->levels[0];
  const Bsr& A = H->K->A;
  point_dinv_kernel<<<grid_for(L.n_rows, TPB), TPB, 0, s>>>(A.row_ptr.p, A.col_idx.p, A.vals.p, L.n_rows, L.bs,
                                                            L.dinv.p);
  TAM_LAUNCH_CHECK();
  // the iteration graph reads the level's arrays through their pointers: it
  // stays valid unless a layout is rebuilt in new memory (the lanes-per-row
  // store); the SELL values (refreshed in place by the caller), D^-1 and the
  // block-CSR split copy (same size, same buffer) keep theirs
  bool moved = false;
  if (L.Aop.L) {
    build_lpr_store(A, L.Aop.L->lpr, L.Aop.df, L.AL, s);
    moved = true;
  } else if (L.Aop.lpr != 0 && L.Aop.df) {
    const float2* before = H->K->A.vals_df.p;
    build_df_values(H->K->A, s);
    moved = H->K->A.vals_df.p != before;
  }
  if (moved && H->iter_exec) {
    cudaGraphExecDestroy(H->iter_exec);
    H->iter_exec = nullptr;
  }
  H->multi.reset();  // its FP32 copies and batch graph belong to the old operator
}

}  // namespace tam
