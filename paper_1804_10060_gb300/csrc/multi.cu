// Many load cases at once: block of independent preconditioned CGs whose
// SpMVs are multi-vector products (SpMM), plus a multi-system driver that
// advances several meshes in one CUDA-graph launch per iteration.
//
// Each RHS keeps its own CG scalars and stopping test (a converged RHS is
// frozen while the others continue).  The outer SpMM with K has FP64 vectors
// and double-float products (K's split values); the
// V-cycle runs in FP32 (BF16 finest values when the hierarchy was built with
// level_precision 2) with one matrix read serving `tm` right-hand sides per
// thread -- the V-cycle is bandwidth-bound in FP32, so reading the matrix
// once for several load cases is where the batch gains.  `tm` (the RHS tile
// per thread) is chosen per operator by timing the candidates once per
// hierarchy and RHS count (the autotuner below).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>

#include "handles.cuh"

namespace tam {
namespace {

constexpr int TPB = 256;
constexpr int TMAX = 8;    // RHS per thread, compile-time register tile
constexpr int MPMAX = 16;  // RHS per system
constexpr int MT_MIN_THREADS = 64, MT_MAX_THREADS = 256;  // CTA sizes the autotuner tries
enum { S_RHO = 0, S_ALPHA, S_BETA, S_RR, S_TOL2, S_BB, S_DONE, S_ITER, S_SCALE, S_COUNT };

// 2^e for |e| <= 1000, built from its bits (exact)
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

unsigned vgrid(long long n) { return stride_grid(n, TPB, 8); }

// -------------------------------------------------------------------------
// layout conversion
// -------------------------------------------------------------------------
__global__ void interleave_kernel(const double* __restrict__ src, double* __restrict__ dst, int m, int mp, long long n3) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n3 * mp; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / mp;
    const int j = (int)(e % mp);
    dst[e] = j < m ? src[(size_t)j * n3 + i] : 0.0;
  }
}

// back to one vector per RHS, undoing each RHS's power-of-two scaling
__global__ void deinterleave_kernel(const double* __restrict__ src, double* __restrict__ dst, int m, int mp,
                                    long long n3, const double* __restrict__ sc) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n3 * m; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / n3);
    const long long i = e % n3;
    dst[e] = src[i * mp + j] * pow2((int)sc[S_SCALE * mp + j]);
  }
}

// b and x of every RHS into the solve's scaling (b 2^-e_j, x 2^-e_j; see mstart_kernel)
__global__ void mscale_in_kernel(double* __restrict__ b, double* __restrict__ x, long long n3, int mp,
                                 const double* __restrict__ sc) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n3 * mp; e += (long long)gridDim.x * blockDim.x) {
    const double f = pow2(-(int)sc[S_SCALE * mp + (int)(e % mp)]);
    b[e] *= f;
    x[e] *= f;
  }
}

// -------------------------------------------------------------------------
// per-RHS reductions: every thread holds up to MPMAX partial sums
// -------------------------------------------------------------------------
__device__ bool reduce_rhs(GridReduce gr, double (&v)[MPMAX], double (&tot)[MPMAX], double* sh) {
  return grid_reduce<MPMAX>(gr, v, tot, sh);
}

// Per RHS: ||b||^2, and the power of two e_j the solve divides b_j and x_j by
// (b_j's RMS entry moved to about 2^half_exp, half K's largest entry exponent,
// so that every vector the double-float and FP32 products see stays far inside
// FP32's exponent range; exact, see pcg_solve); tolerances in scaled units.
__global__ void mstart_kernel(const double* __restrict__ b, long long n3, int m, int mp, double rtol, double atol,
                              int max_iter, int half_exp, GridReduce gr, double* __restrict__ sc,
                              int* __restrict__ flags) {
  __shared__ double sh[32];
  double acc[MPMAX];
#pragma unroll
  for (int j = 0; j < MPMAX; ++j) acc[j] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int j = 0; j < MPMAX; ++j)
      if (j < mp) {
        const double v = b[i * mp + j];
        acc[j] += v * v;
      }
  double tot[MPMAX];
  if (reduce_rhs(gr, acc, tot, sh) && threadIdx.x == 0) {
    for (int j = 0; j < mp; ++j) {
      int e = 0;
      if (tot[j] > 0.0 && isfinite(tot[j])) {
        e = ilogb(sqrt(tot[j] / (double)n3)) - half_exp;
        e = e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
      }
      const double inv = pow2(-e);
      sc[S_SCALE * mp + j] = (double)e;
      sc[S_BB * mp + j] = tot[j] * inv * inv;
      const double t = fmax(rtol * sqrt(tot[j]), atol) * inv;
      sc[S_TOL2 * mp + j] = t * t;
      sc[S_DONE * mp + j] = j < m ? 0.0 : 1.0;
      sc[S_ITER * mp + j] = 0.0;
      sc[S_RHO * mp + j] = sc[S_ALPHA * mp + j] = sc[S_BETA * mp + j] = 0.0;
    }
    flags[0] = 0;
    flags[1] = 0;
    flags[2] = max_iter;
    flags[3] = TAM_OK;
  }
}

// stop when every RHS is done or the iteration cap is reached
__global__ void mcheck_kernel(const double* __restrict__ sc, int mp, int* __restrict__ flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool all = true;
  for (int j = 0; j < mp; ++j) all = all && sc[S_DONE * mp + j] != 0.0;
  if (all || flags[1] >= flags[2] || flags[3] != TAM_OK) flags[0] = 1;
}

__global__ void mupdate_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                               const double* __restrict__ q, long long n3, int mp, GridReduce gr,
                               double* __restrict__ sc, int* __restrict__ flags) {
  __shared__ double sh[32];
  if (flags[0]) return;
  double acc[MPMAX];
#pragma unroll
  for (int j = 0; j < MPMAX; ++j) acc[j] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int j = 0; j < MPMAX; ++j)
      if (j < mp && sc[S_DONE * mp + j] == 0.0) {
        const double a = sc[S_ALPHA * mp + j];
        const long long k = i * mp + j;
        x[k] += a * p[k];
        const double rk = r[k] - a * q[k];
        r[k] = rk;
        acc[j] += rk * rk;
      }
  double tot[MPMAX];
  if (reduce_rhs(gr, acc, tot, sh) && threadIdx.x == 0) {
    bool all = true;
    for (int j = 0; j < mp; ++j) {
      if (sc[S_DONE * mp + j] == 0.0) {
        sc[S_RR * mp + j] = tot[j];
        sc[S_ITER * mp + j] += 1.0;
        if (!isfinite(tot[j])) flags[3] = TAM_ERR_NAN;
        else if (tot[j] <= sc[S_TOL2 * mp + j]) sc[S_DONE * mp + j] = 1.0;
      }
      all = all && sc[S_DONE * mp + j] != 0.0;
    }
    flags[1] += 1;
    if (all || flags[1] >= flags[2] || flags[3] != TAM_OK) flags[0] = 1;
  }
}

__global__ void mrz_kernel(const double* __restrict__ r, const double* __restrict__ z, double* __restrict__ p,
                           long long n3, int mp, int first, GridReduce gr, double* __restrict__ sc,
                           int* __restrict__ flags) {
  __shared__ double sh[32];
  if (flags[0]) return;
  double acc[MPMAX];
#pragma unroll
  for (int j = 0; j < MPMAX; ++j) acc[j] = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
#pragma unroll
    for (int j = 0; j < MPMAX; ++j)
      if (j < mp) {
        const long long k = i * mp + j;
        acc[j] += r[k] * z[k];
        if (first) p[k] = z[k];
      }
  double tot[MPMAX];
  if (reduce_rhs(gr, acc, tot, sh) && threadIdx.x == 0) {
    for (int j = 0; j < mp; ++j) {
      if (sc[S_DONE * mp + j] != 0.0) continue;
      const double rz = tot[j];
      if (!isfinite(rz)) { flags[3] = TAM_ERR_NAN; continue; }
      if (!(rz > 0.0)) { flags[3] = TAM_ERR_INDEFINITE_PRECOND; continue; }
      if (!first) sc[S_BETA * mp + j] = rz / sc[S_RHO * mp + j];
      sc[S_RHO * mp + j] = rz;
    }
    if (flags[3] != TAM_OK) flags[0] = 1;
  }
}

__global__ void mdir_kernel(const double* __restrict__ z, double* __restrict__ p, long long n3, int mp,
                            const double* __restrict__ sc, const int* __restrict__ flags) {
  if (flags[0]) return;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n3 * mp; e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % mp);
    if (sc[S_DONE * mp + j] == 0.0) p[e] = z[e] + sc[S_BETA * mp + j] * p[e];
  }
}

// -------------------------------------------------------------------------
// SpMM with K (SELL-32, thread per row, RHS chunk per blockIdx.y)
// -------------------------------------------------------------------------
// DF: double-float products on K's split values (each value feeds tm
// right-hand sides, so the FP64 version is far past GB300's FP64 rate).
template <class Epi, bool DF>
__global__ void __launch_bounds__(MT_MAX_THREADS)
kspmm_kernel(SellView A, const double* __restrict__ x, int mp, int tm, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  const int slice = pos >> 5, lane = pos & 31;
  const int row = sell_row(A.perm, pos, A.n_rows);
  const int j0 = blockIdx.y * tm;
  double acc[3][TMAX];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < TMAX; ++k) acc[r][k] = 0.0;
  if constexpr (DF) {
    if (slice < A.n_slices) {
      float2 ad[3][TMAX];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < TMAX; ++k) ad[r][k] = make_float2(0.f, 0.f);
      const int k0 = A.slice_ptr[slice], k1 = A.slice_ptr[slice + 1];
      for (int s = k0; s < k1; ++s) {
        const int c = __ldg(A.cols + (size_t)s * 32 + lane);
        const float2* __restrict__ vp = A.vals_df + (size_t)s * 32 * 9 + lane;
        float2 v[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) v[e] = __ldg(vp + e * 32);
#pragma unroll
        for (int jc = 0; jc < 3; ++jc) {
          const double* xr = x + ((size_t)c * 3 + jc) * mp + j0;
#pragma unroll
          for (int k = 0; k < TMAX; ++k)
            if (k < tm) {
              const float2 xv = split_bits(__ldg(xr + k));
#pragma unroll
              for (int r = 0; r < 3; ++r) df_fma(ad[r][k], v[r * 3 + jc], xv);
            }
        }
      }
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < TMAX; ++k) acc[r][k] = df_to_double(ad[r][k]);
    }
    epi(row, j0, tm, acc, sh);
    return;
  }
  if (slice < A.n_slices) {
    const int k0 = A.slice_ptr[slice], k1 = A.slice_ptr[slice + 1];
    for (int s = k0; s < k1; ++s) {
      const int c = __ldg(A.cols + (size_t)s * 32 + lane);
      const double* __restrict__ vp = A.vals + (size_t)s * 32 * 9 + lane;
      double v[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) v[e] = __ldg(vp + e * 32);
#pragma unroll
      for (int jc = 0; jc < 3; ++jc) {
        const double* xr = x + ((size_t)c * 3 + jc) * mp + j0;
#pragma unroll
        for (int k = 0; k < TMAX; ++k)
          if (k < tm) {
            const double xv = __ldg(xr + k);
#pragma unroll
            for (int r = 0; r < 3; ++r) acc[r][k] = fma(v[r * 3 + jc], xv, acc[r][k]);
          }
      }
    }
  }
  epi(row, j0, tm, acc, sh);
}

// q = K p, per-RHS p.q -> alpha
struct EpiPqM {
  const double* p;
  double* q;
  int n_rows, mp;
  GridReduce gr;  // partials/tickets indexed by chunk (blockIdx.y)
  double* sc;
  int* flags;
  __device__ bool skip() const { return flags[0]; }
  __device__ void operator()(int row, int j0, int tm, const double (&acc)[3][TMAX], double* sh) const {
    double s[TMAX];
#pragma unroll
    for (int k = 0; k < TMAX; ++k) s[k] = 0.0;
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < TMAX; ++k)
          if (k < tm) {
            const size_t i = ((size_t)row * 3 + r) * mp + j0 + k;
            q[i] = acc[r][k];
            s[k] += p[i] * acc[r][k];
          }
    GridReduce g{gr.partials + (size_t)blockIdx.y * gridDim.x * TMAX, gr.ticket + blockIdx.y};
    double tot[TMAX];
    if (grid_reduce<TMAX>(g, s, tot, sh) && threadIdx.x == 0) {
      for (int k = 0; k < tm; ++k) {
        const int j = j0 + k;
        if (sc[S_DONE * mp + j] != 0.0) { sc[S_ALPHA * mp + j] = 0.0; continue; }
        const double pq = tot[k];
        if (!isfinite(pq)) { flags[3] = TAM_ERR_NAN; continue; }
        if (!(pq > 0.0)) { flags[3] = TAM_ERR_BREAKDOWN; continue; }
        sc[S_ALPHA * mp + j] = sc[S_RHO * mp + j] / pq;
      }
    }
  }
};

// r = b - K x and ||r||^2 per RHS (initial residual; marks converged RHS)
struct EpiResInitM {
  const double* b;
  double* r;
  int n_rows, mp;
  GridReduce gr;
  double* sc;
  double* out;  // if non-null: store ||b - Kx||^2 here instead (final residual)
  int* flags;
  __device__ bool skip() const { return false; }
  __device__ void operator()(int row, int j0, int tm, const double (&acc)[3][TMAX], double* sh) const {
    double s[TMAX];
#pragma unroll
    for (int k = 0; k < TMAX; ++k) s[k] = 0.0;
    if (row < n_rows)
#pragma unroll
      for (int rr = 0; rr < 3; ++rr)
#pragma unroll
        for (int k = 0; k < TMAX; ++k)
          if (k < tm) {
            const size_t i = ((size_t)row * 3 + rr) * mp + j0 + k;
            const double v = b[i] - acc[rr][k];
            if (r) r[i] = v;
            s[k] += v * v;
          }
    GridReduce g{gr.partials + (size_t)blockIdx.y * gridDim.x * TMAX, gr.ticket + blockIdx.y};
    double tot[TMAX];
    if (grid_reduce<TMAX>(g, s, tot, sh) && threadIdx.x == 0) {
      for (int k = 0; k < tm; ++k) {
        const int j = j0 + k;
        if (out) { out[j] = tot[k]; continue; }
        sc[S_RR * mp + j] = tot[k];
        if (!isfinite(tot[k])) flags[3] = TAM_ERR_NAN;
        else if (tot[k] <= sc[S_TOL2 * mp + j]) sc[S_DONE * mp + j] = 1.0;
      }
    }
  }
};

struct EpiStoreKM {
  double* y;
  int n_rows, mp;
  __device__ bool skip() const { return false; }
  __device__ void operator()(int row, int j0, int tm, const double (&acc)[3][TMAX], double*) const {
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < TMAX; ++k)
          if (k < tm) y[((size_t)row * 3 + r) * mp + j0 + k] = acc[r][k];
  }
};

// df: the double-float kernel on K's split values (the hierarchy's level-0
// choice, amg_params.spmv_fp64); false: plain FP64.
template <class Epi>
void kspmm(const Sell& S, const double* x, int mp, const MTile& t, Epi epi, cudaStream_t s, bool df) {
  dim3 g(grid_for((long long)S.n_slices * 32, t.threads), mp / t.tm);
  if (df && S.vals_df.p)
    kspmm_kernel<Epi, true><<<g, t.threads, 0, s>>>(view(S), x, mp, t.tm, epi);
  else
    kspmm_kernel<Epi, false><<<g, t.threads, 0, s>>>(view(S), x, mp, t.tm, epi);
  TAM_LAUNCH_CHECK();
}

// -------------------------------------------------------------------------
// FP32 multi-vector SpMM for the V-cycle (SELL or lanes-per-row layouts)
// -------------------------------------------------------------------------
template <int BR, int BC, typename TV, class Epi>
__global__ void __launch_bounds__(MT_MAX_THREADS)
msell_kernel(int n_slices, const int* __restrict__ slice_ptr, const int* __restrict__ cols, const TV* __restrict__ vals,
             const float* __restrict__ x, int mp, int tm, const int* __restrict__ perm, Epi epi) {
  if (epi.skip()) return;
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  const int slice = pos >> 5, lane = pos & 31;
  const int row = sell_row(perm, pos, epi.n_rows);
  const int j0 = blockIdx.y * tm;
  float acc[BR][TMAX];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int k = 0; k < TMAX; ++k) acc[r][k] = 0.f;
  if (slice < n_slices) {
    const int k0 = slice_ptr[slice], k1 = slice_ptr[slice + 1];
    for (int s = k0; s < k1; ++s) {
      const TV* __restrict__ vp = vals + (size_t)s * 32 * BR * BC + lane;
      TV vv[BR * BC];  // the slot's values first, then the gathers
#pragma unroll
      for (int e = 0; e < BR * BC; ++e) vv[e] = vp[e * 32];
      const int c = __ldg(cols + (size_t)s * 32 + lane);
#pragma unroll
      for (int jc = 0; jc < BC; ++jc) {
        const float* xr = x + ((size_t)c * BC + jc) * mp + j0;
        float xv[TMAX];
#pragma unroll
        for (int k = 0; k < TMAX; ++k) xv[k] = k < tm ? __ldg(xr + k) : 0.f;
#pragma unroll
        for (int r = 0; r < BR; ++r) {
          const float a = to_f32(vv[r * BC + jc]);
#pragma unroll
          for (int k = 0; k < TMAX; ++k) acc[r][k] = fmaf(a, xv[k], acc[r][k]);
        }
      }
    }
  }
  if (row < epi.n_rows) epi(row, j0, tm, acc);
}

template <int BR, int BC, typename TV, class Epi>
__global__ void __launch_bounds__(MT_MAX_THREADS)
mvec_kernel(int n_rows, const int* __restrict__ rp, const int* __restrict__ ci, const TV* __restrict__ v,
            const float* __restrict__ x, int mp, int tm, int lpr_log2, Epi epi) {
  if (epi.skip()) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int lpr = 1 << lpr_log2;
  const int row = t >> lpr_log2, sub = t & (lpr - 1);
  const int j0 = blockIdx.y * tm;
  float acc[BR][TMAX];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int k = 0; k < TMAX; ++k) acc[r][k] = 0.f;
  if (row < n_rows) {
    const int pe = rp[row + 1];
    for (int p = rp[row] + sub; p < pe; p += lpr) {
      const TV* __restrict__ vb = v + (size_t)p * BR * BC;
      TV vv[BR * BC];  // the block's values first, then the gathers
#pragma unroll
      for (int e = 0; e < BR * BC; ++e) vv[e] = vb[e];
      const int c = ci[p];
#pragma unroll
      for (int jc = 0; jc < BC; ++jc) {
        const float* xr = x + ((size_t)c * BC + jc) * mp + j0;
        float xv[TMAX];
#pragma unroll
        for (int k = 0; k < TMAX; ++k) xv[k] = k < tm ? __ldg(xr + k) : 0.f;
#pragma unroll
        for (int r = 0; r < BR; ++r) {
          const float a = to_f32(vv[r * BC + jc]);
#pragma unroll
          for (int k = 0; k < TMAX; ++k) acc[r][k] = fmaf(a, xv[k], acc[r][k]);
        }
      }
    }
  }
  for (int o = lpr >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int k = 0; k < TMAX; ++k) acc[r][k] += __shfl_xor_sync(0xffffffffu, acc[r][k], o);
  if (sub == 0 && row < n_rows) epi(row, j0, tm, acc);
}

template <int BR, typename TB, typename TO>
struct EpiChebMF {
  const TB* b;
  const float* x;
  const float* dinv;
  const float* coef;
  float* d;
  TO* xn;
  int n_rows, mp;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, int j0, int tm, const float (&acc)[BR][TMAX]) const {
    const float cd = coef[0], cr = coef[1];
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      const float dr = dinv[(size_t)row * BR + r];
#pragma unroll
      for (int k = 0; k < TMAX; ++k)
        if (k < tm) {
          const size_t i = ((size_t)row * BR + r) * mp + j0 + k;
          const float res = dr * ((float)b[i] - acc[r][k]);
          const float di = cd != 0.f ? cd * d[i] + cr * res : cr * res;
          d[i] = di;
          xn[i] = (TO)(x[i] + di);
        }
    }
  }
};

template <int BR, typename TB>
struct EpiResMF {
  const TB* b;
  float* t;
  int n_rows, mp;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, int j0, int tm, const float (&acc)[BR][TMAX]) const {
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int k = 0; k < TMAX; ++k)
        if (k < tm) {
          const size_t i = ((size_t)row * BR + r) * mp + j0 + k;
          t[i] = (float)b[i] - acc[r][k];
        }
  }
};

template <int BR, bool ADD>
struct EpiPutMF {
  float* y;
  int n_rows, mp;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, int j0, int tm, const float (&acc)[BR][TMAX]) const {
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int k = 0; k < TMAX; ++k)
        if (k < tm) {
          const size_t i = ((size_t)row * BR + r) * mp + j0 + k;
          y[i] = ADD ? y[i] + acc[r][k] : acc[r][k];
        }
  }
};

template <int BR, int BC, typename TV, class Epi>
void mspmm(const SpOpLow<TV>& o, const float* x, int mp, const MTile& t, Epi epi, cudaStream_t s) {
  const SpOp& op = o.op;
  if (op.lpr == 0) {
    const Sell& S = *op.S;
    dim3 g(grid_for((long long)S.n_slices * 32, t.threads), mp / t.tm);
    msell_kernel<BR, BC, TV, Epi><<<g, t.threads, 0, s>>>(S.n_slices, S.slice_ptr.p, S.cols.p, o.vals, x, mp, t.tm,
                                                          S.perm.p, epi);
  } else {
    const Bsr& B = *op.B;
    const int lpr = t.lpr ? t.lpr : op.lpr;
    int lg = 0;
    while ((1 << lg) < lpr) ++lg;
    dim3 g(grid_for((long long)B.n_rows << lg, t.threads), mp / t.tm);
    mvec_kernel<BR, BC, TV, Epi><<<g, t.threads, 0, s>>>(B.n_rows, B.row_ptr.p, B.col_idx.p, o.vals, x, mp, t.tm, lg,
                                                         epi);
  }
  TAM_LAUNCH_CHECK();
}

template <typename TB>
__global__ void mfirst_kernel(const TB* __restrict__ b, const float* __restrict__ dinv, const float* __restrict__ consts,
                              float* __restrict__ d, float* __restrict__ x, long long N, int mp,
                              const int* __restrict__ stop) {
  if (stop && *stop) return;
  const float cr = consts[3];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N * mp; e += (long long)gridDim.x * blockDim.x) {
    const float di = cr * dinv[e / mp] * (float)b[e];
    d[e] = di;
    x[e] = di;
  }
}

template <typename TI, typename TO>
__global__ void mcoarse_kernel(const double* __restrict__ A, const TI* __restrict__ b, TO* __restrict__ y, int N, int mp,
                               const int* __restrict__ stop) {
  if (stop && *stop) return;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N * mp) return;
  const int i = (int)(t / mp), k = (int)(t % mp);
  const double* a = A + (size_t)i * N;
  double s = 0.0;
  for (int j = 0; j < N; ++j) s = fma(a[j], (double)b[(size_t)j * mp + k], s);
  y[t] = (TO)s;
}

// A x on a level with its FP32 / BF16 values
template <int BS, class Epi>
void level_mspmm(const Level& L, const float* x, int mp, const MTile& t, Epi epi, cudaStream_t s) {
  if (L.A16.vals) mspmm<BS, BS, __nv_bfloat16>(L.A16, x, mp, t, epi, s);
  else mspmm<BS, BS, float>(L.A32, x, mp, t, epi, s);
}

template <typename TB, typename TO>
void mcheb(const Level& L, const MultiLevel& ML, const TB* b, const float* x, TO* xn, int step, int mp,
           const int* stop, cudaStream_t s) {
  const float* coef = L.consts32.p + 2 + 2 * step;
  if (L.bs == 3)
    level_mspmm<3>(L, x, mp, ML.tA, EpiChebMF<3, TB, TO>{b, x, L.dinv32.p, coef, ML.d.p, xn, L.n_rows, mp, stop}, s);
  else
    level_mspmm<6>(L, x, mp, ML.tA, EpiChebMF<6, TB, TO>{b, x, L.dinv32.p, coef, ML.d.p, xn, L.n_rows, mp, stop}, s);
}

template <typename TB>
void mresidual(const Level& L, const MultiLevel& ML, const TB* b, const float* x, int mp, const int* stop,
               cudaStream_t s) {
  if (L.bs == 3) level_mspmm<3>(L, x, mp, ML.tA, EpiResMF<3, TB>{b, ML.t.p, L.n_rows, mp, stop}, s);
  else level_mspmm<6>(L, x, mp, ML.tA, EpiResMF<6, TB>{b, ML.t.p, L.n_rows, mp, stop}, s);
}

void mrestrict(const Level& L, const MultiLevel& ML, float* bc, int mp, const int* stop, cudaStream_t s) {
  const int nr = L.R.n_rows;
  if (L.kdim == 6 && L.bs == 3) mspmm<6, 3, float>(L.R32, ML.t.p, mp, ML.tR, EpiPutMF<6, false>{bc, nr, mp, stop}, s);
  else if (L.kdim == 6) mspmm<6, 6, float>(L.R32, ML.t.p, mp, ML.tR, EpiPutMF<6, false>{bc, nr, mp, stop}, s);
  else mspmm<3, 3, float>(L.R32, ML.t.p, mp, ML.tR, EpiPutMF<3, false>{bc, nr, mp, stop}, s);
}

void mprolong(const Level& L, const MultiLevel& ML, const float* xc, float* x, int mp, const int* stop,
              cudaStream_t s) {
  const int nr = L.P.n_rows;
  if (L.kdim == 6 && L.bs == 3) mspmm<3, 6, float>(L.P32, xc, mp, ML.tP, EpiPutMF<3, true>{x, nr, mp, stop}, s);
  else if (L.kdim == 6) mspmm<6, 6, float>(L.P32, xc, mp, ML.tP, EpiPutMF<6, true>{x, nr, mp, stop}, s);
  else mspmm<3, 3, float>(L.P32, xc, mp, ML.tP, EpiPutMF<3, true>{x, nr, mp, stop}, s);
}

template <typename TB, typename TO>
void mvcycle(tam_amg_s* H, int l, const TB* b, TO* out, const int* stop, cudaStream_t s) {
  MultiState& MS = *H->multi;
  const int mp = MS.mp;
  Level& L = H->levels[l];
  MultiLevel& ML = MS.lv[l];
  if (l == (int)H->levels.size() - 1) {
    mcoarse_kernel<TB, TO><<<grid_for((long long)H->n_coarse * mp, TPB), TPB, 0, s>>>(H->coarse_inv.p, b, out,
                                                                                      H->n_coarse, mp, stop);
    TAM_LAUNCH_CHECK();
    return;
  }
  const long long N = (long long)L.n_rows * L.bs;
  float* xa = ML.xa.p;
  float* xb = ML.xb.p;
  mfirst_kernel<TB><<<vgrid(N * mp), TPB, 0, s>>>(b, L.dinv32.p, L.consts32.p, ML.d.p, xa, N, mp, stop);
  TAM_LAUNCH_CHECK();
  for (int k = 1; k < L.deg; ++k) {
    mcheb<TB, float>(L, ML, b, xa, xb, k, mp, stop, s);
    std::swap(xa, xb);
  }
  mresidual<TB>(L, ML, b, xa, mp, stop, s);
  MultiLevel& MC = MS.lv[l + 1];
  mrestrict(L, ML, MC.b.p, mp, stop, s);
  mvcycle<float, float>(H, l + 1, MC.b.p, MC.y.p, stop, s);
  mprolong(L, ML, MC.y.p, xa, mp, stop, s);
  for (int k = 0; k < L.deg; ++k) {
    if (k == L.deg - 1) {
      mcheb<TB, TO>(L, ML, b, xa, out, k, mp, stop, s);
    } else {
      mcheb<TB, float>(L, ML, b, xa, xb, k, mp, stop, s);
      std::swap(xa, xb);
    }
  }
}

// ---------------------------------------------------------------------------
// Autotuner: RHS tile per thread for every operator, by timing
// ---------------------------------------------------------------------------
template <class F>
float time_ms(F&& launch, cudaStream_t s) {
  cudaEvent_t a, b;
  TAM_CUDA(cudaEventCreate(&a));
  TAM_CUDA(cudaEventCreate(&b));
  launch();  // warm
  TAM_CUDA(cudaEventRecord(a, s));
  for (int i = 0; i < 3; ++i) launch();
  TAM_CUDA(cudaEventRecord(b, s));
  TAM_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

// Coordinate search over the launch shape of one operator: RHS per thread
// (1, 2, 4, 8), then threads per CTA (64, 128, 256), then -- for the
// block-CSR layout -- lanes per block row (half, the planned, double), each
// candidate timed once (warm-up + 3 launches) with the others fixed.
template <class F>
MTile pick_tile(int mp, int planned_lpr, F&& run, cudaStream_t s) {
  MTile best;
  float best_ms = 1e30f;
  auto consider = [&](MTile t) {
    const float ms = time_ms([&] { run(t); }, s);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  };
  MTile t0;
  for (int tm : {1, 2, 4, 8}) {
    if (tm > mp || mp % tm) continue;
    MTile t = t0;
    t.tm = tm;
    consider(t);
  }
  const MTile after_tm = best;
  for (int th : {MT_MIN_THREADS, 128, MT_MAX_THREADS}) {
    if (th == after_tm.threads) continue;
    MTile t = after_tm;
    t.threads = th;
    consider(t);
  }
  if (planned_lpr > 0) {
    const MTile after_th = best;
    for (int l : {planned_lpr / 2, planned_lpr * 2}) {
      if (l < 1 || l > 32) continue;
      MTile t = after_th;
      t.lpr = l;
      consider(t);
    }
  }
  return best;
}

void autotune(tam_amg_s* H, cudaStream_t s) {
  MultiState& MS = *H->multi;
  const int mp = MS.mp;
  auto t0 = std::chrono::steady_clock::now();
  MS.tK = pick_tile(mp, 0, [&](const MTile& t) {
    kspmm(H->K->S, MS.p.p, mp, t, EpiStoreKM{MS.q.p, H->K->n_nodes, mp}, s, H->levels[0].Aop.df);
  }, s);
  for (size_t l = 0; l + 1 < H->levels.size(); ++l) {
    Level& L = H->levels[l];
    MultiLevel& ML = MS.lv[l];
    MultiLevel& MC = MS.lv[l + 1];
    ML.tA = pick_tile(mp, L.A32.op.lpr, [&](const MTile& t) {
      if (L.bs == 3) level_mspmm<3>(L, ML.xa.p, mp, t, EpiPutMF<3, false>{ML.t.p, L.n_rows, mp, nullptr}, s);
      else level_mspmm<6>(L, ML.xa.p, mp, t, EpiPutMF<6, false>{ML.t.p, L.n_rows, mp, nullptr}, s);
    }, s);
    ML.tR = pick_tile(mp, L.R32.op.lpr, [&](const MTile& t) {
      const int nr = L.R.n_rows;
      if (L.kdim == 6 && L.bs == 3) mspmm<6, 3, float>(L.R32, ML.t.p, mp, t, EpiPutMF<6, false>{MC.b.p, nr, mp, nullptr}, s);
      else if (L.kdim == 6) mspmm<6, 6, float>(L.R32, ML.t.p, mp, t, EpiPutMF<6, false>{MC.b.p, nr, mp, nullptr}, s);
      else mspmm<3, 3, float>(L.R32, ML.t.p, mp, t, EpiPutMF<3, false>{MC.b.p, nr, mp, nullptr}, s);
    }, s);
    ML.tP = pick_tile(mp, L.P32.op.lpr, [&](const MTile& t) {
      const int nr = L.P.n_rows;
      if (L.kdim == 6 && L.bs == 3) mspmm<3, 6, float>(L.P32, MC.y.p, mp, t, EpiPutMF<3, false>{ML.xb.p, nr, mp, nullptr}, s);
      else if (L.kdim == 6) mspmm<6, 6, float>(L.P32, MC.y.p, mp, t, EpiPutMF<6, false>{ML.xb.p, nr, mp, nullptr}, s);
      else mspmm<3, 3, float>(L.P32, MC.y.p, mp, t, EpiPutMF<3, false>{ML.xb.p, nr, mp, nullptr}, s);
    }, s);
  }
  MS.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void ensure_multi(tam_amg_s* H, int mp, cudaStream_t s) {
  if (!H->levels[0].dinv32.p) build_low_precision(H, s);
  if (H->multi && H->multi->mp == mp) return;
  static std::atomic<unsigned long long> serials{0};
  H->multi.reset(new MultiState());
  MultiState& MS = *H->multi;
  MS.mp = mp;
  MS.serial = ++serials;
  const size_t n3 = (size_t)H->K->n_nodes * 3;
  for (auto* v : {&MS.b, &MS.x, &MS.r, &MS.z, &MS.p, &MS.q}) {
    *v = DBuf<double>(n3 * mp, s);
    v->zero();
  }
  MS.sc = DBuf<double>(S_COUNT * (size_t)mp, s);
  MS.flags = DBuf<int>(4, s);
  MS.flags.zero();
  const unsigned g = std::max<unsigned>(grid_for((long long)H->K->S.n_slices * 32, MT_MIN_THREADS),
                                        (unsigned)sm_count() * 8u);
  MS.partials = DBuf<double>((size_t)g * std::max(TMAX, MPMAX) * (MPMAX / 1 + 1), s);
  MS.tickets = DBuf<unsigned int>(MPMAX + 1, s);
  MS.tickets.zero();
  MS.lv.resize(H->levels.size());
  for (size_t l = 0; l < H->levels.size(); ++l) {
    const size_t N = (size_t)H->levels[l].n_rows * H->levels[l].bs * mp;
    MultiLevel& ML = MS.lv[l];
    for (auto* v : {&ML.b, &ML.xa, &ML.xb, &ML.d, &ML.t, &ML.y}) {
      *v = DBuf<float>(N, s);
      v->zero();
    }
  }
  autotune(H, s);
}

void enqueue_multi_iteration(tam_amg_s* H, cudaStream_t s) {
  MultiState& MS = *H->multi;
  const int mp = MS.mp;
  const long long n3 = (long long)H->K->n_nodes * 3;
  int* flags = MS.flags.p;
  GridReduce gk{MS.partials.p, MS.tickets.p};
  kspmm(H->K->S, MS.p.p, mp, MS.tK, EpiPqM{MS.p.p, MS.q.p, H->K->n_nodes, mp, gk, MS.sc.p, flags}, s, H->levels[0].Aop.df);
  GridReduce ge{MS.partials.p, MS.tickets.p + MPMAX};
  mupdate_kernel<<<vgrid(n3), TPB, 0, s>>>(MS.x.p, MS.r.p, MS.p.p, MS.q.p, n3, mp, ge, MS.sc.p, flags);
  TAM_LAUNCH_CHECK();
  mvcycle<double, double>(H, 0, MS.r.p, MS.z.p, flags, s);
  mrz_kernel<<<vgrid(n3), TPB, 0, s>>>(MS.r.p, MS.z.p, MS.p.p, n3, mp, 0, ge, MS.sc.p, flags);
  TAM_LAUNCH_CHECK();
  mdir_kernel<<<vgrid(n3 * mp), TPB, 0, s>>>(MS.z.p, MS.p.p, n3, mp, MS.sc.p, flags);
  TAM_LAUNCH_CHECK();
}

// everything before the loop: residual, first V-cycle, first direction
void start_multi(tam_amg_s* H, int m, const double* B, const double* X, double rtol, double atol, int max_iter,
                 cudaStream_t s) {
  const int mp = ((m + 7) / 8) * 8;
  ensure_multi(H, mp, s);
  MultiState& MS = *H->multi;
  const long long n3 = (long long)H->K->n_nodes * 3;
  interleave_kernel<<<vgrid(n3 * mp), TPB, 0, s>>>(B, MS.b.p, m, mp, n3);
  interleave_kernel<<<vgrid(n3 * mp), TPB, 0, s>>>(X, MS.x.p, m, mp, n3);
  TAM_LAUNCH_CHECK();
  GridReduce ge{MS.partials.p, MS.tickets.p + MPMAX};
  mstart_kernel<<<vgrid(n3), TPB, 0, s>>>(MS.b.p, n3, m, mp, rtol, atol, max_iter, H->K->vmax_exp / 2, ge, MS.sc.p,
                                          MS.flags.p);
  TAM_LAUNCH_CHECK();
  mscale_in_kernel<<<vgrid(n3 * mp), TPB, 0, s>>>(MS.b.p, MS.x.p, n3, mp, MS.sc.p);
  TAM_LAUNCH_CHECK();
  GridReduce gk{MS.partials.p, MS.tickets.p};
  kspmm(H->K->S, MS.x.p, mp, MS.tK,
        EpiResInitM{MS.b.p, MS.r.p, H->K->n_nodes, mp, gk, MS.sc.p, nullptr, MS.flags.p}, s, H->levels[0].Aop.df);
  mcheck_kernel<<<1, 32, 0, s>>>(MS.sc.p, mp, MS.flags.p);
  TAM_LAUNCH_CHECK();
  mvcycle<double, double>(H, 0, MS.r.p, MS.z.p, MS.flags.p, s);
  mrz_kernel<<<vgrid(n3), TPB, 0, s>>>(MS.r.p, MS.z.p, MS.p.p, n3, mp, 1, ge, MS.sc.p, MS.flags.p);
  TAM_LAUNCH_CHECK();
}

int finish_multi(tam_amg_s* H, int m, const double* B, double* X, int* iters, double* rel, cudaStream_t s) {
  MultiState& MS = *H->multi;
  const int mp = MS.mp;
  const long long n3 = (long long)H->K->n_nodes * 3;
  DBuf<double> rn(mp, s);
  GridReduce gk{MS.partials.p, MS.tickets.p};
  // the reported true residual is always a plain FP64 product
  kspmm(H->K->S, MS.x.p, mp, MS.tK, EpiResInitM{MS.b.p, nullptr, H->K->n_nodes, mp, gk, MS.sc.p, rn.p, MS.flags.p},
        s, false);
  deinterleave_kernel<<<vgrid(n3 * m), TPB, 0, s>>>(MS.x.p, X, m, mp, n3, MS.sc.p);
  TAM_LAUNCH_CHECK();
  std::vector<double> sc(S_COUNT * (size_t)mp), r2(mp);
  int flags[4];
  TAM_CUDA(cudaMemcpyAsync(sc.data(), MS.sc.p, sizeof(double) * sc.size(), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaMemcpyAsync(r2.data(), rn.p, sizeof(double) * mp, cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaMemcpyAsync(flags, MS.flags.p, sizeof(flags), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaStreamSynchronize(s));
  bool all = true;
  for (int j = 0; j < m; ++j) {
    if (iters) iters[j] = (int)sc[S_ITER * mp + j];
    const double nb = std::sqrt(sc[S_BB * mp + j]);
    if (rel) rel[j] = nb > 0 ? std::sqrt(r2[j]) / nb : std::sqrt(r2[j]);
    all = all && sc[S_DONE * mp + j] != 0.0;
  }
  if (flags[3] != TAM_OK) return flags[3];
  return all ? TAM_OK : TAM_ERR_NOT_CONVERGED;
}

__global__ void all_stop_kernel(int* const* __restrict__ flags, int n, int* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int all = 1;
  for (int i = 0; i < n; ++i) all &= flags[i][0] != 0;
  *out = all;
}

}  // namespace

int pcg_solve_batch(int n_sys, tam_amg_s* const* H, const int* m, const double* const* B, double* const* X,
                    double rtol, double atol, int max_iter, int* iters, double* rel, cudaStream_t s) {
  NvtxRange nvtx("tam: batched AMG-PCG solve");
  TAM_CHECK(n_sys >= 1 && n_sys <= 64 && rtol >= 0 && atol >= 0 && max_iter >= 0, TAM_ERR_INVALID_ARG,
            "batch solve: bad argument");
  for (int i = 0; i < n_sys; ++i)
    TAM_CHECK(H[i] && m[i] >= 1 && m[i] <= MPMAX && B[i] && X[i], TAM_ERR_INVALID_ARG,
              "batch solve: each system needs a hierarchy and 1..16 right-hand sides");
  for (int i = 0; i < n_sys; ++i)
    for (int k = 0; k < i; ++k) TAM_CHECK(H[i] != H[k], TAM_ERR_INVALID_ARG, "batch solve: a hierarchy appears twice");
  for (int i = 0; i < n_sys; ++i)
    TAM_CHECK(H[i]->K->A.br == 3, TAM_ERR_UNSUPPORTED, "batch solve: 3x3-block (elastic) systems only");
  for (int i = 0; i < n_sys; ++i)
    TAM_CHECK(H[i]->K->df_ok, TAM_ERR_INVALID_ARG,
              "batch solve: the FP32 V-cycle needs K's largest entry within 2^-" + std::to_string(kDfExpLimit) +
                  "..2^" + std::to_string(kDfExpLimit) + " (it is 2^" + std::to_string(H[i]->K->vmax_exp) + ")");
  for (int i = 0; i < n_sys; ++i) start_multi(H[i], m[i], B[i], X[i], rtol, atol, max_iter, s);
  // one graph: a device-side WHILE loop whose body advances every system by
  // one iteration (each system on its own branch, joined), then a flag telling
  // whether all systems have stopped -- one launch for the whole batch solve;
  // built once per set of systems and kept by the first one
  std::vector<unsigned long long> key(n_sys);
  for (int i = 0; i < n_sys; ++i) key[i] = H[i]->multi->serial;
  auto& G = H[0]->multi->batch;
  if (!G || G->key != key) {
    G.reset();
    std::unique_ptr<MultiState::BatchGraph> g(new MultiState::BatchGraph());
    g->key = key;
    g->fl = DBuf<int*>(n_sys, s);
    g->all = DBuf<int>(2, s);
    std::vector<int*> hf(n_sys);
    for (int i = 0; i < n_sys; ++i) hf[i] = H[i]->multi->flags.p;
    TAM_CUDA(cudaMemcpyAsync(g->fl.p, hf.data(), sizeof(int*) * n_sys, cudaMemcpyHostToDevice, s));
    std::vector<cudaStream_t> br(n_sys, nullptr);
    std::vector<cudaEvent_t> ev(n_sys + 1, nullptr);
    auto cleanup = [&] {
      for (auto& e : ev)
        if (e) cudaEventDestroy(e);
      for (auto& b : br)
        if (b) cudaStreamDestroy(b);
    };
    try {
      for (int i = 0; i < n_sys; ++i) TAM_CUDA(cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking));
      for (auto& e : ev) TAM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      int* const* fl = g->fl.p;
      int* all = g->all.p;
      g->exec = build_loop_graph(
          [&](cudaStream_t cs) {
            TAM_CUDA(cudaEventRecord(ev[n_sys], cs));
            for (int i = 0; i < n_sys; ++i) {
              TAM_CUDA(cudaStreamWaitEvent(br[i], ev[n_sys], 0));
              enqueue_multi_iteration(H[i], br[i]);
              TAM_CUDA(cudaEventRecord(ev[i], br[i]));
              TAM_CUDA(cudaStreamWaitEvent(cs, ev[i], 0));
            }
            all_stop_kernel<<<1, 32, 0, cs>>>(fl, n_sys, all);
            TAM_LAUNCH_CHECK();
          },
          all, all + 1, H[0]->multi->flags.p + 2, 2, &g->kernels);
    } catch (...) {
      cudaGetLastError();
      cleanup();
      throw;
    }
    cleanup();
    G = std::move(g);
  }
  TAM_CUDA(cudaMemsetAsync(G->all.p, 0, 2 * sizeof(int), s));
  TAM_CUDA(cudaGraphLaunch(G->exec, s));
  int loops = 0;
  TAM_CUDA(cudaMemcpyAsync(&loops, G->all.p + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaStreamSynchronize(s));
  count_graph_launch(G->kernels * loops);
  int status = TAM_OK, off = 0;
  for (int i = 0; i < n_sys; ++i) {
    const int st = finish_multi(H[i], m[i], B[i], X[i], iters ? iters + off : nullptr, rel ? rel + off : nullptr, s);
    if (status == TAM_OK) status = st;
    off += m[i];
  }
  return status;
}

double multi_tune_ms(tam_amg_s* H) { return H->multi ? H->multi->tune_ms : 0.0; }
void multi_tiles(tam_amg_s* H, int* out, int cap) {
  int k = 0;
  if (!H->multi) return;
  auto put = [&](const MTile& t) {
    if (k + 3 > cap) return;
    out[k++] = t.tm;
    out[k++] = t.threads;
    out[k++] = t.lpr;
  };
  put(H->multi->tK);
  for (size_t l = 0; l + 1 < H->multi->lv.size(); ++l) {
    put(H->multi->lv[l].tA);
    put(H->multi->lv[l].tP);
    put(H->multi->lv[l].tR);
  }
}

}  // namespace tam
