// Reduced-precision V-cycle inside FP64 CG.
//
// The hierarchy is built in FP64 (amg_setup); this file stores a copy of
// every level's A, P and R values in FP32 -- or, for level_precision 2, the
// finest level's A in BF16 -- and runs the V-cycle with FP32 vectors and FP32
// accumulation.  The V-cycle reads the FP64 CG residual and writes the FP64
// preconditioned residual; the coarsest dense solve stays FP64.  The outer
// CG (its SpMV with K, residuals, dot products, stopping test) is untouched.
//
// Why: GB300 runs FP64 FMAs at ~2/clk/SM but FP32 at 128/clk/SM, so the
// FP64 SpMV is bound by the FP64 pipe; in FP32 (40 bytes per 3x3 block instead
// of 76) or BF16 values (22 bytes) the smoother SpMVs become HBM-bound and
// move half or less of the bytes.  A preconditioner only has to be a fixed
// SPD-like operator, so its rounding error costs at most a few iterations.
#include <algorithm>

#include "handles.cuh"

namespace tam {
namespace {

constexpr int TPB = 256;

template <typename T>
__device__ __forceinline__ float f32(T v) { return (float)v; }

template <typename TB>
__global__ void cheb_first_zero_f32_kernel(const TB* __restrict__ b, const float* __restrict__ dinv,
                                           const float* __restrict__ consts, float* __restrict__ d,
                                           float* __restrict__ x, long long N, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const float cr = consts[3];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    float di = cr * dinv[i] * f32(b[i]);
    d[i] = di;
    x[i] = di;
  }
}

// One Chebyshev step fused into the FP32 SpMV of x.
template <int BR, typename TB, typename TO>
struct EpiChebF {
  const TB* b;
  const float* x;
  const float* dinv;
  const float* coef;
  float* d;
  TO* xn;
  int n_rows;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const float (&acc)[BR], double*) const {
    if (row >= n_rows) return;
    const float cd = coef[0], cr = coef[1];
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      size_t i = (size_t)row * BR + r;
      float res = dinv[i] * (f32(b[i]) - acc[r]);
      float di = cd != 0.f ? cd * d[i] + cr * res : cr * res;
      d[i] = di;
      xn[i] = (TO)(x[i] + di);
    }
  }
};

template <int BR, typename TB>
struct EpiResidualF {
  const TB* b;
  float* t;
  int n_rows;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const float (&acc)[BR], double*) const {
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        size_t i = (size_t)row * BR + r;
        t[i] = f32(b[i]) - acc[r];
      }
  }
};

template <int BR>
struct EpiStoreF {
  float* y;
  int n_rows;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const float (&acc)[BR], double*) const {
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < BR; ++r) y[(size_t)row * BR + r] = acc[r];
  }
};

template <int BR>
struct EpiAddF {
  float* y;
  int n_rows;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const float (&acc)[BR], double*) const {
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < BR; ++r) y[(size_t)row * BR + r] += acc[r];
  }
};

// coarsest level: FP64 dense inverse applied to an FP32 (or FP64) vector, FP64 dot products
template <typename TI, typename TO>
__global__ void dense_gemv_mixed_kernel(const double* __restrict__ A, const TI* __restrict__ b, TO* __restrict__ y,
                                        int N, const int* __restrict__ stop) {
  if (stop && *stop) return;
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= N) return;
  const double* a = A + (size_t)row * N;
  double s = 0.0;
  for (int j = lane; j < N; j += 32) s = fma(a[j], (double)b[j], s);
  s = warp_sum(s);
  if (lane == 0) y[row] = (TO)s;
}

__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

unsigned vgrid(long long N) { return stride_grid(N, TPB, 8); }

// A x with the level's reduced-precision values: BF16 on the finest level in
// mode 2, FP32 otherwise.
template <int BS, class Epi>
void level_spmv(const Level& L, const float* x, Epi epi, cudaStream_t s) {
  if (L.A16.vals) spop_apply_f32<BS, BS, __nv_bfloat16>(L.A16, x, epi, s);
  else spop_apply_f32<BS, BS, float>(L.A32, x, epi, s);
}

template <typename TB, typename TO>
void cheb_step_f(const Level& L, const TB* b, const float* x, TO* xn, int step, const int* stop, cudaStream_t s) {
  const float* coef = L.consts32.p + 2 + 2 * step;
  if (L.bs == 3)
    level_spmv<3>(L, x, EpiChebF<3, TB, TO>{b, x, L.dinv32.p, coef, L.d32.p, xn, L.n_rows, stop}, s);
  else
    level_spmv<6>(L, x, EpiChebF<6, TB, TO>{b, x, L.dinv32.p, coef, L.d32.p, xn, L.n_rows, stop}, s);
}

template <typename TB>
void residual_f(const Level& L, const TB* b, const float* x, float* t, const int* stop, cudaStream_t s) {
  if (L.bs == 3) level_spmv<3>(L, x, EpiResidualF<3, TB>{b, t, L.n_rows, stop}, s);
  else level_spmv<6>(L, x, EpiResidualF<6, TB>{b, t, L.n_rows, stop}, s);
}

void restrict_f(const Level& L, const float* t, float* bc, const int* stop, cudaStream_t s) {
  const int nr = L.R.n_rows;
  if (L.kdim == 6 && L.bs == 3) spop_apply_f32<6, 3, float>(L.R32, t, EpiStoreF<6>{bc, nr, stop}, s);
  else if (L.kdim == 6) spop_apply_f32<6, 6, float>(L.R32, t, EpiStoreF<6>{bc, nr, stop}, s);
  else spop_apply_f32<3, 3, float>(L.R32, t, EpiStoreF<3>{bc, nr, stop}, s);
}

void prolong_f(const Level& L, const float* xc, float* x, const int* stop, cudaStream_t s) {
  const int nr = L.P.n_rows;
  if (L.kdim == 6 && L.bs == 3) spop_apply_f32<3, 6, float>(L.P32, xc, EpiAddF<3>{x, nr, stop}, s);
  else if (L.kdim == 6) spop_apply_f32<6, 6, float>(L.P32, xc, EpiAddF<6>{x, nr, stop}, s);
  else spop_apply_f32<3, 3, float>(L.P32, xc, EpiAddF<3>{x, nr, stop}, s);
}

template <typename TB, typename TO>
void vcycle_low(tam_amg_s* H, int l, const TB* b, TO* out, const int* stop, cudaStream_t s) {
  Level& L = H->levels[l];
  const long long N = (long long)L.n_rows * L.bs;
  if (l == (int)H->levels.size() - 1) {
    dense_gemv_mixed_kernel<TB, TO><<<grid_for((long long)H->n_coarse * 32, TPB), TPB, 0, s>>>(
        H->coarse_inv.p, b, out, H->n_coarse, stop);
    TAM_LAUNCH_CHECK();
    return;
  }
  const int deg = L.deg;
  float* xa = L.xa32.p;
  float* xb = L.xb32.p;
  cheb_first_zero_f32_kernel<TB><<<vgrid(N), TPB, 0, s>>>(b, L.dinv32.p, L.consts32.p, L.d32.p, xa, N, stop);
  TAM_LAUNCH_CHECK();
  for (int k = 1; k < deg; ++k) {
    cheb_step_f<TB, float>(L, b, xa, xb, k, stop, s);
    std::swap(xa, xb);
  }
  residual_f<TB>(L, b, xa, L.t32.p, stop, s);
  Level& C = H->levels[l + 1];
  restrict_f(L, L.t32.p, C.b32.p, stop, s);
  vcycle_low<float, float>(H, l + 1, C.b32.p, C.y32.p, stop, s);
  prolong_f(L, C.y32.p, xa, stop, s);
  for (int k = 0; k < deg; ++k) {
    if (k == deg - 1) {
      cheb_step_f<TB, TO>(L, b, xa, out, k, stop, s);
    } else {
      cheb_step_f<TB, float>(L, b, xa, xb, k, stop, s);
      std::swap(xa, xb);
    }
  }
}

}  // namespace

void vcycle_apply_low(tam_amg_s* H, const double* r, double* z, const int* stop, cudaStream_t s) {
  vcycle_low<double, double>(H, 0, r, z, stop, s);
}

void build_low_precision(tam_amg_s* H, cudaStream_t s) {
  const int mode = H->prm.level_precision;
  for (size_t l = 0; l < H->levels.size(); ++l) {
    Level& L = H->levels[l];
    const size_t N = (size_t)L.n_rows * L.bs;
    const bool coarsest = (l + 1 == H->levels.size());
    L.dinv32 = DBuf<float>(N, s);
    to_f32_kernel<<<vgrid((long long)N), TPB, 0, s>>>(L.dinv.p, L.dinv32.p, (long long)N);
    TAM_LAUNCH_CHECK();
    const size_t nc = 2 + 2 * (size_t)std::max(L.deg, 1);
    L.consts32 = DBuf<float>(nc, s);
    to_f32_kernel<<<1, 32, 0, s>>>(L.consts.p, L.consts32.p, (long long)nc);
    TAM_LAUNCH_CHECK();
    L.b32 = DBuf<float>(N, s);
    L.y32 = DBuf<float>(N, s);
    if (coarsest) continue;
    L.xa32 = DBuf<float>(N, s);
    L.xb32 = DBuf<float>(N, s);
    L.d32 = DBuf<float>(N, s);
    L.t32 = DBuf<float>(N, s);
    if (l == 0 && mode == 2) {
      convert_values_bf16(L.Aop, L.A16v, s);
      L.A16 = SpOpLow<__nv_bfloat16>{L.Aop, L.A16v.p};
    } else {
      convert_values_f32(L.Aop, L.A32v, s);
      L.A32 = SpOpLow<float>{L.Aop, L.A32v.p};
    }
    convert_values_f32(L.Pop, L.P32v, s);
    L.P32 = SpOpLow<float>{L.Pop, L.P32v.p};
    convert_values_f32(L.Rop, L.R32v, s);
    L.R32 = SpOpLow<float>{L.Rop, L.R32v.p};
  }
}

}  // namespace tam
