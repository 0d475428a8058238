// Block sparse matrices on the device.
//
// Bsr  -- canonical block-CSR (row_ptr, sorted col_idx, row-major br x bc
//         blocks): the form assembly writes and the AMG setup reads.
// Sell -- the SpMV form: SELL-32 (sliced ELLPACK, slices of 32 block rows,
//         each slice padded to its longest row).  Within a slice, block slot
//         k of lane t (row 32*s + t) stores its br*bc values element-major:
//         vals[((slice_ptr[s] + k) * br*bc + e) * 32 + t].  A warp therefore
//         reads each block element of its 32 rows as one 256-byte coalesced
//         line, and every thread accumulates its own row with exactly br*bc
//         FMAs per block and no cross-lane reduction -- the FP64 FMA pipe, not
//         a shuffle tree, is the only arithmetic cost.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace tam {

struct Bsr {
  int n_rows = 0, n_cols = 0, br = 0, bc = 0;
  long long nnzb = 0;
  DBuf<int> row_ptr, col_idx;
  DBuf<double> vals;
  size_t block_elems() const { return (size_t)br * bc; }
};

struct Sell {
  int n_rows = 0, n_slices = 0, br = 0, bc = 0;
  long long n_slots = 0;  // block columns (each 32 blocks wide)
  DBuf<int> slice_ptr;    // [n_slices + 1]
  DBuf<int> cols;         // [n_slots * 32]
  DBuf<double> vals;      // [n_slots * 32 * br * bc]
};

struct SellView {
  int n_rows, n_slices;
  const int* __restrict__ slice_ptr;
  const int* __restrict__ cols;
  const double* __restrict__ vals;
};

inline SellView view(const Sell& s) {
  return SellView{s.n_rows, s.n_slices, s.slice_ptr.p, s.cols.p, s.vals.p};
}

// Builds the SELL-32 copy of a Bsr (pattern + values).
void bsr_to_sell(const Bsr& A, Sell& S, cudaStream_t s);
// Refreshes only the values of an existing SELL copy built from A.
void sell_refresh_values(const Bsr& A, Sell& S, cudaStream_t s);

// Transpose (block transpose included): R = A^T.  Rows of R sorted by column.
void bsr_transpose(const Bsr& A, Bsr& R, cudaStream_t s);

// C = X * Y for block sparse X (m x k blocks) and Y (k x n blocks).
// Arithmetic of the SpGEMM numeric pass: plain FP64, or double-float (each
// FP64 operand split into two FP32 values, products and sums in FP32 with
// error-free transforms, about 2^-48 relative; FP64 in and out).
enum class SpgemmArith { kFp64, kDoubleFloat };
// Double-float operands and result kept split: x / y are X's / Y's values
// already split (NULL: split here); c (not NULL): C's values are written split
// into *c and C.vals stays empty (for a product that only feeds another
// double-float product).  Ignored for kFp64.
struct SpgemmSplit {
  const float2* x = nullptr;
  const float2* y = nullptr;
  DBuf<float2>* c = nullptr;
};
// FP64 values split into (hi, lo) FP32 pairs with integer operations only.
DBuf<float2> split_values(const Bsr& B, cudaStream_t s);
// C = X Y (block shapes 3/6).
void bsr_spgemm(const Bsr& X, const Bsr& Y, Bsr& C, cudaStream_t s, SpgemmArith arith = SpgemmArith::kDoubleFloat,
                const SpgemmSplit& sp = SpgemmSplit());

// ---------------------------------------------------------------------------
// Thread-per-row SELL SpMV with a fused epilogue.
//   Epi::skip()                      -- uniform early exit (solver stop flag)
//   Epi::operator()(row, acc, sh)    -- consumes the row's BR results; called by
//                                      every thread (row >= n_rows included)
//                                      so that epilogues may reduce over the block.
// ---------------------------------------------------------------------------
constexpr int SPMV_THREADS = 128;

template <int BR, int BC, class Epi>
__global__ void __launch_bounds__(SPMV_THREADS)
sell_spmv_kernel(SellView A, const double* __restrict__ x, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int row = blockIdx.x * SPMV_THREADS + threadIdx.x;
  const int slice = row >> 5, lane = row & 31;
  double acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.0;
  if (slice < A.n_slices) {
    const int k0 = A.slice_ptr[slice], k1 = A.slice_ptr[slice + 1];
    const int* __restrict__ cp = A.cols + (size_t)k0 * 32 + lane;
    const double* __restrict__ vp = A.vals + (size_t)k0 * 32 * BR * BC + lane;
#pragma unroll 2
    for (int k = k0; k < k1; ++k) {
      const int c = __ldg(cp);
      double xv[BC];
#pragma unroll
      for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int j = 0; j < BC; ++j) acc[r] = fma(__ldg(vp + (r * BC + j) * 32), xv[j], acc[r]);
      cp += 32;
      vp += 32 * BR * BC;
    }
  }
  epi(row, acc, sh);
}

template <int BR, int BC, class Epi>
void sell_spmv(const Sell& A, const double* x, Epi epi, cudaStream_t s) {
  unsigned grid = grid_for((long long)A.n_slices * 32, SPMV_THREADS);
  sell_spmv_kernel<BR, BC, Epi><<<grid, SPMV_THREADS, 0, s>>>(view(A), x, epi);
  TAM_LAUNCH_CHECK();
}

inline unsigned sell_grid(const Sell& A) { return grid_for((long long)A.n_slices * 32, SPMV_THREADS); }

// ---------------------------------------------------------------------------
// LPR lanes per block row over the Bsr arrays, for operators whose rows are
// few or long (coarse levels, restriction): thread-per-row would leave most
// SMs idle there.  Lanes stride over the row's blocks, then reduce with
// shuffles (the FP64 adds this costs are irrelevant: these launches are
// latency-, not throughput-bound).
// ---------------------------------------------------------------------------
struct BsrView {
  int n_rows;
  const int* __restrict__ rp;
  const int* __restrict__ ci;
  const double* __restrict__ v;
};

template <int BR, int BC, int LPR, class Epi>
__global__ void __launch_bounds__(SPMV_THREADS)
bsr_vector_kernel(BsrView A, const double* __restrict__ x, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int t = blockIdx.x * SPMV_THREADS + threadIdx.x;
  const int row = t / LPR, sub = t % LPR;
  double acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.0;
  if (row < A.n_rows) {
    const int pe = A.rp[row + 1];
    for (int p = A.rp[row] + sub; p < pe; p += LPR) {
      const int c = A.ci[p];
      const double* __restrict__ vb = A.v + (size_t)p * BR * BC;
      double xv[BC];
#pragma unroll
      for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int j = 0; j < BC; ++j) acc[r] = fma(__ldg(vb + r * BC + j), xv[j], acc[r]);
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  epi((sub == 0 && row < A.n_rows) ? row : A.n_rows, acc, sh);
}

// A sparse operator with its SpMV strategy: SELL-32 thread-per-row (lpr == 0)
// or LPR lanes per row over the Bsr arrays.
struct SpOp {
  const Bsr* B = nullptr;
  const Sell* S = nullptr;
  int lpr = 0;
};

// Strategy: thread-per-row SELL for many short rows, else lanes per row.
// Each lane should own >= ~16 blocks: the closing shuffle reduction costs
// log2(LPR) FP64 adds per output per lane, and on GB300 the FP64 pipe (not
// bandwidth) is the limit, so a wide LPR on medium rows wastes it.
inline int choose_lpr(const Bsr& A) {
  const double avg = A.n_rows > 0 ? (double)A.nnzb / A.n_rows : 0.0;
  if (A.n_rows >= 65536 && avg <= 48.0) return 0;
  int l = 2;
  while (l < 32 && 16 * l < avg) l <<= 1;
  if (A.n_rows < 8192) l = std::max(l, 16);  // few rows: spread them over more lanes
  return l;
}

inline unsigned spop_grid(const SpOp& op) {
  if (op.lpr == 0) return sell_grid(*op.S);
  return grid_for((long long)op.B->n_rows * op.lpr, SPMV_THREADS);
}

template <int BR, int BC, class Epi>
void spop_apply(const SpOp& op, const double* x, Epi epi, cudaStream_t s) {
  if (op.lpr == 0) {
    sell_spmv<BR, BC>(*op.S, x, epi, s);
    return;
  }
  const BsrView v{op.B->n_rows, op.B->row_ptr.p, op.B->col_idx.p, op.B->vals.p};
  const unsigned g = spop_grid(op);
  switch (op.lpr) {
    case 2: bsr_vector_kernel<BR, BC, 2, Epi><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 4: bsr_vector_kernel<BR, BC, 4, Epi><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 8: bsr_vector_kernel<BR, BC, 8, Epi><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 16: bsr_vector_kernel<BR, BC, 16, Epi><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    default: bsr_vector_kernel<BR, BC, 32, Epi><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
  }
  TAM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Reduced-precision copies for the V-cycle (FP32 values, or BF16 values on the
// finest level), FP32 vectors and FP32 accumulation.  Same two layouts and the
// same thread/lane mapping as the FP64 kernels above.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <int BR, int BC, typename TV, class Epi>
__global__ void __launch_bounds__(SPMV_THREADS)
sell_spmv_f32_kernel(int n_slices, const int* __restrict__ slice_ptr, const int* __restrict__ cols,
                     const TV* __restrict__ vals, const float* __restrict__ x, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int row = blockIdx.x * SPMV_THREADS + threadIdx.x;
  const int slice = row >> 5, lane = row & 31;
  float acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.f;
  if (slice < n_slices) {
    const int k0 = slice_ptr[slice], k1 = slice_ptr[slice + 1];
    const int* __restrict__ cp = cols + (size_t)k0 * 32 + lane;
    const TV* __restrict__ vp = vals + (size_t)k0 * 32 * BR * BC + lane;
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
      const int c = __ldg(cp);
      float xv[BC];
#pragma unroll
      for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int j = 0; j < BC; ++j) acc[r] = fmaf(to_f32(vp[(r * BC + j) * 32]), xv[j], acc[r]);
      cp += 32;
      vp += 32 * BR * BC;
    }
  }
  epi(row, acc, sh);
}

template <int BR, int BC, int LPR, typename TV, class Epi>
__global__ void __launch_bounds__(SPMV_THREADS)
bsr_vector_f32_kernel(int n_rows, const int* __restrict__ rp, const int* __restrict__ ci, const TV* __restrict__ v,
                      const float* __restrict__ x, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int t = blockIdx.x * SPMV_THREADS + threadIdx.x;
  const int row = t / LPR, sub = t % LPR;
  float acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.f;
  if (row < n_rows) {
    const int pe = rp[row + 1];
    for (int p = rp[row] + sub; p < pe; p += LPR) {
      const int c = ci[p];
      const TV* __restrict__ vb = v + (size_t)p * BR * BC;
      float xv[BC];
#pragma unroll
      for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int j = 0; j < BC; ++j) acc[r] = fmaf(to_f32(vb[r * BC + j]), xv[j], acc[r]);
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  epi((sub == 0 && row < n_rows) ? row : n_rows, acc, sh);
}

// A reduced-precision operator: the pattern of `op` with values `vals`
// (same layout as op's FP64 values: SELL when op.lpr == 0, else Bsr).
template <typename TV>
struct SpOpLow {
  SpOp op;
  const TV* vals = nullptr;
};

template <int BR, int BC, typename TV, class Epi>
void spop_apply_f32(const SpOpLow<TV>& o, const float* x, Epi epi, cudaStream_t s) {
  const unsigned g = spop_grid(o.op);
  if (o.op.lpr == 0) {
    const Sell& S = *o.op.S;
    sell_spmv_f32_kernel<BR, BC, TV, Epi><<<g, SPMV_THREADS, 0, s>>>(S.n_slices, S.slice_ptr.p, S.cols.p, o.vals, x,
                                                                     epi);
  } else {
    const Bsr& B = *o.op.B;
    switch (o.op.lpr) {
      case 2: bsr_vector_f32_kernel<BR, BC, 2, TV, Epi><<<g, SPMV_THREADS, 0, s>>>(B.n_rows, B.row_ptr.p, B.col_idx.p, o.vals, x, epi); break;
      case 4: bsr_vector_f32_kernel<BR, BC, 4, TV, Epi><<<g, SPMV_THREADS, 0, s>>>(B.n_rows, B.row_ptr.p, B.col_idx.p, o.vals, x, epi); break;
      case 8: bsr_vector_f32_kernel<BR, BC, 8, TV, Epi><<<g, SPMV_THREADS, 0, s>>>(B.n_rows, B.row_ptr.p, B.col_idx.p, o.vals, x, epi); break;
      case 16: bsr_vector_f32_kernel<BR, BC, 16, TV, Epi><<<g, SPMV_THREADS, 0, s>>>(B.n_rows, B.row_ptr.p, B.col_idx.p, o.vals, x, epi); break;
      default: bsr_vector_f32_kernel<BR, BC, 32, TV, Epi><<<g, SPMV_THREADS, 0, s>>>(B.n_rows, B.row_ptr.p, B.col_idx.p, o.vals, x, epi); break;
    }
  }
  TAM_LAUNCH_CHECK();
}

// Values of `op` (whichever layout it uses) as a reduced-precision copy.
void convert_values_f32(const SpOp& op, DBuf<float>& out, cudaStream_t s);
void convert_values_bf16(const SpOp& op, DBuf<__nv_bfloat16>& out, cudaStream_t s);

// --- common epilogues ------------------------------------------------------
struct NoStop {
  __device__ bool skip() const { return false; }
};

// y = A x
template <int BR>
struct EpiStore {
  double* y;
  int n_rows;
  const int* stop;  // may be null
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const double (&acc)[BR], double*) const {
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < BR; ++r) y[(size_t)row * BR + r] = acc[r];
  }
};

// y += A x
template <int BR>
struct EpiAdd {
  double* y;
  int n_rows;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const double (&acc)[BR], double*) const {
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < BR; ++r) y[(size_t)row * BR + r] += acc[r];
  }
};

// t = b - A x
template <int BR>
struct EpiResidual {
  const double* b;
  double* t;
  int n_rows;
  const int* stop;
  __device__ bool skip() const { return stop && *stop; }
  __device__ void operator()(int row, const double (&acc)[BR], double*) const {
    if (row < n_rows)
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        size_t i = (size_t)row * BR + r;
        t[i] = b[i] - acc[r];
      }
  }
};

}  // namespace tam
