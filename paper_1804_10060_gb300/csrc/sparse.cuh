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
void bsr_spgemm(const Bsr& X, const Bsr& Y, Bsr& C, cudaStream_t s);

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
