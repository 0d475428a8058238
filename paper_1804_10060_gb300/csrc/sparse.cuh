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
//
// Double-float ("DF"): either form may also hold vals_df, its values split
// into (hi, lo) FP32 pairs (same 8 bytes per value).  The SpMV kernels then
// multiply in FP32 with error-free transforms (about 2^-47 relative), which
// GB300 issues at 64 times its FP64 FMA rate, so the SpMV is bound by memory
// instead of the FP64 pipe; vectors and epilogues stay FP64.
#pragma once

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace tam {

// IEEE-754 bit manipulations (integer pipe only: GB300's FP64 pipe, which also
// executes FP64<->FP32 conversions, is the scarce resource here).
//
// split_bits: v = hi + lo with hi = v rounded to FP32's 24-bit significand
// (to nearest on the first discarded bit) and lo = v - hi (at most 29 bits,
// |lo| <= 2^-24 |v|) rounded to 24 bits the same way: |v - hi - lo| <=
// 2^-49 |v| for 2^-78 <= |v| < 2^126, with no sign bias.  Below 2^-78 the
// remainder may fall under FP32's normal range and is dropped (absolute error
// < 2^-126); |v| < 2^-126 (zero, FP64 values below FP32's normal range)
// gives (0, 0) and values that round to 2^128 give (+-inf, 0).  The library
// splits only matrices whose largest entry lies within 2^-90..2^90
// (kDfExpLimit), with the CG vectors scaled by a power of two to match (see
// pcg_solve), so that products and sums stay far from both ends.
__device__ __forceinline__ float2 split_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int ef = (int)((b >> 52) & 0x7ff) - 1023 + 127;  // FP32 biased exponent of hi
  if (ef <= 0) return make_float2(0.f, 0.f);
  if (ef >= 255) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
  const unsigned long long m = b & 0xfffffffffffffull;
  const unsigned up = (unsigned)(m >> 28) & 1u;            // first bit below hi's 24
  // a carry out of the significand moves into the exponent field (2^128 -> inf)
  const unsigned hb = (((unsigned)ef << 23) | (unsigned)(m >> 29)) + up;
  const float hi = __uint_as_float(sign | (hb < 0x7f800000u ? hb : 0x7f800000u));
  // v - hi in units of 2^(E - 52): the 29-bit tail, less 2^29 when hi was rounded up
  const int t = (int)(m & 0x1fffffffull) - (int)(up << 29);
  if (t == 0) return make_float2(hi, 0.f);
  const unsigned at = (unsigned)(t < 0 ? -t : t);           // 1 .. 2^28
  const unsigned lsign = t < 0 ? (sign ^ 0x80000000u) : sign;
  const int nb = 32 - __clz(at);                            // significant bits of the tail, 1..29
  int el = ef - 53 + nb;                                    // FP32 biased exponent of lo
  unsigned mant;
  if (nb <= 24) {
    mant = at << (24 - nb);
  } else {
    const int sh = nb - 24;                                  // 1..5 bits dropped, rounded to nearest
    mant = (at + (1u << (sh - 1))) >> sh;
    if (mant >> 24) { mant >>= 1; ++el; }
  }
  if (el <= 0) return make_float2(hi, 0.f);
  return make_float2(hi, __uint_as_float(lsign | ((unsigned)el << 23) | (mant & 0x7fffffu)));
}

// Exact FP32 -> FP64 (zero and FP32 subnormals give 0; inf/nan keep their class).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xff;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ed = e == 255 ? 0x7ffull : (unsigned long long)(e - 127 + 1023);
  return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// a += x * y in double-float: the product of the high parts made exact with
// an FMA, the two cross terms added to its error (lo * lo, below 2^-48 of the
// product, dropped), the sum with the accumulator by Knuth's TwoSum.
// __fadd_rn / __fmul_rn keep the compiler from contracting the transforms.
__device__ __forceinline__ void df_fma(float2& a, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = fmaf(x.x, y.x, -p);        // exact: x.x * y.x = p + e
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  const float s = __fadd_rn(a.x, p);   // TwoSum(a.x, p) = s + err exactly
  const float bp = __fadd_rn(s, -a.x);
  const float err = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(s, -bp)), __fadd_rn(p, -bp));
  a.x = s;
  a.y = __fadd_rn(a.y, __fadd_rn(err, e));
}

// df_fma with the lo * lo product kept as well (the accurate SpMV: the dropped
// term is otherwise up to 2^-48 of each product)
__device__ __forceinline__ void df_fma4(float2& a, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  e = fmaf(x.y, y.y, e);
  const float s = __fadd_rn(a.x, p);
  const float bp = __fadd_rn(s, -a.x);
  const float err = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(s, -bp)), __fadd_rn(p, -bp));
  a.x = s;
  a.y = __fadd_rn(a.y, __fadd_rn(err, e));
}

// a += b for two unevaluated sums hi + lo: TwoSum of the high parts, the
// low parts and the rounding error added to the low part.
__device__ __forceinline__ void df_add(float2& a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bp = __fadd_rn(s, -a.x);
  const float err = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(s, -bp)), __fadd_rn(b.x, -bp));
  a.x = s;
  a.y = __fadd_rn(a.y, __fadd_rn(err, b.y));
}

__device__ __forceinline__ double df_to_double(float2 a) { return f2d_bits(a.x) + f2d_bits(a.y); }

// a += b for two double-float values, the accurate form: TwoSum of the high
// parts and of the low parts, the errors folded in with two renormalisations
// (Fast2Sum), relative error a few 2^-48 whatever the magnitudes' order --
// the double-word addition with the tight bound of Joldes, Muller and
// Popescu (2017).  The accurate SpMV folds each slot's products in with it.
__device__ __forceinline__ void df_add_accurate(float2& a, float2 b) {
  float sh = __fadd_rn(a.x, b.x);
  float t = __fadd_rn(sh, -a.x);
  float sl = __fadd_rn(__fadd_rn(a.x, -__fadd_rn(sh, -t)), __fadd_rn(b.x, -t));
  const float th = __fadd_rn(a.y, b.y);
  t = __fadd_rn(th, -a.y);
  const float tl = __fadd_rn(__fadd_rn(a.y, -__fadd_rn(th, -t)), __fadd_rn(b.y, -t));
  sl = __fadd_rn(sl, th);
  float h = __fadd_rn(sh, sl);
  sl = __fadd_rn(sl, -__fadd_rn(h, -sh));
  sl = __fadd_rn(sl, tl);
  a.x = __fadd_rn(h, sl);
  a.y = __fadd_rn(sl, -__fadd_rn(a.x, -h));
}

// Largest |binary exponent| of a matrix's largest entry for which the
// double-float products are used (amg_params.spmv_fp64 / setup_fp64 fall back
// to FP64 outside it).
constexpr int kDfExpLimit = 90;

struct Bsr;
// Binary exponent of A's largest |entry| (floor(log2 max |A_ij|); 0 when there
// is none) into *max_exp, over the block rows that hold more than their
// diagonal block (identity rows of Dirichlet and cell-less nodes do not set
// the scale), and whether every entry is finite.  Synchronising.
void operator_exponent_range(const Bsr& A, int* max_exp, bool* finite, cudaStream_t s);

struct Bsr {
  int n_rows = 0, n_cols = 0, br = 0, bc = 0;
  long long nnzb = 0;
  DBuf<int> row_ptr, col_idx;
  DBuf<double> vals;
  DBuf<float2> vals_df;   // optional split copy of vals (SpMV only)
  size_t block_elems() const { return (size_t)br * bc; }
};

struct Sell {
  int n_rows = 0, n_slices = 0, br = 0, bc = 0;
  long long n_slots = 0;  // block columns (each 32 blocks wide)
  DBuf<int> slice_ptr;    // [n_slices + 1]
  DBuf<int> cols;         // [n_slots * 32]
  DBuf<double> vals;      // [n_slots * 32 * br * bc]
  DBuf<float2> vals_df;   // optional split copy of vals
  // optional row order (SELL-C-sigma): slot position p holds row perm[p]; rows
  // are sorted by length within windows of 256 so that a slice's rows have
  // similar lengths (P2 meshes interleave long vertex rows with short edge
  // rows: 40% padding unsorted, 8% sorted).  Empty: position p holds row p.
  DBuf<int> perm;
};

struct SellView {
  int n_rows, n_slices;
  const int* __restrict__ slice_ptr;
  const int* __restrict__ cols;
  const double* __restrict__ vals;
  const float2* __restrict__ vals_df;
  const int* __restrict__ perm;
};

inline SellView view(const Sell& s) {
  return SellView{s.n_rows, s.n_slices, s.slice_ptr.p, s.cols.p, s.vals.p, s.vals_df.p, s.perm.p};
}

// Row held by slot position pos (positions past the last row stay out of range).
__device__ __forceinline__ int sell_row(const int* __restrict__ perm, int pos, int n_rows) {
  return (perm && pos < n_rows) ? __ldg(perm + pos) : pos;
}

// (Re)builds the split copy vals_df from vals (integer operations only).
void build_df_values(Sell& S, cudaStream_t s);
void build_df_values(Bsr& B, cudaStream_t s);

// Builds the SELL-32 copy of a Bsr (pattern + values).
void bsr_to_sell(const Bsr& A, Sell& S, cudaStream_t s, bool df = false);  // df: the split copy too
// Refreshes only the values of an existing SELL copy built from A (and its
// split copy, when it has one).
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
  // C known to be symmetric (square blocks, R (A P) with R = P^T): only the
  // blocks on or above the diagonal are multiplied, the rest mirrored.
  bool symmetric = false;
};
// FP64 values split into (hi, lo) FP32 pairs with integer operations only.
DBuf<float2> split_values(const Bsr& B, cudaStream_t s);
// C = X Y (block shapes 3/6).
void bsr_spgemm(const Bsr& X, const Bsr& Y, Bsr& C, cudaStream_t s, SpgemmArith arith = SpgemmArith::kDoubleFloat,
                const SpgemmSplit& sp = SpgemmSplit());
// C = X P_tent for a tentative prolongator (one block per aggregated row k, in
// column agg[k]; agg[k] < 0: an empty row), xs: X's split values or NULL.
// Returns false, with C untouched, for block shapes other than 3x3.3x6,
// 6x6.6x6, 1x1.1x1 or a row of X longer than 256 blocks (use bsr_spgemm).
bool bsr_spgemm_tentative(const Bsr& X, const Bsr& Pt, const int* agg, Bsr& C, cudaStream_t s, SpgemmArith arith,
                          const float2* xs);

// ---------------------------------------------------------------------------
// Thread-per-row SELL SpMV with a fused epilogue.
//   Epi::skip()                      -- uniform early exit (solver stop flag)
//   Epi::operator()(row, acc, sh)    -- consumes the row's BR results; called by
//                                      every thread (row >= n_rows included)
//                                      so that epilogues may reduce over the block.
// ---------------------------------------------------------------------------
constexpr int SPMV_THREADS = 128;


template <int BR, int BC, class Epi, bool DF, bool ACC = false>
__global__ void __launch_bounds__(SPMV_THREADS)
sell_spmv_kernel(SellView A, const double* __restrict__ x, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int pos = blockIdx.x * SPMV_THREADS + threadIdx.x;
  const int slice = pos >> 5, lane = pos & 31;
  double acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.0;
  if (slice < A.n_slices) {
    const int k0 = A.slice_ptr[slice], k1 = A.slice_ptr[slice + 1];
    const int* __restrict__ cp = A.cols + (size_t)k0 * 32 + lane;
    if constexpr (DF) {
      const float2* __restrict__ vp = A.vals_df + (size_t)k0 * 32 * BR * BC + lane;
      float2 ad[BR], run[BR];
#pragma unroll
      for (int r = 0; r < BR; ++r) ad[r] = run[r] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int k = k0; k < k1; ++k) {
        float2 vv[BR * BC];  // the slot's values first, then the gather
#pragma unroll
        for (int e = 0; e < BR * BC; ++e) vv[e] = __ldg(vp + e * 32);
        const int c = __ldg(cp);
        float2 xv[BC];
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[j] = split_bits(__ldg(x + (size_t)c * BC + j));
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int j = 0; j < BC; ++j) {
            if constexpr (ACC) df_fma4(ad[r], vv[r * BC + j], xv[j]);
            else df_fma(ad[r], vv[r * BC + j], xv[j]);
          }
        if constexpr (ACC) {
          // ACC: each slot's double-float partial sum (its BC products) is
          // added into the row's running sum with the accurate double-word
          // addition, so that the low part never carries more than one
          // slot's rounding: a few 2^-48 of sum_j |A_ij x_j| per row whatever
          // the row's length (the plain running double-float sum drifts to
          // ~2^-45 on long P2 rows); FP32 work only (an FP64 sum every two
          // slots cost 1.5 FP64 adds per row and slot pair on GB300's slow
          // FP64 pipe)
#pragma unroll
          for (int r = 0; r < BR; ++r) {
            df_add_accurate(run[r], ad[r]);
            ad[r] = make_float2(0.f, 0.f);
          }
        }
        cp += 32;
        vp += 32 * BR * BC;
      }
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        if constexpr (ACC) acc[r] = df_to_double(run[r]);
        else acc[r] += df_to_double(ad[r]);
      }
    } else {
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
  }
  epi(sell_row(A.perm, pos, A.n_rows), acc, sh);
}

// df: use the split copy when the matrix has one (false: plain FP64).
// acc: the accurate double-float accumulation (outer CG products with K and
// tam_matrix_spmv; the V-cycle's smoothing SpMVs keep the faster running sum).
template <int BR, int BC, class Epi>
void sell_spmv(const Sell& A, const double* x, Epi epi, cudaStream_t s, bool df = true, bool acc = false) {
  unsigned grid = grid_for((long long)A.n_slices * 32, SPMV_THREADS);
  if (df && A.vals_df.p && acc)
    sell_spmv_kernel<BR, BC, Epi, true, true><<<grid, SPMV_THREADS, 0, s>>>(view(A), x, epi);
  else if (df && A.vals_df.p)
    sell_spmv_kernel<BR, BC, Epi, true><<<grid, SPMV_THREADS, 0, s>>>(view(A), x, epi);
  else
    sell_spmv_kernel<BR, BC, Epi, false><<<grid, SPMV_THREADS, 0, s>>>(view(A), x, epi);
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
  const float2* __restrict__ v_df;
};

// CNT consecutive 8-byte values of one block into registers: 16-byte loads
// when CNT is even (block starts are then 16-byte aligned: CNT * 8 * p),
// else 8-byte loads.
template <int CNT, typename V>
__device__ __forceinline__ void block_load(const V* __restrict__ p, V (&out)[CNT]) {
  static_assert(sizeof(V) == 8, "block_load: 8-byte values");
  if constexpr (CNT % 2 == 0) {
    if constexpr (std::is_same<V, double>::value) {
      const double2* __restrict__ p2 = reinterpret_cast<const double2*>(p);
#pragma unroll
      for (int i = 0; i < CNT / 2; ++i) {
        const double2 v = __ldg(p2 + i);
        out[2 * i] = v.x;
        out[2 * i + 1] = v.y;
      }
    } else {
      const float4* __restrict__ p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
      for (int i = 0; i < CNT / 2; ++i) {
        const float4 v = __ldg(p4 + i);
        out[2 * i] = make_float2(v.x, v.y);
        out[2 * i + 1] = make_float2(v.z, v.w);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < CNT; ++i) out[i] = __ldg(p + i);
  }
}

template <int BR, int BC, int LPR, class Epi, bool DF>
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
    if constexpr (DF) {
      float2 ad[BR];
#pragma unroll
      for (int r = 0; r < BR; ++r) ad[r] = make_float2(0.f, 0.f);
      for (int p = A.rp[row] + sub; p < pe; p += LPR) {
        float2 vv[BR * BC];  // the whole block first (16-byte loads), then the gather
        block_load<BR * BC>(A.v_df + (size_t)p * BR * BC, vv);
        const int c = A.ci[p];
        float2 xv[BC];
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[j] = split_bits(__ldg(x + (size_t)c * BC + j));
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int j = 0; j < BC; ++j) df_fma(ad[r], vv[r * BC + j], xv[j]);
      }
#pragma unroll
      for (int r = 0; r < BR; ++r) acc[r] = df_to_double(ad[r]);
    } else {
      for (int p = A.rp[row] + sub; p < pe; p += LPR) {
        double vv[BR * BC];
        block_load<BR * BC>(A.v + (size_t)p * BR * BC, vv);
        const int c = A.ci[p];
        double xv[BC];
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int j = 0; j < BC; ++j) acc[r] = fma(vv[r * BC + j], xv[j], acc[r]);
      }
    }
  }
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1)
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  epi((sub == 0 && row < A.n_rows) ? row : A.n_rows, acc, sh);
}

// Lanes-per-row storage: each row's blocks in groups of lpr, a group stored
// element-major (value e of the group's block j at vals[(g * bb + e) * lpr + j])
// so that the lpr lanes of a row read lpr consecutive values per load -- with
// the plain block-CSR arrays each lane reads its own block and a warp's load
// touches 32 separate sectors.  Rows are padded to whole groups with zero
// blocks whose column is the row's last (so no new column is read).
struct LprStore {
  int lpr = 0, n_rows = 0, br = 0, bc = 0;
  long long n_groups = 0;
  DBuf<int> grp_ptr;     // [n_rows + 1], in groups
  DBuf<int> cols;        // [n_groups * lpr]
  DBuf<double> vals;     // [n_groups * lpr * br * bc]
  DBuf<float2> vals_df;  // optional split copy
};

// Builds L from A for lanes-per-row width lpr (and the split copy when df).
void build_lpr_store(const Bsr& A, int lpr, bool df, LprStore& L, cudaStream_t s);
// The interleaved store pays for 2..8 lanes per row (level-1 Chebyshev 177 ->
// 111 us on the 3.2M-DOF box); the 16- and 32-lane launches on the smallest
// levels ran 1.6x slower with it and keep the block-CSR arrays.
inline bool lpr_store_pays(int lpr) { return lpr >= 2 && lpr <= 8; }

struct LprView {
  int n_rows;
  const int* __restrict__ gp;
  const int* __restrict__ cols;
  const double* __restrict__ v;
  const float2* __restrict__ v_df;
};

template <int BR, int BC, int LPR, class Epi, bool DF>
__global__ void __launch_bounds__(SPMV_THREADS)
lpr_spmv_kernel(LprView A, const double* __restrict__ x, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int t = blockIdx.x * SPMV_THREADS + threadIdx.x;
  const int row = t / LPR, sub = t % LPR;
  constexpr int BB = BR * BC;
  double acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.0;
  [[maybe_unused]] float2 ad[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) ad[r] = make_float2(0.f, 0.f);
  if (row < A.n_rows) {
    const int g0 = A.gp[row], g1 = A.gp[row + 1];
    if constexpr (DF) {
      // the x gather runs one group ahead: the next group's column and x
      // entries are requested before this group's products, so that they
      // arrive together with the next group's values (one memory round trip
      // per group instead of values, then column and gather)
      double xg[BC];
      if (g0 < g1) {
        const int c = __ldg(A.cols + (size_t)g0 * LPR + sub);
#pragma unroll
        for (int j = 0; j < BC; ++j) xg[j] = __ldg(x + (size_t)c * BC + j);
      }
      for (int g = g0; g < g1; ++g) {
        const float2* __restrict__ vb = A.v_df + (size_t)g * BB * LPR + sub;
        float2 vv[BB];
#pragma unroll
        for (int e = 0; e < BB; ++e) vv[e] = __ldg(vb + e * LPR);
        float2 xv[BC];
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[j] = split_bits(xg[j]);
        if (g + 1 < g1) {
          const int c = __ldg(A.cols + (size_t)(g + 1) * LPR + sub);
#pragma unroll
          for (int j = 0; j < BC; ++j) xg[j] = __ldg(x + (size_t)c * BC + j);
        }
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int j = 0; j < BC; ++j) df_fma(ad[r], vv[r * BC + j], xv[j]);
      }
    } else {
      for (int g = g0; g < g1; ++g) {
        const double* __restrict__ vb = A.v + (size_t)g * BB * LPR + sub;
        double vv[BB];
#pragma unroll
        for (int e = 0; e < BB; ++e) vv[e] = __ldg(vb + e * LPR);
        const int c = __ldg(A.cols + (size_t)g * LPR + sub);
        double xv[BC];
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int j = 0; j < BC; ++j) acc[r] = fma(vv[r * BC + j], xv[j], acc[r]);
      }
    }
  }
  if constexpr (DF) {
    // the lanes' partial sums combined in double-float (FP32 work: an FP64
    // butterfly costs every lane log2(LPR) FP64 adds per row component)
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < BR; ++r)
        df_add(ad[r], make_float2(__shfl_xor_sync(0xffffffffu, ad[r].x, o), __shfl_xor_sync(0xffffffffu, ad[r].y, o)));
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] = df_to_double(ad[r]);
  } else {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  }
  epi((sub == 0 && row < A.n_rows) ? row : A.n_rows, acc, sh);
}

// Few long rows (the coarse operators and their transfer operators): TPR
// threads per row -- one to eight whole warps -- over the 8-lane interleaved
// store, so that a level of a few hundred or thousand rows still spreads over
// the SMs and every load is sector-coalesced.  Thread sub of a row takes lane
// sub % 8 of the row's groups sub / 8, sub / 8 + TPR / 8, ...; each warp
// reduces with shuffles and the row's warps meet in shared memory, summed in
// warp order (deterministic).
constexpr int ROWS_LPR = 8;
constexpr int SPMV_ROW_THREADS = 256;

template <int BR, int BC, int TPR, class Epi, bool DF>
__global__ void __launch_bounds__(SPMV_ROW_THREADS)
lpr_rows_kernel(LprView A, const double* __restrict__ x, Epi epi) {
  static_assert(TPR % 32 == 0 && SPMV_ROW_THREADS % TPR == 0, "lpr_rows_kernel: whole warps per row");
  constexpr int BB = BR * BC, GS = TPR / ROWS_LPR;
  using P = typename std::conditional<DF, float2, double>::type;  // partial sums
  __shared__ double sh[32];
  __shared__ P part[SPMV_ROW_THREADS / 32][BR];
  if (epi.skip()) return;  // block-uniform (a device flag)
  const int row = blockIdx.x * (SPMV_ROW_THREADS / TPR) + threadIdx.x / TPR;
  const int sub = threadIdx.x % TPR, ln = sub % ROWS_LPR, wid = threadIdx.x >> 5;
  double acc[BR];
  if constexpr (DF) {
    // the closing reduction stays in double-float too: FP64 adds would make
    // the FP64 pipe the limit again on these short per-thread sums
    float2 ad[BR];
#pragma unroll
    for (int r = 0; r < BR; ++r) ad[r] = make_float2(0.f, 0.f);
    if (row < A.n_rows) {
      const int g1 = A.gp[row + 1];
      for (int g = A.gp[row] + sub / ROWS_LPR; g < g1; g += GS) {
        const float2* __restrict__ vb = A.v_df + (size_t)g * BB * ROWS_LPR + ln;
        float2 vv[BB];
#pragma unroll
        for (int e = 0; e < BB; ++e) vv[e] = __ldg(vb + e * ROWS_LPR);
        const int c = __ldg(A.cols + (size_t)g * ROWS_LPR + ln);
        float2 xv[BC];
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[j] = split_bits(__ldg(x + (size_t)c * BC + j));
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int j = 0; j < BC; ++j) df_fma(ad[r], vv[r * BC + j], xv[j]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < BR; ++r)
        df_add(ad[r], make_float2(__shfl_xor_sync(0xffffffffu, ad[r].x, o), __shfl_xor_sync(0xffffffffu, ad[r].y, o)));
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int r = 0; r < BR; ++r) part[wid][r] = ad[r];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < BR; ++r) {
      acc[r] = 0.0;
      if (sub == 0) {  // the row's first warp: part[wid .. wid + TPR / 32) are its warps
        float2 t = part[wid][r];
#pragma unroll
        for (int w = 1; w < TPR / 32; ++w) df_add(t, part[wid + w][r]);
        acc[r] = df_to_double(t);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < BR; ++r) acc[r] = 0.0;
    if (row < A.n_rows) {
      const int g1 = A.gp[row + 1];
      for (int g = A.gp[row] + sub / ROWS_LPR; g < g1; g += GS) {
        const double* __restrict__ vb = A.v + (size_t)g * BB * ROWS_LPR + ln;
        double vv[BB];
#pragma unroll
        for (int e = 0; e < BB; ++e) vv[e] = __ldg(vb + e * ROWS_LPR);
        const int c = __ldg(A.cols + (size_t)g * ROWS_LPR + ln);
        double xv[BC];
#pragma unroll
        for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
        for (int r = 0; r < BR; ++r)
#pragma unroll
          for (int j = 0; j < BC; ++j) acc[r] = fma(vv[r * BC + j], xv[j], acc[r]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < BR; ++r) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int r = 0; r < BR; ++r) part[wid][r] = acc[r];
    __syncthreads();
    if (sub == 0)
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        double t = part[wid][r];
#pragma unroll
        for (int w = 1; w < TPR / 32; ++w) t += part[wid + w][r];
        acc[r] = t;
      }
  }
  epi((sub == 0 && row < A.n_rows) ? row : A.n_rows, acc, sh);
}

// Block-row lanes (the coarse levels' 6x6 operators): BR lanes per block,
// lane r of a group multiplies row r of the block by x_c, so a warp step
// covers G = 32 / BR consecutive blocks of a row, each lane reading its BC
// values with 16-byte loads from the block-CSR arrays (a row's blocks are
// contiguous: one coalesced span per step).  Lane r of a group loads and
// splits x_c[r] only; the group shares the column's BC entries by shuffles.
// Used for the 6x6 operators with few long rows (coarse levels, restrictions)
// or short rows (coarse prolongations); the level-1-like operators with many
// medium rows keep the 8-lane store, whose six independent row sums per lane
// ran 20% faster there.
// WPR warps per row take every WPR-th step.  No thread holds a whole block,
// so the kernel runs at ~50 registers and many warps per SM hide the gather
// latency (the 8-lane and whole-warp-row kernels hold 36 values per thread:
// 128 registers, a quarter of the warps).  Sums: a lane's own blocks in
// order (even and odd columns apart, then together), then the groups of a
// warp in order, then the row's warps in order.
constexpr int BLOCKROW_THREADS = 256;

template <int BR, int BC, int WPR, class Epi, bool DF>
__global__ void __launch_bounds__(BLOCKROW_THREADS)
blockrow_spmv_kernel(BsrView A, const double* __restrict__ x, Epi epi) {
  static_assert(BC <= BR && BR <= 32 && (BLOCKROW_THREADS / 32) % WPR == 0, "blockrow_spmv_kernel: shape");
  constexpr int G = 32 / BR, W = BLOCKROW_THREADS / 32, RPB = W / WPR, BB = BR * BC;
  using P = typename std::conditional<DF, float2, double>::type;
  __shared__ double sh[32];
  __shared__ P part[W][BR];
  if (epi.skip()) return;  // block-uniform (a device flag)
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * RPB + wid / WPR, wr = wid % WPR;
  const int g = lane / BR, r = lane - g * BR;
  const bool act = g < G;
  P ad;
  if constexpr (DF) ad = make_float2(0.f, 0.f);
  else ad = 0.0;
  if (row < A.n_rows) {  // warp-uniform
    // two accumulators (even and odd j) halve the dependent chain of
    // double-float updates per step
    P ad1;
    if constexpr (DF) ad1 = make_float2(0.f, 0.f);
    else ad1 = 0.0;
    const int p1 = A.rp[row + 1];
    // x entry one step ahead: the next step's column and x are requested
    // before this step's products
    double xn = 0.0;
    {
      const int pf = A.rp[row] + wr * G + g;
      if (act && pf < p1 && r < BC) xn = __ldg(x + (size_t)__ldg(A.ci + pf) * BC + r);
    }
    for (int base = A.rp[row] + wr * G; base < p1; base += WPR * G) {
      const int p = base + g;
      const bool has = act && p < p1;
      const double xr = xn;
      {
        const int pf = p + WPR * G;
        xn = 0.0;
        if (act && pf < p1 && r < BC) xn = __ldg(x + (size_t)__ldg(A.ci + pf) * BC + r);
      }
      if constexpr (DF) {
        float2 v[BC];
        if (has) block_load<BC>(A.v_df + (size_t)p * BB + r * BC, v);
        const float2 xs = split_bits(xr);
#pragma unroll
        for (int j = 0; j < BC; ++j) {
          const float2 xj = make_float2(__shfl_sync(0xffffffffu, xs.x, g * BR + j),
                                        __shfl_sync(0xffffffffu, xs.y, g * BR + j));
          if (has) df_fma((j & 1) ? ad1 : ad, v[j], xj);
        }
      } else {
        double v[BC];
        if (has) block_load<BC>(A.v + (size_t)p * BB + r * BC, v);
#pragma unroll
        for (int j = 0; j < BC; ++j) {
          const double xj = __shfl_sync(0xffffffffu, xr, g * BR + j);
          if (has) {
            if (j & 1) ad1 = fma(v[j], xj, ad1);
            else ad = fma(v[j], xj, ad);
          }
        }
      }
    }
    if constexpr (DF) df_add(ad, ad1);
    else ad += ad1;
  }
  // groups of the warp, in order, into lanes 0 .. BR-1
#pragma unroll
  for (int gg = 1; gg < G; ++gg) {
    if constexpr (DF) {
      const float2 o = make_float2(__shfl_sync(0xffffffffu, ad.x, gg * BR + r),
                                   __shfl_sync(0xffffffffu, ad.y, gg * BR + r));
      if (lane < BR) df_add(ad, o);
    } else {
      const double o = __shfl_sync(0xffffffffu, ad, gg * BR + r);
      if (lane < BR) ad += o;
    }
  }
  if constexpr (WPR > 1) {
    if (lane < BR) part[wid][lane] = ad;
    __syncthreads();
    if (wr == 0 && lane < BR)
#pragma unroll
      for (int w = 1; w < WPR; ++w) {
        if constexpr (DF) df_add(ad, part[wid + w][lane]);
        else ad += part[wid + w][lane];
      }
  }
  double acc[BR];
#pragma unroll
  for (int k = 0; k < BR; ++k) {
    if constexpr (DF) {
      const float2 t = make_float2(__shfl_sync(0xffffffffu, ad.x, k), __shfl_sync(0xffffffffu, ad.y, k));
      acc[k] = df_to_double(t);
    } else {
      acc[k] = __shfl_sync(0xffffffffu, ad, k);
    }
  }
  const bool lead = wr == 0 && lane == 0 && row < A.n_rows;
  epi(lead ? row : A.n_rows, acc, sh);
}

// Warps per row for blockrow_spmv_kernel: enough warps for two waves of 32
// resident warps per SM, while each warp keeps at least four steps.
inline int blockrow_wpr(int n_rows, long long nnzb, int br) {
  if (n_rows <= 0) return 1;
  const long long want = 2LL * sm_count() * 32;
  const double steps = (double)nnzb / n_rows / (32 / br);
  int w = 1;
  while (w < 8 && (long long)n_rows * w < want && steps / (2 * w) >= 4.0) w <<= 1;
  return w;
}

// A sparse operator with its SpMV strategy: SELL-32 thread-per-row (lpr == 0)
// or LPR lanes per row (over the interleaved store L when built, else over the
// Bsr arrays).
struct SpOp {
  const Bsr* B = nullptr;
  const Sell* S = nullptr;
  int lpr = 0;
  bool df = true;  // use the storage's split copy when it has one
  const LprStore* L = nullptr;
  int tpr = 0;     // > 0: lpr_rows_kernel with tpr threads per row over L (an 8-lane store)
  int brw = 0;     // > 0: blockrow_spmv_kernel with brw warps per row over B (lpr and L unused)
};

// Threads that fill the GPU (1,024 per SM) for the SpMV layout choices.
inline long long spmv_fill_threads() {
  static long long fill = 0;
  if (fill == 0) {
    int dev = 0, n_sm = 0;
    TAM_CUDA(cudaGetDevice(&dev));
    TAM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    fill = (long long)std::max(1, n_sm) * 1024;
  }
  return fill;
}

// Threads per row for lpr_rows_kernel, or 0: whole warps per row for the
// operators that choose_lpr leaves at 16-32 lanes (too few rows to fill the
// GPU at 8 lanes each), as many warps as fill it while every thread keeps at
// least one block.
inline int rows_tpr(int n_rows, long long nnzb, int lpr) {
  const long long fill = spmv_fill_threads();
  if (lpr < 16 || n_rows <= 0) return 0;
  const double avg = (double)nnzb / n_rows;
  int t = 0;
  for (int c = 32; c <= SPMV_ROW_THREADS && avg >= c; c <<= 1) {
    t = c;
    if ((long long)n_rows * c >= fill) break;
  }
  return t;
}

// Double-float pays where an operator is large enough to be bound by memory;
// on small operators (coarse levels) each lane's short dependent chain makes
// the 12x FP32 instruction count a latency cost (measured up to 2x slower).
// mode: amg_params.spmv_fp64 (0 auto, 1 never, 2 always).
inline bool use_df(const Bsr& A, int mode) {
  if (mode == 1) return false;
  if (mode == 2) return true;
  return A.nnzb >= (1LL << 20);
}

// Strategy: thread-per-row SELL for many short rows, else lanes per row.
// Each lane should own >= ~16 blocks: the closing shuffle reduction costs
// log2(LPR) FP64 adds per output per lane, and on GB300 the FP64 pipe (not
// bandwidth) is the limit, so a wide LPR on medium rows wastes it.
inline int choose_lpr(const Bsr& A) {
  const double avg = A.n_rows > 0 ? (double)A.nnzb / A.n_rows : 0.0;
  if (A.n_rows >= 65536 && avg <= 48.0) return 0;
  int l = 2;
  // few rows (coarse levels): at least 8 blocks per lane is enough to hide
  // the reduction; the extra lanes are what keeps the SMs busy there
  const int per_lane = A.n_rows < 65536 ? 8 : 16;
  while (l < 32 && per_lane * l < avg) l <<= 1;
  if (A.n_rows < 8192) l = std::max(l, 16);  // few rows: spread them over more lanes
  // rows enough to fill the GPU at 8 lanes each: the coalesced 8-lane
  // interleaved store beats 16-32 lanes over the block-CSR arrays
  if (l > 8 && (long long)A.n_rows * 8 >= spmv_fill_threads()) l = 8;
  return l;
}

inline unsigned spop_grid(const SpOp& op) {
  if (op.lpr == 0) return sell_grid(*op.S);
  return grid_for((long long)op.B->n_rows * op.lpr, SPMV_THREADS);
}

template <int BR, int BC, class Epi, bool DF>
void bsr_vector_launch(const SpOp& op, const BsrView& v, const double* x, Epi epi, cudaStream_t s) {
  const unsigned g = spop_grid(op);
  switch (op.lpr) {
    case 2: bsr_vector_kernel<BR, BC, 2, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 4: bsr_vector_kernel<BR, BC, 4, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 8: bsr_vector_kernel<BR, BC, 8, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 16: bsr_vector_kernel<BR, BC, 16, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    default: bsr_vector_kernel<BR, BC, 32, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
  }
  TAM_LAUNCH_CHECK();
}

template <int BR, int BC, class Epi, bool DF>
void lpr_launch(const SpOp& op, const LprView& v, const double* x, Epi epi, cudaStream_t s) {
  const unsigned g = spop_grid(op);
  switch (op.lpr) {
    case 2: lpr_spmv_kernel<BR, BC, 2, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 4: lpr_spmv_kernel<BR, BC, 4, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 8: lpr_spmv_kernel<BR, BC, 8, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    case 16: lpr_spmv_kernel<BR, BC, 16, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
    default: lpr_spmv_kernel<BR, BC, 32, Epi, DF><<<g, SPMV_THREADS, 0, s>>>(v, x, epi); break;
  }
  TAM_LAUNCH_CHECK();
}

template <int BR, int BC, class Epi, bool DF>
void rows_launch(const SpOp& op, const LprView& v, const double* x, Epi epi, cudaStream_t s) {
  TAM_CHECK(op.L->lpr == ROWS_LPR, TAM_ERR_INTERNAL, "spmv: whole-warp rows need the 8-lane store");
  const unsigned g = grid_for(v.n_rows, SPMV_ROW_THREADS / op.tpr);
  switch (op.tpr) {
    case 32: lpr_rows_kernel<BR, BC, 32, Epi, DF><<<g, SPMV_ROW_THREADS, 0, s>>>(v, x, epi); break;
    case 64: lpr_rows_kernel<BR, BC, 64, Epi, DF><<<g, SPMV_ROW_THREADS, 0, s>>>(v, x, epi); break;
    case 128: lpr_rows_kernel<BR, BC, 128, Epi, DF><<<g, SPMV_ROW_THREADS, 0, s>>>(v, x, epi); break;
    case 256: lpr_rows_kernel<BR, BC, 256, Epi, DF><<<g, SPMV_ROW_THREADS, 0, s>>>(v, x, epi); break;
    default: throw Error(TAM_ERR_INTERNAL, "spmv: threads per row must be 32, 64, 128 or 256");
  }
  TAM_LAUNCH_CHECK();
}

template <int BR, int BC, class Epi, bool DF>
void blockrow_launch(const SpOp& op, const BsrView& v, const double* x, Epi epi, cudaStream_t s) {
  if constexpr (BC <= BR && BR >= 2) {
    const unsigned g = grid_for(v.n_rows, (BLOCKROW_THREADS / 32) / op.brw);
    switch (op.brw) {
      case 1: blockrow_spmv_kernel<BR, BC, 1, Epi, DF><<<g, BLOCKROW_THREADS, 0, s>>>(v, x, epi); break;
      case 2: blockrow_spmv_kernel<BR, BC, 2, Epi, DF><<<g, BLOCKROW_THREADS, 0, s>>>(v, x, epi); break;
      case 4: blockrow_spmv_kernel<BR, BC, 4, Epi, DF><<<g, BLOCKROW_THREADS, 0, s>>>(v, x, epi); break;
      case 8: blockrow_spmv_kernel<BR, BC, 8, Epi, DF><<<g, BLOCKROW_THREADS, 0, s>>>(v, x, epi); break;
      default: throw Error(TAM_ERR_INTERNAL, "spmv: block-row lanes need 1, 2, 4 or 8 warps per row");
    }
    TAM_LAUNCH_CHECK();
  } else {
    throw Error(TAM_ERR_INTERNAL, "spmv: block-row lanes need a block at least as tall as wide");
  }
}

template <int BR, int BC, class Epi>
void spop_apply(const SpOp& op, const double* x, Epi epi, cudaStream_t s) {
  if (op.brw) {
    const BsrView v{op.B->n_rows, op.B->row_ptr.p, op.B->col_idx.p, op.B->vals.p, op.B->vals_df.p};
    if (op.df && v.v_df)
      blockrow_launch<BR, BC, Epi, true>(op, v, x, epi, s);
    else
      blockrow_launch<BR, BC, Epi, false>(op, v, x, epi, s);
    return;
  }
  if (op.lpr == 0) {
    sell_spmv<BR, BC>(*op.S, x, epi, s, op.df);
    return;
  }
  if (op.L && op.tpr) {
    const LprView v{op.L->n_rows, op.L->grp_ptr.p, op.L->cols.p, op.L->vals.p, op.L->vals_df.p};
    if (op.df && v.v_df)
      rows_launch<BR, BC, Epi, true>(op, v, x, epi, s);
    else
      rows_launch<BR, BC, Epi, false>(op, v, x, epi, s);
    return;
  }
  if (op.L) {
    const LprView v{op.L->n_rows, op.L->grp_ptr.p, op.L->cols.p, op.L->vals.p, op.L->vals_df.p};
    if (op.df && v.v_df)
      lpr_launch<BR, BC, Epi, true>(op, v, x, epi, s);
    else
      lpr_launch<BR, BC, Epi, false>(op, v, x, epi, s);
    return;
  }
  const BsrView v{op.B->n_rows, op.B->row_ptr.p, op.B->col_idx.p, op.B->vals.p, op.B->vals_df.p};
  if (op.df && v.v_df)
    bsr_vector_launch<BR, BC, Epi, true>(op, v, x, epi, s);
  else
    bsr_vector_launch<BR, BC, Epi, false>(op, v, x, epi, s);
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
                     const TV* __restrict__ vals, const float* __restrict__ x, const int* __restrict__ perm,
                     int n_rows, Epi epi) {
  __shared__ double sh[32];
  if (epi.skip()) return;
  const int pos = blockIdx.x * SPMV_THREADS + threadIdx.x;
  const int slice = pos >> 5, lane = pos & 31;
  float acc[BR];
#pragma unroll
  for (int r = 0; r < BR; ++r) acc[r] = 0.f;
  if (slice < n_slices) {
    const int k0 = slice_ptr[slice], k1 = slice_ptr[slice + 1];
    const int* __restrict__ cp = cols + (size_t)k0 * 32 + lane;
    const TV* __restrict__ vp = vals + (size_t)k0 * 32 * BR * BC + lane;
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
      TV vv[BR * BC];  // the slot's values first, then the gather
#pragma unroll
      for (int e = 0; e < BR * BC; ++e) vv[e] = vp[e * 32];
      const int c = __ldg(cp);
      float xv[BC];
#pragma unroll
      for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int j = 0; j < BC; ++j) acc[r] = fmaf(to_f32(vv[r * BC + j]), xv[j], acc[r]);
      cp += 32;
      vp += 32 * BR * BC;
    }
  }
  epi(sell_row(perm, pos, n_rows), acc, sh);
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
      const TV* __restrict__ vb = v + (size_t)p * BR * BC;
      TV vv[BR * BC];  // the block's values first, then the gather
#pragma unroll
      for (int e = 0; e < BR * BC; ++e) vv[e] = vb[e];
      const int c = ci[p];
      float xv[BC];
#pragma unroll
      for (int j = 0; j < BC; ++j) xv[j] = __ldg(x + (size_t)c * BC + j);
#pragma unroll
      for (int r = 0; r < BR; ++r)
#pragma unroll
        for (int j = 0; j < BC; ++j) acc[r] = fmaf(to_f32(vv[r * BC + j]), xv[j], acc[r]);
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
                                                                     S.perm.p, S.n_rows, epi);
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
