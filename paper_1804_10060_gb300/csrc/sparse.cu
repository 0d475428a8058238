// Block-sparse building blocks of the AMG setup: SELL-32 conversion, block
// transpose and the block SpGEMM C = X * Y used for A P_tent and R (A P).
#include <algorithm>

#include <type_traits>

#include "sparse.cuh"

namespace tam {

// ---------------------------------------------------------------------------
// SELL-32 conversion
// ---------------------------------------------------------------------------
namespace {

__global__ void sell_slice_len_kernel(const int* __restrict__ row_ptr, int n_rows, int n_slices,
                                      const int* __restrict__ perm, int* __restrict__ len) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slices) return;
  int m = 0;
  int p1 = min(32 * s + 32, n_rows);
  for (int p = 32 * s; p < p1; ++p) {
    const int r = perm ? perm[p] : p;
    m = max(m, row_ptr[r + 1] - row_ptr[r]);
  }
  len[s] = m;
}

// Row order for SELL-C-sigma: within each window of 256 positions, rows by
// decreasing length (ties by row index, so the order is deterministic).  One
// block of 256 threads per window; each thread ranks its row by counting.
__global__ void __launch_bounds__(256) sell_sort_window_kernel(const int* __restrict__ row_ptr, int n_rows,
                                                               int* __restrict__ perm) {
  __shared__ int slen[256];
  const int base = blockIdx.x * 256, t = threadIdx.x, r = base + t;
  const int len = r < n_rows ? row_ptr[r + 1] - row_ptr[r] : -1;
  slen[t] = len;
  __syncthreads();
  if (r >= n_rows) return;
  int rank = 0;
  for (int j = 0; j < 256; ++j) {
    const int lj = slen[j];
    rank += (lj > len) || (lj == len && j < t);
  }
  perm[base + rank] = r;
}

// One thread per (slice, lane).  Pads a row with zero blocks pointing at the
// row's last real column (keeps the padded x reads local).
__global__ void sell_fill_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                                 const double* __restrict__ vals, int n_rows, int n_slices, int bb,
                                 const int* __restrict__ slice_ptr, const int* __restrict__ perm,
                                 int* __restrict__ scols, double* __restrict__ svals, float2* __restrict__ svals_df,
                                 bool with_pattern) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int s = t >> 5, lane = t & 31;
  if (s >= n_slices) return;
  int row = (perm && t < n_rows) ? perm[t] : t;
  int rp = 0, len = 0;
  if (row < n_rows) {
    rp = row_ptr[row];
    len = row_ptr[row + 1] - rp;
  }
  int k0 = slice_ptr[s], K = slice_ptr[s + 1] - k0;
  int lastc = len > 0 ? col_idx[rp + len - 1] : 0;
  for (int k = 0; k < K; ++k) {
    size_t slot = (size_t)(k0 + k);
    if (with_pattern) scols[slot * 32 + lane] = k < len ? col_idx[rp + k] : lastc;
    for (int e = 0; e < bb; ++e) {
      const double x = k < len ? vals[((size_t)rp + k) * bb + e] : 0.0;
      svals[(slot * bb + e) * 32 + lane] = x;
      if (svals_df) svals_df[(slot * bb + e) * 32 + lane] = split_bits(x);  // the split copy in the same pass
    }
  }
}

}  // namespace

void bsr_to_sell(const Bsr& A, Sell& S, cudaStream_t s, bool df) {
  TAM_CHECK(A.n_cols > 0, TAM_ERR_INTERNAL, "SELL of a matrix without columns");
  S.n_rows = A.n_rows;
  S.br = A.br;
  S.bc = A.bc;
  S.n_slices = (A.n_rows + 31) / 32;
  S.slice_ptr = DBuf<int>((size_t)S.n_slices + 1, s);
  sell_slice_len_kernel<<<grid_for(S.n_slices, 256), 256, 0, s>>>(A.row_ptr.p, A.n_rows, S.n_slices, nullptr,
                                                                  S.slice_ptr.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i32(S.slice_ptr.p, S.slice_ptr.p, S.n_slices, s);
  S.n_slots = read_back_int(S.slice_ptr.p + S.n_slices, s);
  if ((double)S.n_slots * 32.0 > 1.10 * (double)A.nnzb) {
    // more than 10% padding in row order: sort rows by length within windows
    S.perm = DBuf<int>((size_t)A.n_rows, s);
    sell_sort_window_kernel<<<(A.n_rows + 255) / 256, 256, 0, s>>>(A.row_ptr.p, A.n_rows, S.perm.p);
    TAM_LAUNCH_CHECK();
    sell_slice_len_kernel<<<grid_for(S.n_slices, 256), 256, 0, s>>>(A.row_ptr.p, A.n_rows, S.n_slices, S.perm.p,
                                                                    S.slice_ptr.p);
    TAM_LAUNCH_CHECK();
    exclusive_scan_i32(S.slice_ptr.p, S.slice_ptr.p, S.n_slices, s);
    S.n_slots = read_back_int(S.slice_ptr.p + S.n_slices, s);
  }
  S.cols = DBuf<int>((size_t)S.n_slots * 32, s);
  S.vals = DBuf<double>((size_t)S.n_slots * 32 * A.block_elems(), s);
  if (df) S.vals_df = DBuf<float2>((size_t)std::max(1LL, S.n_slots * 32 * (long long)A.block_elems()), s);
  sell_fill_kernel<<<grid_for((long long)S.n_slices * 32, 256), 256, 0, s>>>(
      A.row_ptr.p, A.col_idx.p, A.vals.p, A.n_rows, S.n_slices, (int)A.block_elems(),
      S.slice_ptr.p, S.perm.p, S.cols.p, S.vals.p, df ? S.vals_df.p : nullptr, true);
  TAM_LAUNCH_CHECK();
}

void sell_refresh_values(const Bsr& A, Sell& S, cudaStream_t s) {
  sell_fill_kernel<<<grid_for((long long)S.n_slices * 32, 256), 256, 0, s>>>(
      A.row_ptr.p, A.col_idx.p, A.vals.p, A.n_rows, S.n_slices, (int)A.block_elems(),
      S.slice_ptr.p, S.perm.p, S.cols.p, S.vals.p, S.vals_df.p, false);
  TAM_LAUNCH_CHECK();
}

namespace {
// Largest biased FP64 exponent (out[0]; 0: none) of the entries of a
// block-CSR matrix and an inf/NaN flag (out[1]), leaving out rows that hold only their diagonal block (Dirichlet and cell-less nodes:
// identity rows whose 1.0 says nothing about the operator's scale); inf/NaN
// are flagged in every row.
__global__ void row_exponent_range_kernel(const int* __restrict__ rp, const double* __restrict__ v, int n_rows,
                                          int bb, int* __restrict__ out) {
  int emax = 0, bad = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_rows; i += gridDim.x * blockDim.x) {
    const int p0 = rp[i], p1 = rp[i + 1];
    const bool scale_row = p1 - p0 > 1;
    for (long long k = (long long)p0 * bb; k < (long long)p1 * bb; ++k) {
      const int e = (int)(((unsigned long long)__double_as_longlong(v[k]) >> 52) & 0x7ff);
      if (e == 0x7ff) bad = 1;
      else if (scale_row) emax = max(emax, e);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (emax) atomicMax(out, emax);
    if (bad) atomicOr(out + 1, 1);
  }
}
}  // namespace

void operator_exponent_range(const Bsr& A, int* max_exp, bool* finite, cudaStream_t s) {
  DBuf<int> out(2, s);
  out.zero();
  if (A.n_rows > 0) {
    row_exponent_range_kernel<<<stride_grid(A.n_rows, 256, 8), 256, 0, s>>>(A.row_ptr.p, A.vals.p, A.n_rows,
                                                                           (int)A.block_elems(), out.p);
    TAM_LAUNCH_CHECK();
  }
  int e = 0, bad = 0;
  read_back_int2(out.p, out.p + 1, &e, &bad, s);
  *max_exp = e ? e - 1023 : 0;
  *finite = bad == 0;
}

namespace {
__global__ void split_values_kernel(const double* __restrict__ in, float2* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = split_bits(in[i]);
}

void split_into(const double* in, long long n, DBuf<float2>& out, cudaStream_t s) {
  if (out.n != (size_t)std::max(1LL, n)) out = DBuf<float2>((size_t)std::max(1LL, n), s);
  if (n > 0) {
    split_values_kernel<<<stride_grid(n, 256, 16), 256, 0, s>>>(in, out.p, n);
    TAM_LAUNCH_CHECK();
  }
}
}  // namespace

namespace {
__global__ void lpr_count_kernel(const int* __restrict__ rp, int n_rows, int lpr, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_rows) cnt[i] = (rp[i + 1] - rp[i] + lpr - 1) / lpr;
}

// Row of every group (a row's groups are consecutive).
__global__ void lpr_group_row_kernel(const int* __restrict__ gp, int n_rows, int* __restrict__ grow) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  for (int g = gp[i]; g < gp[i + 1]; ++g) grow[g] = i;
}

// One warp per group: the lanes write the group's lpr columns and its
// bb * lpr values in storage order (coalesced writes), gathering from the
// block-CSR arrays; the split copy, when asked for, in the same pass.
__global__ void lpr_fill_kernel(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                                int lpr, int bb, const int* __restrict__ gp, const int* __restrict__ grow,
                                long long n_groups, int* __restrict__ cols, double* __restrict__ vals,
                                float2* __restrict__ vals_df) {
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_groups) return;
  const int i = grow[w];
  const int s0 = rp[i] + (int)(w - gp[i]) * lpr, e0 = rp[i + 1];
  const int lastc = e0 > rp[i] ? ci[e0 - 1] : 0;
  if (lane < lpr) cols[w * lpr + lane] = s0 + lane < e0 ? ci[s0 + lane] : lastc;
  const int sh = __ffs(lpr) - 1, n = bb * lpr;  // lpr a power of two
  for (int e = lane; e < n; e += 32) {
    const int idx = s0 + (e & (lpr - 1));
    const double x = idx < e0 ? v[(size_t)idx * bb + (e >> sh)] : 0.0;
    vals[w * n + e] = x;
    if (vals_df) vals_df[w * n + e] = split_bits(x);
  }
}
}  // namespace

void build_lpr_store(const Bsr& A, int lpr, bool df, LprStore& L, cudaStream_t s) {
  TAM_CHECK(lpr >= 2 && lpr <= 32 && (lpr & (lpr - 1)) == 0, TAM_ERR_INTERNAL, "lanes-per-row width must be 2..32");
  L.lpr = lpr;
  L.n_rows = A.n_rows;
  L.br = A.br;
  L.bc = A.bc;
  L.grp_ptr = DBuf<int>((size_t)A.n_rows + 1, s);
  lpr_count_kernel<<<grid_for(A.n_rows, 256), 256, 0, s>>>(A.row_ptr.p, A.n_rows, lpr, L.grp_ptr.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i32(L.grp_ptr.p, L.grp_ptr.p, A.n_rows, s);
  L.n_groups = read_back_int(L.grp_ptr.p + A.n_rows, s);
  const long long n = L.n_groups * lpr, nv = n * (long long)A.block_elems();
  L.cols = DBuf<int>((size_t)std::max(1LL, n), s);
  L.vals = DBuf<double>((size_t)std::max(1LL, nv), s);
  if (df) L.vals_df = DBuf<float2>((size_t)std::max(1LL, nv), s);
  if (L.n_groups == 0) return;
  DBuf<int> grow((size_t)L.n_groups, s);
  lpr_group_row_kernel<<<grid_for(A.n_rows, 256), 256, 0, s>>>(L.grp_ptr.p, A.n_rows, grow.p);
  TAM_LAUNCH_CHECK();
  lpr_fill_kernel<<<grid_for(L.n_groups * 32, 256), 256, 0, s>>>(
      A.row_ptr.p, A.col_idx.p, A.vals.p, lpr, (int)A.block_elems(), L.grp_ptr.p, grow.p, L.n_groups, L.cols.p,
      L.vals.p, df ? L.vals_df.p : nullptr);
  TAM_LAUNCH_CHECK();
}

void build_df_values(Sell& S, cudaStream_t s) {
  split_into(S.vals.p, S.n_slots * 32 * (long long)S.br * S.bc, S.vals_df, s);
}

void build_df_values(Bsr& B, cudaStream_t s) {
  split_into(B.vals.p, B.nnzb * (long long)B.block_elems(), B.vals_df, s);
}

// ---------------------------------------------------------------------------
// Transpose
// ---------------------------------------------------------------------------
namespace {

__global__ void count_cols_kernel(const int* __restrict__ col_idx, long long nnzb, int* __restrict__ cnt) {
  long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nnzb) atomicAdd(&cnt[col_idx[b]], 1);
}

__global__ void transpose_scatter_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                                         int n_rows, const int* __restrict__ rt_ptr, int* __restrict__ cursor,
                                         int* __restrict__ tkey, int* __restrict__ tsrc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
    int c = col_idx[b];
    int pos = rt_ptr[c] + atomicAdd(&cursor[c], 1);
    tkey[pos] = i;
    tsrc[pos] = b;
  }
}

// Warp per transposed row: the rank of each (unique) key among its row gives
// its sorted slot -- deterministic regardless of the scatter order.
__global__ void transpose_rank_kernel(const int* __restrict__ rt_ptr, int n_rt, const int* __restrict__ tkey,
                                      const int* __restrict__ tsrc, int* __restrict__ out_col,
                                      int* __restrict__ out_src) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n_rt) return;
  int s = rt_ptr[w], e = rt_ptr[w + 1];
  for (int p = s + lane; p < e; p += 32) {
    int key = tkey[p];
    int rank = 0;
    for (int q = s; q < e; ++q) rank += (tkey[q] < key);
    out_col[s + rank] = key;
    out_src[s + rank] = tsrc[p];
  }
}

// the block shape as template parameters: the index arithmetic divides by
// constants (a 64-bit division by a runtime value costs ~100 instructions)
template <int BR, int BC>
__global__ void transpose_vals_kernel(const double* __restrict__ vals, const int* __restrict__ src, long long nnzb,
                                      double* __restrict__ out) {
  constexpr int BB = BR * BC;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzb * BB) return;
  const long long b = t / BB;
  const int e = (int)(t - b * BB);
  const int r = e / BR, c = e - r * BR;  // output block is BC x BR: element (r, c) = input (c, r)
  out[t] = vals[(size_t)src[b] * BB + (size_t)c * BC + r];
}

}  // namespace

void bsr_transpose(const Bsr& A, Bsr& R, cudaStream_t s) {
  R.n_rows = A.n_cols;
  R.n_cols = A.n_rows;
  R.br = A.bc;
  R.bc = A.br;
  R.nnzb = A.nnzb;
  R.row_ptr = DBuf<int>((size_t)R.n_rows + 1, s);
  R.row_ptr.zero();
  count_cols_kernel<<<grid_for(A.nnzb, 256), 256, 0, s>>>(A.col_idx.p, A.nnzb, R.row_ptr.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i32(R.row_ptr.p, R.row_ptr.p, R.n_rows, s);
  DBuf<int> cursor((size_t)R.n_rows, s), tkey((size_t)A.nnzb, s), tsrc((size_t)A.nnzb, s), src((size_t)A.nnzb, s);
  cursor.zero();
  transpose_scatter_kernel<<<grid_for(A.n_rows, 256), 256, 0, s>>>(A.row_ptr.p, A.col_idx.p, A.n_rows,
                                                                  R.row_ptr.p, cursor.p, tkey.p, tsrc.p);
  TAM_LAUNCH_CHECK();
  R.col_idx = DBuf<int>((size_t)A.nnzb, s);
  transpose_rank_kernel<<<grid_for((long long)R.n_rows * 32, 256), 256, 0, s>>>(R.row_ptr.p, R.n_rows, tkey.p,
                                                                                tsrc.p, R.col_idx.p, src.p);
  TAM_LAUNCH_CHECK();
  R.vals = DBuf<double>((size_t)A.nnzb * A.block_elems(), s);
  const unsigned g = grid_for(A.nnzb * (long long)A.block_elems(), 256);
  if (A.br == 3 && A.bc == 6) transpose_vals_kernel<3, 6><<<g, 256, 0, s>>>(A.vals.p, src.p, A.nnzb, R.vals.p);
  else if (A.br == 6 && A.bc == 6) transpose_vals_kernel<6, 6><<<g, 256, 0, s>>>(A.vals.p, src.p, A.nnzb, R.vals.p);
  else if (A.br == 1 && A.bc == 1) transpose_vals_kernel<1, 1><<<g, 256, 0, s>>>(A.vals.p, src.p, A.nnzb, R.vals.p);
  else if (A.br == 3 && A.bc == 3) transpose_vals_kernel<3, 3><<<g, 256, 0, s>>>(A.vals.p, src.p, A.nnzb, R.vals.p);
  else if (A.br == 6 && A.bc == 3) transpose_vals_kernel<6, 3><<<g, 256, 0, s>>>(A.vals.p, src.p, A.nnzb, R.vals.p);
  else throw Error(TAM_ERR_UNSUPPORTED, "transpose: block shape not instantiated");
  TAM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// SpGEMM C = X Y.  Symbolic: one warp per row inserts the candidate columns
// into a shared-memory hash set (open addressing), counts, and in the fill
// pass compacts and bitonic-sorts them; narrow outputs use a column bitmap.
// Numeric: one thread per output block for 3-row blocks
// (spgemm_numeric_os_kernel), a warp per output row window otherwise
// (spgemm_numeric_rs_kernel).
// ---------------------------------------------------------------------------
namespace {

constexpr int SG_WARPS = 4;
constexpr int HT = 2048;            // hash slots per warp
constexpr int HT_MAX = 1536;        // max unique columns per row (load 0.75)
constexpr int HT_SMALL = 256;       // slots per warp when every row's bound is <= 128

// Open addressing in a table of hsz (a power of two <= HT) slots.
__device__ __forceinline__ bool ht_insert(int* tab, int col, int hsz) {
  const unsigned mask = (unsigned)hsz - 1u;
  unsigned h = ((unsigned)col * 2654435761u) & mask;
  int key = col + 1;
  for (int probe = 0; probe < hsz; ++probe) {
    int prev = atomicCAS(&tab[h], 0, key);
    if (prev == 0) return true;
    if (prev == key) return false;
    h = (h + 1) & mask;
  }
  return false;  // table full: caught by the count check
}

// HTT slots per warp: HT, or HT_SMALL when every row's bound fits (the finest
// levels: an eighth of the shared memory, so several times the resident warps).
template <bool FILL, int HTT>
__global__ void __launch_bounds__(SG_WARPS * 32)
spgemm_symbolic_kernel(const int* __restrict__ xrp, const int* __restrict__ xci, int n_rows,
                       const int* __restrict__ yrp, const int* __restrict__ yci, int n_cols,
                       int* __restrict__ row_cnt, const int* __restrict__ crp, int* __restrict__ cci,
                       int* __restrict__ overflow) {
  __shared__ int tab_all[SG_WARPS][HTT];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * SG_WARPS + wid;
  if (row >= n_rows) return;
  int* tab = tab_all[wid];
  const int xs = xrp[row], xe = xrp[row + 1];
  // table sized for this row: at least twice the sum of the Y row lengths (an
  // upper bound of the distinct columns), so that short rows -- most of them --
  // do not clear and scan all HT slots
  int bound = 0;
  for (int p = xs + lane; p < xe; p += 32) {
    const int j = xci[p];
    bound += yrp[j + 1] - yrp[j];
  }
  bound = warp_sum_i(bound);
  int hsz = 32;
  while (hsz < 2 * bound && hsz < HTT) hsz <<= 1;
  // Narrow outputs (the coarse levels: few columns, long rows): a bitmap of
  // the n_cols columns instead of the hash set when it has no more words than
  // the table has slots -- no probing, no column limit, and the set bits come
  // out already sorted.
  const int words = (n_cols + 31) >> 5;
  if (words <= hsz) {
    for (int i = lane; i < words; i += 32) tab[i] = 0;
    __syncwarp();
    // sub-groups of W lanes: 32 / W X entries in flight at once, the W lanes
    // of each striding its Y row (coalesced)
    const int W = bound >= 8 * (xe - xs) ? 8 : 1;
    const int sg = lane / W, l = lane % W, nsg = 32 / W;
    for (int p = xs + sg; p < xe; p += nsg) {
      const int j = xci[p];
      for (int q = yrp[j] + l; q < yrp[j + 1]; q += W) {
        const int c = yci[q];
        atomicOr(reinterpret_cast<unsigned*>(tab) + (c >> 5), 1u << (c & 31));
      }
    }
    __syncwarp();
    if (!FILL) {
      int cnt = 0;
      for (int i = lane; i < words; i += 32) cnt += __popc((unsigned)tab[i]);
      cnt = warp_sum_i(cnt);
      if (lane == 0) row_cnt[row] = cnt;
      return;
    }
    int base = crp[row];
    for (int i0 = 0; i0 < words; i0 += 32) {
      unsigned w = i0 + lane < words ? (unsigned)tab[i0 + lane] : 0u;
      const int c = __popc(w);
      int off = c;  // inclusive scan of the lanes' counts
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, off, d);
        if (lane >= d) off += t;
      }
      const int total = __shfl_sync(0xffffffffu, off, 31);
      off = base + off - c;
      while (w) {
        cci[off++] = ((i0 + lane) << 5) + (__ffs(w) - 1);
        w &= w - 1u;
      }
      base += total;
    }
    if (row_cnt && lane == 0) row_cnt[row] = base - crp[row];
    return;
  }
  for (int i = lane; i < hsz; i += 32) tab[i] = 0;
  __syncwarp();
  int ins = 0;
  for (int p = xs + lane; p < xe; p += 32) {
    int j = xci[p];
    for (int q = yrp[j]; q < yrp[j + 1]; ++q) ins += ht_insert(tab, yci[q], hsz) ? 1 : 0;
  }
  __syncwarp();
  int cnt = warp_sum_i(ins);
  if (cnt > HTT / 4 * 3) {
    if (lane == 0) atomicExch(overflow, 1);
    if (row_cnt && lane == 0) row_cnt[row] = 0;
    return;
  }
  if (!FILL) {
    if (lane == 0) row_cnt[row] = cnt;
    return;
  }
  // compact non-empty slots (decoded) to the front, pad, sort
  int base = 0;
  for (int i0 = 0; i0 < hsz; i0 += 32) {
    int v = tab[i0 + lane];
    bool keep = v != 0;
    unsigned m = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    if (keep) tab[base + __popc(m & ((1u << lane) - 1u))] = v - 1;
    base += __popc(m);
    __syncwarp();
  }
  int n2 = next_pow2(cnt);
  for (int i = cnt + lane; i < n2; i += 32) tab[i] = 0x7fffffff;
  __syncwarp();
  warp_bitonic_sort<false>(tab, nullptr, n2);
  const int c0 = crp[row];
  for (int i = lane; i < cnt; i += 32) cci[c0 + i] = tab[i];
  if (row_cnt && lane == 0) row_cnt[row] = cnt;
}

// Single-pass symbolic: each row's bound (the sum of its X entries' Y row
// lengths, at least its distinct columns) ...
__global__ void spgemm_bound_kernel(const int* __restrict__ xrp, const int* __restrict__ xci, int n_rows,
                                    const int* __restrict__ yrp, long long* __restrict__ bound,
                                    int* __restrict__ max_bound) {
  const int row = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  int b = 0;
  for (int p = xrp[row] + lane; p < xrp[row + 1]; p += 32) {
    const int j = xci[p];
    b += yrp[j + 1] - yrp[j];
  }
  b = warp_sum_i(b);
  if (lane == 0) {
    bound[row] = b;
    atomicMax(max_bound, b);
  }
}

// ... as 32-bit offsets of the rows' scratch ranges (total checked < 2^31) ...
__global__ void offsets_to_i32_kernel(const long long* __restrict__ in, long long n, int* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= n) out[i] = (int)in[i];
}

// ... and, once the fill pass has written each row's sorted columns to the
// front of its scratch range and its count, the rows packed into C.
__global__ void spgemm_pack_kernel(const int* __restrict__ soff, const int* __restrict__ scratch, int n_rows,
                                   const int* __restrict__ crp, int* __restrict__ cci) {
  const int row = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  const int s0 = soff[row], c0 = crp[row], n = crp[row + 1] - c0;
  for (int i = lane; i < n; i += 32) cci[c0 + i] = scratch[s0 + i];
}

// Output-stationary numeric pass: one thread per output block C_ic.  It walks
// X's row i, finds column c in Y's row j by binary search and accumulates
// X_ij Y_jc in registers -- every FP64 FMA is useful work, nothing is shared
// between threads (no atomics, no shared-memory windows), and the threads of
// one output row read the same X row (L1 broadcast).
__global__ void expand_rows_kernel(const int* __restrict__ rp, int n_rows, int* __restrict__ row_of) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_rows) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) row_of[p] = i;
}

// Arithmetic of the numeric passes.
//
// Both policies read operands of type V and accumulate in A; out() gives the
// FP64 result.  F64 is plain FP64.  DF ("double-float") keeps every operand
// as an unevaluated sum hi + lo of two FP32 values (split once, before the
// product) and accumulates in the same form: the product of the high parts is
// made exact with an FMA, the two cross terms are added to its error, and the
// sum with the accumulator uses Knuth's TwoSum, so each product-accumulate is
// accurate to about 2^-48 of the magnitudes involved.  GB300 issues FP32 FMAs
// at 64 times its FP64 rate, and these kernels run the FP64 pipe at ~98% in
// the F64 form, so the ~12 FP32 operations per multiply-add are the cheaper
// way to the same accuracy class.  __fadd_rn/__fmul_rn keep the compiler from
// contracting the error-free transforms into FMAs.
struct ArithF64 {
  using V = double;
  using A = double;
  __device__ static A zero() { return 0.0; }
  __device__ static void fma(A& a, V x, V y) { a = ::fma(x, y, a); }
  __device__ static void add(A& a, A b) { a += b; }
  __device__ static void store(double* p, A a) { *p = a; }
};

struct ArithDF {
  using V = float2;
  using A = float2;
  __device__ static A zero() { return make_float2(0.f, 0.f); }
  __device__ static void fma(A& a, V x, V y) { df_fma(a, x, y); }
  __device__ static void add(A& a, A b) { df_fma(a, b, make_float2(1.f, 0.f)); }  // b * 1 is exact
  __device__ static void store(double* p, A a) { *p = f2d_bits(a.x) + f2d_bits(a.y); }
  // kept split for a following double-float product: renormalised (Fast2Sum)
  __device__ static void store(float2* p, A a) {
    const float s = __fadd_rn(a.x, a.y);
    *p = make_float2(s, __fadd_rn(a.y, -__fadd_rn(s, -a.x)));
  }
};

template <int M, int K, int N, class Ar, typename OutT>
__global__ void __launch_bounds__(128, 6)
spgemm_numeric_os_kernel(const int* __restrict__ xrp, const int* __restrict__ xci, const typename Ar::V* __restrict__ xv,
                         const int* __restrict__ yrp, const int* __restrict__ yci, const typename Ar::V* __restrict__ yv,
                         const int* __restrict__ crow, const int* __restrict__ cci, long long nnzc,
                         OutT* __restrict__ cv) {
  using V = typename Ar::V;
  using A = typename Ar::A;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nnzc) return;
  const int i = crow[t], c = cci[t];
  A acc[M * N];
#pragma unroll
  for (int e = 0; e < M * N; ++e) acc[e] = Ar::zero();
  const int pe = xrp[i + 1];
  for (int p = xrp[i]; p < pe; ++p) {
    const int j = xci[p];
    int lo = yrp[j], hi = yrp[j + 1];
    const int end = hi;
    if (hi - lo <= 8) {
      // short Y rows (prolongators): all candidates loaded at once, one
      // memory round trip instead of a chain of dependent probes
      int f = end;
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (lo + t < end && yci[lo + t] == c) f = lo + t;
      lo = f;
    } else {
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (yci[mid] < c) lo = mid + 1; else hi = mid;
      }
    }
    if (lo < end && yci[lo] == c) {
      const V* __restrict__ xb = xv + (size_t)p * M * K;
      const V* __restrict__ yb = yv + (size_t)lo * K * N;
      V xr[M * K];
#pragma unroll
      for (int e = 0; e < M * K; ++e) xr[e] = xb[e];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        V yr[N];
#pragma unroll
        for (int s2 = 0; s2 < N; ++s2) yr[s2] = yb[k * N + s2];
#pragma unroll
        for (int r = 0; r < M; ++r)
#pragma unroll
          for (int s2 = 0; s2 < N; ++s2) Ar::fma(acc[r * N + s2], xr[r * K + k], yr[s2]);
      }
    }
  }
  OutT* out = cv + (size_t)t * M * N;
#pragma unroll
  for (int e = 0; e < M * N; ++e) Ar::store(out + e, acc[e]);
}

// Row-stationary numeric pass for tall X blocks (M = 6: R (A P) and the coarse
// levels): one warp per output row, the row's output blocks accumulated in
// shared memory a window of W columns at a time.  For each X entry (i, j) the
// lanes take the (Y-row entry q, block row r) items: item (q, r) computes row
// r of X_ij Y_jq (K*N multiply-adds) and adds it to output block col(q).
// Columns in a Y row are distinct, so the items of one X entry never touch the
// same accumulator element and no atomics are needed; X entries are processed
// one after the other.  Most of the warp does useful work (items = M * |Y row|).
// CNT consecutive 8-byte values (double or float2) into registers with
// 16-byte loads (CNT even; p 16-byte aligned: block sizes 18 and 36 values).
template <int CNT, typename V>
__device__ __forceinline__ void load_block(const V* __restrict__ p, V (&out)[CNT]) {
  static_assert(sizeof(V) == 8 && CNT % 2 == 0, "load_block: 8-byte values, even count");
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
}

constexpr int RS_WARPS = 8;
constexpr int RS_ACC_BYTES = 8192;

template <int M, int K, int N, class Ar, typename OutT>
__global__ void __launch_bounds__(RS_WARPS * 32, 3)
spgemm_numeric_rs_kernel(const int* __restrict__ xrp, const int* __restrict__ xci, const typename Ar::V* __restrict__ xv,
                         int n_rows, const int* __restrict__ yrp, const int* __restrict__ yci,
                         const typename Ar::V* __restrict__ yv, const int* __restrict__ crp, const int* __restrict__ cci,
                         OutT* __restrict__ cv, int upper, const int* __restrict__ win_row,
                         const int* __restrict__ win_w0, int n_win, int split) {
  using V = typename Ar::V;
  using A = typename Ar::A;
  constexpr int MN = M * N;
  constexpr int W = RS_ACC_BYTES / (MN * (int)sizeof(A));
  extern __shared__ double sm_d[];
  A* sm = reinterpret_cast<A*>(sm_d);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one warp per (output row, column window); with split, one block per
  // window, its warps taking every RS_WARPS-th X entry of the row (block-uniform
  // exit: the partial windows are summed after a __syncthreads)
  const int win = split ? (int)blockIdx.x : (int)blockIdx.x * RS_WARPS + wid;
  const int p0 = split ? wid : 0, pstep = split ? RS_WARPS : 1;
  if (win >= n_win) return;
  const int row = win_row[win];
  A* acc = sm + (size_t)wid * (RS_ACC_BYTES / sizeof(A));
  int* wcols = reinterpret_cast<int*>(sm + (size_t)RS_WARPS * (RS_ACC_BYTES / sizeof(A))) + wid * W;
  int cs = crp[row];
  const int ce = crp[row + 1];
  if (upper) {  // symmetric C: only the blocks with column >= row (mirrored afterwards)
    int lo = cs, hi = ce;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cci[mid] < row) lo = mid + 1; else hi = mid;
    }
    cs = lo;
  }
  const int xs = xrp[row], xe = xrp[row + 1];
  {
    const int w0 = win_w0[win];
    const int wn = min(W, ce - w0);
    for (int i = lane; i < wn; i += 32) wcols[i] = cci[w0 + i];
    for (int i = lane; i < wn * MN; i += 32) acc[i] = Ar::zero();
    __syncwarp();
    const int clo = wcols[0], chi = wcols[wn - 1];
    for (int p = xs + p0; p < xe; p += pstep) {
      const int j = xci[p];
      int qs = yrp[j], qe = yrp[j + 1];
      if (upper || wn < ce - cs) {
        // restrict Y's row to the window's column range: the warp reads the
        // (short, sorted) row 32 columns at a time and ballots, one memory
        // round trip per 32 entries instead of two dependent binary searches
        int first = qe, last = qs - 1;
        for (int b0 = qs; b0 < qe; b0 += 32) {
          const int q = b0 + lane;
          const int cq = q < qe ? yci[q] : 0x7fffffff;
          const unsigned ge = __ballot_sync(0xffffffffu, q < qe && cq >= clo);
          const unsigned le = __ballot_sync(0xffffffffu, q < qe && cq <= chi);
          if (first == qe && ge) first = b0 + __ffs(ge) - 1;
          if (le) last = b0 + 31 - __clz(le);
          if (le != 0xffffffffu) break;  // the columns <= chi form a prefix
        }
        qs = first;
        qe = last + 1 > first ? last + 1 : first;
      }
      const V* __restrict__ xb = xv + (size_t)p * M * K;
      // G groups of M lanes: group g takes Y entry qs + q0 + g, lane r of the
      // group its block row r.  One lane per group finds the entry's window
      // slot and shares it; each lane then loads the whole Y block at once
      // and accumulates row r of X_ij Y_jq.  Three blocks per SM (80
      // registers, no spills; 3 x 66 KB of windows): 10-21% faster than the
      // two that 117 registers allowed.
      constexpr int G = 32 / M;
      const int g = lane / M, r = lane % M;
      const int nq = qe - qs;
      for (int q0 = 0; q0 < nq; q0 += G) {
        const int qi = q0 + g;
        const bool has = g < G && qi < nq;
        int pos = 0;
        if (has && r == 0) {
          const int c = yci[qs + qi];
          int lo = 0, hi = wn - 1;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (wcols[mid] < c) lo = mid + 1; else hi = mid;
          }
          pos = lo;
        }
        pos = __shfl_sync(0xffffffffu, pos, min(g * M, 31));
        if (has) {
          V xr[K];
#pragma unroll
          for (int k = 0; k < K; ++k) xr[k] = xb[r * K + k];
          V yr[K * N];
          load_block<K * N>(yv + (size_t)(qs + qi) * K * N, yr);
          A* a = acc + pos * MN + r * N;
#pragma unroll
          for (int s2 = 0; s2 < N; ++s2) {
            A t = a[s2];
#pragma unroll
            for (int k = 0; k < K; ++k) Ar::fma(t, xr[k], yr[k * N + s2]);
            a[s2] = t;
          }
        }
      }
      __syncwarp();
    }
    if (!split) {
      for (int i = lane; i < wn * MN; i += 32) Ar::store(cv + (size_t)w0 * MN + i, acc[i]);
      return;
    }
    __syncthreads();
    constexpr int STRIDE = RS_ACC_BYTES / sizeof(A);
    for (int i = threadIdx.x; i < wn * MN; i += RS_WARPS * 32) {
      A t = sm[i];
#pragma unroll
      for (int w = 1; w < RS_WARPS; ++w) Ar::add(t, sm[(size_t)w * STRIDE + i]);
      Ar::store(cv + (size_t)w0 * MN + i, t);
    }
  }
}

// Column windows of the output rows (W blocks each; from the diagonal on for
// a symmetric C): one warp per window, so that a long row -- the few, long rows
// of a coarse Galerkin product -- is spread over many warps.
__device__ __forceinline__ int rs_row_start(const int* __restrict__ crp, const int* __restrict__ cci, int row,
                                            int upper) {
  int lo = crp[row], hi = crp[row + 1];
  if (!upper) return lo;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cci[mid] < row) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void rs_window_count_kernel(const int* __restrict__ crp, const int* __restrict__ cci, int n_rows, int upper,
                                       int W, int* __restrict__ cnt) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  const int len = crp[row + 1] - rs_row_start(crp, cci, row, upper);
  cnt[row] = (len + W - 1) / W;
}

__global__ void rs_window_list_kernel(const int* __restrict__ wptr, const int* __restrict__ crp,
                                      const int* __restrict__ cci, int n_rows, int upper, int W,
                                      int* __restrict__ win_row, int* __restrict__ win_w0) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n_rows) return;
  const int cs = rs_row_start(crp, cci, row, upper);
  for (int k = 0, w = wptr[row]; w < wptr[row + 1]; ++k, ++w) {
    win_row[w] = row;
    win_w0[w] = cs + k * W;
  }
}

// Lower blocks of a symmetric C from their upper partners: C_ic = C_ci^T.
// A missing partner (a pattern that is not symmetric) is reported, not read.
template <int M>
__global__ void mirror_lower_kernel(const int* __restrict__ crp, const int* __restrict__ cci, int n_rows,
                                    double* __restrict__ cv, int* __restrict__ bad) {
  const int row = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  for (int p = crp[row] + lane; p < crp[row + 1]; p += 32) {
    const int c = cci[p];
    if (c >= row) break;  // sorted: the rest of this lane's entries are upper
    int lo = crp[c], hi = crp[c + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cci[mid] < row) lo = mid + 1; else hi = mid;
    }
    if (lo >= crp[c + 1] || cci[lo] != row) {
      atomicExch(bad, 1);
      continue;
    }
    const double* __restrict__ src = cv + (size_t)lo * M * M;  // block (c, row)
    double* __restrict__ dst = cv + (size_t)p * M * M;
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
      for (int k = 0; k < M; ++k) dst[r * M + k] = src[k * M + r];
  }
}

// Windows below which a window gets a whole block: the warps two resident
// blocks per SM hold.
int rs_split_windows() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, n_sm = 0;
    TAM_CUDA(cudaGetDevice(&dev));
    TAM_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    n = std::max(1, n_sm) * 2 * RS_WARPS;
  }
  return n;
}

template <int M, int K, int N, class Ar, typename OutT>
void launch_numeric(const Bsr& X, const typename Ar::V* xv, const Bsr& Y, const typename Ar::V* yv, Bsr& C,
                    OutT* cv, bool symmetric, cudaStream_t s) {
  if (C.nnzb == 0) return;
  // 3-row blocks (A P_tent, A P on the finest level) keep the output-stationary
  // pass: with only 3 rows per item the row-stationary warp idles (measured
  // 2x slower on the 256x64x64 box).
  if constexpr (M == 6) {
    constexpr int W = RS_ACC_BYTES / (M * N * (int)sizeof(typename Ar::A));
    const size_t smem = (size_t)RS_WARPS * (RS_ACC_BYTES + W * 4);
    static bool attr_set = false;
    if (!attr_set) {
      TAM_CUDA(cudaFuncSetAttribute(spgemm_numeric_rs_kernel<M, K, N, Ar, OutT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr_set = true;
    }
    const bool upper = symmetric && M == N && std::is_same<OutT, double>::value;
    DBuf<int> wptr((size_t)C.n_rows + 1, s);
    rs_window_count_kernel<<<grid_for(C.n_rows, 256), 256, 0, s>>>(C.row_ptr.p, C.col_idx.p, C.n_rows, upper ? 1 : 0,
                                                                    W, wptr.p);
    TAM_LAUNCH_CHECK();
    exclusive_scan_i32(wptr.p, wptr.p, C.n_rows, s);
    const int n_win = read_back_int(wptr.p + C.n_rows, s);
    if (n_win > 0) {
      DBuf<int> win_row((size_t)n_win, s), win_w0((size_t)n_win, s);
      rs_window_list_kernel<<<grid_for(C.n_rows, 256), 256, 0, s>>>(wptr.p, C.row_ptr.p, C.col_idx.p, C.n_rows,
                                                                     upper ? 1 : 0, W, win_row.p, win_w0.p);
      TAM_LAUNCH_CHECK();
      // Few windows (the coarse levels' products): a block per window, so
      // that its long X row is shared by RS_WARPS warps instead of one.
      const int split = n_win < rs_split_windows() ? 1 : 0;
      spgemm_numeric_rs_kernel<M, K, N, Ar, OutT>
          <<<split ? (unsigned)n_win : grid_for(n_win, RS_WARPS), RS_WARPS * 32, smem, s>>>(
              X.row_ptr.p, X.col_idx.p, xv, X.n_rows, Y.row_ptr.p, Y.col_idx.p, yv, C.row_ptr.p, C.col_idx.p, cv,
              upper ? 1 : 0, win_row.p, win_w0.p, n_win, split);
      TAM_LAUNCH_CHECK();
    }
    if constexpr (M == N && std::is_same<OutT, double>::value) {
      if (upper) {
        DBuf<int> bad(1, s);
        bad.zero();
        mirror_lower_kernel<M><<<grid_for((long long)C.n_rows * 32, 256), 256, 0, s>>>(C.row_ptr.p, C.col_idx.p,
                                                                                         C.n_rows, cv, bad.p);
        TAM_LAUNCH_CHECK();
        TAM_CHECK(read_back_int(bad.p, s) == 0, TAM_ERR_INTERNAL, "spgemm: symmetric product with an unsymmetric pattern");
      }
    }
  } else {
    DBuf<int> crow((size_t)C.nnzb, s);
    expand_rows_kernel<<<grid_for(C.n_rows, 256), 256, 0, s>>>(C.row_ptr.p, C.n_rows, crow.p);
    TAM_LAUNCH_CHECK();
    spgemm_numeric_os_kernel<M, K, N, Ar, OutT><<<grid_for(C.nnzb, 128), 128, 0, s>>>(
        X.row_ptr.p, X.col_idx.p, xv, Y.row_ptr.p, Y.col_idx.p, yv, crow.p, C.col_idx.p, C.nnzb, cv);
    TAM_LAUNCH_CHECK();
  }
}

}  // namespace

DBuf<float2> split_values(const Bsr& B, cudaStream_t s) {
  DBuf<float2> out;
  split_into(B.vals.p, B.nnzb * (long long)B.block_elems(), out, s);
  return out;
}

template <int M, int K, int N>
void launch_numeric_any(const Bsr& X, const Bsr& Y, Bsr& C, SpgemmArith arith, const SpgemmSplit& sp,
                        cudaStream_t s) {
  if (arith == SpgemmArith::kFp64) {
    C.vals = DBuf<double>((size_t)C.nnzb * C.block_elems(), s);
    launch_numeric<M, K, N, ArithF64>(X, X.vals.p, Y, Y.vals.p, C, C.vals.p, sp.symmetric, s);
    return;
  }
  DBuf<float2> xs, ys;
  const float2* xv = sp.x;
  const float2* yv = sp.y;
  if (!xv) xs = split_values(X, s), xv = xs.p;
  if (!yv) ys = split_values(Y, s), yv = ys.p;
  if (sp.c) {
    *sp.c = DBuf<float2>((size_t)std::max<long long>(1, C.nnzb * (long long)C.block_elems()), s);
    launch_numeric<M, K, N, ArithDF>(X, xv, Y, yv, C, sp.c->p, false, s);
  } else {
    C.vals = DBuf<double>((size_t)C.nnzb * C.block_elems(), s);
    launch_numeric<M, K, N, ArithDF>(X, xv, Y, yv, C, C.vals.p, sp.symmetric, s);
  }
}

void bsr_spgemm(const Bsr& X, const Bsr& Y, Bsr& C, cudaStream_t s, SpgemmArith arith, const SpgemmSplit& sp) {
  TAM_CHECK(X.bc == Y.br && X.n_cols == Y.n_rows, TAM_ERR_INTERNAL, "spgemm: shape mismatch");
  C.n_rows = X.n_rows;
  C.n_cols = Y.n_cols;
  C.br = X.br;
  C.bc = Y.bc;
  C.row_ptr = DBuf<int>((size_t)C.n_rows + 1, s);
  DBuf<int> overflow(1, s);
  overflow.zero();
  const unsigned grid = grid_for(X.n_rows, SG_WARPS);
  // one pass when the rows' bounds sum below 2^31: the fill kernel writes each
  // row's sorted columns into a scratch range of its bound and its count, and
  // a pack kernel moves them into C; otherwise a counting pass first
  DBuf<long long> b64((size_t)X.n_rows + 1, s);
  DBuf<int> max_bound(1, s);
  max_bound.zero();
  spgemm_bound_kernel<<<grid_for((long long)X.n_rows * 32, 256), 256, 0, s>>>(X.row_ptr.p, X.col_idx.p, X.n_rows,
                                                                              Y.row_ptr.p, b64.p, max_bound.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i64(b64.p, b64.p, X.n_rows, s);
  long long total_bound = 0;
  int max_b = 0;
  read_back_ll_int(b64.p + X.n_rows, max_bound.p, &total_bound, &max_b, s);
  const bool small_tab = 2 * max_b <= HT_SMALL;
  if (total_bound < (1LL << 31) - 1) {
    DBuf<int> soff((size_t)X.n_rows + 1, s);
    offsets_to_i32_kernel<<<grid_for((long long)X.n_rows + 1, 256), 256, 0, s>>>(b64.p, X.n_rows, soff.p);
    TAM_LAUNCH_CHECK();
    b64.reset();
    DBuf<int> scratch((size_t)std::max(1LL, total_bound), s);
    if (small_tab)
      spgemm_symbolic_kernel<true, HT_SMALL><<<grid, SG_WARPS * 32, 0, s>>>(
          X.row_ptr.p, X.col_idx.p, X.n_rows, Y.row_ptr.p, Y.col_idx.p, Y.n_cols, C.row_ptr.p, soff.p, scratch.p,
          overflow.p);
    else
      spgemm_symbolic_kernel<true, HT><<<grid, SG_WARPS * 32, 0, s>>>(
          X.row_ptr.p, X.col_idx.p, X.n_rows, Y.row_ptr.p, Y.col_idx.p, Y.n_cols, C.row_ptr.p, soff.p, scratch.p,
          overflow.p);
    TAM_LAUNCH_CHECK();
    exclusive_scan_i32(C.row_ptr.p, C.row_ptr.p, C.n_rows, s);
    int nnzb = 0, ovf = 0;
    read_back_int2(C.row_ptr.p + C.n_rows, overflow.p, &nnzb, &ovf, s);
    C.nnzb = nnzb;
    TAM_CHECK(ovf == 0, TAM_ERR_INTERNAL, "spgemm: an output row exceeds 1536 blocks");
    C.col_idx = DBuf<int>((size_t)std::max(1LL, C.nnzb), s);
    spgemm_pack_kernel<<<grid_for((long long)X.n_rows * 32, 256), 256, 0, s>>>(soff.p, scratch.p, X.n_rows,
                                                                               C.row_ptr.p, C.col_idx.p);
    TAM_LAUNCH_CHECK();
  } else {
    b64.reset();
    spgemm_symbolic_kernel<false, HT><<<grid, SG_WARPS * 32, 0, s>>>(X.row_ptr.p, X.col_idx.p, X.n_rows, Y.row_ptr.p,
                                                               Y.col_idx.p, Y.n_cols, C.row_ptr.p, nullptr, nullptr,
                                                               overflow.p);
    TAM_LAUNCH_CHECK();
    exclusive_scan_i32(C.row_ptr.p, C.row_ptr.p, C.n_rows, s);
    C.nnzb = read_back_int(C.row_ptr.p + C.n_rows, s);
    TAM_CHECK(read_back_int(overflow.p, s) == 0, TAM_ERR_INTERNAL,
              "spgemm: an output row exceeds 1536 blocks");
    C.col_idx = DBuf<int>((size_t)C.nnzb, s);
    spgemm_symbolic_kernel<true, HT><<<grid, SG_WARPS * 32, 0, s>>>(X.row_ptr.p, X.col_idx.p, X.n_rows, Y.row_ptr.p,
                                                              Y.col_idx.p, Y.n_cols, nullptr, C.row_ptr.p,
                                                              C.col_idx.p, overflow.p);
    TAM_LAUNCH_CHECK();
  }
  const int m = X.br, k = X.bc, n = Y.bc;
  if (m == 3 && k == 3 && n == 6) launch_numeric_any<3, 3, 6>(X, Y, C, arith, sp, s);
  else if (m == 6 && k == 3 && n == 6) launch_numeric_any<6, 3, 6>(X, Y, C, arith, sp, s);
  else if (m == 6 && k == 6 && n == 6) launch_numeric_any<6, 6, 6>(X, Y, C, arith, sp, s);
  else if (m == 3 && k == 3 && n == 3) launch_numeric_any<3, 3, 3>(X, Y, C, arith, sp, s);
  else if (m == 6 && k == 6 && n == 3) launch_numeric_any<6, 6, 3>(X, Y, C, arith, sp, s);
  else if (m == 3 && k == 6 && n == 6) launch_numeric_any<3, 6, 6>(X, Y, C, arith, sp, s);
  else if (m == 1 && k == 1 && n == 1) launch_numeric_any<1, 1, 1>(X, Y, C, arith, sp, s);
  else throw Error(TAM_ERR_UNSUPPORTED, "spgemm: block shape not instantiated");
}

// ---------------------------------------------------------------------------
// C = A P_tent.  P_tent has one block per aggregated row (row k: column
// agg[k]), so C's row i holds the distinct aggregates of A's row i: a warp
// sorts them in shared memory (no hash set, no bound pass), and the numeric
// pass sums, per output element, the products of the entries whose column
// lies in that aggregate -- in A's row order and the inner index's order,
// the same operations as the general output-stationary pass.
// ---------------------------------------------------------------------------
namespace {

constexpr int AT_WARPS = 4;
constexpr int AT_CAP = 256;  // longest row of A handled here (else the general product)

__global__ void __launch_bounds__(AT_WARPS * 32)
aptent_symbolic_kernel(const int* __restrict__ xrp, const int* __restrict__ xci, int n_rows,
                       const int* __restrict__ agg, int* __restrict__ row_cnt, int* __restrict__ scratch,
                       int* __restrict__ overflow) {
  __shared__ int tab[AT_WARPS][AT_CAP];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * AT_WARPS + wid;
  if (row >= n_rows) return;  // warp-uniform
  const int p0 = xrp[row], len = xrp[row + 1] - p0;
  if (len > AT_CAP) {
    if (lane == 0) {
      atomicExch(overflow, 1);
      row_cnt[row] = 0;
    }
    return;
  }
  int* t = tab[wid];
  const int n2 = next_pow2(len);
  for (int i = lane; i < n2; i += 32) {
    int v = 0x7fffffff;
    if (i < len) {
      const int a = agg[xci[p0 + i]];
      if (a >= 0) v = a;
    }
    t[i] = v;
  }
  __syncwarp();
  warp_bitonic_sort<false>(t, nullptr, n2);
  int base = 0;
  for (int i0 = 0; i0 < n2; i0 += 32) {
    const int i = i0 + lane;
    const int v = t[i];
    const bool keep = v != 0x7fffffff && (i == 0 || t[i - 1] != v);
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) scratch[p0 + base + __popc(m & ((1u << lane) - 1u))] = v;
    base += __popc(m);
  }
  if (lane == 0) row_cnt[row] = base;
}

template <int M, int K, int N, class Ar>
__global__ void __launch_bounds__(AT_WARPS * 32)
aptent_numeric_kernel(const int* __restrict__ xrp, const int* __restrict__ xci, const typename Ar::V* __restrict__ xv,
                      int n_rows, const int* __restrict__ agg, const int* __restrict__ ptrp,
                      const typename Ar::V* __restrict__ ptv, const int* __restrict__ crp,
                      const int* __restrict__ cci, double* __restrict__ cv) {
  using V = typename Ar::V;
  using A = typename Ar::A;
  constexpr int MN = M * N;
  __shared__ int pos[AT_WARPS][AT_CAP];
  __shared__ int ord[AT_WARPS][AT_CAP];
  __shared__ int qst[AT_WARPS][AT_CAP + 1];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * AT_WARPS + wid;
  if (row >= n_rows) return;  // warp-uniform
  const int p0 = xrp[row], len = xrp[row + 1] - p0;
  const int c0 = crp[row], nc = crp[row + 1] - c0;
  int* ps = pos[wid];
  int* od = ord[wid];
  int* qs = qst[wid];
  // the output position of each entry's aggregate (-1: an unaggregated column)
  for (int i = lane; i < len; i += 32) {
    const int a = agg[xci[p0 + i]];
    int q = -1;
    if (a >= 0) {
      int lo = 0, hi = nc;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cci[c0 + mid] < a) lo = mid + 1; else hi = mid;
      }
      q = lo;
    }
    ps[i] = q;
  }
  __syncwarp();
  // the entries grouped by output position, each group in row order: qs[q] =
  // entries with a smaller position, then each entry's rank in its group
  for (int q = lane; q <= nc; q += 32) {
    int c = 0;
    for (int i = 0; i < len; ++i) c += (ps[i] >= 0 && ps[i] < q) ? 1 : 0;
    qs[q] = c;
  }
  __syncwarp();
  for (int i = lane; i < len; i += 32) {
    const int q = ps[i];
    if (q < 0) continue;
    int rank = 0;
    for (int j = 0; j < i; ++j) rank += ps[j] == q ? 1 : 0;
    od[qs[q] + rank] = i;
  }
  __syncwarp();
  for (int it = lane; it < nc * MN; it += 32) {
    const int q = it / MN, e = it - q * MN, r = e / N, s2 = e - r * N;
    A acc = Ar::zero();
    for (int t = qs[q]; t < qs[q + 1]; ++t) {
      const int i = od[t];
      const V* __restrict__ xb = xv + (size_t)(p0 + i) * M * K + r * K;
      const V* __restrict__ yb = ptv + (size_t)ptrp[xci[p0 + i]] * K * N + s2;
#pragma unroll
      for (int k = 0; k < K; ++k) Ar::fma(acc, xb[k], yb[k * N]);
    }
    Ar::store(cv + (size_t)(c0 + q) * MN + e, acc);
  }
}

template <int M, int K, int N, class Ar>
void aptent_numeric(const Bsr& X, const typename Ar::V* xv, const Bsr& Pt, const typename Ar::V* pv, const int* agg,
                    Bsr& C, cudaStream_t s) {
  aptent_numeric_kernel<M, K, N, Ar><<<grid_for(X.n_rows, AT_WARPS), AT_WARPS * 32, 0, s>>>(
      X.row_ptr.p, X.col_idx.p, xv, X.n_rows, agg, Pt.row_ptr.p, pv, C.row_ptr.p, C.col_idx.p, C.vals.p);
  TAM_LAUNCH_CHECK();
}

template <int M, int K, int N>
void aptent_numeric_any(const Bsr& X, const Bsr& Pt, const int* agg, Bsr& C, SpgemmArith arith, const float2* xs,
                        cudaStream_t s) {
  if (arith == SpgemmArith::kFp64) {
    aptent_numeric<M, K, N, ArithF64>(X, X.vals.p, Pt, Pt.vals.p, agg, C, s);
    return;
  }
  DBuf<float2> xo;
  if (!xs) xo = split_values(X, s), xs = xo.p;
  DBuf<float2> ps = split_values(Pt, s);
  aptent_numeric<M, K, N, ArithDF>(X, xs, Pt, ps.p, agg, C, s);
}

}  // namespace

bool bsr_spgemm_tentative(const Bsr& X, const Bsr& Pt, const int* agg, Bsr& C, cudaStream_t s, SpgemmArith arith,
                          const float2* xs) {
  TAM_CHECK(X.bc == Pt.br && X.n_cols == Pt.n_rows, TAM_ERR_INTERNAL, "spgemm: shape mismatch");
  const int m = X.br, k = X.bc, n = Pt.bc;
  if (!((m == 3 && k == 3 && n == 6) || (m == 6 && k == 6 && n == 6) || (m == 1 && k == 1 && n == 1))) return false;
  Bsr T;
  T.n_rows = X.n_rows;
  T.n_cols = Pt.n_cols;
  T.br = m;
  T.bc = n;
  T.row_ptr = DBuf<int>((size_t)T.n_rows + 1, s);
  DBuf<int> scratch((size_t)std::max(1LL, X.nnzb), s), overflow(1, s);
  overflow.zero();
  aptent_symbolic_kernel<<<grid_for(X.n_rows, AT_WARPS), AT_WARPS * 32, 0, s>>>(
      X.row_ptr.p, X.col_idx.p, X.n_rows, agg, T.row_ptr.p, scratch.p, overflow.p);
  TAM_LAUNCH_CHECK();
  exclusive_scan_i32(T.row_ptr.p, T.row_ptr.p, T.n_rows, s);
  int nnzb = 0, ovf = 0;
  read_back_int2(T.row_ptr.p + T.n_rows, overflow.p, &nnzb, &ovf, s);
  if (ovf) return false;  // a row longer than the shared-memory list: the general product
  T.nnzb = nnzb;
  T.col_idx = DBuf<int>((size_t)std::max(1LL, T.nnzb), s);
  spgemm_pack_kernel<<<grid_for((long long)X.n_rows * 32, 256), 256, 0, s>>>(X.row_ptr.p, scratch.p, X.n_rows,
                                                                             T.row_ptr.p, T.col_idx.p);
  TAM_LAUNCH_CHECK();
  // 6x6 blocks: a warp per row over the row's output elements; the short
  // 3-row products keep the output-stationary pass (a thread per output
  // block), which measured faster there (1.9 vs 2.2 ms on the 3.2M-DOF box)
  if (m == 6) {
    T.vals = DBuf<double>((size_t)std::max(1LL, T.nnzb * (long long)T.block_elems()), s);
    if (T.nnzb > 0) aptent_numeric_any<6, 6, 6>(X, Pt, agg, T, arith, xs, s);
  } else {
    SpgemmSplit sp;
    sp.x = xs;
    if (m == 3) launch_numeric_any<3, 3, 6>(X, Pt, T, arith, sp, s);
    else launch_numeric_any<1, 1, 1>(X, Pt, T, arith, sp, s);
  }
  C = std::move(T);
  return true;
}

// ---------------------------------------------------------------------------
// Reduced-precision value copies
// ---------------------------------------------------------------------------
namespace {
template <typename T>
__global__ void convert_kernel(const double* __restrict__ in, T* __restrict__ out, long long n);
template <>
__global__ void convert_kernel<float>(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}
template <>
__global__ void convert_kernel<__nv_bfloat16>(const double* __restrict__ in, __nv_bfloat16* __restrict__ out,
                                              long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __double2bfloat16(in[i]);
}

template <typename T>
void convert_values(const SpOp& op, DBuf<T>& out, cudaStream_t s) {
  const double* src;
  long long n;
  if (op.lpr == 0) {
    src = op.S->vals.p;
    n = op.S->n_slots * 32 * (long long)op.S->br * op.S->bc;
  } else {
    src = op.B->vals.p;
    n = op.B->nnzb * (long long)op.B->block_elems();
  }
  out = DBuf<T>((size_t)std::max(1LL, n), s);
  if (n > 0) {
    convert_kernel<T><<<stride_grid(n, 256, 16), 256, 0, s>>>(src, out.p, n);
    TAM_LAUNCH_CHECK();
  }
}
}  // namespace

void convert_values_f32(const SpOp& op, DBuf<float>& out, cudaStream_t s) { convert_values<float>(op, out, s); }
void convert_values_bf16(const SpOp& op, DBuf<__nv_bfloat16>& out, cudaStream_t s) {
  convert_values<__nv_bfloat16>(op, out, s);
}

}  // namespace tam
