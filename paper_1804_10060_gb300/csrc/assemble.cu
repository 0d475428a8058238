// Assembly of the thermoelastic system (paper Sec. 3, Eq. wf_elastic, steady,
// traction free, with the Dirichlet condition of Eq. u-dbc).
//
//   K[(a,i),(b,j)] = int lambda d_i phi_a d_j phi_b + mu d_j phi_a d_i phi_b
//                        + mu delta_ij grad phi_a . grad phi_b
//   f[(a,i)]       = int (3 lambda + 2 mu) alpha (T_h - T_ref) d_i phi_a + int f_h,i phi_a
//
// (isotropic C, eps_T = alpha (T - T_ref) I, so C:eps_T = (3 lambda + 2 mu) alpha (T - T_ref) I).
//
// Pipeline: cell-node incidence (count, scan, fill) -> block-CSR pattern, one
// warp per node (gather, bitonic sort, unique) -> element kernels with FP64
// atomic scatter -> Dirichlet rows.  Dirichlet couplings never enter the
// pattern: an element block K_ab with a free row a and a Dirichlet column b
// is lifted straight into the load (f_a -= K_ab u_b) and rows of Dirichlet
// nodes become identity rows -- the symmetric elimination of Eq. u-dbc.
#include <cstdlib>

#include <atomic>

#include "handles.cuh"
#include "tet.cuh"

namespace tam {
namespace {

constexpr int PAT_WARPS = 4;
constexpr int PAT_CAP = 1024;  // candidate node ids per row (incident cells x nodes per cell + 1)

__global__ void validate_kernel(const int* __restrict__ cells, long long n_entries, int npc, int n_nodes,
                                const int* __restrict__ mat, int n_cells, int n_mat, int* __restrict__ bad) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_entries) {
    int v = cells[t];
    if (v < 0 || v >= n_nodes) atomicExch(bad, 1);
  }
  if (mat && t < n_cells) {
    int m = mat[t];
    if (m < 0 || m >= n_mat) atomicExch(bad, 2);
  }
}

__global__ void incidence_count_kernel(const int* __restrict__ cells, long long n_entries, int* __restrict__ cnt) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_entries) atomicAdd(&cnt[cells[t]], 1);
}

__global__ void incidence_fill_kernel(const int* __restrict__ cells, long long n_entries, int npc,
                                      const int* __restrict__ ptr, int* __restrict__ cursor,
                                      int* __restrict__ inc) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_entries) return;
  int v = cells[t];
  inc[ptr[v] + atomicAdd(&cursor[v], 1)] = (int)(t / npc);
}

// One warp per node: candidate columns = self + all nodes of incident cells,
// minus Dirichlet nodes (a Dirichlet row keeps only its diagonal).
// Open-addressing insert of node j into a table of hsz (a power of two)
// slots; true if j was new.  The table has room for every candidate.
__device__ __forceinline__ bool pat_insert(int* tab, int j, int hsz) {
  const unsigned mask = (unsigned)hsz - 1u;
  unsigned h = ((unsigned)j * 2654435761u) & mask;
  const int key = j + 1;
  for (int probe = 0; probe < hsz; ++probe) {
    const int prev = atomicCAS(&tab[h], 0, key);
    if (prev == 0) return true;
    if (prev == key) return false;
    h = (h + 1) & mask;
  }
  return false;
}

template <bool FILL>
__global__ void __launch_bounds__(PAT_WARPS * 32)
pattern_kernel(int n_nodes, int npc, const int* __restrict__ cells, const int* __restrict__ inc_ptr,
               const int* __restrict__ inc, const unsigned char* __restrict__ dmask,
               int* __restrict__ row_cnt, const int* __restrict__ row_ptr, int* __restrict__ col_idx,
               int* __restrict__ overflow, int* __restrict__ big_list = nullptr, int big_cap = 0) {
  __shared__ int buf_all[PAT_WARPS][PAT_CAP];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * PAT_WARPS + wid;
  if (i >= n_nodes) return;
  int* buf = buf_all[wid];
  const bool di = dmask[i] != 0;
  const int s = inc_ptr[i], e = inc_ptr[i + 1];
  const int n_cand = di ? 1 : 1 + (e - s) * npc;
  if (n_cand > PAT_CAP) {
    if (lane == 0) {
      // rows beyond the shared-memory capacity: to pattern_big_kernel when a
      // list is given (it writes the count), else reported
      const int k = big_list ? atomicAdd(overflow + 1, 1) : -1;
      if (k >= 0 && k < big_cap) big_list[k] = i;
      else atomicExch(overflow, 1);
      if (row_cnt) row_cnt[i] = FILL ? 0 : 1;
    }
    return;
  }
  // distinct candidates through a shared-memory hash set (open addressing,
  // keys stored + 1, 0 empty), so that only the row's distinct columns --
  // ~15 of ~97 candidates for a P1 row, ~60 of ~400 for P2 -- are sorted
  int hsz = 32;
  while (hsz < 2 * n_cand && hsz < PAT_CAP) hsz <<= 1;
  for (int t = lane; t < hsz; t += 32) buf[t] = 0;
  __syncwarp();
  int ins = lane == 0 ? (pat_insert(buf, i, hsz) ? 1 : 0) : 0;
  if (!di) {
    for (int t = lane; t < (e - s) * npc; t += 32) {
      const int c = inc[s + t / npc];
      const int j = cells[(size_t)c * npc + (t % npc)];
      if (!dmask[j]) ins += pat_insert(buf, j, hsz) ? 1 : 0;
    }
  }
  __syncwarp();
  const int cnt = warp_sum_i(ins);
  int base = 0;  // compact the occupied slots (decoded) to the front
  for (int t0 = 0; t0 < hsz; t0 += 32) {
    const int v = buf[t0 + lane];
    const unsigned m = __ballot_sync(0xffffffffu, v != 0);
    __syncwarp();
    if (v != 0) buf[base + __popc(m & ((1u << lane) - 1u))] = v - 1;
    base += __popc(m);
    __syncwarp();
  }
  const int n2 = next_pow2(cnt);
  for (int t = cnt + lane; t < n2; t += 32) buf[t] = 0x7fffffff;
  __syncwarp();
  warp_bitonic_sort<false>(buf, nullptr, n2);
  __syncwarp();
  if (!FILL) {
    if (lane == 0) row_cnt[i] = cnt;
  } else {
    const int r0 = row_ptr[i];
    for (int t = lane; t < cnt; t += 32) col_idx[r0 + t] = buf[t];
    if (lane == 0 && row_cnt) row_cnt[i] = cnt;
  }
}

// Candidate count of each row (upper bound of its pattern length): self plus
// the nodes of its incident cells; 1 for a Dirichlet row.  A row with more
// candidates than the warp builder's shared memory holds (PAT_CAP) gets three
// times that room: its candidates are sorted in global memory in the upper
// two thirds (padded to a power of two) and its columns written to the front.
__global__ void pattern_bound_kernel(int n_nodes, int npc, const int* __restrict__ inc_ptr,
                                     const unsigned char* __restrict__ dmask, int* __restrict__ bound) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const int b = dmask[i] ? 1 : 1 + (inc_ptr[i + 1] - inc_ptr[i]) * npc;
  bound[i] = b > PAT_CAP ? 3 * b : b;
}

// One block per row whose candidates exceed PAT_CAP (the list built by
// pattern_kernel): candidates gathered into the row's scratch range, padded
// with INT_MAX to a power of two, bitonic-sorted by the block in global
// memory, then the distinct ones compacted to the front of the range
// (block-wide scan of the keep flags) and the count written to row_cnt.
constexpr int BIG_THREADS = 256;

__global__ void __launch_bounds__(BIG_THREADS)
pattern_big_kernel(const int* __restrict__ list, int npc, const int* __restrict__ cells,
                   const int* __restrict__ inc_ptr, const int* __restrict__ inc, const unsigned char* __restrict__ dmask,
                   const int* __restrict__ bptr, int* __restrict__ tmp, int* __restrict__ row_cnt) {
  __shared__ int wsum[BIG_THREADS / 32];
  __shared__ int carry;
  const int i = list[blockIdx.x];
  const int s = inc_ptr[i], e = inc_ptr[i + 1];
  const int n = 1 + (e - s) * npc;
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  int* cand = tmp + bptr[i] + n;  // [n, n + n2) of the 3n range
  int* outp = tmp + bptr[i];
  for (int t = threadIdx.x; t < n2; t += BIG_THREADS) {
    int v = 0x7fffffff;
    if (t == 0) v = i;
    else if (t < n) {
      const int j = cells[(size_t)inc[s + (t - 1) / npc] * npc + (t - 1) % npc];
      if (!dmask[j]) v = j;
    }
    cand[t] = v;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n2; t += BIG_THREADS) {
        const int x = t ^ j;
        if (x > t) {
          const int a = cand[t], b = cand[x];
          if ((a > b) == ((t & k) == 0)) {
            cand[t] = b;
            cand[x] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n2; base += BIG_THREADS) {
    const int t = base + threadIdx.x;
    const int v = t < n2 ? cand[t] : 0x7fffffff;
    const int keep = (v != 0x7fffffff) && (t == 0 || cand[t - 1] != v);
    int x = keep;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int off = carry;
    for (int w = 0; w < wid; ++w) off += wsum[w];
    if (keep) outp[off + x - 1] = v;
    __syncthreads();
    if (threadIdx.x == BIG_THREADS - 1) carry = off + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) row_cnt[i] = carry;
}

// Rows written at their bound offsets in tmp, packed into col_idx (warp per row).
__global__ void pattern_pack_kernel(int n_nodes, const int* __restrict__ bptr, const int* __restrict__ tmp,
                                    const int* __restrict__ row_ptr, int* __restrict__ col_idx) {
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= n_nodes) return;
  const int src = bptr[i], dst = row_ptr[i], cnt = row_ptr[i + 1] - dst;
  for (int t = lane; t < cnt; t += 32) col_idx[dst + t] = tmp[src + t];
}

__device__ __forceinline__ void lame(double E, double nu, double& lam, double& mu) {
  mu = E / (2.0 * (1.0 + nu));
  lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

struct AsmArgs {
  const double* coords;
  const int* cells;
  const int* mat;
  const double* props;
  const double* T;
  double T_ref;
  const double* body;
  const unsigned char* dmask;
  const double* ud;
  const int* row_ptr;
  const int* col_idx;
  double* vals;
  double* rhs;
  int n_cells;
  int* bad_cell;
  int loads_only;  // 1: only the load vector (K of this mesh exists already)
  // deterministic mode (non-null): every element block and load goes to its
  // own slot, ck[((c npc + a) npc + b) 9 + e] and cf[(c npc + a) 3 + d], and
  // gather_kernel sums them per node in cell order (no atomics)
  double* ck = nullptr;
  double* cf = nullptr;
  int npc = 0;
};

// Does the element block (row na, column nb) contribute anything?  In
// loads-only mode only Dirichlet columns with prescribed values do (lifting).
__device__ __forceinline__ bool block_needed(const AsmArgs& A, int nb) {
  return !A.loads_only || (A.dmask[nb] && A.ud);
}

// Scatter one 3x3 block (row node na, col node nb; local a, b of cell c) or
// lift it into the load; in deterministic mode store it in its slot.
__device__ __forceinline__ void scatter_block(const AsmArgs& A, int c, int a, int b, int na, int nb,
                                              const double k[9]) {
  if (A.ck) {
    double* dst = A.ck + (((size_t)c * A.npc + a) * A.npc + b) * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) dst[e] = k[e];
    return;
  }
  if (A.dmask[nb]) {
    if (A.ud) {
      const double* u = A.ud + 3 * (size_t)nb;
      for (int r = 0; r < 3; ++r)
        atomicAdd(&A.rhs[3 * (size_t)na + r], -(k[3 * r] * u[0] + k[3 * r + 1] * u[1] + k[3 * r + 2] * u[2]));
    }
    return;
  }
  if (A.loads_only) return;
  int slot = bsearch_i32(A.col_idx, A.row_ptr[na], A.row_ptr[na + 1], nb);
  double* dst = A.vals + (size_t)slot * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) atomicAdd(dst + e, k[e]);
}

// P1: constant gradients, one thread per cell.
__global__ void __launch_bounds__(128) assemble_p1_kernel(AsmArgs A) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= A.n_cells) return;
  int v[4];
  for (int a = 0; a < 4; ++a) v[a] = A.cells[4 * (size_t)c + a];
  double g[4][3], vol;
  if (!tet_geometry(A.coords, v, g, vol)) {
    atomicExch(A.bad_cell, 1);
    return;
  }
  const int m = A.mat[c];
  double lam, mu;
  lame(A.props[3 * m], A.props[3 * m + 1], lam, mu);
  const double alpha = A.props[3 * m + 2];
  // thermal: int (T_h - T_ref) d_i phi_a = vol (mean vertex T - T_ref) g_a[i]
  double cT = 0.0;
  if (A.T) cT = (3.0 * lam + 2.0 * mu) * alpha * vol * (0.25 * (A.T[v[0]] + A.T[v[1]] + A.T[v[2]] + A.T[v[3]]) - A.T_ref);
  double fsum[3] = {0, 0, 0};
  if (A.body)
    for (int b = 0; b < 4; ++b)
      for (int d = 0; d < 3; ++d) fsum[d] += A.body[3 * (size_t)v[b] + d];
  // K_ab[i][j] = lg_a[i] g_b[j] + mg_a[j] g_b[i] + delta_ij (mg_a . g_b) with
  // lg = lam vol g, mg = mu vol g; K_ba = K_ab^T, so only a <= b is formed
  // (FP64 is GB300's scarce pipe) and the transpose is scattered for b > a.
  double lg[4][3], mg[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      lg[a][i] = lam * vol * g[a][i];
      mg[a][i] = mu * vol * g[a][i];
    }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = a; b < 4; ++b) {
      const bool ab = !A.dmask[v[a]] && block_needed(A, v[b]);
      const bool ba = b != a && !A.dmask[v[b]] && block_needed(A, v[a]);
      if (!ab && !ba) continue;
      const double mgg = mg[a][0] * g[b][0] + mg[a][1] * g[b][1] + mg[a][2] * g[b][2];
      double k[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) k[3 * i + j] = fma(lg[a][i], g[b][j], mg[a][j] * g[b][i]) + (i == j ? mgg : 0.0);
      if (ab) scatter_block(A, c, a, b, v[a], v[b], k);
      if (ba) {
        const double kt[9] = {k[0], k[3], k[6], k[1], k[4], k[7], k[2], k[5], k[8]};
        scatter_block(A, c, b, a, v[b], v[a], kt);
      }
    }
  }
  for (int a = 0; a < 4; ++a) {
    const int na = v[a];
    if (A.dmask[na]) continue;
    // body: int f_h phi_a = vol/20 (sum_b f_b + f_a) (P1 mass matrix vol (1 + delta_ab)/20)
    for (int i = 0; i < 3; ++i) {
      double f = cT * g[a][i];
      if (A.body) f += vol / 20.0 * (fsum[i] + A.body[3 * (size_t)na + i]);
      if (A.cf) A.cf[((size_t)c * 4 + a) * 3 + i] = f;
      else atomicAdd(&A.rhs[3 * (size_t)na + i], f);
    }
  }
}

// P2 quadrature.  Stiffness integrand is degree 2: 4-point rule with
// barycentric points (A,B,B,B) and permutations, A = (5+3 sqrt5)/20,
// B = (5-sqrt5)/20, equal weights 1/4.  Loads are degree 3 (thermal) and 4
// (body): Keast's 11-point degree-4 rule (weights normalised to sum 1).
__constant__ double c_q4[4][4] = {
    {0.5854101966249685, 0.1381966011250105, 0.1381966011250105, 0.1381966011250105},
    {0.1381966011250105, 0.5854101966249685, 0.1381966011250105, 0.1381966011250105},
    {0.1381966011250105, 0.1381966011250105, 0.5854101966249685, 0.1381966011250105},
    {0.1381966011250105, 0.1381966011250105, 0.1381966011250105, 0.5854101966249685}};
__constant__ double c_k11[11][5] = {  // l0, l1, l2, l3, weight
    {0.25, 0.25, 0.25, 0.25, -0.078933333333333333},
    {0.7857142857142857, 0.0714285714285714, 0.0714285714285714, 0.0714285714285714, 0.045733333333333333},
    {0.0714285714285714, 0.7857142857142857, 0.0714285714285714, 0.0714285714285714, 0.045733333333333333},
    {0.0714285714285714, 0.0714285714285714, 0.7857142857142857, 0.0714285714285714, 0.045733333333333333},
    {0.0714285714285714, 0.0714285714285714, 0.0714285714285714, 0.7857142857142857, 0.045733333333333333},
    {0.3994035761667992, 0.3994035761667992, 0.1005964238332008, 0.1005964238332008, 0.149333333333333333},
    {0.3994035761667992, 0.1005964238332008, 0.3994035761667992, 0.1005964238332008, 0.149333333333333333},
    {0.3994035761667992, 0.1005964238332008, 0.1005964238332008, 0.3994035761667992, 0.149333333333333333},
    {0.1005964238332008, 0.3994035761667992, 0.3994035761667992, 0.1005964238332008, 0.149333333333333333},
    {0.1005964238332008, 0.3994035761667992, 0.1005964238332008, 0.3994035761667992, 0.149333333333333333},
    {0.1005964238332008, 0.1005964238332008, 0.3994035761667992, 0.3994035761667992, 0.149333333333333333}};
__constant__ int c_edge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

__device__ __forceinline__ double p2_phi(int a, const double* l) {
  if (a < 4) return l[a] * (2.0 * l[a] - 1.0);
  return 4.0 * l[c_edge[a - 4][0]] * l[c_edge[a - 4][1]];
}

__device__ __forceinline__ void p2_grad(int a, const double* l, const double g[4][3], double out[3]) {
  if (a < 4) {
    double s = 4.0 * l[a] - 1.0;
    for (int d = 0; d < 3; ++d) out[d] = s * g[a][d];
  } else {
    int p = c_edge[a - 4][0], q = c_edge[a - 4][1];
    for (int d = 0; d < 3; ++d) out[d] = 4.0 * (l[q] * g[p][d] + l[p] * g[q][d]);
  }
}

constexpr int P2_WARPS = 4;

// P2: one warp per cell.  Lane 0 computes the geometry; the 4x10 gradient
// table goes to shared memory; lanes then take the 100 (a,b) blocks.
__global__ void __launch_bounds__(P2_WARPS * 32) assemble_p2_kernel(AsmArgs A) {
  __shared__ double sg[P2_WARPS][4][10][3];  // basis gradients at the 4 stiffness points
  __shared__ double sgeo[P2_WARPS][4][3];
  __shared__ double svol[P2_WARPS];
  __shared__ double sq[P2_WARPS][11][4];     // per load point: T_h - T_ref, f_h
  __shared__ int sv[P2_WARPS][10];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * P2_WARPS + wid;
  if (c >= A.n_cells) return;
  if (lane < 10) sv[wid][lane] = A.cells[10 * (size_t)c + lane];
  __syncwarp();
  int ok = 1;
  if (lane == 0) {
    double g[4][3], vol;
    ok = tet_geometry(A.coords, sv[wid], g, vol) ? 1 : 0;
    for (int k = 0; k < 4; ++k)
      for (int d = 0; d < 3; ++d) sgeo[wid][k][d] = g[k][d];
    svol[wid] = vol;
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) {
    if (lane == 0) atomicExch(A.bad_cell, 1);
    return;
  }
  __syncwarp();
  double g[4][3];
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) g[k][d] = sgeo[wid][k][d];
  const double vol = svol[wid];
  for (int t = lane; t < 40; t += 32) {
    int q = t / 10, a = t % 10;
    double gr[3];
    p2_grad(a, c_q4[q], g, gr);
    for (int d = 0; d < 3; ++d) sg[wid][q][a][d] = gr[d];
  }
  const int m = A.mat[c];
  double lam, mu;
  lame(A.props[3 * m], A.props[3 * m + 1], lam, mu);
  const double alpha = A.props[3 * m + 2];
  // load values at the 11 load points, one lane each
  const bool loads = A.T || A.body;
  if (loads && lane < 11) {
    const double* l = c_k11[lane];
    double Th = 0.0, fh[3] = {0, 0, 0};
    for (int ci = 0; ci < 10; ++ci) {
      const double ph = p2_phi(ci, l);
      const int nc = sv[wid][ci];
      if (A.T) Th += ph * A.T[nc];
      if (A.body)
        for (int d = 0; d < 3; ++d) fh[d] += ph * A.body[3 * (size_t)nc + d];
    }
    sq[wid][lane][0] = A.T ? Th - A.T_ref : 0.0;
    for (int d = 0; d < 3; ++d) sq[wid][lane][1 + d] = fh[d];
  }
  __syncwarp();
  // stiffness, 4-point rule: K_ab = sum_q w (lam g_a g_b^T + mu g_b g_a^T + mu (g_a . g_b) I)
  // for the 55 pairs a <= b, with the gradients pre-scaled by w lam and w mu;
  // K_ba = K_ab^T is scattered for b > a (FP64 is GB300's scarce pipe)
  const double wl = 0.25 * vol * lam, wm = 0.25 * vol * mu;
  for (int pidx = lane; pidx < 55; pidx += 32) {
    int a = 0, r = pidx;
    while (r >= 10 - a) {
      r -= 10 - a;
      ++a;
    }
    const int b = a + r;
    const int na = sv[wid][a], nb = sv[wid][b];
    const bool ab = !A.dmask[na] && block_needed(A, nb);
    const bool ba = b != a && !A.dmask[nb] && block_needed(A, na);
    if (!ab && !ba) continue;
    double k[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) k[e] = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double* ga = sg[wid][q][a];
      const double* gb = sg[wid][q][b];
      const double gb0 = gb[0], gb1 = gb[1], gb2 = gb[2];
      const double lga[3] = {wl * ga[0], wl * ga[1], wl * ga[2]};
      const double mga[3] = {wm * ga[0], wm * ga[1], wm * ga[2]};
      const double gbv[3] = {gb0, gb1, gb2};
      const double mgg = mga[0] * gb0 + mga[1] * gb1 + mga[2] * gb2;
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
          k[3 * ii + jj] += fma(lga[ii], gbv[jj], mga[jj] * gbv[ii]) + (ii == jj ? mgg : 0.0);
    }
    if (ab) scatter_block(A, c, a, b, na, nb, k);
    if (ba) {
      const double kt[9] = {k[0], k[3], k[6], k[1], k[4], k[7], k[2], k[5], k[8]};
      scatter_block(A, c, b, a, nb, na, kt);
    }
  }
  // loads, Keast 11-point rule: lane 3a + d sums component d of node a over the points
  if (loads && lane < 30) {
    const int a = lane / 3, d = lane % 3, na = sv[wid][a];
    if (!A.dmask[na]) {
      const double kT = (3.0 * lam + 2.0 * mu) * alpha;
      double f = 0.0;
      for (int q = 0; q < 11; ++q) {
        const double* l = c_k11[q];
        const double wq = l[4] * vol;
        double gr[3];
        p2_grad(a, l, g, gr);
        if (A.T) f += wq * kT * sq[wid][q][0] * gr[d];
        if (A.body) f += wq * p2_phi(a, l) * sq[wid][q][1 + d];
      }
      if (A.cf) A.cf[((size_t)c * 10 + a) * 3 + d] = f;
      else atomicAdd(&A.rhs[3 * (size_t)na + d], f);
    }
  }
}

// ---------------------------------------------------------------------------
// Deterministic assembly: the element kernels store every block and load in
// its own slot; per node, a warp sums its cells' slots in increasing cell id
// order into the node's row of K and its load (Dirichlet columns lifted) --
// the same sums as the atomic scatter, in an order fixed by the mesh, so two
// runs give bitwise equal K and f.
// ---------------------------------------------------------------------------
constexpr int DET_WARPS = 4;
constexpr int DET_CAP = 1024;  // cells per node the sorting pass handles

// each node's incident cells in increasing id (warp per node, shared-memory
// bitonic sort); a node in more than DET_CAP cells sets *bad
__global__ void __launch_bounds__(DET_WARPS * 32)
incidence_sort_kernel(int n_nodes, const int* __restrict__ ptr, int* __restrict__ inc, int* __restrict__ bad) {
  __shared__ int tab[DET_WARPS][DET_CAP];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * DET_WARPS + wid;
  if (v >= n_nodes) return;  // warp-uniform
  const int p0 = ptr[v], len = ptr[v + 1] - p0;
  if (len > DET_CAP) {
    if (lane == 0) atomicExch(bad, 1);
    return;
  }
  int* t = tab[wid];
  const int n2 = next_pow2(len);
  for (int i = lane; i < n2; i += 32) t[i] = i < len ? inc[p0 + i] : 0x7fffffff;
  __syncwarp();
  warp_bitonic_sort<false>(t, nullptr, n2);
  for (int i = lane; i < len; i += 32) inc[p0 + i] = t[i];
}

__global__ void __launch_bounds__(DET_WARPS * 32)
gather_kernel(int n_nodes, int npc, const int* __restrict__ cells, const int* __restrict__ ptr,
              const int* __restrict__ inc, const unsigned char* __restrict__ dmask, const double* __restrict__ ud,
              const int* __restrict__ rp, const int* __restrict__ ci, double* __restrict__ vals,
              double* __restrict__ rhs, const double* __restrict__ ck, const double* __restrict__ cf, int has_loads) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * DET_WARPS + wid;
  if (i >= n_nodes || dmask[i]) return;  // warp-uniform; Dirichlet rows: dirichlet_rows_kernel
  double f = 0.0;  // lane d < 3: component d of the node's load
  for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
    const int c = inc[p];
    const int* cn = cells + (size_t)c * npc;
    const unsigned m = __ballot_sync(0xffffffffu, lane < npc && cn[lane] == i);
    const int a = __ffs(m) - 1;  // the node's local index in cell c
    const double* kc = ck + ((size_t)c * npc + a) * npc * 9;
    if (has_loads && lane < 3) f += cf[((size_t)c * npc + a) * 3 + lane];
    if (vals)
      for (int it = lane; it < npc * 9; it += 32) {
        const int b = it / 9, e = it - b * 9, j = cn[b];
        if (dmask[j]) continue;
        const int slot = bsearch_i32(ci, rp[i], rp[i + 1], j);
        vals[(size_t)slot * 9 + e] += kc[it];
      }
    if (ud && lane < 3)
      for (int b = 0; b < npc; ++b) {
        const int j = cn[b];
        if (!dmask[j]) continue;
        const double* kb = kc + b * 9;
        const double* u = ud + 3 * (size_t)j;
        f -= kb[3 * lane] * u[0] + kb[3 * lane + 1] * u[1] + kb[3 * lane + 2] * u[2];
      }
    __syncwarp();
  }
  if (lane < 3) rhs[3 * (size_t)i + lane] = f;
}

// Dirichlet (and cell-less) rows: identity diagonal block, load = u_D.
__global__ void dirichlet_rows_kernel(int n, const unsigned char* __restrict__ dmask,
                                      const int* __restrict__ inc_ptr, const double* __restrict__ ud,
                                      const int* __restrict__ row_ptr, const int* __restrict__ col_idx,
                                      double* __restrict__ vals, double* __restrict__ rhs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool orphan = inc_ptr && inc_ptr[i + 1] == inc_ptr[i];
  if (!dmask[i] && !orphan) return;
  if (vals) {  // loads-only assembly leaves the existing K alone
    int slot = bsearch_i32(col_idx, row_ptr[i], row_ptr[i + 1], i);
    double* d = vals + (size_t)slot * 9;
    for (int e = 0; e < 9; ++e) d[e] = (e % 4 == 0) ? 1.0 : 0.0;
  }
  for (int r = 0; r < 3; ++r) rhs[3 * (size_t)i + r] = (dmask[i] && ud) ? ud[3 * (size_t)i + r] : 0.0;
}

}  // namespace

// Node and material ids of a mesh in range (INVALID_ARG otherwise).  Synchronising.
void validate_mesh(int n_nodes, int n_cells, int npc, const int* cells, const int* mat, int n_mat, const char* who,
                   cudaStream_t s) {
  if (n_cells <= 0) return;
  const long long n_entries = (long long)n_cells * npc;
  DBuf<int> bad(1, s);
  bad.zero();
  validate_kernel<<<grid_for(n_entries, 256), 256, 0, s>>>(cells, n_entries, npc, n_nodes, mat, n_cells, n_mat,
                                                            bad.p);
  TAM_LAUNCH_CHECK();
  const int b = read_back_int(bad.p, s);
  TAM_CHECK(b == 0, TAM_ERR_INVALID_ARG,
            std::string(who) + (b == 1 ? ": cell node id out of range" : ": material id out of range"));
}

// Node-adjacency pattern of a mesh: block row i holds i and every node that
// shares a cell with it, sorted, without the Dirichlet nodes (dmask) -- whose
// own rows keep only the diagonal.  Fills A.n_rows/n_cols, row_ptr, col_idx
// and nnzb (block sizes are the caller's), and returns the cell-node
// incidence (inc_ptr[n_nodes + 1], inc) that the pattern came from.  flag[1]
// is set when a node has too many incident cells for the shared-memory
// builder.  Synchronising.
// 64-bit sum of per-row counts (overflow check before an int32 scan)
__global__ void count_sum_kernel(const int* __restrict__ cnt, int n, unsigned long long* __restrict__ out) {
  unsigned long long v = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v += (unsigned long long)(unsigned)cnt[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

void build_node_pattern(int n_nodes, int n_cells, int npc, const int* cells, const unsigned char* dmask, Bsr& A,
                        DBuf<int>& inc_ptr, DBuf<int>& inc, int* flag, cudaStream_t s) {
  const long long n_entries = (long long)n_cells * npc;
  // cell-node incidence
  inc_ptr = DBuf<int>((size_t)n_nodes + 1, s);
  inc = DBuf<int>((size_t)std::max(1LL, n_entries), s);
  DBuf<int> cursor((size_t)n_nodes, s);
  inc_ptr.zero();
  cursor.zero();
  if (n_cells > 0) {
    incidence_count_kernel<<<grid_for(n_entries, 256), 256, 0, s>>>(cells, n_entries, inc_ptr.p);
    TAM_LAUNCH_CHECK();
  }
  exclusive_scan_i32(inc_ptr.p, inc_ptr.p, n_nodes, s);
  if (n_cells > 0) {
    incidence_fill_kernel<<<grid_for(n_entries, 256), 256, 0, s>>>(cells, n_entries, npc, inc_ptr.p, cursor.p,
                                                                   inc.p);
    TAM_LAUNCH_CHECK();
  }
  // pattern
  A.n_rows = A.n_cols = n_nodes;
  A.row_ptr = DBuf<int>((size_t)n_nodes + 1, s);
  unsigned pg = grid_for(n_nodes, PAT_WARPS);
  if (3 * ((long long)n_nodes + (long long)npc * npc * n_cells) < (1LL << 31)) {
    // one sort pass: each row's sorted unique columns go to its candidate-
    // bound offset in a scratch array (the bounds' sum, at most
    // 3 (n_nodes + npc^2 n_cells), fits the int32 scan), the counts give
    // row_ptr, then pack
    DBuf<int> bptr((size_t)n_nodes + 1, s);
    pattern_bound_kernel<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, npc, inc_ptr.p, dmask, bptr.p);
    TAM_LAUNCH_CHECK();
    exclusive_scan_i32(bptr.p, bptr.p, n_nodes, s);
    const long long total = read_back_int(bptr.p + n_nodes, s);
    DBuf<int> tmp((size_t)std::max(1LL, total), s);
    // flag[1]: overflow beyond the list; big[0]: rows listed for pattern_big_kernel
    const int big_cap = std::max(1, std::min(n_nodes, 1 << 20));
    DBuf<int> big_list((size_t)big_cap, s), big(2, s);
    big.zero();
    pattern_kernel<true><<<pg, PAT_WARPS * 32, 0, s>>>(n_nodes, npc, cells, inc_ptr.p, inc.p, dmask, A.row_ptr.p,
                                                      bptr.p, tmp.p, big.p, big_list.p, big_cap);
    TAM_LAUNCH_CHECK();
    int n_big = 0, big_over = 0;
    read_back_int2(big.p + 1, big.p, &n_big, &big_over, s);
    TAM_CHECK(big_over == 0, TAM_ERR_UNSUPPORTED, "fem_assemble: too many high-valence nodes for the pattern builder");
    if (n_big > 0) {
      pattern_big_kernel<<<n_big, BIG_THREADS, 0, s>>>(big_list.p, npc, cells, inc_ptr.p, inc.p, dmask, bptr.p, tmp.p,
                                                      A.row_ptr.p);
      TAM_LAUNCH_CHECK();
    }
    exclusive_scan_i32(A.row_ptr.p, A.row_ptr.p, n_nodes, s);
    A.nnzb = read_back_int(A.row_ptr.p + n_nodes, s);
    A.col_idx = DBuf<int>((size_t)std::max(1LL, A.nnzb), s);
    pattern_pack_kernel<<<grid_for((long long)n_nodes * 32, 256), 256, 0, s>>>(n_nodes, bptr.p, tmp.p,
                                                                               A.row_ptr.p, A.col_idx.p);
    TAM_LAUNCH_CHECK();
  } else {
    // very large meshes: count pass, then fill pass (no scratch)
    pattern_kernel<false><<<pg, PAT_WARPS * 32, 0, s>>>(n_nodes, npc, cells, inc_ptr.p, inc.p, dmask, A.row_ptr.p,
                                                       nullptr, nullptr, flag + 1);
    TAM_LAUNCH_CHECK();
    {
      // block counts are int32 (K's arrays): refuse a pattern of 2^31 blocks or more
      DBuf<unsigned long long> tot(1, s);
      tot.zero();
      count_sum_kernel<<<stride_grid(n_nodes, 256, 8), 256, 0, s>>>(A.row_ptr.p, n_nodes, tot.p);
      TAM_LAUNCH_CHECK();
      TAM_CHECK(read_back_ll(reinterpret_cast<const long long*>(tot.p), s) < (1LL << 31), TAM_ERR_UNSUPPORTED,
                "fem_assemble: K would have 2^31 or more 3x3 blocks (int32 indices)");
    }
    exclusive_scan_i32(A.row_ptr.p, A.row_ptr.p, n_nodes, s);
    A.nnzb = read_back_int(A.row_ptr.p + n_nodes, s);
    TAM_CHECK(read_back_int(flag + 1, s) == 0, TAM_ERR_UNSUPPORTED,
              "fem_assemble: a node has too many incident cells for the pattern builder");
    A.col_idx = DBuf<int>((size_t)A.nnzb, s);
    pattern_kernel<true><<<pg, PAT_WARPS * 32, 0, s>>>(n_nodes, npc, cells, inc_ptr.p, inc.p, dmask, nullptr,
                                                      A.row_ptr.p, A.col_idx.p, flag + 1);
    TAM_LAUNCH_CHECK();
  }
}

std::atomic<int> g_deterministic_assembly{0};

// Deterministic assembly's second pass: sort the incidence lists, sum the
// slots per node (vals may be null: loads only).
static void gather_assembly(const AsmArgs& args, int n_nodes, int npc, const int* cells, const int* inc_ptr,
                            int* inc, const unsigned char* dmask, double* vals, double* rhs, bool has_loads,
                            cudaStream_t s) {
  DBuf<int> bad(1, s);
  bad.zero();
  incidence_sort_kernel<<<grid_for(n_nodes, DET_WARPS), DET_WARPS * 32, 0, s>>>(n_nodes, inc_ptr, inc, bad.p);
  TAM_LAUNCH_CHECK();
  TAM_CHECK(read_back_int(bad.p, s) == 0, TAM_ERR_UNSUPPORTED,
            "fem_assemble: deterministic assembly handles nodes in at most 1024 cells");
  gather_kernel<<<grid_for(n_nodes, DET_WARPS), DET_WARPS * 32, 0, s>>>(
      n_nodes, npc, cells, inc_ptr, inc, dmask, args.ud, args.row_ptr, args.col_idx, vals, rhs, args.ck, args.cf,
      has_loads ? 1 : 0);
  TAM_LAUNCH_CHECK();
}

tam_matrix_s* assemble_elasticity(int n_nodes, const double* coords, int n_cells, int npc, const int* cells,
                                  const int* mat, int n_mat, const double* props, const double* T,
                                  double T_ref, const double* body, const unsigned char* dmask,
                                  const double* ud, double* rhs, cudaStream_t s) {
  NvtxRange nvtx("tam: assemble K and f");
  TAM_CHECK(n_nodes > 0 && n_cells >= 0 && n_mat > 0, TAM_ERR_INVALID_ARG, "fem_assemble: bad sizes");
  TAM_CHECK(npc == 4 || npc == 10, TAM_ERR_INVALID_ARG, "fem_assemble: nodes_per_cell must be 4 or 10");
  TAM_CHECK(coords && (cells || n_cells == 0) && (mat || n_cells == 0) && props && dmask && rhs,
            TAM_ERR_INVALID_ARG, "fem_assemble: null pointer");
  auto M = new tam_matrix_s();
  M->nodes_per_cell = npc;
  try {
    M->n_nodes = n_nodes;
    const long long n_entries = (long long)n_cells * npc;
    DBuf<int> flag(2, s);
    flag.zero();
    if (n_cells > 0) {
      validate_kernel<<<grid_for(n_entries, 256), 256, 0, s>>>(cells, n_entries, npc, n_nodes, mat, n_cells,
                                                                n_mat, flag.p);
      TAM_LAUNCH_CHECK();
      int bad = read_back_int(flag.p, s);
      TAM_CHECK(bad == 0, TAM_ERR_INVALID_ARG,
                bad == 1 ? "fem_assemble: cell node id out of range" : "fem_assemble: material id out of range");
    }
    // cell-node incidence and block pattern
    Bsr& A = M->A;
    A.br = A.bc = 3;
    DBuf<int> inc_ptr, inc;
    build_node_pattern(n_nodes, n_cells, npc, cells, dmask, A, inc_ptr, inc, flag.p, s);
    // numeric
    A.vals = DBuf<double>((size_t)A.nnzb * 9, s);
    A.vals.zero();
    TAM_CUDA(cudaMemsetAsync(rhs, 0, sizeof(double) * 3 * (size_t)n_nodes, s));
    AsmArgs args{coords, cells, mat, props, T, T_ref, body, dmask, ud, A.row_ptr.p, A.col_idx.p,
                 A.vals.p, rhs, n_cells, flag.p, 0};
    const bool det = g_deterministic_assembly.load() != 0 && n_cells > 0;
    DBuf<double> ck, cf;
    if (det) {
      ck = DBuf<double>((size_t)n_cells * npc * npc * 9, s);
      cf = DBuf<double>((size_t)n_cells * npc * 3, s);
      args.ck = ck.p;
      args.cf = cf.p;
      args.npc = npc;
    }
    if (n_cells > 0) {
      if (npc == 4)
        assemble_p1_kernel<<<grid_for(n_cells, 128), 128, 0, s>>>(args);
      else
        assemble_p2_kernel<<<grid_for(n_cells, P2_WARPS), P2_WARPS * 32, 0, s>>>(args);
      TAM_LAUNCH_CHECK();
    }
    if (det) gather_assembly(args, n_nodes, npc, cells, inc_ptr.p, inc.p, dmask, A.vals.p, rhs, T || body, s);
    dirichlet_rows_kernel<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, dmask, inc_ptr.p, ud, A.row_ptr.p,
                                                                 A.col_idx.p, A.vals.p, rhs);
    TAM_LAUNCH_CHECK();
    TAM_CHECK(read_back_int(flag.p, s) == 0, TAM_ERR_DEGENERATE_CELL,
              "fem_assemble: a cell has non-positive or non-finite volume");
    {
      operator_exponent_range(A, &M->vmax_exp, &M->finite, s);
      M->df_ok = M->finite && std::abs(M->vmax_exp) <= kDfExpLimit;
    }
    M->dmask = DBuf<unsigned char>((size_t)n_nodes, s);
    TAM_CUDA(cudaMemcpyAsync(M->dmask.p, dmask, n_nodes, cudaMemcpyDeviceToDevice, s));
    // split copies for the double-float SpMV: SELL always (the CG's own SpMVs
    // with K use it; written by the SELL fill), the block-CSR only where K's
    // operator runs on it
    // (none when K is outside the double-float range: every product is FP64)
    bsr_to_sell(A, M->S, s, M->df_ok);
    if (M->df_ok && choose_lpr(A) != 0) build_df_values(A, s);
    TAM_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    delete M;
    throw;
  }
  return M;
}

// Load vector of another load case on the mesh of an existing K: thermal and
// body loads (and the lifting of prescribed displacements), Dirichlet rows
// set to u_D; K itself is not touched.
void assemble_loads(tam_matrix_s* K, const double* coords, int n_cells, int npc, const int* cells, const int* mat,
                    int n_mat, const double* props, const double* T, double T_ref, const double* body,
                    const double* ud, double* rhs, cudaStream_t s) {
  NvtxRange nvtx("tam: assemble f");
  TAM_CHECK(K && coords && props && rhs && n_mat > 0 && n_cells >= 0 && (npc == 4 || npc == 10) &&
                (cells || n_cells == 0) && (mat || n_cells == 0),
            TAM_ERR_INVALID_ARG, "fem_assemble_load: bad argument");
  const int n_nodes = K->n_nodes;
  DBuf<int> flag(2, s);
  flag.zero();
  const long long n_entries = (long long)n_cells * npc;
  if (n_cells > 0) {
    validate_kernel<<<grid_for(n_entries, 256), 256, 0, s>>>(cells, n_entries, npc, n_nodes, mat, n_cells, n_mat,
                                                              flag.p);
    TAM_LAUNCH_CHECK();
    TAM_CHECK(read_back_int(flag.p, s) == 0, TAM_ERR_INVALID_ARG, "fem_assemble_load: cell or material id out of range");
  }
  TAM_CUDA(cudaMemsetAsync(rhs, 0, sizeof(double) * 3 * (size_t)n_nodes, s));
  AsmArgs args{coords, cells, mat, props, T, T_ref, body, K->dmask.p, ud, K->A.row_ptr.p, K->A.col_idx.p,
               nullptr, rhs, n_cells, flag.p + 1, 1};
  const bool det = g_deterministic_assembly.load() != 0 && n_cells > 0;
  DBuf<double> ck, cf;
  DBuf<int> inc_ptr, inc;
  if (det) {
    ck = DBuf<double>((size_t)n_cells * npc * npc * 9, s);
    cf = DBuf<double>((size_t)n_cells * npc * 3, s);
    args.ck = ck.p;
    args.cf = cf.p;
    args.npc = npc;
    inc_ptr = DBuf<int>((size_t)n_nodes + 1, s);
    inc = DBuf<int>((size_t)n_entries, s);
    DBuf<int> cursor((size_t)n_nodes, s);
    inc_ptr.zero();
    cursor.zero();
    incidence_count_kernel<<<grid_for(n_entries, 256), 256, 0, s>>>(cells, n_entries, inc_ptr.p);
    TAM_LAUNCH_CHECK();
    exclusive_scan_i32(inc_ptr.p, inc_ptr.p, n_nodes, s);
    incidence_fill_kernel<<<grid_for(n_entries, 256), 256, 0, s>>>(cells, n_entries, npc, inc_ptr.p, cursor.p,
                                                                   inc.p);
    TAM_LAUNCH_CHECK();
  }
  if (n_cells > 0) {
    if (npc == 4)
      assemble_p1_kernel<<<grid_for(n_cells, 128), 128, 0, s>>>(args);
    else
      assemble_p2_kernel<<<grid_for(n_cells, P2_WARPS), P2_WARPS * 32, 0, s>>>(args);
    TAM_LAUNCH_CHECK();
  }
  if (det) gather_assembly(args, n_nodes, npc, cells, inc_ptr.p, inc.p, K->dmask.p, nullptr, rhs, T || body, s);
  dirichlet_rows_kernel<<<grid_for(n_nodes, 256), 256, 0, s>>>(n_nodes, K->dmask.p, nullptr, ud, nullptr, nullptr,
                                                               nullptr, rhs);
  TAM_LAUNCH_CHECK();
  TAM_CHECK(read_back_int(flag.p + 1, s) == 0, TAM_ERR_DEGENERATE_CELL,
            "fem_assemble_load: a cell has non-positive or non-finite volume");
}

}  // namespace tam
