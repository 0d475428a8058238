// Opaque handle types behind the C ABI and the internal entry points that
// the C ABI wraps.
#pragma once

#include <atomic>
#include <functional>
#include <memory>
#include <vector>

#include "sparse.cuh"

struct tam_matrix_s {
  int n_nodes = 0;
  int nodes_per_cell = 0;              // 4 (P1) or 10 (P2) tetrahedra
  // floor(log2 max |K_ij|) over the rows with off-diagonal blocks, and whether
  // K is finite and within the double-float range (|exponent| <= kDfExpLimit):
  // else every product with K is plain FP64
  int vmax_exp = 0;
  bool finite = true;
  bool df_ok = true;
  tam::Bsr A;                          // 3x3 blocks, Dirichlet rows are identity rows
  tam::Sell S;                         // SELL-32 copy used by every SpMV with K
  tam::DBuf<unsigned char> dmask;      // Dirichlet mask [n_nodes]
};

namespace tam {

// Device-side state of one PCG solve (one per hierarchy).
struct PcgScalars {
  double rho;       // r . z of the current iterate
  double alpha, beta;
  double rr;        // ||r||^2
  double tol2;      // stop when rr <= tol2
  double bb;        // ||b||^2
  int iter;
  int max_iter;
  int stop;         // nonzero: every solver kernel returns at entry
  int status;       // TAM_OK or a TAM_ERR_* code
  int scale_exp;    // the solve runs on b 2^-scale_exp and x 2^-scale_exp (exact)
  int loops;        // iterations the device-side loop has run (its failsafe count)
};

struct Level {
  int n_rows = 0;     // block rows
  int bs = 0;         // block size of A on this level
  int kdim = 0;       // near-nullspace columns (block size of the next level)
  int deg = 2;        // Chebyshev degree used on this level
  const Bsr* A = nullptr;   // level 0: the matrix handle's K
  const Sell* AS = nullptr;
  Bsr A_own;
  Sell AS_own;
  DBuf<double> dinv;        // point-Jacobi inverse diagonal [n_rows*bs] (0 on zero diagonals)
  DBuf<double> consts;      // [0] lambda_max, [1] omega, [2..] Chebyshev (c_d, c_r) per step
  DBuf<int> agg;            // aggregate id per block row (-1 = none)
  int n_agg = 0;
  Bsr Pt, P, R;             // tentative prolongator, smoothed prolongator, R = P^T
  Sell PS, RS;
  SpOp Aop, Pop, Rop;       // SpMV strategy per operator (SELL thread-per-row or lanes per row)
  LprStore AL, PL, RL;      // interleaved lanes-per-row copies of the operators that use lanes per row
  // V-cycle work vectors (n_rows*bs each)
  DBuf<double> b, xa, xb, d, t, y;  // y: the level's V-cycle result (never an internal buffer)
  double lambda_host = 0.0;
  // reduced-precision V-cycle (level_precision 1: FP32; 2: FP32 with BF16 finest-level values)
  DBuf<float> dinv32, consts32, b32, xa32, xb32, d32, t32, y32;
  DBuf<float> A32v, P32v, R32v;
  DBuf<__nv_bfloat16> A16v;
  SpOpLow<float> A32, P32, R32;
  SpOpLow<__nv_bfloat16> A16;
};

// Multi-right-hand-side solve state (block of independent CGs sharing every
// SpMV as a multi-vector product).  Vectors are interleaved [rows][bs][mp]
// with the RHS index fastest; mp = RHS count padded to a multiple of 8.
// Launch shape of one multi-RHS SpMM, picked by the autotuner: right-hand
// sides per thread, threads per CTA (rows per CTA for thread-per-row SELL),
// and lanes per block row for the block-CSR layout (0: the operator's own).
struct MTile {
  int tm = 8, threads = 128, lpr = 0;
};

struct MultiLevel {
  DBuf<float> b, xa, xb, d, t, y;
  MTile tA, tP, tR;
};

struct MultiState {
  int mp = 0;
  DBuf<double> b, x, r, z, p, q;  // FP64 CG vectors [3n][mp]
  DBuf<double> sc;                // per-RHS scalars [8][mp]
  DBuf<int> flags;                // [0] stop, [1] iteration, [2] max_iter, [3] status
  DBuf<double> partials;
  DBuf<unsigned int> tickets;     // one per RHS chunk
  std::vector<MultiLevel> lv;
  MTile tK;
  double tune_ms = 0.0;
  unsigned long long serial = 0;  // unique per workspace: batch graphs are keyed on it
  // the last batch solve's loop graph, kept by the batch's first system: valid
  // while the batch names the same workspaces (serials) in the same order
  struct BatchGraph {
    std::vector<unsigned long long> key;
    cudaGraphExec_t exec = nullptr;
    DBuf<int*> fl;   // the systems' flag arrays
    DBuf<int> all;   // [0] all stopped, [1] loop count
    long long kernels = 0;
    ~BatchGraph() {
      if (exec) cudaGraphExecDestroy(exec);
    }
  };
  std::unique_ptr<BatchGraph> batch;
};

}  // namespace tam

struct tam_amg_s {
  tam_matrix_s* K = nullptr;
  amg_params prm{};
  std::vector<tam::Level> levels;
  int n_coarse = 0;                      // dense coarsest size (scalars)
  tam::DBuf<double> coarse_inv;          // [n_coarse * n_coarse]
  // PCG workspace
  tam::DBuf<double> r, z, p, q;
  tam::DBuf<double> bs, xs;              // b and x scaled by the solve's power of two
  tam::DBuf<double> hist;                // ||r_k||^2 of the last solve (scaled), k = 0 .. hist_len - 1
  long long hist_len = 0;
  int hist_scale_exp = 0;
  tam::DBuf<tam::PcgScalars> sc;
  tam::DBuf<double> partials;            // grid-reduction partials
  tam::DBuf<unsigned int> ticket;
  int max_grid = 0;
  // captured V-cycle + iteration graph (on the hierarchy's own vectors; rebuilt
  // when the finest level is refreshed)
  cudaGraphExec_t iter_exec = nullptr;
  long long graph_kernels = 0;           // kernel nodes in iter_exec
  double setup_ms[8] = {};               // setup phase times, see amg_setup_stats
  // Chebyshev coefficients of the last smooth_fine call (degree, interval)
  tam::DBuf<double> smooth_coef;
  int smooth_deg = 0;
  double smooth_lo = 0.0, smooth_hi = 0.0;
  std::unique_ptr<tam::MultiState> multi;  // multi-RHS workspace (built on first use)
  ~tam_amg_s();
};

namespace tam {

// Mesh topology shared by the elastic and the thermal assembly (assemble.cu).
// Process-wide assembly mode: nonzero sums element contributions per node in
// cell order (bitwise reproducible) instead of scattering them with atomics.
extern std::atomic<int> g_deterministic_assembly;

void validate_mesh(int n_nodes, int n_cells, int npc, const int* cells, const int* mat, int n_mat, const char* who,
                   cudaStream_t s);
void build_node_pattern(int n_nodes, int n_cells, int npc, const int* cells, const unsigned char* dmask, Bsr& A,
                        DBuf<int>& inc_ptr, DBuf<int>& inc, int* flag, cudaStream_t s);

tam_matrix_s* assemble_elasticity(int n_nodes, const double* coords, int n_cells, int npc, const int* cells,
                                  const int* mat, int n_mat, const double* props, const double* T,
                                  double T_ref, const double* body, const unsigned char* dmask,
                                  const double* ud, double* rhs, cudaStream_t s);

void assemble_loads(tam_matrix_s* K, const double* coords, int n_cells, int npc, const int* cells, const int* mat,
                    int n_mat, const double* props, const double* T, double T_ref, const double* body,
                    const double* ud, double* rhs, cudaStream_t s);

tam_amg_s* amg_build(tam_matrix_s* K, const double* coords, const amg_params& prm, cudaStream_t s);
// Finest-level data of H refreshed after K's values changed in place.
void amg_refresh_finest(tam_amg_s* H, cudaStream_t s);

// One V-cycle z = M^-1 r on level 0 (r, z device vectors of the fine size).
void vcycle_apply(tam_amg_s* H, const double* r, double* z, const int* stop, cudaStream_t s);
// The reduced-precision V-cycle (FP32 vectors and arithmetic; FP64 in/out on
// level 0 and FP64 dense coarsest solve), and its set-up after amg_build.
void vcycle_apply_low(tam_amg_s* H, const double* r, double* z, const int* stop, cudaStream_t s);
void build_low_precision(tam_amg_s* H, cudaStream_t s);
// x <- degree Chebyshev-Jacobi steps on K x = b from x over [lo, hi] * lambda_max(D^-1 K)
void smooth_fine(tam_amg_s* H, const double* b, double* x, int degree, double lo, double hi, cudaStream_t s);

int pcg_solve_batch(int n_sys, tam_amg_s* const* H, const int* m, const double* const* B, double* const* X,
                    double rtol, double atol, int max_iter, int* iters, double* rel, cudaStream_t s);
double multi_tune_ms(tam_amg_s* H);
void multi_tiles(tam_amg_s* H, int* out, int cap);

int pcg_solve(tam_amg_s* H, const double* b, double* x, double rtol, double atol, int max_iter, int* iters,
              double* rel, cudaStream_t s);

// A CUDA graph whose one conditional WHILE node repeats the work enqueue(s)
// puts on a stream (captured once as the node's body, followed by a one-thread
// kernel that sets the loop condition) for as long as the device flag *stop is
// 0 -- no host round trip per iteration.  Failsafe: at most *limit + limit_add
// passes, counted in *count, which must be zero when the graph is launched.
// *body_kernels receives the body's kernel count.
cudaGraphExec_t build_loop_graph(const std::function<void(cudaStream_t)>& enqueue, const int* stop, int* count,
                                 const int* limit, int limit_add, long long* body_kernels);

void spmv_K(tam_matrix_s* K, const double* x, double* y, cudaStream_t s);
double residual_norm_K(tam_matrix_s* K, const double* b, const double* x, cudaStream_t s);

long long launches_total();
long long captured_and_reset();

}  // namespace tam
