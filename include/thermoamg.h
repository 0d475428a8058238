/*
 * thermoamg.h -- C ABI of the GB300 (sm_103a) thermoelastic solver.
 *
 * The library solves the steady linear-elastic part of the paper's
 * thermomechanical model (Sec. 3: Eqs. elasticity_bvp, u-dbc and the weak
 * form wf_elastic with the thermal strain eps_T = alpha (T - T_ref) I) on
 * P1/P2 Lagrange tetrahedra, by conjugate gradients (Sec. 2.1, "Iterative
 * solvers") preconditioned with a smoothed-aggregation AMG V-cycle whose
 * near-nullspace is the six rigid-body modes (Sec. 2.1, "Multigrid
 * preconditioned iterative solvers"; Sec. 5.1, "Solver configuration":
 * Chebyshev smoothing with estimated lambda_max, controlled coarsening and a
 * direct coarsest-grid solve).
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: TAM_OK (0) or a negative TAM_ERR_*
 *    code.  tam_last_error() gives a message for the calling thread's last
 *    failure.  No entry point aborts the process.
 *  - Array arguments are DEVICE pointers unless the name ends in _host.  They
 *    are owned by the caller and only read (const) or written in place.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; calls documented as "synchronising"
 *    wait for it before returning.
 *  - Node ids and cell ids are int32.  Vectors of displacement DOFs are
 *    node-major: dof = 3*node + component.
 *  - Handles (tam_matrix, tam_amg) own device memory allocated by the library
 *    (stream-ordered from the device's default memory pool) and release it in
 *    *_destroy.  A handle must be used from one host thread at a time.
 */
#ifndef THERMOAMG_H
#define THERMOAMG_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TAM_OK = 0,
  TAM_ERR_INVALID_ARG = -1,        /* bad pointer, size, index or parameter       */
  TAM_ERR_CUDA = -2,               /* a CUDA runtime call failed                  */
  TAM_ERR_OOM = -3,                /* device allocation failed                    */
  TAM_ERR_DEGENERATE_CELL = -4,    /* a cell has non-positive or non-finite volume */
  TAM_ERR_NOT_CONVERGED = -5,      /* max_iter reached before the tolerance        */
  TAM_ERR_BREAKDOWN = -6,          /* CG: p^T K p <= 0                            */
  TAM_ERR_INDEFINITE_PRECOND = -7, /* CG: r^T M^-1 r <= 0 (bad Chebyshev bounds)  */
  TAM_ERR_NAN = -8,                /* NaN/Inf met in the solve                    */
  TAM_ERR_INTERNAL = -9,           /* internal capacity/consistency check failed   */
  TAM_ERR_UNSUPPORTED = -10        /* valid request this build does not support    */
};

typedef struct tam_matrix_s* tam_matrix; /* assembled 3x3-block sparse K (+ metadata) */
typedef struct tam_amg_s* tam_amg;       /* SA-AMG hierarchy bound to one tam_matrix  */

/* Message for the calling thread's last failing call ("" if none). */
const char* tam_last_error(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (kernels replayed from its CUDA graphs included).  Instrumentation for
 * benchmarks; never fails. */
long long tam_kernel_launches(void);

/* Measured FMA throughput of the current device's FP64 and FP32 pipes in
 * TFLOP/s (2 flops per FMA; best of 5 launches of 8 independent FMA chains
 * per thread, 8 blocks of 256 threads per SM), into host doubles (either may
 * be NULL).  Instrumentation: the rate that decides whether a matrix product
 * is bound by memory or by the FP64 pipe; the paper has no counterpart.
 * Synchronising.  Errors: INVALID_ARG, CUDA. */
int tam_fma_throughput(double* fp64_tflops_host, double* fp32_tflops_host, void* stream);

/* ------------------------------------------------------------------------
 * Assembly (Sec. 3, Eq. wf_elastic, steady, traction free; Eq. u-dbc).
 *
 * Builds the block-CSR pattern of K from the cell-node incidence, evaluates
 * the element stiffness int C:eps(u):eps(v), the thermal load
 * int C:eps_T(T_h):eps(v) and the body load int f_h.v on every cell
 * (T_h, f_h: nodal interpolants in the same P1/P2 space), scatters them,
 * then eliminates the Dirichlet nodes symmetrically: the load is lifted by
 * -K_{:,D} u_D, rows and columns of Dirichlet nodes are zeroed, their
 * diagonal block becomes I and their load entries u_D.  A node in no cell
 * gets an identity row and a zero load (u_D if it is a Dirichlet node);
 * n_cells = 0 gives K = I.
 *
 *  n_nodes, coords[n_nodes*3]      node coordinates (float64, xyz per node)
 *  n_cells, nodes_per_cell          4 (P1) or 10 (P2; vertices 0-3 then the
 *                                   mid-edge nodes of edges 01,02,03,12,13,23)
 *  cells[n_cells*nodes_per_cell]    node ids (int32), positively oriented
 *  cell_material[n_cells]           material id in [0, n_mat)
 *  mat_props[n_mat*3]               E, nu, alpha per material (float64)
 *  T[n_nodes] (may be NULL)         nodal temperature; NULL = T_ref everywhere
 *  T_ref                            reference temperature
 *  body_force[n_nodes*3] (NULL = 0) nodal body-force density
 *  dirichlet_mask[n_nodes]          uint8, nonzero = all 3 components fixed
 *  u_dirichlet[n_nodes*3] (NULL = 0) prescribed displacement on masked nodes
 *  K_out                            receives the new matrix handle
 *  rhs_out[n_nodes*3]               receives the load vector (written)
 * Synchronising (the pattern size is read back).  Errors: INVALID_ARG for
 * bad sizes/pointers, DEGENERATE_CELL if any cell volume is <= 0 or not
 * finite (no handle is returned), OOM, CUDA.
 */
int fem_assemble_elasticity(int n_nodes, const double* coords, int n_cells, int nodes_per_cell,
                            const int* cells, const int* cell_material, int n_mat,
                            const double* mat_props, const double* T, double T_ref,
                            const double* body_force, const unsigned char* dirichlet_mask,
                            const double* u_dirichlet, tam_matrix* K_out, double* rhs_out,
                            void* stream);

/* Assembly mode for fem_assemble_elasticity / fem_assemble_load (process-wide,
 * default 0).  0: element blocks and loads are scattered with FP64 atomics
 * (fastest; the summation order, hence the last bits of K and f, may differ
 * between runs).  1: deterministic -- every element block and load is stored
 * in its own slot (n_cells * npc^2 * 9 + n_cells * npc * 3 doubles of
 * temporary device memory) and each node's warp sums its cells' slots in
 * increasing cell id, so two runs give bitwise equal K and f (the element
 * contributions are the same; only the order of the sums is fixed).  Nodes in
 * more than 1024 cells return UNSUPPORTED in mode 1.  *previous (may be NULL)
 * receives the old mode.  Not tied to a stream; set it between calls. */
int tam_set_deterministic_assembly(int on, int* previous);

/* Load vector of another load case on the mesh of an existing K (same
 * coords/cells/materials/Dirichlet mask as K was assembled with): thermal and
 * body loads of Eq. wf_elastic plus the lifting of u_dirichlet, Dirichlet
 * entries = u_D; K is not modified.  Argument meaning as in
 * fem_assemble_elasticity; rhs_out[n_nodes*3] is written.  Synchronising.
 * Errors: INVALID_ARG, DEGENERATE_CELL, CUDA. */
int fem_assemble_load(tam_matrix K, const double* coords, int n_cells, int nodes_per_cell,
                      const int* cells, const int* cell_material, int n_mat, const double* mat_props,
                      const double* T, double T_ref, const double* body_force,
                      const double* u_dirichlet, double* rhs_out, void* stream);

/* Sizes of K: block rows (= n_nodes), stored 3x3 blocks, block size (3). */
int tam_matrix_info(tam_matrix K, int* n_block_rows, long long* nnzb, int* block_size);

/* Copies K in block-CSR form: row_ptr[n+1], col_idx[nnzb] (sorted per row),
 * vals[nnzb*9] (row-major 3x3 blocks).  Device pointers; synchronising. */
int tam_matrix_export_bsr(tam_matrix K, int* row_ptr, int* col_idx, double* vals, void* stream);

/* y = K x (x, y: [3n] float64 device vectors, must not overlap).  The
 * product is the solve's own: double-float products on K's split values
 * (see amg_params.spmv_fp64), FP64 vectors in and out. */
int tam_matrix_spmv(tam_matrix K, const double* x, double* y, void* stream);

/* ||b - K x||_2 into *norm_host (host double): the true residual of a
 * candidate displacement, the quantity the CG stopping test of Sec. 2.1 is
 * measured by.  b, x: [3n] float64 device vectors.  One fused SpMV + grid
 * reduction in plain FP64 arithmetic; its per-block partial sums live in
 * scratch memory the call allocates stream-ordered and frees again.
 * Synchronising.
 * Errors: INVALID_ARG, OOM, CUDA. */
int tam_matrix_residual_norm(tam_matrix K, const double* b, const double* x, double* norm_host,
                             void* stream);

/* Same result as tam_matrix_residual_norm, for callers that must not
 * allocate device memory (code inside a custom allocator or pool callback,
 * applications with a device-memory budget fixed at start-up, paths that
 * cannot take cudaMalloc's implicit synchronisation).  The paper has no
 * counterpart; this is a library-integration entry point.
 *  - Allocates nothing: the reduction scratch is a 128 KiB file-scope device
 *    array that every device loading the library keeps until exit.
 *  - Limit: K with at most 2,097,152 block rows (16384 blocks of 128 rows);
 *    larger K returns INVALID_ARG without launching anything.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it; make that call before any stream
 *    capture begins.  The cache does not survive cudaDeviceReset: do not call
 *    this entry point on a device after resetting it.
 *  - All calls share the array: calls whose work overlaps on the GPU race.
 * b, x: [3n] float64 device vectors; *norm_host receives ||b - K x||_2.
 * Synchronising.  Errors: INVALID_ARG, CUDA. */
int tam_matrix_residual_norm_noalloc(tam_matrix K, const double* b, const double* x,
                                     double* norm_host, void* stream);

/* Releases K (an AMG built on K must be destroyed first). */
int tam_matrix_destroy(tam_matrix K);

/* ------------------------------------------------------------------------
 * Smoothed-aggregation AMG (Sec. 2.1 and Sec. 5.1).  The paper fixes the
 * method (SA-AMG with the rigid-body near-nullspace, Chebyshev smoothing
 * with estimated lambda_max, controllable coarsening, a larger coarsest grid
 * for robustness) but not its constants; these are the knobs.
 */
typedef struct amg_params {
  double strength_theta;   /* block (i,j) strong if |A_ij|_F >= theta sqrt(|A_ii|_F |A_jj|_F); default 0.02 */
  int smoother_degree;     /* Chebyshev degree, pre and post; default 2                               */
  double cheb_lo;          /* smoothing interval [cheb_lo, cheb_hi] * lambda_max(D^-1 A); 0.1       */
  double cheb_hi;          /* 1.1                                                                    */
  int eig_iters;           /* Lanczos steps for lambda_max(D^-1 A); default 10                        */
  int coarse_max_dofs;     /* stop coarsening at or below this many DOFs; default 2000                */
  int aggressive_levels;   /* levels aggregated with distance-2 roots (fast coarsening); distance-1
                              roots below; default 1                                                */
  int coarse_min_dofs;     /* redo a distance-2 aggregation with distance-1 roots when it would give
                              fewer coarse DOFs than this (0 = never); default 500                  */
  int small_level_dofs;    /* smoothed levels with at most this many DOFs use ...                     */
  int small_level_degree;  /* ... this Chebyshev degree instead of smoother_degree; default 0 (off), 16 */
  int max_levels;          /* including the finest; default 10                                       */
  int use_rotations;       /* 1: six rigid-body modes; 0: three translations only; default 1         */
  int level_precision;     /* V-cycle storage/arithmetic: 0 FP64; 1 FP32; 2 FP32 with BF16 finest-level
                              values (P1 meshes; a P2 K keeps FP32 there, as BF16's 8-bit mantissa
                              doubles its iterations).  The outer CG and the coarsest dense solve stay
                              FP64; default 0 */
  double strength_theta_scale; /* level l uses strength_theta * strength_theta_scale^l; default 0.5    */
  int setup_fp64;          /* products of the setup (A P_tent, A P, R (A P)) in plain FP64 arithmetic (1)
                              or in double-float, two FP32 values per operand with error-free transforms,
                              about 2^-47 relative, faster on GB300 (0, default)                     */
  int spmv_fp64;           /* products of the solve's SpMVs (outer CG, V-cycle operators): 0 (default)
                              double-float, on split copies of the matrix values (same 8 bytes per
                              value, each split to within 2^-49, bound by memory instead of GB300's
                              FP64 pipe), for operators of at least 2^20 blocks and for the coarse
                              operators of a few long rows run with whole warps per row, plain FP64
                              on the others; 1 plain FP64 everywhere; 2 double-float everywhere.
                              The outer CG's product with K accumulates accurately (within about
                              1e-14 of sum_j |K_ij x_j| per row), the V-cycle's more loosely (a few
                              1e-14).  Vectors and all other arithmetic stay FP64.
                              Exponent range: double-float and the FP32 V-cycle need K's largest
                              entry (over rows with off-diagonal blocks) within 2^-90..2^90; outside
                              it amg_setup runs every product in FP64 (spmv_fp64 0 and setup_fp64 0
                              fall back) and refuses spmv_fp64 = 2 and level_precision 1/2 with
                              INVALID_ARG.  The loads may have any scale (see amg_pcg_solve)      */
} amg_params;

/* Fills *p with the defaults above. */
int amg_params_default(amg_params* p);

/* Builds the hierarchy for K.  coords[n*3] (device) gives the rigid-body
 * modes (translations and rotations about the node centroid; zero on
 * Dirichlet nodes).  Per level: Lanczos estimate of lambda_max(D^-1 A),
 * strength graph, aggregation (distance-2 maximal independent set by
 * SplitMix64 priority), tentative prolongator by modified Gram-Schmidt,
 * P = (I - 4/(3 lambda) D^-1 A) P_tent, R = P^T, A_c = R A P; the coarsest
 * operator is inverted densely.  K must outlive the handle.  Synchronising.
 * Errors: INVALID_ARG, OOM, CUDA, INTERNAL. */
int amg_setup(tam_matrix K, const double* coords, const amg_params* params, tam_amg* amg_out,
              void* stream);

/* Level sizes: n_levels, and per level (arrays of length >= n_levels, host
 * memory, each may be NULL): block rows, stored blocks, block size, the
 * lambda_max estimate; op_complexity = sum nnz(A_l) / nnz(A_0) in scalars. */
int amg_info(tam_amg amg, int* n_levels, long long* level_rows_host, long long* level_nnzb_host,
             int* level_block_host, double* level_lambda_host, double* op_complexity);

/* Device time of the setup phases summed over levels, in milliseconds, into
 * phase_ms_host[8] (host): 0 diagonal + Lanczos lambda_max, 1 strength +
 * aggregation, 2 tentative prolongator, 3 A P_tent + smoothing, 4 R = P^T,
 * 5 Galerkin product (A P, R (A P)), 6 SpMV-layout conversions, 7 coarsest
 * dense inverse.  Measured with CUDA events; never synchronises. */
int amg_setup_stats(tam_amg amg, double* phase_ms_host);

/* Aggregate id of every block row of `level` (-1 = not aggregated) into
 * agg[n_rows] (device int32).  Synchronising. */
int amg_level_aggregates(tam_amg amg, int level, int* agg, void* stream);

/* Block-CSR export of one operator of `level`: which = 0 A_level, 1 P
 * (prolongator to level+1), 2 R = P^T, 3 tentative prolongator.  Call first
 * with row_ptr == NULL to get the sizes (host ints), then with device arrays
 * row_ptr[n_rows+1], col_idx[nnzb], vals[nnzb*br*bc].  Synchronising. */
int amg_level_export(tam_amg amg, int level, int which, int* n_rows, int* n_cols, int* br, int* bc,
                     long long* nnzb, int* row_ptr, int* col_idx, double* vals, void* stream);

/* Residual history of the last amg_pcg_solve with this hierarchy (not the
 * batched solve): hist_host[k] = ||r_k||_2, the recursively updated residual
 * the stopping test reads (Sec. 2.1; r_0 = b - K x_0), for k = 0 .. iters, in
 * the caller's units; at most cap entries are written (host array), *n_host
 * (may be NULL) = iters + 1, or 0 before the first solve.  Recorded on the
 * device by the iteration kernels (one store per iteration) and copied out
 * here; synchronising.  Errors: INVALID_ARG. */
int amg_residual_history(tam_amg amg, double* hist_host, int cap, int* n_host, void* stream);

/* SpMV layout the setup chose for one operator of `level` (which = 0 A_level,
 * 1 P, 2 R), host ints: *kind 0 = SELL-32, one thread per block row; 1 =
 * lanes per row over the interleaved lanes-per-row store; 2 = lanes per row
 * over the block-CSR arrays; 3 = whole warps per row over the 8-lane store;
 * 4 = block-row lanes over the block-CSR arrays (one lane per row of each
 * block, 6-row blocks).  *lanes = lanes (kinds 1, 2) or threads (kinds 3, 4)
 * per row, 1 for kind 0;
 * *df = 1 when its products run in double-float on split values.  The
 * layouts differ only in arithmetic order, not in the operator (Sec. 2.1
 * V-cycle); exposed so that parity tests can name the kernel they cover.
 * Level 0's A is K (the outer CG's SpMV).  Errors: INVALID_ARG. */
int amg_level_spmv_plan(tam_amg amg, int level, int which, int* kind, int* lanes, int* df);

/* Algorithmic bytes of one V-cycle and of one PCG iteration (Sec. 2.1: CG
 * preconditioned by the V-cycle), host doubles, either may be NULL: every
 * array each kernel of this implementation must touch, counted once per
 * kernel, without SELL padding or cache re-reads -- matrix values (8 B FP64 /
 * double-float, 4 B FP32, 2 B BF16) and 4 B column indices per block, plus
 * the vectors of the fused epilogues.  Per smoothed level: a zero-start
 * Chebyshev step (4 vectors), 2*degree - 1 fused SpMV Chebyshev steps (matrix +
 * 6 vectors), the residual (matrix + 3), restriction (R + fine + coarse
 * vector), prolongation (P + coarse + 2 fine); the coarsest level's dense
 * inverse (N^2 * 8 B); the outer CG adds K (8 B values) and 13 vectors of 3n
 * FP64.  Divided by the measured time this gives the solve phase's achieved
 * bandwidth.  Errors: INVALID_ARG. */
int amg_solve_bytes(tam_amg amg, double* vcycle_bytes, double* iteration_bytes);

/* x <- `degree` (1..64) Chebyshev-Jacobi steps on K x = b from the given x,
 * over [cheb_lo, cheb_hi] * lambda_max(D^-1 K) of the hierarchy's parameters:
 * the finest level's smoother of the V-cycle (Sec. 5.1, "Solver
 * configuration"; Chebyshev with an estimated lambda_max), each step one fused
 * SpMV kernel (res = D^-1 (b - K x), d = c_d d + c_r res, x += d) in the
 * V-cycle's arithmetic.  b, x: [3n] device vectors, must not overlap.  The
 * first call with a new degree uploads its coefficients (synchronising);
 * later calls are asynchronous.  Errors: INVALID_ARG. */
int amg_smooth(tam_amg amg, const double* b, double* x, int degree, void* stream);

/* z = M^-1 r: one V-cycle (the preconditioner), r and z [3n] device. */
int amg_vcycle(tam_amg amg, const double* r, double* z, void* stream);

/* Preconditioned CG on K x = b from the initial guess in x.  Stops when the
 * recursively updated residual satisfies ||r||_2 <= max(rtol ||b||_2, atol)
 * or after max_iter iterations.  iters_out and final_rel_resid_out (host,
 * may be NULL) receive the iteration count and ||b - K x||_2 / ||b||_2
 * (recomputed at the end in plain FP64).  Internally the solve runs on b and
 * x divided by a power of two chosen from ||b|| and K's largest entry, so that
 * the vectors the double-float and FP32 products see sit inside FP32's
 * exponent range whatever the units of the problem; the scaling is exact (in
 * range the iterates are the unscaled ones times that power of two) and x is
 * scaled back before return.  The iterations run as one CUDA graph launch (a
 * device-side loop over one captured iteration, ended by the stopping test),
 * so the host waits once per solve.  Synchronising.
 * Errors: NOT_CONVERGED (x holds the last iterate), BREAKDOWN,
 * INDEFINITE_PRECOND, NAN, INVALID_ARG, CUDA.  (With TAM_PCG_HOST_LOOP=1 in
 * the environment the same iterations run as plain launches from a host loop
 * that reads the stop flag after each one: for profilers that do not trace
 * kernels inside conditional graph nodes.) */
int amg_pcg_solve(tam_amg amg, const double* b, double* x, double rtol, double atol, int max_iter,
                  int* iters_out, double* final_rel_resid_out, void* stream);

/* Releases the hierarchy. */
int amg_destroy(tam_amg amg);

/* ------------------------------------------------------------------------
 * Many load cases at once (an extension of the paper's per-load-case solve;
 * the paper reuses the elastic preconditioner across time steps, Sec. 5.3).
 * Each system i (hierarchy amg[i]) has n_rhs[i] (1..16) right-hand sides,
 * B[i] and X[i] device arrays [n_rhs[i] x 3n_i] (one displacement vector per
 * row; X holds the initial guesses in, the solutions out).  Every right-hand
 * side runs its own CG with its own stopping test ||r|| <= max(rtol ||b||,
 * atol); all SpMVs are multi-vector products: FP64 with K, FP32 in the
 * V-cycle (BF16 finest values for a hierarchy built with level_precision 2;
 * FP64 coarsest solve).  One CUDA graph launch runs the whole batch: a
 * device-side loop whose body advances every system by one iteration (systems
 * on parallel branches) until all have stopped.  The first call for a hierarchy and RHS count builds the FP32
 * copies and workspaces and tunes the launch shape of every operator by
 * timing candidates: right-hand sides per thread (1, 2, 4, 8), threads per
 * CTA (64, 128, 256) and, for the block-CSR layouts, lanes per block row.
 * iters_host / rel_host (may be NULL): per right-hand side, systems in order.
 * Synchronising.  Errors: INVALID_ARG, NOT_CONVERGED, BREAKDOWN,
 * INDEFINITE_PRECOND, NAN, CUDA. */
int amg_pcg_solve_batch(int n_systems, const tam_amg* amg, const int* n_rhs, const double* const* B,
                        double* const* X, double rtol, double atol, int max_iter, int* iters_host,
                        double* rel_host, void* stream);

/* Launch shapes chosen by the autotuner for `amg`, as triples (right-hand
 * sides per thread, threads per CTA, lanes per block row or 0 = as planned):
 * K first, then (A, P, R) per smoothed level; *n receives the number of ints
 * written (at most cap) and *tune_ms_host the tuning time. */
int amg_batch_tiles(tam_amg amg, int* tiles_host, int cap, int* n, double* tune_ms_host);

/* ------------------------------------------------------------------------
 * Learned initial guess (an extension; the paper has no learned component).
 * A node-wise multilayer perceptron maps per-node features to a displacement
 * guess that seeds amg_pcg_solve; CG always iterates to the tolerance, so the
 * network changes the iteration count, never the answer.  Network: n_in
 * inputs, `depth` tanh layers of `width`, linear n_out outputs; inputs are
 * standardised (x - shift) * scale, outputs multiplied by out_scale.
 * Parameters: FP32, per layer W [fan_in x fan_out] row-major then bias, layers
 * in order (Glorot-uniform init from SplitMix64(seed)).  Training minimises
 * the mean squared error with Adam (beta 0.9, 0.999, eps 1e-8).
 * All array arguments are device pointers unless named *_host.
 */
typedef struct tam_mlp_s* tam_mlp;

int tam_mlp_create(int n_in, int width, int depth, int n_out, unsigned long long seed, tam_mlp* out);
int tam_mlp_destroy(tam_mlp mlp);
/* number of FP32 parameters and of layers */
int tam_mlp_info(tam_mlp mlp, long long* n_params, int* n_layers);
/* host arrays shift[n_in], scale[n_in], out_scale[n_out] */
int tam_mlp_set_normalization(tam_mlp mlp, const float* shift_host, const float* scale_host,
                              const float* out_scale_host);
/* copy all parameters out of / into host memory (n_params floats) */
int tam_mlp_get_params(tam_mlp mlp, float* theta_host);
int tam_mlp_set_params(tam_mlp mlp, const float* theta_host);
/* Y[n x n_out] = net(X[n x n_in]) (device arrays, row-major).  bf16 = 0: FP32
 * weights and activations, one kernel per layer; 1: BF16 weights and
 * BF16-rounded activations on the tensor cores with FP32 accumulation, the
 * whole network in one kernel (activations never leave the SM; nets of at
 * most 8 layers of width <= 128, else layer by layer); 2: the same BF16
 * arithmetic one kernel per layer (bitwise the same results as 1). */
int tam_mlp_forward(tam_mlp mlp, long long n, const float* X, float* Y, int bf16, void* stream);
/* mean squared error of net(X) against Yt and its gradient (grad_host: n_params
 * floats, may be NULL); synchronising */
int tam_mlp_loss_grad(tam_mlp mlp, long long n, const float* X, const float* Yt, double* loss_host,
                      float* grad_host, void* stream);
/* one Adam step on the batch (X, Yt) with learning rate lr; synchronising */
int tam_mlp_train_step(tam_mlp mlp, long long n, const float* X, const float* Yt, float lr,
                       double* loss_host, void* stream);

/* Node features[n_nodes x 8] (FP32): x, y, z, T, grad T (volume-weighted mean
 * of the cells' centroid gradients of the temperature interpolant), dist.
 * T and dist (distance to the clamped boundary, [n_nodes]) may be NULL (0).
 * Synchronising. */
int tam_node_features(int n_nodes, const double* coords, int n_cells, int nodes_per_cell,
                      const int* cells, const double* T, const double* dist, float* features,
                      void* stream);

/* x[3n] = the network's guess for K x = rhs (K of the hierarchy `amg`; 8
 * features in, 3 displacements out), Dirichlet rows set to their prescribed
 * values, then smooth_degree (0..64; 0 = none) Chebyshev-Jacobi steps on
 * K x = rhs over [0.1, 1.1] lambda_max(D^-1 K), which remove the rough part of
 * the network's error.  The guess is kept only if its preconditioned residual energy
 * <r, M r> (r = rhs - K x, M one V-cycle of `amg`) is below <rhs, M rhs>, the
 * zero guess's; otherwise x = 0.  used_host (may be NULL) tells which;
 * energy_ratio_host (may be NULL) receives <r, M r> / <rhs, M rhs>.
 * Synchronising. */
int tam_learned_guess(tam_mlp mlp, tam_amg amg, const float* features, const double* rhs, int bf16,
                      int smooth_degree, double* x, int* used_host, double* energy_ratio_host,
                      void* stream);

/* ------------------------------------------------------------------------
 * The thermal half of the model (Sec. 3): the heat equation
 *   rho c_v dT/dt - div(kappa grad T) = 0 in Omega,
 *   kappa grad T . n = beta (T - T_bc)  on the Robin faces,
 * discretised by the theta-method (Eq. wf_thermal) on the same P1/P2 meshes,
 * solved by Newton's method on the full linearisation (Sec. 3, "Solution
 * strategy": the Jacobian is non-symmetric when kappa depends on T; as in the
 * paper each Newton step is solved by CG), each step preconditioned by the
 * smoothed-aggregation AMG of this library on the scalar operator (constant
 * near-nullspace; the paper uses classical AMG there), with the adaptive time
 * step of Eq. dt_spec.  Materials: c_v(T) = c0 + c1 T, kappa(T) = k0 + k1 T.
 * beta follows the paper's sign: beta <= 0 is a cooling film.  T fields are
 * nodal [n_nodes] float64 device vectors (interpolants in the cells' space).
 */
typedef struct tam_thermal_s* tam_thermal;

/* Thermal problem on a mesh.  coords, cells, cell_material, faces: device
 * arrays that must outlive the handle (not copied).  thermal_props_host
 * [n_mat*5] (host): rho, c0, c1, k0, k1 per material.  faces[n_faces*nf]:
 * the Robin faces, nf = 3 (P1: vertices) or 6 (P2: vertices v0 v1 v2, then
 * the mid-edge nodes of v0v1, v1v2, v2v0).  dirichlet_mask[n_nodes] (device,
 * may be NULL): nodes whose temperature is prescribed.  params: AMG knobs for
 * the Newton steps (NULL = defaults; level_precision must be 0).  Builds the
 * scalar pattern; synchronising.  Errors: INVALID_ARG, OOM, CUDA,
 * UNSUPPORTED. */
int tam_thermal_create(int n_nodes, const double* coords, int n_cells, int nodes_per_cell, const int* cells,
                       const int* cell_material, int n_mat, const double* thermal_props_host, int n_faces,
                       const int* faces, const unsigned char* dirichlet_mask, const amg_params* params,
                       tam_thermal* out, void* stream);

/* Residual F(T)[n_nodes] of Eq. wf_thermal at the iterate T of T_{m+1}
 * (T_old = T_m, NULL = the steady problem with theta = 1), with per-face
 * beta[n_faces] and nodal T_bc[n_nodes] at the theta-weighted time; Dirichlet
 * entries 0.  The Jacobian dF/dT is assembled alongside (see export).
 * Synchronising.  Errors: INVALID_ARG, DEGENERATE_CELL, CUDA. */
int tam_thermal_residual(tam_thermal th, const double* T, const double* T_old, double dt, double theta,
                         const double* beta, const double* T_bc, double* F_out, void* stream);

/* The last assembled Jacobian in CSR form: *nnz_host (host) always; with
 * row_ptr != NULL also row_ptr[n+1], col_idx[nnz], vals[nnz] (device).
 * Dirichlet rows are identity rows.  Synchronising. */
int tam_thermal_export_jacobian(tam_thermal th, int* row_ptr, int* col_idx, double* vals, long long* nnz_host,
                                void* stream);

/* Newton's method on F(T) = 0 from the guess in T (overwritten with the
 * solution): stops when ||F||_2 <= rtol ||F(T_0)||_2 (the paper's steady runs
 * use 1e-9) or after max_newton steps.  Each step solves J delta = F by CG to
 * lin_rtol (at most lin_max_iter iterations) preconditioned by an AMG
 * hierarchy: with reuse = 0 a new one every step, with reuse = 1 the
 * hierarchy of an earlier Jacobian (from an earlier step or call) with its
 * finest level refreshed, rebuilt only when that solve fails -- the paper's
 * transient runs rebuild the thermal preconditioner only at some steps
 * (Sec. 5.3).  T_dirichlet (may be NULL) sets the masked nodes first.
 * Outputs (host, may be NULL): Newton steps, CG iterations in all, hierarchies
 * built, final ||F|| / ||F_0||.  Synchronising.  Errors: NOT_CONVERGED, NAN,
 * BREAKDOWN, INDEFINITE_PRECOND, INVALID_ARG, CUDA. */
int tam_thermal_newton(tam_thermal th, double* T, const double* T_old, double dt, double theta, const double* beta,
                       const double* T_bc, const double* T_dirichlet, double rtol, int max_newton, double lin_rtol,
                       int lin_max_iter, int reuse, int* newton_iters, int* linear_iters, int* setups,
                       double* rel_resid, void* stream);

/* max_i |a_i - b_i| into *max_host (a, b: device [n]).  Synchronising. */
int tam_thermal_max_change(const double* a, const double* b, long long n, double* max_host, void* stream);

/* Eq. dt_spec: the step with max |T_{m+1} - T_m| = max_change is accepted when
 * max_change <= dT_max, and then dt_next = eps dT_max / max_change * dt (twice
 * dt when nothing changed); otherwise it is rejected and dt_next = dt / 2 (the
 * step is repeated).  Host arithmetic only. */
int tam_thermal_next_dt(double dt, double max_change, double dT_max, double eps, double* dt_next_host,
                        int* accepted_host);

/* Releases the handle (and the hierarchy it holds). */
int tam_thermal_destroy(tam_thermal th);

/* ------------------------------------------------------------------------
 * One-call host-buffer path: copies the mesh and fields from host memory
 * (pinned memory gives the fastest copies), assembles, builds the AMG, solves
 * to rtol and copies the displacement back into u_host[n_nodes*3].  Same
 * argument meaning as fem_assemble_elasticity / amg_pcg_solve; params may be
 * NULL (defaults).  Synchronising; all device memory is released on return.
 */
int tam_solve_elasticity_host(int n_nodes, const double* coords_host, int n_cells,
                              int nodes_per_cell, const int* cells_host,
                              const int* cell_material_host, int n_mat,
                              const double* mat_props_host, const double* T_host, double T_ref,
                              const double* body_force_host,
                              const unsigned char* dirichlet_mask_host,
                              const double* u_dirichlet_host, const amg_params* params,
                              double rtol, int max_iter, double* u_host, int* iters_out,
                              double* final_rel_resid_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* THERMOAMG_H */
