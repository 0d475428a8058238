// C ABI of the thermoamg library (declared in include/thermoamg.h).  Every
// entry point converts internal exceptions into a status code and a message
// for tam_last_error(); none aborts the process.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "handles.cuh"

namespace tam {
const char* last_error_cstr();
}

using namespace tam;

tam_amg_s::~tam_amg_s() {
  if (iter_exec) cudaGraphExecDestroy(iter_exec);
}

namespace {

template <class F>
int guarded(F&& f) {
  try {
    set_last_error("");
    return f();
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return TAM_ERR_OOM;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return TAM_ERR_INTERNAL;
  } catch (...) {
    set_last_error("unknown failure");
    return TAM_ERR_INTERNAL;
  }
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void export_bsr(const Bsr& A, int* rp, int* ci, double* v, cudaStream_t s) {
  TAM_CUDA(cudaMemcpyAsync(rp, A.row_ptr.p, sizeof(int) * ((size_t)A.n_rows + 1), cudaMemcpyDeviceToDevice, s));
  if (A.nnzb > 0) {
    TAM_CUDA(cudaMemcpyAsync(ci, A.col_idx.p, sizeof(int) * (size_t)A.nnzb, cudaMemcpyDeviceToDevice, s));
    TAM_CUDA(cudaMemcpyAsync(v, A.vals.p, sizeof(double) * (size_t)A.nnzb * A.block_elems(),
                             cudaMemcpyDeviceToDevice, s));
  }
  TAM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

const char* tam_last_error(void) { return last_error_cstr(); }

long long tam_kernel_launches(void) { return launches_total(); }

int fem_assemble_elasticity(int n_nodes, const double* coords, int n_cells, int nodes_per_cell, const int* cells,
                            const int* cell_material, int n_mat, const double* mat_props, const double* T,
                            double T_ref, const double* body_force, const unsigned char* dirichlet_mask,
                            const double* u_dirichlet, tam_matrix* K_out, double* rhs_out, void* stream) {
  return guarded([&] {
    TAM_CHECK(K_out, TAM_ERR_INVALID_ARG, "fem_assemble: K_out is NULL");
    *K_out = nullptr;
    *K_out = assemble_elasticity(n_nodes, coords, n_cells, nodes_per_cell, cells, cell_material, n_mat, mat_props, T,
                                 T_ref, body_force, dirichlet_mask, u_dirichlet, rhs_out, as_stream(stream));
    return TAM_OK;
  });
}

int tam_set_deterministic_assembly(int on, int* previous) {
  return guarded([&] {
    const int old = g_deterministic_assembly.exchange(on ? 1 : 0);
    if (previous) *previous = old;
    return TAM_OK;
  });
}

int fem_assemble_load(tam_matrix K, const double* coords, int n_cells, int nodes_per_cell, const int* cells,
                      const int* cell_material, int n_mat, const double* mat_props, const double* T, double T_ref,
                      const double* body_force, const double* u_dirichlet, double* rhs_out, void* stream) {
  return guarded([&] {
    assemble_loads(K, coords, n_cells, nodes_per_cell, cells, cell_material, n_mat, mat_props, T, T_ref, body_force,
                   u_dirichlet, rhs_out, as_stream(stream));
    TAM_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return TAM_OK;
  });
}

int tam_matrix_info(tam_matrix K, int* n_block_rows, long long* nnzb, int* block_size) {
  return guarded([&] {
    TAM_CHECK(K, TAM_ERR_INVALID_ARG, "tam_matrix_info: NULL handle");
    if (n_block_rows) *n_block_rows = K->A.n_rows;
    if (nnzb) *nnzb = K->A.nnzb;
    if (block_size) *block_size = K->A.br;
    return TAM_OK;
  });
}

int tam_matrix_export_bsr(tam_matrix K, int* row_ptr, int* col_idx, double* vals, void* stream) {
  return guarded([&] {
    TAM_CHECK(K && row_ptr && col_idx && vals, TAM_ERR_INVALID_ARG, "tam_matrix_export_bsr: NULL argument");
    export_bsr(K->A, row_ptr, col_idx, vals, as_stream(stream));
    return TAM_OK;
  });
}

int tam_matrix_spmv(tam_matrix K, const double* x, double* y, void* stream) {
  return guarded([&] {
    TAM_CHECK(K && x && y && x != y, TAM_ERR_INVALID_ARG, "tam_matrix_spmv: bad argument");
    spmv_K(K, x, y, as_stream(stream));
    return TAM_OK;
  });
}

int tam_matrix_residual_norm(tam_matrix K, const double* b, const double* x, double* norm_host, void* stream) {
  return guarded([&] {
    TAM_CHECK(K && b && x && norm_host, TAM_ERR_INVALID_ARG, "tam_matrix_residual_norm: NULL argument");
    *norm_host = residual_norm_K(K, b, x, as_stream(stream));
    return TAM_OK;
  });
}

int tam_matrix_destroy(tam_matrix K) {
  return guarded([&] {
    delete K;
    return TAM_OK;
  });
}

int amg_params_default(amg_params* p) {
  return guarded([&] {
    TAM_CHECK(p, TAM_ERR_INVALID_ARG, "amg_params_default: NULL");
    p->strength_theta = 0.02;
    p->smoother_degree = 2;
    p->cheb_lo = 0.1;
    p->cheb_hi = 1.1;
    p->eig_iters = 10;
    p->coarse_max_dofs = 2000;
    p->aggressive_levels = 1;
    p->coarse_min_dofs = 500;
    p->small_level_dofs = 0;
    p->small_level_degree = 16;
    p->max_levels = 10;
    p->use_rotations = 1;
    p->level_precision = 0;
    p->strength_theta_scale = 0.5;
    p->setup_fp64 = 0;
    p->spmv_fp64 = 0;
    return TAM_OK;
  });
}

int amg_setup(tam_matrix K, const double* coords, const amg_params* params, tam_amg* amg_out, void* stream) {
  return guarded([&] {
    TAM_CHECK(K && coords && amg_out, TAM_ERR_INVALID_ARG, "amg_setup: NULL argument");
    *amg_out = nullptr;
    amg_params prm;
    if (params) prm = *params; else amg_params_default(&prm);
    *amg_out = amg_build(K, coords, prm, as_stream(stream));
    return TAM_OK;
  });
}

int amg_info(tam_amg amg, int* n_levels, long long* level_rows, long long* level_nnzb, int* level_block,
             double* level_lambda, double* op_complexity) {
  return guarded([&] {
    TAM_CHECK(amg, TAM_ERR_INVALID_ARG, "amg_info: NULL handle");
    const int L = (int)amg->levels.size();
    if (n_levels) *n_levels = L;
    double tot = 0.0, fine = 0.0;
    for (int l = 0; l < L; ++l) {
      const Level& lv = amg->levels[l];
      if (level_rows) level_rows[l] = lv.n_rows;
      if (level_nnzb) level_nnzb[l] = lv.A->nnzb;
      if (level_block) level_block[l] = lv.bs;
      if (level_lambda) level_lambda[l] = lv.lambda_host;
      double nz = (double)lv.A->nnzb * lv.bs * lv.bs;
      tot += nz;
      if (l == 0) fine = nz;
    }
    if (op_complexity) *op_complexity = fine > 0 ? tot / fine : 0.0;
    return TAM_OK;
  });
}

int amg_setup_stats(tam_amg amg, double* phase_ms_host) {
  return guarded([&] {
    TAM_CHECK(amg && phase_ms_host, TAM_ERR_INVALID_ARG, "amg_setup_stats: NULL argument");
    for (int i = 0; i < 8; ++i) phase_ms_host[i] = amg->setup_ms[i];
    return TAM_OK;
  });
}

int amg_residual_history(tam_amg amg, double* hist_host, int cap, int* n_host, void* stream) {
  return guarded([&] {
    TAM_CHECK(amg && cap >= 0 && (hist_host || cap == 0), TAM_ERR_INVALID_ARG, "amg_residual_history: bad argument");
    const long long n = std::min<long long>(amg->hist_len, cap);
    if (n_host) *n_host = (int)amg->hist_len;
    if (n > 0) {
      cudaStream_t s = as_stream(stream);
      TAM_CUDA(cudaMemcpyAsync(hist_host, amg->hist.p, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
      TAM_CUDA(cudaStreamSynchronize(s));
      const double f = std::ldexp(1.0, amg->hist_scale_exp);
      for (long long k = 0; k < n; ++k) hist_host[k] = std::sqrt(hist_host[k]) * f;
    }
    return TAM_OK;
  });
}

int amg_level_aggregates(tam_amg amg, int level, int* agg, void* stream) {
  return guarded([&] {
    TAM_CHECK(amg && agg && level >= 0 && level < (int)amg->levels.size(), TAM_ERR_INVALID_ARG,
              "amg_level_aggregates: bad argument");
    const Level& L = amg->levels[level];
    cudaStream_t s = as_stream(stream);
    if (L.agg.p)
      TAM_CUDA(cudaMemcpyAsync(agg, L.agg.p, sizeof(int) * L.n_rows, cudaMemcpyDeviceToDevice, s));
    else
      TAM_CUDA(cudaMemsetAsync(agg, 0xff, sizeof(int) * L.n_rows, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    return TAM_OK;
  });
}

int amg_level_export(tam_amg amg, int level, int which, int* n_rows, int* n_cols, int* br, int* bc, long long* nnzb,
                     int* row_ptr, int* col_idx, double* vals, void* stream) {
  return guarded([&] {
    TAM_CHECK(amg && level >= 0 && level < (int)amg->levels.size() && which >= 0 && which <= 3,
              TAM_ERR_INVALID_ARG, "amg_level_export: bad argument");
    const Level& L = amg->levels[level];
    const Bsr* M = which == 0 ? L.A : which == 1 ? &L.P : which == 2 ? &L.R : &L.Pt;
    TAM_CHECK(which == 0 || L.n_agg > 0, TAM_ERR_INVALID_ARG, "amg_level_export: the coarsest level has no P/R");
    if (n_rows) *n_rows = M->n_rows;
    if (n_cols) *n_cols = M->n_cols;
    if (br) *br = M->br;
    if (bc) *bc = M->bc;
    if (nnzb) *nnzb = M->nnzb;
    if (row_ptr) {
      TAM_CHECK(col_idx && vals, TAM_ERR_INVALID_ARG, "amg_level_export: NULL array");
      export_bsr(*M, row_ptr, col_idx, vals, as_stream(stream));
    }
    return TAM_OK;
  });
}

int amg_level_spmv_plan(tam_amg amg, int level, int which, int* kind, int* lanes, int* df) {
  return guarded([&] {
    TAM_CHECK(amg && level >= 0 && level < (int)amg->levels.size() && which >= 0 && which <= 2,
              TAM_ERR_INVALID_ARG, "amg_level_spmv_plan: bad argument");
    const Level& L = amg->levels[level];
    TAM_CHECK(which == 0 || L.n_agg > 0, TAM_ERR_INVALID_ARG, "amg_level_spmv_plan: the coarsest level has no P/R");
    const SpOp& op = which == 0 ? L.Aop : which == 1 ? L.Pop : L.Rop;
    int k = 0, ln = 0;
    if (op.brw) {
      k = 4;
      ln = op.brw * 32;
    } else if (op.lpr == 0) {
      k = 0;
      ln = 1;
    } else if (op.L && op.tpr) {
      k = 3;
      ln = op.tpr;
    } else if (op.L) {
      k = 1;
      ln = op.lpr;
    } else {
      k = 2;
      ln = op.lpr;
    }
    bool split = false;
    if (op.brw) split = op.df && op.B && op.B->vals_df.p;
    else if (op.lpr == 0) split = op.df && op.S && op.S->vals_df.p;
    else if (op.L) split = op.df && op.L->vals_df.p;
    else split = op.df && op.B && op.B->vals_df.p;
    if (kind) *kind = k;
    if (lanes) *lanes = ln;
    if (df) *df = split ? 1 : 0;
    return TAM_OK;
  });
}

// Algorithmic bytes (the data the method itself must move, each array once per
// kernel, no padding or re-reads) of one V-cycle and of one PCG iteration of
// this implementation, from the hierarchy's sizes and precision.
int amg_solve_bytes(tam_amg amg, double* vcycle_bytes, double* iteration_bytes) {
  return guarded([&] {
    TAM_CHECK(amg, TAM_ERR_INVALID_ARG, "amg_solve_bytes: NULL handle");
    const int prec = amg->prm.level_precision;
    const int nl = (int)amg->levels.size();
    auto mat = [](const Bsr& B, double vb) { return (double)B.nnzb * ((double)B.br * B.bc * vb + 4.0); };
    double v = 0.0;
    for (int l = 0; l < nl; ++l) {
      const Level& L = amg->levels[l];
      const double ws = prec > 0 ? 4.0 : 8.0;                    // V-cycle vector word
      const double n = (double)L.n_rows * L.bs;                  // this level's vector length
      if (l == nl - 1) {                                         // dense inverse, b in, y out
        v += (double)amg->n_coarse * amg->n_coarse * 8.0 + 2.0 * amg->n_coarse * ws;
        break;
      }
      const double va = prec == 0 ? 8.0 : (prec == 2 && l == 0 ? 2.0 : 4.0);
      const double vp = prec == 0 ? 8.0 : 4.0;
      const double A = mat(*L.A, va), P = mat(L.P, vp), R = mat(L.R, vp);
      const double nc = (double)L.P.n_cols * L.P.bc;
      const int deg = std::max(L.deg, 1);
      // pre-smoothing: first step from zero (b, dinv in; d, x out), deg - 1 fused
      // SpMV steps (x, b, dinv, d in; d, x' out); residual (x, b in; t out);
      // restriction (t in; b_c out); prolongation (x_c in; x in/out);
      // post-smoothing: deg fused SpMV steps
      v += 4.0 * n * ws;
      v += (double)(2 * deg - 1) * (A + 6.0 * n * ws);
      v += A + 3.0 * n * ws;
      v += R + n * ws + nc * ws;
      v += P + nc * ws + 2.0 * n * ws;
    }
    const double n0 = (double)amg->K->n_nodes * amg->K->A.br;
    if (prec > 0) v += 2.0 * n0 * 4.0;  // FP64 r in / z out at level 0
    // outer CG: q = K p (p in, q out), x/r update (x, r in/out; p, q in),
    // r.z (r, z in), p = z + beta p (z in, p in/out)
    const double it = v + mat(amg->K->A, 8.0) + 13.0 * n0 * 8.0;
    if (vcycle_bytes) *vcycle_bytes = v;
    if (iteration_bytes) *iteration_bytes = it;
    return TAM_OK;
  });
}

int amg_smooth(tam_amg amg, const double* b, double* x, int degree, void* stream) {
  return guarded([&] {
    TAM_CHECK(amg && b && x && b != x, TAM_ERR_INVALID_ARG, "amg_smooth: bad argument");
    smooth_fine(amg, b, x, degree, amg->prm.cheb_lo, amg->prm.cheb_hi, as_stream(stream));
    return TAM_OK;
  });
}

int amg_vcycle(tam_amg amg, const double* r, double* z, void* stream) {
  return guarded([&] {
    TAM_CHECK(amg && r && z && r != z, TAM_ERR_INVALID_ARG, "amg_vcycle: bad argument");
    vcycle_apply(amg, r, z, nullptr, as_stream(stream));
    return TAM_OK;
  });
}

int amg_pcg_solve(tam_amg amg, const double* b, double* x, double rtol, double atol, int max_iter, int* iters_out,
                  double* final_rel_resid_out, void* stream) {
  return guarded([&] {
    TAM_CHECK(amg, TAM_ERR_INVALID_ARG, "amg_pcg_solve: NULL handle");
    int st = pcg_solve(amg, b, x, rtol, atol, max_iter, iters_out, final_rel_resid_out, as_stream(stream));
    if (st != TAM_OK) {
      const char* msg = st == TAM_ERR_NOT_CONVERGED   ? "amg_pcg_solve: max_iter reached"
                        : st == TAM_ERR_BREAKDOWN      ? "amg_pcg_solve: p^T K p <= 0"
                        : st == TAM_ERR_INDEFINITE_PRECOND ? "amg_pcg_solve: r^T M^-1 r <= 0 (indefinite preconditioner)"
                        : st == TAM_ERR_NAN            ? "amg_pcg_solve: NaN/Inf encountered"
                                                      : "amg_pcg_solve: failed";
      set_last_error(msg);
    }
    return st;
  });
}

int amg_pcg_solve_batch(int n_systems, const tam_amg* amg, const int* n_rhs, const double* const* B, double* const* X,
                        double rtol, double atol, int max_iter, int* iters_host, double* rel_host, void* stream) {
  return guarded([&] {
    TAM_CHECK(amg && n_rhs && B && X, TAM_ERR_INVALID_ARG, "amg_pcg_solve_batch: NULL argument");
    int st = pcg_solve_batch(n_systems, amg, n_rhs, B, X, rtol, atol, max_iter, iters_host, rel_host,
                             as_stream(stream));
    if (st != TAM_OK) set_last_error("amg_pcg_solve_batch: a right-hand side did not converge (status per code)");
    return st;
  });
}

int amg_batch_tiles(tam_amg amg, int* tiles_host, int cap, int* n, double* tune_ms_host) {
  return guarded([&] {
    TAM_CHECK(amg, TAM_ERR_INVALID_ARG, "amg_batch_tiles: NULL handle");
    int count = amg->multi ? 3 * (1 + 3 * (int)(amg->levels.size() - 1)) : 0;
    if (tiles_host) multi_tiles(amg, tiles_host, cap);
    if (n) *n = std::min(count, cap);
    if (tune_ms_host) *tune_ms_host = multi_tune_ms(amg);
    return TAM_OK;
  });
}

int amg_destroy(tam_amg amg) {
  return guarded([&] {
    delete amg;
    return TAM_OK;
  });
}

int tam_solve_elasticity_host(int n_nodes, const double* coords_h, int n_cells, int npc, const int* cells_h,
                              const int* mat_h, int n_mat, const double* props_h, const double* T_h, double T_ref,
                              const double* body_h, const unsigned char* dmask_h, const double* ud_h,
                              const amg_params* params, double rtol, int max_iter, double* u_h, int* iters_out,
                              double* rel_out, void* stream) {
  return guarded([&] {
    TAM_CHECK(n_nodes > 0 && n_cells >= 0 && (npc == 4 || npc == 10) && n_mat > 0, TAM_ERR_INVALID_ARG,
              "tam_solve_elasticity_host: bad sizes");
    TAM_CHECK(coords_h && (cells_h || !n_cells) && (mat_h || !n_cells) && props_h && dmask_h && u_h,
              TAM_ERR_INVALID_ARG, "tam_solve_elasticity_host: NULL argument");
    cudaStream_t s = as_stream(stream);
    const size_t n3 = (size_t)n_nodes * 3, ne = (size_t)n_cells * npc;
    DBuf<double> X(n3, s), Td(T_h ? n_nodes : 0, s), Bd(body_h ? n3 : 0, s), Ud(ud_h ? n3 : 0, s),
        props(3 * (size_t)n_mat, s), rhs(n3, s), u(n3, s);
    DBuf<int> C(std::max<size_t>(ne, 1), s), M(std::max<size_t>(n_cells, 1), s);
    DBuf<unsigned char> D(n_nodes, s);
    TAM_CUDA(cudaMemcpyAsync(X.p, coords_h, n3 * 8, cudaMemcpyHostToDevice, s));
    if (ne) TAM_CUDA(cudaMemcpyAsync(C.p, cells_h, ne * 4, cudaMemcpyHostToDevice, s));
    if (n_cells) TAM_CUDA(cudaMemcpyAsync(M.p, mat_h, (size_t)n_cells * 4, cudaMemcpyHostToDevice, s));
    TAM_CUDA(cudaMemcpyAsync(props.p, props_h, 24 * (size_t)n_mat, cudaMemcpyHostToDevice, s));
    if (T_h) TAM_CUDA(cudaMemcpyAsync(Td.p, T_h, (size_t)n_nodes * 8, cudaMemcpyHostToDevice, s));
    if (body_h) TAM_CUDA(cudaMemcpyAsync(Bd.p, body_h, n3 * 8, cudaMemcpyHostToDevice, s));
    if (ud_h) TAM_CUDA(cudaMemcpyAsync(Ud.p, ud_h, n3 * 8, cudaMemcpyHostToDevice, s));
    TAM_CUDA(cudaMemcpyAsync(D.p, dmask_h, (size_t)n_nodes, cudaMemcpyHostToDevice, s));
    tam_matrix_s* K = assemble_elasticity(n_nodes, X.p, n_cells, npc, C.p, M.p, n_mat, props.p, Td.p, T_ref, Bd.p, D.p,
                                          Ud.p, rhs.p, s);
    int st = TAM_OK;
    try {
      amg_params prm;
      if (params) prm = *params; else amg_params_default(&prm);
      tam_amg_s* H = amg_build(K, X.p, prm, s);
      try {
        u.zero();
        st = pcg_solve(H, rhs.p, u.p, rtol, 0.0, max_iter, iters_out, rel_out, s);
      } catch (...) {
        delete H;
        throw;
      }
      delete H;
    } catch (...) {
      delete K;
      throw;
    }
    delete K;
    TAM_CUDA(cudaMemcpyAsync(u_h, u.p, n3 * 8, cudaMemcpyDeviceToHost, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    if (st != TAM_OK) set_last_error("tam_solve_elasticity_host: PCG did not reach the tolerance");
    return st;
  });
}

}  // extern "C"
