"""Python binding of libthermoamg.so (C ABI in include/thermoamg.h).

Argument marshalling only: every computation runs in the CUDA library.  The
functions keep the C names; device arrays are torch CUDA tensors (float64,
int32 or uint8, contiguous) and `stream` is a torch.cuda.Stream (default: the
current stream).  Importing this module loads the library and raises
ImportError when it has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libthermoamg.so")

TAM_OK = 0
STATUS_NAMES = {
    0: "OK", -1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "DEGENERATE_CELL", -5: "NOT_CONVERGED",
    -6: "BREAKDOWN", -7: "INDEFINITE_PRECOND", -8: "NAN", -9: "INTERNAL", -10: "UNSUPPORTED",
}


class TamError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class AmgParams(ctypes.Structure):
    _fields_ = [
        ("strength_theta", ctypes.c_double),
        ("smoother_degree", ctypes.c_int),
        ("cheb_lo", ctypes.c_double),
        ("cheb_hi", ctypes.c_double),
        ("eig_iters", ctypes.c_int),
        ("coarse_max_dofs", ctypes.c_int),
        ("aggressive_levels", ctypes.c_int),
        ("coarse_min_dofs", ctypes.c_int),
        ("small_level_dofs", ctypes.c_int),
        ("small_level_degree", ctypes.c_int),
        ("max_levels", ctypes.c_int),
        ("use_rotations", ctypes.c_int),
        ("level_precision", ctypes.c_int),
        ("strength_theta_scale", ctypes.c_double),
        ("setup_fp64", ctypes.c_int),
        ("spmv_fp64", ctypes.c_int),
    ]


_vp, _i, _d, _ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_pi, _pd, _pll = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)

_SIGNATURES = {
    "tam_last_error": ([], ctypes.c_char_p),
    "tam_kernel_launches": ([], ctypes.c_longlong),
    "tam_fma_throughput": ([_pd, _pd, _vp], _i),
    "fem_assemble_elasticity": ([_i, _vp, _i, _i, _vp, _vp, _i, _vp, _vp, _d, _vp, _vp, _vp,
                                 ctypes.POINTER(_vp), _vp, _vp], _i),
    "tam_matrix_info": ([_vp, _pi, _pll, _pi], _i),
    "tam_matrix_export_bsr": ([_vp, _vp, _vp, _vp, _vp], _i),
    "tam_matrix_spmv": ([_vp, _vp, _vp, _vp], _i),
    "tam_matrix_residual_norm": ([_vp, _vp, _vp, _pd, _vp], _i),
    "tam_matrix_residual_norm_noalloc": ([_vp, _vp, _vp, _pd, _vp], _i),
    "tam_matrix_destroy": ([_vp], _i),
    "amg_params_default": ([ctypes.POINTER(AmgParams)], _i),
    "amg_setup": ([_vp, _vp, ctypes.POINTER(AmgParams), ctypes.POINTER(_vp), _vp], _i),
    "amg_info": ([_vp, _pi, _pll, _pll, _pi, _pd, _pd], _i),
    "amg_setup_stats": ([_vp, _pd], _i),
    "amg_level_aggregates": ([_vp, _i, _vp, _vp], _i),
    "amg_level_export": ([_vp, _i, _i, _pi, _pi, _pi, _pi, _pll, _vp, _vp, _vp, _vp], _i),
    "amg_level_spmv_plan": ([_vp, _i, _i, _pi, _pi, _pi], _i),
    "amg_residual_history": ([_vp, _vp, _i, _pi, _vp], _i),
    "tam_set_deterministic_assembly": ([_i, _pi], _i),
    "amg_smooth": ([_vp, _vp, _vp, _i, _vp], _i),
    "amg_solve_bytes": ([_vp, _pd, _pd], _i),
    "amg_vcycle": ([_vp, _vp, _vp, _vp], _i),
    "amg_pcg_solve": ([_vp, _vp, _vp, _d, _d, _i, _pi, _pd, _vp], _i),
    "amg_destroy": ([_vp], _i),
    "fem_assemble_load": ([_vp, _vp, _i, _i, _vp, _vp, _i, _vp, _vp, _d, _vp, _vp, _vp, _vp], _i),
    "amg_pcg_solve_batch": ([_i, _vp, _vp, _vp, _vp, _d, _d, _i, _vp, _vp, _vp], _i),
    "amg_batch_tiles": ([_vp, _vp, _i, _pi, _pd], _i),
    "tam_mlp_create": ([_i, _i, _i, _i, ctypes.c_ulonglong, ctypes.POINTER(_vp)], _i),
    "tam_mlp_destroy": ([_vp], _i),
    "tam_mlp_info": ([_vp, _pll, _pi], _i),
    "tam_mlp_set_normalization": ([_vp, _vp, _vp, _vp], _i),
    "tam_mlp_get_params": ([_vp, _vp], _i),
    "tam_mlp_set_params": ([_vp, _vp], _i),
    "tam_mlp_forward": ([_vp, _ll, _vp, _vp, _i, _vp], _i),
    "tam_mlp_loss_grad": ([_vp, _ll, _vp, _vp, _pd, _vp, _vp], _i),
    "tam_mlp_train_step": ([_vp, _ll, _vp, _vp, ctypes.c_float, _pd, _vp], _i),
    "tam_node_features": ([_i, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "tam_learned_guess": ([_vp, _vp, _vp, _vp, _i, _i, _vp, _pi, _pd, _vp], _i),
    "tam_thermal_create": ([_i, _vp, _i, _i, _vp, _vp, _i, _vp, _i, _vp, _vp, ctypes.POINTER(AmgParams),
                            ctypes.POINTER(_vp), _vp], _i),
    "tam_thermal_residual": ([_vp, _vp, _vp, _d, _d, _vp, _vp, _vp, _vp], _i),
    "tam_thermal_export_jacobian": ([_vp, _vp, _vp, _vp, _pll, _vp], _i),
    "tam_thermal_newton": ([_vp, _vp, _vp, _d, _d, _vp, _vp, _vp, _d, _i, _d, _i, _i, _pi, _pi, _pi, _pd, _vp],
                           _i),
    "tam_thermal_max_change": ([_vp, _vp, _ll, _pd, _vp], _i),
    "tam_thermal_next_dt": ([_d, _d, _d, _d, _pd, _pi], _i),
    "tam_thermal_destroy": ([_vp], _i),
    "tam_solve_elasticity_host": ([_i, _vp, _i, _i, _vp, _vp, _i, _vp, _vp, _d, _vp, _vp, _vp,
                                   ctypes.POINTER(AmgParams), _d, _i, _vp, _pi, _pd, _vp], _i),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_1804_10060_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def last_error() -> str:
    return lib.tam_last_error().decode()


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process (graph replays included)."""
    return int(lib.tam_kernel_launches())


def fma_throughput(stream=None) -> dict:
    """Measured FP64 / FP32 FMA throughput of the current device (TFLOP/s)."""
    f64, f32 = ctypes.c_double(), ctypes.c_double()
    _check(lib.tam_fma_throughput(ctypes.byref(f64), ctypes.byref(f32), _stream(stream)))
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value}


def _check(status, allow=()):
    if status != TAM_OK and status not in allow:
        raise TamError(status, last_error())
    return status


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _dev(t, dtype, name, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")
    return _vp(t.data_ptr())


class Matrix:
    """Handle of an assembled 3x3-block system matrix K."""

    def __init__(self, handle, n_nodes):
        self.handle = handle
        self.n_nodes = n_nodes

    def info(self):
        n, nnzb, bs = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
        _check(lib.tam_matrix_info(self.handle, ctypes.byref(n), ctypes.byref(nnzb), ctypes.byref(bs)))
        return n.value, nnzb.value, bs.value

    def destroy(self):
        if self.handle:
            lib.tam_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Amg:
    """Handle of an SA-AMG hierarchy (keeps its matrix alive)."""

    def __init__(self, handle, K):
        self.handle = handle
        self.K = K

    def destroy(self):
        if self.handle:
            lib.amg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fem_assemble_elasticity(coords, cells, cell_material, mat_props, T=None, T_ref=0.0, body_force=None,
                            dirichlet_mask=None, u_dirichlet=None, stream=None):
    """Assemble K and the load; returns (Matrix, rhs[n,3] float64 CUDA tensor)."""
    n_nodes = coords.shape[0]
    n_cells, npc = cells.shape
    rhs = torch.empty((n_nodes, 3), dtype=torch.float64, device=coords.device)
    h = _vp()
    _check(lib.fem_assemble_elasticity(
        n_nodes, _dev(coords, torch.float64, "coords"), n_cells, npc, _dev(cells, torch.int32, "cells"),
        _dev(cell_material, torch.int32, "cell_material"), mat_props.shape[0],
        _dev(mat_props, torch.float64, "mat_props"), _dev(T, torch.float64, "T", True), float(T_ref),
        _dev(body_force, torch.float64, "body_force", True), _dev(dirichlet_mask, torch.uint8, "dirichlet_mask"),
        _dev(u_dirichlet, torch.float64, "u_dirichlet", True), ctypes.byref(h), _vp(rhs.data_ptr()),
        _stream(stream)))
    return Matrix(h, n_nodes), rhs


def tam_matrix_export_bsr(K: Matrix, stream=None):
    n, nnzb, bs = K.info()
    dev = torch.device("cuda")
    rp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(nnzb, dtype=torch.int32, device=dev)
    v = torch.empty((nnzb, bs, bs), dtype=torch.float64, device=dev)
    _check(lib.tam_matrix_export_bsr(K.handle, _vp(rp.data_ptr()), _vp(ci.data_ptr()), _vp(v.data_ptr()),
                                     _stream(stream)))
    return rp, ci, v


def tam_matrix_spmv(K: Matrix, x, y=None, stream=None):
    if y is None:
        y = torch.empty_like(x)
    _check(lib.tam_matrix_spmv(K.handle, _dev(x, torch.float64, "x"), _dev(y, torch.float64, "y"),
                               _stream(stream)))
    return y


def tam_matrix_residual_norm(K: Matrix, b, x, stream=None) -> float:
    """||b - K x||_2 (host float)."""
    out = ctypes.c_double()
    _check(lib.tam_matrix_residual_norm(K.handle, _dev(b, torch.float64, "b"), _dev(x, torch.float64, "x"),
                                        ctypes.byref(out), _stream(stream)))
    return out.value


def tam_matrix_residual_norm_noalloc(K: Matrix, b, x, stream=None) -> float:
    """||b - K x||_2 without any device allocation (static 128 KiB scratch; see the C header)."""
    out = ctypes.c_double()
    _check(lib.tam_matrix_residual_norm_noalloc(K.handle, _dev(b, torch.float64, "b"),
                                                _dev(x, torch.float64, "x"), ctypes.byref(out), _stream(stream)))
    return out.value


def amg_params_default(**overrides) -> AmgParams:
    p = AmgParams()
    _check(lib.amg_params_default(ctypes.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def amg_setup(K: Matrix, coords, params: AmgParams | None = None, stream=None) -> Amg:
    h = _vp()
    pp = ctypes.byref(params) if params is not None else None
    _check(lib.amg_setup(K.handle, _dev(coords, torch.float64, "coords"), pp, ctypes.byref(h), _stream(stream)))
    return Amg(h, K)


def amg_info(amg: Amg) -> dict:
    L = ctypes.c_int()
    _check(lib.amg_info(amg.handle, ctypes.byref(L), None, None, None, None, None))
    n = L.value
    rows = (ctypes.c_longlong * n)()
    nnzb = (ctypes.c_longlong * n)()
    blk = (ctypes.c_int * n)()
    lam = (ctypes.c_double * n)()
    oc = ctypes.c_double()
    _check(lib.amg_info(amg.handle, ctypes.byref(L), rows, nnzb, blk, lam, ctypes.byref(oc)))
    return {"n_levels": n, "rows": list(rows), "nnzb": list(nnzb), "block": list(blk), "lambda": list(lam),
            "op_complexity": oc.value}


SETUP_PHASES = ("lambda_max", "aggregation", "tentative", "smoothing", "transpose", "galerkin", "layout",
                "coarse_inverse")


def amg_setup_stats(amg: Amg) -> dict:
    """Setup phase device times in ms (CUDA events), keyed by phase name."""
    buf = (ctypes.c_double * 8)()
    _check(lib.amg_setup_stats(amg.handle, buf))
    return dict(zip(SETUP_PHASES, list(buf)))


def amg_level_aggregates(amg: Amg, level: int, stream=None):
    info = amg_info(amg)
    agg = torch.empty(info["rows"][level], dtype=torch.int32, device="cuda")
    _check(lib.amg_level_aggregates(amg.handle, level, _vp(agg.data_ptr()), _stream(stream)))
    return agg


def amg_level_export(amg: Amg, level: int, which: int, stream=None) -> dict:
    nr, nc, br, bc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nnzb = ctypes.c_longlong()
    args = [ctypes.byref(x) for x in (nr, nc, br, bc, nnzb)]
    _check(lib.amg_level_export(amg.handle, level, which, *args, None, None, None, _stream(stream)))
    rp = torch.empty(nr.value + 1, dtype=torch.int32, device="cuda")
    ci = torch.empty(max(nnzb.value, 1), dtype=torch.int32, device="cuda")
    v = torch.empty((max(nnzb.value, 1), br.value, bc.value), dtype=torch.float64, device="cuda")
    _check(lib.amg_level_export(amg.handle, level, which, *args, _vp(rp.data_ptr()), _vp(ci.data_ptr()),
                                _vp(v.data_ptr()), _stream(stream)))
    return {"n_rows": nr.value, "n_cols": nc.value, "br": br.value, "bc": bc.value, "nnzb": nnzb.value,
            "row_ptr": rp, "col_idx": ci[:nnzb.value], "vals": v[:nnzb.value]}


def set_deterministic_assembly(on: bool) -> bool:
    """Process-wide assembly mode (True: bitwise reproducible sums); returns the previous mode."""
    prev = ctypes.c_int()
    _check(lib.tam_set_deterministic_assembly(int(bool(on)), ctypes.byref(prev)))
    return bool(prev.value)


def amg_residual_history(amg: Amg, stream=None) -> np.ndarray:
    """||r_k||_2, k = 0 .. iterations, of the hierarchy's last single-system solve."""
    n = ctypes.c_int()
    _check(lib.amg_residual_history(amg.handle, None, 0, ctypes.byref(n), _stream(stream)))
    h = np.empty(max(n.value, 1), np.float64)
    _check(lib.amg_residual_history(amg.handle, _vp(h.ctypes.data), n.value, None, _stream(stream)))
    return h[:n.value]


def amg_level_spmv_plan(amg: Amg, level: int, which: int) -> dict:
    """SpMV layout of one operator: kind (0 SELL, 1 lanes/row interleaved store,
    2 lanes/row block-CSR, 3 whole warps/row), lanes per row, double-float flag."""
    k, ln, df = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.amg_level_spmv_plan(amg.handle, int(level), int(which), ctypes.byref(k), ctypes.byref(ln),
                                   ctypes.byref(df)))
    return {"kind": k.value, "lanes": ln.value, "df": bool(df.value)}


def amg_solve_bytes(amg: Amg) -> dict:
    """Algorithmic bytes of one V-cycle and of one PCG iteration of this hierarchy."""
    v, it = ctypes.c_double(), ctypes.c_double()
    _check(lib.amg_solve_bytes(amg.handle, ctypes.byref(v), ctypes.byref(it)))
    return {"vcycle": v.value, "iteration": it.value}


def amg_smooth(amg: Amg, b, x, degree, stream=None):
    """x <- `degree` Chebyshev-Jacobi steps on K x = b (the finest level's smoother), in place."""
    _check(lib.amg_smooth(amg.handle, _dev(b, torch.float64, "b"), _dev(x, torch.float64, "x"), int(degree),
                          _stream(stream)))
    return x


def amg_vcycle(amg: Amg, r, z=None, stream=None):
    if z is None:
        z = torch.empty_like(r)
    _check(lib.amg_vcycle(amg.handle, _dev(r, torch.float64, "r"), _dev(z, torch.float64, "z"), _stream(stream)))
    return z


def amg_pcg_solve(amg: Amg, b, x, rtol=1e-8, atol=0.0, max_iter=1000, stream=None, raise_on_error=True):
    """Returns (iterations, ||b-Kx||/||b||, status)."""
    it, rel = ctypes.c_int(), ctypes.c_double()
    st = lib.amg_pcg_solve(amg.handle, _dev(b, torch.float64, "b"), _dev(x, torch.float64, "x"), float(rtol),
                           float(atol), int(max_iter), ctypes.byref(it), ctypes.byref(rel), _stream(stream))
    if raise_on_error:
        _check(st)
    return it.value, rel.value, st


def _host(a, dtype):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, _vp(arr.ctypes.data)


def tam_solve_elasticity_host(coords, cells, cell_material, mat_props, T, T_ref, body_force, dirichlet_mask,
                              u_dirichlet=None, params: AmgParams | None = None, rtol=1e-8, max_iter=1000,
                              u_out=None, stream=None):
    """Host-buffer path (numpy or pinned CPU torch tensors).  Returns (u[n,3], iters, rel)."""
    def hp(a, dt):
        if a is None:
            return None, None
        if isinstance(a, torch.Tensor):
            assert a.device.type == "cpu" and a.is_contiguous()
            return a, _vp(a.data_ptr())
        return _host(a, dt)
    keep = []
    ptrs = []
    for a, dt in ((coords, np.float64), (cells, np.int32), (cell_material, np.int32), (mat_props, np.float64),
                  (T, np.float64), (body_force, np.float64), (dirichlet_mask, np.uint8), (u_dirichlet, np.float64)):
        arr, p = hp(a, dt)
        keep.append(arr)
        ptrs.append(p)
    n_nodes = coords.shape[0]
    if u_out is None:
        u_out = np.empty((n_nodes, 3), dtype=np.float64)
    up = _vp(u_out.data_ptr()) if isinstance(u_out, torch.Tensor) else _vp(u_out.ctypes.data)
    it, rel = ctypes.c_int(), ctypes.c_double()
    pp = ctypes.byref(params) if params is not None else None
    st = lib.tam_solve_elasticity_host(n_nodes, ptrs[0], cells.shape[0], cells.shape[1], ptrs[1], ptrs[2],
                                       mat_props.shape[0], ptrs[3], ptrs[4], float(T_ref), ptrs[5], ptrs[6], ptrs[7],
                                       pp, float(rtol), int(max_iter), up, ctypes.byref(it), ctypes.byref(rel),
                                       _stream(stream))
    _check(st)
    return u_out, it.value, rel.value


def fem_assemble_load(K: Matrix, coords, cells, cell_material, mat_props, T=None, T_ref=0.0, body_force=None,
                      u_dirichlet=None, dirichlet_mask=None, stream=None, out=None):
    """Load vector [n,3] of another load case on K's mesh (dirichlet_mask is K's; accepted and ignored).

    out: optional contiguous float64 CUDA tensor of n*3 elements to write into.
    """
    if out is None:
        rhs = torch.empty((coords.shape[0], 3), dtype=torch.float64, device=coords.device)
    else:
        if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == 3 * coords.shape[0]):
            raise ValueError("out must be a contiguous float64 CUDA tensor of n*3 elements")
        rhs = out
    _check(lib.fem_assemble_load(
        K.handle, _dev(coords, torch.float64, "coords"), cells.shape[0], cells.shape[1],
        _dev(cells, torch.int32, "cells"), _dev(cell_material, torch.int32, "cell_material"), mat_props.shape[0],
        _dev(mat_props, torch.float64, "mat_props"), _dev(T, torch.float64, "T", True), float(T_ref),
        _dev(body_force, torch.float64, "body_force", True), _dev(u_dirichlet, torch.float64, "u_dirichlet", True),
        _vp(rhs.data_ptr()), _stream(stream)))
    return rhs


def amg_pcg_solve_batch(amgs, Bs, Xs, rtol=1e-8, atol=0.0, max_iter=1000, stream=None, raise_on_error=True):
    """Solve several systems, each with a block of right-hand sides.

    amgs: list of Amg; Bs/Xs: lists of [n_rhs, 3n] float64 CUDA tensors (X: guesses in,
    solutions out).  Returns (iterations per RHS, rel residual per RHS, status).
    """
    n = len(amgs)
    hs = (_vp * n)(*[a.handle for a in amgs])
    m = (ctypes.c_int * n)(*[int(B.shape[0]) for B in Bs])
    bp = (_vp * n)(*[_dev(B, torch.float64, "B") for B in Bs])
    xp = (_vp * n)(*[_dev(X, torch.float64, "X") for X in Xs])
    tot = sum(m)
    it = (ctypes.c_int * tot)()
    rel = (ctypes.c_double * tot)()
    st = lib.amg_pcg_solve_batch(n, hs, m, bp, xp, float(rtol), float(atol), int(max_iter), it, rel, _stream(stream))
    if raise_on_error:
        _check(st)
    return list(it), list(rel), st


def amg_batch_tiles(amg: Amg):
    """(RHS tiles chosen by the autotuner: K then (A, P, R) per level, tuning time ms)."""
    buf = (ctypes.c_int * 64)()
    n, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib.amg_batch_tiles(amg.handle, buf, 64, ctypes.byref(n), ctypes.byref(ms)))
    return list(buf)[:n.value], ms.value


class Mlp:
    """Handle of a node-wise MLP (learned initial guess)."""

    def __init__(self, n_in=8, width=128, depth=3, n_out=3, seed=1):
        h = _vp()
        _check(lib.tam_mlp_create(n_in, width, depth, n_out, seed, ctypes.byref(h)))
        self.handle = h
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out
        npar, nl = ctypes.c_longlong(), ctypes.c_int()
        _check(lib.tam_mlp_info(h, ctypes.byref(npar), ctypes.byref(nl)))
        self.n_params = npar.value

    def set_normalization(self, shift, scale, out_scale):
        a = [np.ascontiguousarray(v, dtype=np.float32) for v in (shift, scale, out_scale)]
        _check(lib.tam_mlp_set_normalization(self.handle, *[_vp(x.ctypes.data) for x in a]))

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        _check(lib.tam_mlp_get_params(self.handle, _vp(out.ctypes.data)))
        return out

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib.tam_mlp_set_params(self.handle, _vp(t.ctypes.data)))

    def forward(self, X, bf16=False, stream=None):
        Y = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device=X.device)
        _check(lib.tam_mlp_forward(self.handle, X.shape[0], _dev(X, torch.float32, "X"),
                                   _vp(Y.data_ptr()), int(bf16), _stream(stream)))
        return Y

    def loss_grad(self, X, Y, stream=None):
        loss = ctypes.c_double()
        g = np.empty(self.n_params, np.float32)
        _check(lib.tam_mlp_loss_grad(self.handle, X.shape[0], _dev(X, torch.float32, "X"),
                                     _dev(Y, torch.float32, "Y"), ctypes.byref(loss), _vp(g.ctypes.data),
                                     _stream(stream)))
        return loss.value, g

    def train_step(self, X, Y, lr, stream=None):
        loss = ctypes.c_double()
        _check(lib.tam_mlp_train_step(self.handle, X.shape[0], _dev(X, torch.float32, "X"),
                                      _dev(Y, torch.float32, "Y"), ctypes.c_float(lr), ctypes.byref(loss),
                                      _stream(stream)))
        return loss.value

    def destroy(self):
        if self.handle:
            lib.tam_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tam_node_features(coords, cells, T=None, dist=None, stream=None):
    F = torch.empty((coords.shape[0], 8), dtype=torch.float32, device=coords.device)
    _check(lib.tam_node_features(coords.shape[0], _dev(coords, torch.float64, "coords"), cells.shape[0],
                                 cells.shape[1], _dev(cells, torch.int32, "cells"), _dev(T, torch.float64, "T", True),
                                 _dev(dist, torch.float64, "dist", True), _vp(F.data_ptr()), _stream(stream)))
    return F


def tam_learned_guess(net: Mlp, amg: Amg, features, rhs, x=None, bf16=True, smooth_degree=8, stream=None):
    """Returns (x, used, <r, M r> / <rhs, M rhs>) after smooth_degree smoothing steps."""
    if x is None:
        x = torch.empty_like(rhs)
    used, rel = ctypes.c_int(), ctypes.c_double()
    _check(lib.tam_learned_guess(net.handle, amg.handle, _dev(features, torch.float32, "features"),
                                 _dev(rhs, torch.float64, "rhs"), int(bf16), int(smooth_degree),
                                 _dev(x, torch.float64, "x"),
                                 ctypes.byref(used), ctypes.byref(rel), _stream(stream)))
    return x, bool(used.value), rel.value


def problem_to_device(pb, device="cuda"):
    """Host arrays of a meshgen.Problem as the device tensors the C ABI takes."""
    t = lambda a, dt: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)
    return dict(coords=t(pb.coords, np.float64), cells=t(pb.cells, np.int32),
                cell_material=t(pb.cell_material, np.int32), mat_props=t(pb.mat_props, np.float64),
                T=t(pb.T, np.float64), T_ref=pb.T_ref, body_force=t(pb.body_force, np.float64),
                dirichlet_mask=t(pb.dirichlet_mask, np.uint8), u_dirichlet=t(pb.u_dirichlet, np.float64))


# ---------------------------------------------------------------------------
# The thermal problem (heat equation, theta-method, Newton)
# ---------------------------------------------------------------------------
class Thermal:
    """Handle of a thermal problem on a mesh (device arrays kept alive here)."""

    def __init__(self, coords, cells, cell_material, thermal_props, faces, dirichlet_mask=None, params=None,
                 stream=None):
        self._keep = [coords, cells, cell_material, faces, dirichlet_mask]
        npc = int(cells.shape[1])
        props = np.ascontiguousarray(np.asarray(thermal_props, dtype=np.float64))
        h = _vp()
        _check(lib.tam_thermal_create(int(coords.shape[0]), _dev(coords, torch.float64, "coords"), int(cells.shape[0]),
                                      npc, _dev(cells, torch.int32, "cells"),
                                      _dev(cell_material, torch.int32, "cell_material"), int(props.shape[0]),
                                      props.ctypes.data_as(_vp), int(faces.shape[0]),
                                      _dev(faces, torch.int32, "faces"),
                                      _dev(dirichlet_mask, torch.uint8, "dirichlet_mask", allow_none=True),
                                      ctypes.byref(params) if params is not None else None, ctypes.byref(h),
                                      _stream(stream)))
        self.handle = h
        self.n = int(coords.shape[0])

    def residual(self, T, T_old=None, dt=0.0, theta=1.0, beta=None, T_bc=None, stream=None):
        F = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(lib.tam_thermal_residual(self.handle, _dev(T, torch.float64, "T"),
                                        _dev(T_old, torch.float64, "T_old", allow_none=True), float(dt), float(theta),
                                        _dev(beta, torch.float64, "beta", allow_none=True),
                                        _dev(T_bc, torch.float64, "T_bc", allow_none=True), _dev(F, torch.float64, "F"),
                                        _stream(stream)))
        return F

    def jacobian(self, stream=None):
        """(row_ptr, col_idx, vals) of the last assembled Jacobian (device tensors)."""
        nnz = ctypes.c_longlong()
        _check(lib.tam_thermal_export_jacobian(self.handle, None, None, None, ctypes.byref(nnz), _stream(stream)))
        rp = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
        v = torch.empty(max(nnz.value, 1), dtype=torch.float64, device="cuda")
        _check(lib.tam_thermal_export_jacobian(self.handle, _vp(rp.data_ptr()), _vp(ci.data_ptr()), _vp(v.data_ptr()),
                                               ctypes.byref(nnz), _stream(stream)))
        return rp, ci[:nnz.value], v[:nnz.value]

    def newton(self, T, T_old=None, dt=0.0, theta=1.0, beta=None, T_bc=None, T_dirichlet=None, rtol=1e-9,
               max_newton=30, lin_rtol=1e-8, lin_max_iter=500, reuse=1, stream=None, raise_on_error=True):
        """Newton on F(T) = 0 in place; returns dict(newton, linear, setups, rel, status)."""
        it, li, su, rel = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        st = lib.tam_thermal_newton(self.handle, _dev(T, torch.float64, "T"),
                                    _dev(T_old, torch.float64, "T_old", allow_none=True), float(dt), float(theta),
                                    _dev(beta, torch.float64, "beta", allow_none=True),
                                    _dev(T_bc, torch.float64, "T_bc", allow_none=True),
                                    _dev(T_dirichlet, torch.float64, "T_dirichlet", allow_none=True), float(rtol),
                                    int(max_newton), float(lin_rtol), int(lin_max_iter), int(reuse),
                                    ctypes.byref(it), ctypes.byref(li), ctypes.byref(su), ctypes.byref(rel),
                                    _stream(stream))
        if raise_on_error:
            _check(st)
        return {"newton": it.value, "linear": li.value, "setups": su.value, "rel": rel.value, "status": st}

    def destroy(self):
        if self.handle:
            lib.tam_thermal_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tam_thermal_max_change(a, b, stream=None) -> float:
    m = ctypes.c_double()
    _check(lib.tam_thermal_max_change(_dev(a, torch.float64, "a"), _dev(b, torch.float64, "b"), int(a.numel()),
                                      ctypes.byref(m), _stream(stream)))
    return m.value


def tam_thermal_next_dt(dt, max_change, dT_max, eps):
    """Eq. dt_spec: (next dt, accepted)."""
    d, ok = ctypes.c_double(), ctypes.c_int()
    _check(lib.tam_thermal_next_dt(float(dt), float(max_change), float(dT_max), float(eps), ctypes.byref(d),
                                   ctypes.byref(ok)))
    return d.value, bool(ok.value)


def thermal_to_device(tp, device="cuda"):
    """Device tensors of a meshgen.ThermalProblem (mesh, faces, beta, T_bc, masks)."""
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)
    out = dict(coords=t(tp.coords, np.float64), cells=t(tp.cells, np.int32), cell_material=t(tp.cell_material, np.int32),
               faces=t(tp.faces, np.int32), beta=t(tp.beta, np.float64), T_bc=t(tp.T_bc, np.float64))
    out["dirichlet_mask"] = t(tp.dirichlet_mask, np.uint8) if tp.dirichlet_mask is not None else None
    out["T_dirichlet"] = t(tp.T_dirichlet, np.float64) if tp.T_dirichlet is not None else None
    return out
