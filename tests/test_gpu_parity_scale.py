"""Parity at the sizes and configurations the benchmark runs.

The method's result is the solution of K u = f (Sec. 2.1, "Iterative
solvers": CG and the AMG preconditioner only reach it faster), so the GPU
displacement is compared with a solution the oracle reaches by itself:

* the full two-material box, 256x64x64 hexes -> 6,291,456 P1 tets,
  3,257,475 DOF (the benchmark workload), against the oracle's own assembly
  and SA-AMG-PCG run to rtol 1e-12 (several minutes on the host cores);
* a reduced P2 bladed disc (12 blades, 29,880 DOF) against a sparse direct
  solve, with the FP64 and the FP32 V-cycle.

At full size the setup picks size-dependent SpMV layouts (SELL-32 for K and
the level-0 prolongator, 8 lanes per row over the interleaved store for the
level-1 operator and the level-0 restriction, whole warps per row for the few
long rows of level 2 and the level-1 restriction, double-float products on
operators of at least 2^20 blocks).  The V-cycle is compared, element by
element, with the oracle's V-cycle (Sec. 5.1: Chebyshev smoothing, Galerkin
coarse levels, exact coarsest solve) applied to the operators the GPU built,
in every precision mode, and the test asserts which layouts ran.
"""
import numpy as np
import pytest

from gpu_util import bsr_to_csr, exact_spmv, need_gpu, torch
from oracle import amg as oamg
from oracle import fem, linsolve
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-6          # displacement rel L2 at rtol 1e-8
VCYCLE_TOL = {0: 1e-9, 1: 1e-5, 2: 5e-2}   # FP64 / FP32 / FP32 with BF16 finest values vs the FP64 oracle


@pytest.fixture(scope="module")
def full_box():
    tam = need_gpu()
    pb = meshgen.slab_box_problem()
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"])
    yield tam, pb, d, K, rhs, H
    H.destroy()
    K.destroy()


def test_full_box_displacement_matches_oracle_solve(full_box):
    tam, pb, d, K, rhs, H = full_box
    assert pb.n_dof == 3_257_475
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-8, max_iter=500)
    assert st == 0 and rel <= 1e-8
    u_gpu = x.cpu().numpy().ravel()
    del x
    Ko, fo = fem.assemble_system(pb)
    u_o, it_o, rel_o, _ = oamg.solve(Ko, fo, pb.coords, pb.dirichlet_mask, rtol=1e-12)
    assert rel_o <= 1e-12
    err = np.linalg.norm(u_gpu - u_o) / np.linalg.norm(u_o)
    assert err <= SOL_TOL, (it, rel, err, it_o)


def _oracle_hierarchy_from(tam, H):
    """The oracle's V-cycle data structure filled with the operators the GPU built."""
    info = tam.amg_info(H)
    levels = []
    for lev in range(info["n_levels"]):
        e = tam.amg_level_export(H, lev, 0)
        A = bsr_to_csr(e["row_ptr"], e["col_idx"], e["vals"], e["n_cols"])
        L = oamg.Level(A=A, bs=info["block"][lev], dinv=oamg.point_dinv(A), lam=info["lambda"][lev])
        if lev + 1 < info["n_levels"]:
            for which, attr in ((1, "P"), (2, "R")):
                e = tam.amg_level_export(H, lev, which)
                setattr(L, attr, bsr_to_csr(e["row_ptr"], e["col_idx"], e["vals"], e["n_cols"]))
        levels.append(L)
    return oamg.Hierarchy(levels=levels, coarse_inv=oamg.coarse_inverse(levels[-1].A), params=dict(oamg.DEFAULTS))


@pytest.fixture(scope="module")
def full_box_oracle_vcycle(full_box):
    tam, pb, d, K, rhs, H = full_box
    return _oracle_hierarchy_from(tam, H)


@pytest.mark.parametrize("precision,spmv_fp64", [(0, 0), (0, 1), (1, 0), (2, 0)])
def test_full_box_vcycle_matches_oracle_on_gpu_operators(full_box, full_box_oracle_vcycle, precision, spmv_fp64):
    tam, pb, d, K, rhs, H0 = full_box
    Ho = full_box_oracle_vcycle
    H = H0 if (precision, spmv_fp64) == (0, 0) else tam.amg_setup(
        K, d["coords"], tam.amg_params_default(level_precision=precision, spmv_fp64=spmv_fp64))
    info = tam.amg_info(H)
    assert [L.A.shape[0] for L in Ho.levels] == [r * b for r, b in zip(info["rows"], info["block"])]
    # the layouts of the full-size plan
    plans = {(lev, w): tam.amg_level_spmv_plan(H, lev, w)
             for lev in range(info["n_levels"] - 1) for w in (0, 1, 2)}
    kinds = {p["kind"] for p in plans.values()}
    assert kinds == {0, 1, 4}, plans                         # SELL-32, 8-lane store, block-row lanes
    assert plans[(0, 0)]["kind"] == 0 and plans[(0, 1)]["kind"] == 0   # K and P_0: SELL-32
    assert plans[(0, 2)]["kind"] == 1 and plans[(0, 2)]["lanes"] == 8  # R_0 (6x3): 8-lane store
    assert plans[(1, 0)]["kind"] == 1 and plans[(1, 0)]["lanes"] == 8  # A_1: 8-lane store
    assert plans[(1, 1)]["kind"] == 4                        # P_1 (short rows): block-row lanes
    assert any(p["kind"] == 4 and p["lanes"] >= 64 for p in plans.values())   # coarse long rows: several warps
    if spmv_fp64 == 0:
        assert plans[(0, 0)]["df"] and plans[(1, 0)]["df"]   # >= 2^20 blocks: double-float products
    else:
        assert not any(p["df"] for p in plans.values())
    rng = np.random.default_rng(7)
    for _ in range(2):
        r = rng.standard_normal(pb.n_dof)
        zg = tam.amg_vcycle(H, torch.from_numpy(r).cuda()).cpu().numpy()
        zo = oamg.vcycle(Ho, r)
        err = np.linalg.norm(zg - zo) / np.linalg.norm(zo)
        assert err <= VCYCLE_TOL[precision], (precision, spmv_fp64, err)
    if H is not H0:
        H.destroy()


def test_full_box_smoother_matches_oracle_chebyshev(full_box):
    """The benchmark's dominant kernel: the level-0 Chebyshev step (Sec. 5.1
    smoother; fused SpMV + update) against the oracle's Chebyshev iteration on
    the exported K, its point diagonal and the GPU's lambda_max estimate."""
    tam, pb, d, K, rhs, H = full_box
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    A = bsr_to_csr(rp, ci, v, pb.n_nodes)
    del rp, ci, v
    lam = tam.amg_info(H)["lambda"][0]
    rng = np.random.default_rng(11)
    x0 = rng.standard_normal(pb.n_dof)
    b = rhs.cpu().numpy().ravel()
    for degree in (1, 4):
        xg = tam.amg_smooth(H, rhs, torch.from_numpy(x0).cuda().reshape(rhs.shape), degree).cpu().numpy().ravel()
        xo = oamg.chebyshev(A, oamg.point_dinv(A), b, x0, 0.1 * lam, 1.1 * lam, degree)
        assert np.linalg.norm(xg - xo) <= 1e-10 * np.linalg.norm(xo), degree
    assert tam.amg_level_spmv_plan(H, 0, 0) == {"kind": 0, "lanes": 1, "df": True}


def test_full_box_outer_spmv_within_1e14_per_row(full_box):
    """A13, the outer CG's y = K x at full size: every sampled row within
    1e-14 of sum_j |K_ij x_j| of the correctly rounded product."""
    tam, pb, d, K, rhs, H = full_box
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    A = bsr_to_csr(rp, ci, v, pb.n_nodes)
    del rp, ci, v
    xs = np.random.default_rng(13).standard_normal((pb.n_nodes, 3))
    y = tam.tam_matrix_spmv(K, torch.from_numpy(xs).cuda()).cpu().numpy().ravel()
    rows = np.unique(np.random.default_rng(12).integers(0, pb.n_dof, 20000))
    y_ex, s = exact_spmv(A[rows], xs.ravel())
    err = np.abs(y[rows] - y_ex)
    assert np.all(err <= 1e-14 * s), (err / np.maximum(s, 1e-300)).max()


def _small_p2_disc():
    return meshgen.bladed_disc_problem(n_r=8, n_theta_per_blade=4, n_z=2, n_blades=12, n_r_blade=3, degree=2)


@pytest.mark.parametrize("precision", [0, 1])
def test_p2_disc_solve_matches_direct_solve(precision):
    tam = need_gpu()
    pb = _small_p2_disc()
    assert pb.n_dof == 29_880
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=precision))
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-8, max_iter=1000)
    assert st == 0 and rel <= 1e-8
    Ko, fo = fem.assemble_system(pb)
    u = linsolve.direct_solve(Ko, fo)
    err = np.linalg.norm(x.cpu().numpy().ravel() - u) / np.linalg.norm(u)
    assert err <= SOL_TOL, (it, rel, err)
