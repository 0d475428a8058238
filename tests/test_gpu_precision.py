"""Reduced-precision V-cycle inside FP64 CG (FP32 hierarchy; BF16 finest values).

The outer CG keeps FP64 residuals, dot products and stopping test, and the
coarsest dense solve stays FP64, so the displacement must still match a direct
FP64 solve to rel L2 <= 1e-6 at rtol 1e-8; the V-cycle itself is compared
with the FP64 V-cycle on the same hierarchy within the precision's own
rounding (FP32: 1e-5, BF16 values: 5e-2 relative).
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import fem, linsolve
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu


def _solve(pb, precision, **prm):
    tam = need_gpu()
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=precision, **prm))
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-8, max_iter=500)
    return tam, K, rhs, H, x, it, rel, st


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("problem", ["slab", "cube_p2"])
def test_low_precision_vcycle_keeps_fp64_accuracy(problem, precision):
    pb = {"slab": lambda: meshgen.slab_box_problem(48, 12, 12),
          "cube_p2": lambda: meshgen.unit_cube_problem(5, 2)}[problem]()
    _, _, _, _, x64, it64, _, st64 = _solve(pb, 0)
    tam, K, rhs, H, x, it, rel, st = _solve(pb, precision)
    assert st == 0 and rel <= 1e-8
    Ko, fo = fem.assemble_system(pb)
    u = linsolve.dense_solve(Ko, fo) if Ko.shape[0] <= 6000 else linsolve.direct_solve(Ko, fo)
    err = np.linalg.norm(x.cpu().numpy().ravel() - u) / np.linalg.norm(u)
    assert err <= 1e-6, (precision, it, err)
    assert it <= it64 + 3, (it, it64)


@pytest.mark.parametrize("precision,tol", [(1, 1e-5), (2, 5e-2)])
def test_low_precision_vcycle_matches_oracle_vcycle(precision, tol):
    """The reduced-precision V-cycle vs the oracle's FP64 V-cycle on the same operators.

    The hierarchy's exported operators (FP64 arrays) feed the oracle's
    V-cycle; the FP32 arithmetic of the V-cycle must agree within its own
    rounding (FP32: 1e-5; BF16 finest values: 5e-2).
    """
    from gpu_util import bsr_to_csr
    from oracle import amg as oamg
    tam = need_gpu()
    pb = meshgen.slab_box_problem(32, 8, 8)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=precision, coarse_max_dofs=60))
    info = tam.amg_info(H)
    nl = info["n_levels"]
    assert nl >= 3

    def ex(lev, which):
        e = tam.amg_level_export(H, lev, which)
        return bsr_to_csr(e["row_ptr"], e["col_idx"], e["vals"], e["n_cols"])

    levels = []
    for lev in range(nl):
        A = ex(lev, 0)
        L = oamg.Level(A=A, bs=info["block"][lev], dinv=oamg.point_dinv(A), lam=info["lambda"][lev])
        if lev < nl - 1:
            L.P, L.R = ex(lev, 1), ex(lev, 2)
        levels.append(L)
    Ho = oamg.Hierarchy(levels=levels, coarse_inv=oamg.coarse_inverse(levels[-1].A), params=dict(oamg.DEFAULTS))
    rng = np.random.default_rng(3)
    r = rng.standard_normal(pb.n_dof)
    z = tam.amg_vcycle(H, torch.from_numpy(r).cuda()).cpu().numpy()
    zo = oamg.vcycle(Ho, r)
    rel = np.linalg.norm(z - zo) / np.linalg.norm(zo)
    assert rel <= tol, rel
    # still a positive operator on random vectors
    assert float(r @ z) > 0


@pytest.mark.parametrize("setup_fp64", [0, 1])
def test_setup_products_match_oracle(setup_fp64):
    """Setup products in double-float (default) or plain FP64 arithmetic.

    Double-float keeps each operand as two FP32 values and forms products and
    sums with error-free transforms (about 2^-48 relative), so the FP32-stored
    hierarchy's operators match the oracle's FP64 formulas applied to the same
    level inputs at the FP64 setup tolerance (1e-10), like the plain FP64
    arithmetic; aggregates and level sizes equal the FP64 setup's.
    """
    from gpu_util import bsr_to_csr, sparse_rel
    from oracle import amg as oamg
    tam = need_gpu()
    pb = meshgen.slab_box_problem(32, 8, 8)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    prm = dict(coarse_max_dofs=60)
    H64 = tam.amg_setup(K, d["coords"], tam.amg_params_default(**prm))
    H32 = tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=1, setup_fp64=setup_fp64, **prm))
    info = tam.amg_info(H32)
    assert info["rows"] == tam.amg_info(H64)["rows"]

    def ex(lev, which):
        e = tam.amg_level_export(H32, lev, which)
        return bsr_to_csr(e["row_ptr"], e["col_idx"], e["vals"], e["n_cols"])

    for lev in range(info["n_levels"] - 1):
        assert np.array_equal(tam.amg_level_aggregates(H32, lev).cpu().numpy(),
                              tam.amg_level_aggregates(H64, lev).cpu().numpy())
        A, Pt, P = ex(lev, 0), ex(lev, 3), ex(lev, 1)
        assert sparse_rel(P, oamg.smooth_prolongator(A, Pt, info["lambda"][lev])) <= 1e-10, lev
        Ac, _ = oamg.galerkin(A, P)
        assert sparse_rel(ex(lev + 1, 0), Ac) <= 1e-10, lev


def test_double_float_spmv_matches_fp64_spmv():
    """SpMVs of the solve in double-float on every operator (spmv_fp64 = 2) vs plain FP64 (1).

    Double-float products are accurate to about 2^-47 of the terms, so both
    arithmetics take the same number of iterations (+-1); their iterates then
    differ by what the stopping point leaves (both stop at ||r|| <= 1e-8
    ||b||; measured 1.4e-9 apart, bound 1e-7), and both match the direct
    solve to 1e-6.
    """
    pb = meshgen.slab_box_problem(48, 12, 12)
    _, _, _, _, xdf, itdf, reldf, stdf = _solve(pb, 0, spmv_fp64=2)
    _, _, _, _, x64, it64, rel64, st64 = _solve(pb, 0, spmv_fp64=1)
    assert stdf == 0 and st64 == 0 and reldf <= 1e-8 and rel64 <= 1e-8
    assert abs(itdf - it64) <= 1, (itdf, it64)
    assert float(torch.linalg.norm(xdf - x64) / torch.linalg.norm(x64)) <= 1e-7
    Ko, fo = fem.assemble_system(pb)
    u = linsolve.direct_solve(Ko, fo)
    for x in (xdf, x64):
        assert np.linalg.norm(x.cpu().numpy().ravel() - u) <= 1e-6 * np.linalg.norm(u)


def test_bf16_request_on_p2_keeps_fp32():
    """BF16 finest-level values double the iterations on P2 matrices (their
    8-bit mantissa weakens the fine smoother), so level_precision 2 on a P2 K
    builds the FP32 hierarchy: the same V-cycle, bit for bit, as level 1."""
    pb = meshgen.unit_cube_problem(5, 2)
    tam = need_gpu()
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    z = [tam.amg_vcycle(tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=p)), rhs.reshape(-1))
         for p in (1, 2)]
    assert torch.equal(z[0], z[1])
