"""Failure statuses of the CG solve, forced by bad host inputs (no GPU fault).

Sec. 2.1 ("Iterative solvers") asks for CG on an SPD system with an SPD
preconditioner, and Sec. 5.1 ("Solver configuration") warns that Chebyshev
smoothing needs an adequate estimate of lambda_max.  Each test breaks one of
those premises with an input the host builds, and checks that the single and
the batched solve both stop with the status that names it:

* a NaN in the load                              -> TAM_ERR_NAN
* a smoothing interval far below lambda_max      -> TAM_ERR_INDEFINITE_PRECOND
  (the Chebyshev polynomial amplifies the upper spectrum, so M^-1 is
  indefinite: r^T M^-1 r < 0 for the first residual)
* a region with a negative Young's modulus       -> TAM_ERR_BREAKDOWN
  (K indefinite: p^T K p < 0 for the first search direction)

The sign each status rests on is first computed with the oracle's V-cycle on
the same problem (its hierarchy is the GPU's: aggregation is unique), and the
margin is asserted, so the GPU's sign cannot flip by rounding.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import amg as oamg
from oracle import fem
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu

TAM_ERR_BREAKDOWN = -6
TAM_ERR_INDEFINITE_PRECOND = -7
TAM_ERR_NAN = -8


def _solve_both(tam, pb, params, b=None, max_iter=200):
    """Status of amg_pcg_solve and of amg_pcg_solve_batch (2 right-hand sides) on pb."""
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], params)
    bb = rhs if b is None else torch.from_numpy(b).cuda().reshape(rhs.shape)
    x = torch.zeros_like(bb)
    it, rel, st = tam.amg_pcg_solve(H, bb, x, rtol=1e-8, max_iter=max_iter, raise_on_error=False)
    B = torch.stack([bb.reshape(-1), 0.5 * bb.reshape(-1)])
    X = torch.zeros_like(B)
    its, rels, st_b = tam.amg_pcg_solve_batch([H], [B], [X], rtol=1e-8, max_iter=max_iter, raise_on_error=False)
    H.destroy()
    K.destroy()
    return st, it, st_b, its


def test_nan_in_load_gives_nan_status():
    tam = need_gpu()
    pb = meshgen.unit_cube_problem(6)
    b = np.asarray(fem.assemble_system(pb)[1], dtype=np.float64).copy()
    b[17] = np.nan
    st, it, st_b, _ = _solve_both(tam, pb, tam.amg_params_default(), b=b)
    assert st == TAM_ERR_NAN and it == 0
    assert st_b == TAM_ERR_NAN


def test_smoothing_interval_below_lambda_max_gives_indefinite_preconditioner():
    tam = need_gpu()
    pb = meshgen.unit_cube_problem(8)
    lo, hi = 0.01, 0.02
    K, f = fem.assemble_system(pb)
    Ho = oamg.setup(K, fem.rigid_body_modes(pb.coords, pb.dirichlet_mask), 3, cheb_lo=lo, cheb_hi=hi,
                    coarse_max_dofs=60)
    # the oracle's V-cycle on the first residual (x0 = 0): f^T M^-1 f < 0, by a wide margin
    z = oamg.vcycle(Ho, f)
    assert f @ z < -0.01 * np.linalg.norm(f) * np.linalg.norm(z)
    prm = tam.amg_params_default(cheb_lo=lo, cheb_hi=hi, coarse_max_dofs=60)
    st, it, st_b, _ = _solve_both(tam, pb, prm)
    assert st == TAM_ERR_INDEFINITE_PRECOND and it == 0
    assert st_b == TAM_ERR_INDEFINITE_PRECOND


def _negative_modulus_cube():
    """Unit cube 8^3, the 5% of cells nearest (0.7, 0.5, 0.5) with E = -10."""
    pb = meshgen.unit_cube_problem(8)
    cen = pb.coords[pb.cells].mean(axis=1)
    d = np.linalg.norm(cen - np.array([0.7, 0.5, 0.5]), axis=1)
    sel = np.argsort(d, kind="stable")[:int(0.05 * d.size)]
    mat = np.zeros(d.size, np.int32)
    mat[sel] = 1
    pb.cell_material = mat
    pb.mat_props = np.array([[1.0, 0.3, 1e-3], [-10.0, 0.3, 1e-3]])
    return pb


def test_negative_modulus_gives_breakdown():
    tam = need_gpu()
    pb = _negative_modulus_cube()
    K, f = fem.assemble_system(pb)
    assert np.linalg.eigvalsh(K.toarray()).min() < 0  # K is indefinite
    Ho = oamg.setup(K, fem.rigid_body_modes(pb.coords, pb.dirichlet_mask), 3, coarse_max_dofs=60)
    p = oamg.vcycle(Ho, f)          # first search direction from x0 = 0
    q = K @ p
    assert f @ p > 0.01 * np.linalg.norm(f) * np.linalg.norm(p)      # rz > 0: the preconditioner passes
    assert p @ q < -0.01 * np.linalg.norm(p) * np.linalg.norm(q)     # p^T K p < 0: breakdown at once
    st, it, st_b, _ = _solve_both(tam, pb, tam.amg_params_default(coarse_max_dofs=60))
    assert st == TAM_ERR_BREAKDOWN and it == 0
    assert st_b == TAM_ERR_BREAKDOWN
