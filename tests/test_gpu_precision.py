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
def test_low_precision_vcycle_matches_fp64_vcycle(precision, tol):
    tam = need_gpu()
    pb = meshgen.slab_box_problem(32, 8, 8)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    prm = dict(coarse_max_dofs=60)
    H64 = tam.amg_setup(K, d["coords"], tam.amg_params_default(**prm))
    Hlo = tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=precision, **prm))
    assert tam.amg_info(H64)["rows"] == tam.amg_info(Hlo)["rows"]
    r = torch.randn(pb.n_nodes, 3, dtype=torch.float64, device="cuda")
    z64 = tam.amg_vcycle(H64, r)
    zlo = tam.amg_vcycle(Hlo, r)
    rel = float(torch.linalg.norm(zlo - z64) / torch.linalg.norm(z64))
    assert rel <= tol, rel
    # still a positive operator on random vectors
    assert float((r * zlo).sum()) > 0
