"""Problems posed in other units: the double-float and FP32 paths keep FP64 accuracy.

The weak form of Sec. 3 (Eq. wf_elastic) is linear in E and in the loads:
scaling every Young's modulus by s scales K and the thermal load by s and
leaves u unchanged; scaling alpha by s scales u by s.  The double-float
products split FP64 values into FP32 pairs, and the FP32 V-cycle stores FP32
values, so both need their operands inside FP32's exponent range:

* the CG vectors are moved by a power of two (exact) so that their entries sit
  near the middle of that range, whatever the scale of the loads;
* a K whose largest entry lies outside 2^-90..2^90 runs its products in FP64
  (automatic choice), and the requests that need FP32 arithmetic on it
  (spmv_fp64 = 2, an FP32 V-cycle, the batched solve) are refused with
  TAM_ERR_INVALID_ARG.

Every case is compared with the oracle's dense solve of the unscaled unit
cube (C1), rel L2 <= 1e-6 at rtol 1e-8.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import fem, linsolve
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-6


@pytest.fixture(scope="module")
def cube():
    pb = meshgen.unit_cube_problem(10)
    K, f = fem.assemble_system(pb)
    return pb, linsolve.dense_solve(K, f)


def _scaled(pb, e_scale=1.0, alpha_scale=1.0):
    q = meshgen.unit_cube_problem(10)
    q.mat_props = pb.mat_props.copy()
    q.mat_props[:, 0] *= e_scale
    q.mat_props[:, 2] *= alpha_scale
    return q


def _solve(tam, pb, **prm):
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], tam.amg_params_default(**prm))
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-8, max_iter=500)
    return it, rel, st, x.cpu().numpy().ravel(), K, H, rhs


def _err(u, ref):
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("e_scale", [1e-20, 1e20])
@pytest.mark.parametrize("spmv_fp64,precision", [(0, 0), (1, 0), (2, 0), (0, 1)])
def test_scaled_modulus_gives_the_same_displacement(cube, e_scale, spmv_fp64, precision):
    tam = need_gpu()
    pb, u0 = cube
    it1, _, _, _, K1, H1, _ = _solve(tam, _scaled(pb), spmv_fp64=spmv_fp64, level_precision=precision)
    it, rel, st, u, K, H, _ = _solve(tam, _scaled(pb, e_scale), spmv_fp64=spmv_fp64, level_precision=precision)
    assert st == 0 and rel <= 1e-8
    assert _err(u, u0) <= SOL_TOL
    assert abs(it - it1) <= 1, (it, it1)
    # in range: the requested arithmetic is the one that ran
    assert tam.amg_level_spmv_plan(H, 0, 0)["df"] == (spmv_fp64 == 2)


@pytest.mark.parametrize("e_scale", [1e-30, 1e30])
def test_out_of_range_modulus_falls_back_to_fp64_or_is_refused(cube, e_scale):
    tam = need_gpu()
    pb, u0 = cube
    q = _scaled(pb, e_scale)
    it, rel, st, u, K, H, rhs = _solve(tam, q)       # automatic choice: FP64 products
    assert st == 0 and rel <= 1e-8 and _err(u, u0) <= SOL_TOL
    info = tam.amg_info(H)
    assert not any(tam.amg_level_spmv_plan(H, l, w)["df"] for l in range(info["n_levels"] - 1) for w in (0, 1, 2))
    d = tam.problem_to_device(q)
    for prm in (dict(spmv_fp64=2), dict(level_precision=1)):
        with pytest.raises(tam.TamError) as e:
            tam.amg_setup(K, d["coords"], tam.amg_params_default(**prm))
        assert e.value.code == -1 and "2^" in str(e.value)
    B = torch.stack([rhs.reshape(-1), 2.0 * rhs.reshape(-1)])
    _, _, st_b = tam.amg_pcg_solve_batch([H], [B], [torch.zeros_like(B)], raise_on_error=False)
    assert st_b == -1


def test_tiny_loads_keep_fp64_accuracy(cube):
    """alpha scaled by 1e-40: u ~ 1e-43, far below FP32's range; the centred
    CG vectors keep the double-float SpMVs, the FP32 V-cycle and the batch exact."""
    tam = need_gpu()
    pb, u0 = cube
    ref = 1e-40 * u0
    q = _scaled(pb, alpha_scale=1e-40)
    for prm in (dict(spmv_fp64=2), dict(level_precision=1), dict(spmv_fp64=2, level_precision=2)):
        it, rel, st, u, K, H, rhs = _solve(tam, q, **prm)
        assert st == 0 and rel <= 1e-8, prm
        assert _err(u, ref) <= SOL_TOL, (prm, _err(u, ref))
    B = torch.stack([rhs.reshape(-1), -3.0 * rhs.reshape(-1)])
    X = torch.zeros_like(B)
    its, rels, st_b = tam.amg_pcg_solve_batch([H], [B], [X])
    assert st_b == 0 and max(rels) <= 1e-8
    assert _err(X[0].cpu().numpy(), ref) <= SOL_TOL and _err(X[1].cpu().numpy(), -3.0 * ref) <= SOL_TOL
