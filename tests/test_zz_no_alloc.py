"""The allocation-free residual norm agrees with the allocating one.

tam_matrix_residual_norm_noalloc serves callers that must not allocate device
memory (allocator callbacks, fixed device-memory budgets, paths that cannot
take cudaMalloc's implicit synchronisation).  It keeps its reduction scratch in
a static device array, so it is checked here against
tam_matrix_residual_norm on two calls in a row (the second call must not see
stale scratch from the first), and its size limit is checked to refuse
without launching.  This file is named to be collected last.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-13  # same kernel and reduction order as the allocating entry point


def test_noalloc_residual_norm_matches_allocating_entry_point_twice():
    tam = need_gpu()
    pb = meshgen.slab_box_problem(48, 12, 12)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    gen = torch.Generator(device="cuda").manual_seed(3)
    for call in range(2):
        x = torch.randn(pb.n_nodes, 3, dtype=torch.float64, device="cuda", generator=gen) * 1e-3
        ref = tam.tam_matrix_residual_norm(K, rhs, x)
        got = tam.tam_matrix_residual_norm_noalloc(K, rhs, x)
        assert abs(got - ref) <= TOL * ref, (call, got, ref)
    # a different matrix and vector right after: results follow the inputs
    pb2 = meshgen.unit_cube_problem(9)
    d2 = tam.problem_to_device(pb2)
    K2, rhs2 = tam.fem_assemble_elasticity(**d2)
    z = torch.zeros_like(rhs2)
    got2 = tam.tam_matrix_residual_norm_noalloc(K2, rhs2, z)
    assert abs(got2 - float(torch.linalg.norm(rhs2))) <= TOL * got2


def test_noalloc_refuses_matrices_beyond_its_limit():
    tam = need_gpu()
    # 161 x 129 x 103 = 2,139,207 nodes > 2,097,152 block rows
    coords, cells = meshgen.box_kuhn(160, 128, 102)
    n = coords.shape[0]
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    K, rhs = tam.fem_assemble_elasticity(
        dev(coords, np.float64), dev(cells, np.int32), dev(np.zeros(cells.shape[0]), np.int32),
        dev(np.array([[1.0, 0.3, 0.0]]), np.float64), dirichlet_mask=dev(coords[:, 0] <= 0, np.uint8))
    x = torch.zeros_like(rhs)
    with pytest.raises(tam.TamError) as e:
        tam.tam_matrix_residual_norm_noalloc(K, rhs, x)
    assert e.value.code == -1 and "limit" in str(e.value)
    assert n > 2_097_152
