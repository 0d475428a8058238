"""Assembly, hierarchy and PCG parity on unstructured meshes (paper Sec. 4 "Meshes",
Sec. 2.2 on cell quality; Sec. 5.1 on robustness on lower-quality meshes).

The meshes are seeded Delaunay tetrahedrisations of the two-material box
(irregular valences, slivers with dihedral angles below 2 degrees kept: the
mesh-quality stress the paper discusses), and one with a node of about 160
incident cells, whose P2 row has more candidates than the pattern builder's
shared memory holds (the global-memory path).  K and f are compared entry by
entry with the oracle's assembly, the hierarchy step by step (aggregates bit
for bit), and the PCG displacement with a direct solve.
"""
import numpy as np
import pytest

from gpu_util import bsr_to_csr, need_gpu, sparse_rel, torch
from oracle import amg as oamg
from oracle import fem, linsolve
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12
OP_TOL = 1e-10
SOL_TOL = 1e-6


@pytest.mark.parametrize("n,degree,hub", [(6, 1, 0), (6, 2, 0), (8, 2, 80)])
def test_unstructured_assembly_matches_oracle(n, degree, hub):
    tam = need_gpu()
    pb = meshgen.delaunay_box_problem(n, degree, hub=hub)
    if hub:
        assert 1 + np.bincount(pb.cells.ravel()).max() * 10 > 1024   # beyond the shared-memory row builder
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    Kg = bsr_to_csr(rp, ci, v, pb.n_nodes)
    Ko, fo = fem.assemble_system(pb)
    assert sparse_rel(Kg, Ko) <= TOL
    assert np.abs(rhs.cpu().numpy().ravel() - fo).max() <= TOL * np.abs(fo).max()
    rpn, cin = rp.cpu().numpy(), ci.cpu().numpy()
    assert all(np.all(np.diff(cin[rpn[i]:rpn[i + 1]]) > 0) for i in range(pb.n_nodes))


def test_unstructured_hierarchy_matches_oracle_step_by_step():
    tam = need_gpu()
    pb = meshgen.delaunay_box_problem(8, 1, seed=4)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], tam.amg_params_default(coarse_max_dofs=60))
    info = tam.amg_info(H)
    assert info["n_levels"] >= 3
    Ko, _ = fem.assemble_system(pb)
    B = fem.rigid_body_modes(pb.coords, pb.dirichlet_mask)
    A_in, bs = Ko, 3
    for lev in range(info["n_levels"] - 1):
        e = tam.amg_level_export(H, lev, 0)
        Ag = bsr_to_csr(e["row_ptr"], e["col_idx"], e["vals"], e["n_cols"])
        assert sparse_rel(Ag, A_in) <= OP_TOL, lev
        nbrs = oamg.strength_graph(Ag, bs, 0.02 * 0.5 ** lev)
        agg_o, n_agg = oamg.aggregate_level(nbrs, lev, 6, 500, aggressive_levels=1)
        assert np.array_equal(tam.amg_level_aggregates(H, lev).cpu().numpy(), agg_o), lev
        e = tam.amg_level_export(H, lev, 1)
        Pg = bsr_to_csr(e["row_ptr"], e["col_idx"], e["vals"], e["n_cols"])
        Pto, Bc = oamg.tentative_prolongator(agg_o, n_agg, B, bs)
        assert sparse_rel(Pg, oamg.smooth_prolongator(Ag, Pto, info["lambda"][lev])) <= OP_TOL, lev
        Aco, _ = oamg.galerkin(Ag, Pg)
        A_in, B, bs = Aco, Bc, 6


@pytest.mark.parametrize("n,degree,hub", [(12, 1, 0), (6, 2, 0), (8, 2, 80)])
def test_unstructured_pcg_matches_direct_solve(n, degree, hub):
    tam = need_gpu()
    pb = meshgen.delaunay_box_problem(n, degree, hub=hub)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"])
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-8, max_iter=1000)
    assert st == 0 and rel <= 1e-8
    Ko, fo = fem.assemble_system(pb)
    u = linsolve.direct_solve(Ko, fo)
    err = np.linalg.norm(x.cpu().numpy().ravel() - u) / np.linalg.norm(u)
    assert err <= SOL_TOL, (it, rel, err, pb.meta)
