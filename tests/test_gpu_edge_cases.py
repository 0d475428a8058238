"""Degenerate meshes and the full-size solve.

Degenerate cases of the method (Sec. 3, Eq. u-dbc): a mesh without cells
(K = I), nodes that belong to no cell (identity rows, zero load), a mesh
whose every node is clamped (K = I, u = u_D).  At the full 256x64x64 box
size the solve is checked on sampled rows: the residual of the GPU
displacement against the oracle's own assembly of those rows must be below
the stopping tolerance (|r_i| <= ||r||_2 <= 1e-8 ||b||_2 for every row i).
"""
import numpy as np
import pytest

from gpu_util import bsr_to_csr, need_gpu, torch
from oracle import fem, linsolve
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu


def _dev(pb, tam):
    return tam.problem_to_device(pb)


def test_mesh_without_cells_is_identity():
    tam = need_gpu()
    rng = np.random.default_rng(1)
    n = 37
    coords = rng.uniform(0, 1, (n, 3))
    mask = np.zeros(n, np.uint8)
    mask[[0, 5, 36]] = 1
    ud = np.zeros((n, 3))
    ud[mask.astype(bool)] = rng.standard_normal((3, 3))
    pb = meshgen.Problem("empty", coords, np.zeros((0, 4), np.int32), np.zeros(0, np.int32),
                         np.array([[1.0, 0.3, 1e-3]]), rng.standard_normal(n), 0.0, rng.standard_normal((n, 3)),
                         mask, ud)
    d = _dev(pb, tam)
    K, rhs = tam.fem_assemble_elasticity(**d)
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    Kg = bsr_to_csr(rp, ci, v, n)
    assert abs(Kg - np.eye(3 * n)).max() == 0.0
    assert np.array_equal(rhs.cpu().numpy(), ud)
    H = tam.amg_setup(K, d["coords"])
    b = torch.randn(n, 3, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    it, rel, st = tam.amg_pcg_solve(H, b, x, rtol=1e-8)
    assert st == 0 and it <= 1 and float((x - b).abs().max()) <= 1e-14 * float(b.abs().max())


def test_nodes_in_no_cell_get_identity_rows():
    tam = need_gpu()
    base = meshgen.slab_box_problem(8, 3, 3)
    rng = np.random.default_rng(2)
    extra = rng.uniform(0, 1, (5, 3)) + np.array([5.0, 0, 0])
    n0 = base.n_nodes
    coords = np.vstack([base.coords, extra])
    mask = np.concatenate([base.dirichlet_mask, np.array([0, 1, 0, 0, 0], np.uint8)])
    ud = np.zeros((coords.shape[0], 3))
    ud[n0 + 1] = [1e-3, -2e-3, 5e-4]
    T = np.concatenate([base.T, rng.standard_normal(5)])
    body = rng.standard_normal((coords.shape[0], 3))
    pb = meshgen.Problem("isolated", coords, base.cells, base.cell_material, base.mat_props, T, base.T_ref, body,
                         mask, ud)
    d = _dev(pb, tam)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], tam.amg_params_default(coarse_max_dofs=60))
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-10)
    assert st == 0
    # reference: the oracle's assembly, identity rows for the nodes in no cell (their load 0)
    Ko, fo = fem.assemble(pb.coords, pb.cells, pb.cell_material, pb.mat_props, pb.T, pb.T_ref, pb.body_force)
    iso = np.setdiff1d(np.arange(coords.shape[0]), np.unique(pb.cells))
    assert np.array_equal(iso, np.arange(n0, n0 + 5))
    dofs = (3 * iso[:, None] + np.arange(3)).ravel()
    Ko = Ko.tolil()
    for k in dofs:
        Ko[k, k] = 1.0
    fo[dofs] = 0.0
    Ko, fo = fem.apply_dirichlet(Ko.tocsr(), fo, pb.dirichlet_mask, pb.u_dirichlet)
    u = linsolve.direct_solve(Ko, fo)
    xs = x.cpu().numpy().ravel()
    assert np.linalg.norm(xs - u) <= 1e-6 * np.linalg.norm(u)
    # the free nodes in no cell stay at zero; the clamped one takes u_D up to its share
    # of the CG residual (an identity row: |x_D - u_D| = |r_D| <= ||r|| <= rtol ||b||)
    bnorm = float(torch.linalg.norm(rhs))
    free_iso = (3 * np.array([n0, n0 + 2, n0 + 3, n0 + 4])[:, None] + np.arange(3)).ravel()
    assert np.abs(xs[free_iso]).max() <= 1e-10 * bnorm
    assert np.abs(xs[3 * (n0 + 1):3 * (n0 + 2)] - ud[n0 + 1]).max() <= 1e-10 * bnorm


def test_all_nodes_clamped():
    tam = need_gpu()
    pb = meshgen.slab_box_problem(6, 2, 2)
    rng = np.random.default_rng(3)
    pb.dirichlet_mask = np.ones(pb.n_nodes, np.uint8)
    pb.u_dirichlet = rng.standard_normal((pb.n_nodes, 3))
    d = _dev(pb, tam)
    K, rhs = tam.fem_assemble_elasticity(**d)
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    assert abs(bsr_to_csr(rp, ci, v, pb.n_nodes) - np.eye(pb.n_dof)).max() == 0.0
    assert np.array_equal(rhs.cpu().numpy(), pb.u_dirichlet)
    H = tam.amg_setup(K, d["coords"])
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-8)
    assert st == 0 and it <= 1
    assert float((x - rhs).abs().max()) <= 1e-14 * float(rhs.abs().max())


def test_full_size_box_solve_sampled_residual():
    """256x64x64 box (3,257,475 DOF), library defaults: residual on sampled rows."""
    tam = need_gpu()
    pb = meshgen.slab_box_problem()
    d = _dev(pb, tam)
    K, rhs = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"])
    x = torch.zeros_like(rhs)
    it, rel, st = tam.amg_pcg_solve(H, rhs, x, rtol=1e-8)
    assert st == 0 and rel <= 1e-8
    true_rel = tam.tam_matrix_residual_norm(K, rhs, x) / float(torch.linalg.norm(rhs))
    assert true_rel <= 1.01e-8
    n = pb.n_nodes
    rng = np.random.default_rng(4)
    nodes = np.unique(np.concatenate([rng.integers(0, n, 200), [1, n - 1, 257 * 65 * 32 + 128]]))
    hit = np.isin(pb.cells, nodes).any(axis=1)
    Ko, fo = fem.assemble(pb.coords, pb.cells[hit], pb.cell_material[hit], pb.mat_props, pb.T, pb.T_ref)
    Ko, fo = fem.apply_dirichlet(Ko, fo, pb.dirichlet_mask)
    u = x.cpu().numpy().ravel()
    bnorm = float(torch.linalg.norm(rhs))
    rows = (3 * nodes[:, None] + np.arange(3)).ravel()
    r = fo[rows] - Ko[rows] @ u
    assert np.abs(r).max() <= 1e-8 * bnorm, (np.abs(r).max(), bnorm)
