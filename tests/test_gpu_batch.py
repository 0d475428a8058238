"""Many load cases at once: loads-only assembly and the batched block PCG.

Each right-hand side of a batch must reach the same answer as its own FP64
solve (rel L2 <= 1e-6 at rtol 1e-8 against the oracle's direct solve), with
about the same iteration count as a single solve with the FP32 V-cycle; the
systems of a batch may have different meshes, sizes, element orders and
right-hand-side counts.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import fem, linsolve
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu


def _cases(pb, n_cases, seed):
    """Load cases on pb's mesh: seeded temperature fields and rotation speeds."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_cases):
        T = pb.T_ref + 50.0 * meshgen.fourier_temperature(pb.coords, seed + k, scale=np.ptp(pb.coords, 0) + 1e-9)
        w = rng.uniform(0.0, 2.0)
        body = w * w * np.stack([pb.coords[:, 0], pb.coords[:, 1], np.zeros(pb.n_nodes)], 1)
        out.append((T, body))
    return out


def _oracle_solution(pb, T, body):
    K, f = fem.assemble(pb.coords, pb.cells, pb.cell_material, pb.mat_props, T, pb.T_ref, body)
    K, f = fem.apply_dirichlet(K, f, pb.dirichlet_mask, pb.u_dirichlet)
    return linsolve.direct_solve(K, f)


def test_loads_only_assembly_matches_full_assembly():
    tam = need_gpu()
    pb = meshgen.slab_box_problem(12, 4, 4)
    rng = np.random.default_rng(2)
    pb.u_dirichlet = np.zeros((pb.n_nodes, 3))
    pb.u_dirichlet[pb.dirichlet_mask.astype(bool)] = 1e-3 * rng.standard_normal((int(pb.dirichlet_mask.sum()), 3))
    d = tam.problem_to_device(pb)
    K, _ = tam.fem_assemble_elasticity(**d)
    for T, body in _cases(pb, 2, 5):
        d2 = dict(d, T=torch.from_numpy(T).cuda(), body_force=torch.from_numpy(body).cuda())
        _, full = tam.fem_assemble_elasticity(**d2)
        only = tam.fem_assemble_load(K, **d2)
        assert torch.allclose(only, full, rtol=0, atol=1e-13 * float(full.abs().max()))


def _batch_inputs(tam, pb, n_cases, seed, precision=0, **prm):
    d = tam.problem_to_device(pb)
    K, _ = tam.fem_assemble_elasticity(**d)
    H = tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=precision, **prm))
    cases = _cases(pb, n_cases, seed)
    B = torch.stack([tam.fem_assemble_load(K, **dict(d, T=torch.from_numpy(T).cuda(),
                                                       body_force=torch.from_numpy(b).cuda())).reshape(-1)
                     for T, b in cases])
    return d, K, H, cases, B


def test_batch_of_load_cases_matches_single_solves():
    tam = need_gpu()
    pb = meshgen.slab_box_problem(32, 8, 8)
    d, K, H, cases, B = _batch_inputs(tam, pb, 5, 11)
    X = torch.zeros_like(B)
    its, rels, st = tam.amg_pcg_solve_batch([H], [B], [X], rtol=1e-8)
    assert st == 0 and all(r <= 1e-8 for r in rels)
    # the same cases one at a time with the FP32 V-cycle
    H32 = tam.amg_setup(K, d["coords"], tam.amg_params_default(level_precision=1))
    for k, (T, body) in enumerate(cases):
        x1 = torch.zeros(pb.n_nodes, 3, dtype=torch.float64, device="cuda")
        it1, _, _ = tam.amg_pcg_solve(H32, B[k].reshape(-1, 3).contiguous(), x1, rtol=1e-8)
        assert abs(its[k] - it1) <= 2, (k, its[k], it1)
        u = _oracle_solution(pb, T, body)
        assert np.linalg.norm(X[k].cpu().numpy() - u) <= 1e-6 * np.linalg.norm(u)
    tiles, tune_ms = tam.amg_batch_tiles(H)
    assert tiles and len(tiles) % 3 == 0 and tune_ms > 0
    for tm, threads, lpr in zip(tiles[0::3], tiles[1::3], tiles[2::3]):
        assert tm in (1, 2, 4, 8) and threads in (64, 128, 256) and lpr in (0, 1, 2, 4, 8, 16, 32)


def test_batch_of_uneven_meshes_in_one_graph():
    tam = need_gpu()
    problems = [(meshgen.slab_box_problem(24, 6, 6), 3, 0),
                (meshgen.unit_cube_problem(4, 2), 8, 2),
                (meshgen.bladed_disc_problem(n_r=6, n_theta_per_blade=4, n_z=2, n_blades=12, n_r_blade=3,
                                             degree=1), 2, 0)]
    sys = [_batch_inputs(tam, pb, m, 20 + i, prec) for i, (pb, m, prec) in enumerate(problems)]
    Xs = [torch.zeros_like(s[4]) for s in sys]
    its, rels, st = tam.amg_pcg_solve_batch([s[2] for s in sys], [s[4] for s in sys], Xs, rtol=1e-8)
    assert st == 0 and all(r <= 1e-8 for r in rels)
    k = 0
    for (pb, m, _), s, X in zip(problems, sys, Xs):
        for j in range(m):
            T, body = s[3][j]
            u = _oracle_solution(pb, T, body)
            assert np.linalg.norm(X[j].cpu().numpy() - u) <= 1e-6 * np.linalg.norm(u), (pb.name, j)
            k += 1


def test_batch_zero_load_and_iteration_cap():
    tam = need_gpu()
    pb = meshgen.slab_box_problem(16, 4, 4)
    # a coarsest level small enough that the preconditioner is not an exact solve
    d, K, H, cases, B = _batch_inputs(tam, pb, 3, 3, coarse_max_dofs=100)
    B[1].zero_()
    X = torch.zeros_like(B)
    its, rels, st = tam.amg_pcg_solve_batch([H], [B], [X], rtol=1e-8)
    assert st == 0 and its[1] == 0 and float(X[1].abs().max()) == 0.0
    X2 = torch.zeros_like(B)
    its, rels, st = tam.amg_pcg_solve_batch([H], [B], [X2], rtol=1e-14, max_iter=2, raise_on_error=False)
    assert st == -5 and max(its) == 2
