"""GPU assembly and SpMV vs the CPU oracle (paper Sec. 3, Eqs. wf_elastic, u-dbc).

K and f from the CUDA path are compared entry by entry with the oracle's
exact-integral assembly on the same seeded inputs (P1 and P2, several
materials, thermal and body loads, nonzero Dirichlet data), at sizes that
span many SELL slices with a ragged last slice; at the full 256x64x64 box
size, sampled block rows are compared with an oracle assembly of their
incident cells.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import bsr_to_csr, exact_spmv, need_gpu, sparse_rel, torch
from oracle import fem
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12  # FP64 assembly: only summation order differs


def _rich_problem(n, degree, seed=5):
    coords, cells = meshgen.box_kuhn(n + 1, n, n - 1, 1.3, 1.0, 0.8)
    coords = meshgen.jitter_interior(coords, 0.8 / n, 0.15, seed)
    if degree == 2:
        coords, cells, _ = meshgen.p1_to_p2(coords, cells)
        coords, cells, _ = meshgen.renumber_nodes(coords, cells, meshgen.spatial_order(coords, 0.8 / n))
    rng = np.random.default_rng(seed)
    xc = meshgen.cell_centroids(coords, cells)
    mat = ((xc[:, 0] > 0.6).astype(np.int32) + (xc[:, 2] > 0.4).astype(np.int32)).astype(np.int32)
    props = np.array([[1.0, 0.3, 1e-3], [10.0, 0.25, 2e-3], [3.0, 0.35, 5e-4]])
    T = meshgen.fourier_temperature(coords, seed, scale=(1.3, 1.0, 0.8)) * 50 + 300
    body = rng.standard_normal((coords.shape[0], 3))
    mask = (coords[:, 0] <= 1e-12) | (coords[:, 2] >= 0.8 - 1e-12)
    ud = np.zeros_like(coords)
    ud[mask] = 1e-3 * rng.standard_normal((mask.sum(), 3))
    return meshgen.Problem("rich", coords, cells, mat, props, T, 290.0, body, mask.astype(np.uint8), ud)


@pytest.mark.parametrize("degree,n", [(1, 7), (2, 4)])
def test_assembly_matches_oracle(degree, n):
    tam = need_gpu()
    pb = _rich_problem(n, degree)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    Kg = bsr_to_csr(rp, ci, v, pb.n_nodes)
    Ko, fo = fem.assemble_system(pb)
    assert Kg.shape == Ko.shape
    assert sparse_rel(Kg, Ko) <= TOL
    f = rhs.cpu().numpy().ravel()
    assert np.abs(f - fo).max() <= TOL * np.abs(fo).max()
    # pattern: sorted columns, diagonal present, no Dirichlet couplings
    rpn, cin = rp.cpu().numpy(), ci.cpu().numpy()
    for i in range(pb.n_nodes):
        row = cin[rpn[i]:rpn[i + 1]]
        assert np.all(np.diff(row) > 0) and i in row
        if pb.dirichlet_mask[i]:
            assert row.tolist() == [i]
        else:
            assert not np.any(pb.dirichlet_mask[row[row != i]])


# Per-row bound of the outer double-float SpMV: |y_i - (K x)_i| <= 1e-14 sum_j |K_ij x_j|.
# Each product's operands are split to within 2^-49 relative (round to
# nearest), every partial product including lo*lo is kept, and the FP32
# rounding of the cross terms and of the low part (restarted every two slots,
# its sum added in FP64) adds a few 2^-48 of the magnitudes involved; the
# errors are unbiased, so a row's total, measured against the sum of the
# magnitudes of its terms (which absorbs cancellation), stays below 1e-14
# (about 2.8 * 2^-48).
SPMV_ROW_TOL = 1e-14


@pytest.mark.parametrize("degree", [1, 2])
def test_spmv_matches_exact_products(degree):
    tam = need_gpu()
    pb = _rich_problem(6 if degree == 1 else 3, degree)
    d = tam.problem_to_device(pb)
    K, _ = tam.fem_assemble_elasticity(**d)
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    Kg = bsr_to_csr(rp, ci, v, pb.n_nodes)
    xs = np.random.default_rng(21 + degree).standard_normal((pb.n_nodes, 3))
    x = torch.from_numpy(xs).cuda()
    y = tam.tam_matrix_spmv(K, x).cpu().numpy().ravel()
    y_ex, s = exact_spmv(Kg, xs.ravel())
    err = np.abs(y - y_ex)
    assert np.all(err <= SPMV_ROW_TOL * s), (err / np.maximum(s, 1e-300)).max()


def test_degenerate_cell_is_reported():
    tam = need_gpu()
    pb = meshgen.unit_cube_problem(3)
    pb.cells = pb.cells.copy()
    pb.cells[5] = pb.cells[5][[0, 2, 1, 3]]  # inverted orientation -> negative volume
    d = tam.problem_to_device(pb)
    with pytest.raises(tam.TamError) as e:
        tam.fem_assemble_elasticity(**d)
    assert e.value.code == -4


def test_out_of_range_node_is_rejected():
    tam = need_gpu()
    pb = meshgen.unit_cube_problem(3)
    pb.cells = pb.cells.copy()
    pb.cells[0, 0] = pb.n_nodes
    d = tam.problem_to_device(pb)
    with pytest.raises(tam.TamError) as e:
        tam.fem_assemble_elasticity(**d)
    assert e.value.code == -1


def test_full_size_box_sampled_rows():
    """256x64x64 two-material box (3,257,475 DOF): sampled block rows vs the oracle."""
    tam = need_gpu()
    pb = meshgen.slab_box_problem()
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    n, nnzb, _ = K.info()
    assert n == 1_085_825 and nnzb <= 15_987_841
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    rpn, cin = rp.cpu().numpy(), ci.cpu().numpy()
    rng = np.random.default_rng(0)
    nodes = np.unique(np.concatenate([rng.integers(0, n, 300), [0, n - 1, 257 * 65 * 32 + 128]]))
    # cells incident to the sampled nodes
    hit = np.isin(pb.cells, nodes).any(axis=1)
    sub = pb.cells[hit]
    Ko, fo = fem.assemble(pb.coords, sub, pb.cell_material[hit], pb.mat_props, pb.T, pb.T_ref)
    Ko, fo = fem.apply_dirichlet(Ko, fo, pb.dirichlet_mask)
    vals = v.cpu().numpy()
    f = rhs.cpu().numpy()
    for i in nodes:
        blocks = {int(c): vals[p] for p, c in zip(range(rpn[i], rpn[i + 1]), cin[rpn[i]:rpn[i + 1]])}
        for r in range(3):
            row = Ko.getrow(3 * i + r)
            ref = dict(zip(row.indices, row.data))
            scale = max(abs(row.data).max(), 1e-300)
            for c, blk in blocks.items():
                for cc in range(3):
                    assert abs(blk[r, cc] - ref.get(3 * c + cc, 0.0)) <= TOL * scale
            assert set(int(c) // 3 for c, val in zip(row.indices, row.data) if val != 0) <= set(blocks)
            assert abs(f[i, r] - fo[3 * i + r]) <= TOL * max(np.abs(fo).max(), 1e-300)


def test_residual_norm_entry_point():
    tam = need_gpu()
    pb = _rich_problem(6, 1)
    d = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**d)
    rp, ci, v = tam.tam_matrix_export_bsr(K)
    Kg = bsr_to_csr(rp, ci, v, pb.n_nodes)
    x = torch.randn(pb.n_nodes, 3, dtype=torch.float64, device="cuda")
    got = tam.tam_matrix_residual_norm(K, rhs, x)
    ref = np.linalg.norm(rhs.cpu().numpy().ravel() - Kg @ x.cpu().numpy().ravel())
    assert abs(got - ref) <= 1e-12 * ref


@pytest.mark.parametrize("degree", [1, 2])
def test_deterministic_assembly_is_bitwise_reproducible(degree):
    """tam_set_deterministic_assembly(1): per-node sums of the element slots in
    cell order -- two runs bitwise equal (K and f, loads-only path included),
    the same operator as the atomic scatter to rounding and the oracle's to 1e-12;
    prescribed displacements exercise the lifting."""
    tam = need_gpu()
    pb = meshgen.slab_box_problem(12, 4, 4) if degree == 1 else meshgen.unit_cube_problem(4, 2)
    rng = np.random.default_rng(9)
    pb.u_dirichlet = 1e-3 * rng.standard_normal((pb.n_nodes, 3)) * pb.dirichlet_mask[:, None]
    d = tam.problem_to_device(pb)
    prev = tam.set_deterministic_assembly(True)
    try:
        runs = []
        for _ in range(2):
            K, rhs = tam.fem_assemble_elasticity(**d)
            rp, ci, v = tam.tam_matrix_export_bsr(K)
            b2 = tam.fem_assemble_load(K, **d)
            runs.append((rp.cpu().numpy(), ci.cpu().numpy(), v.cpu().numpy(), rhs.cpu().numpy(), b2.cpu().numpy()))
    finally:
        tam.set_deterministic_assembly(prev)
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
    K0, rhs0 = tam.fem_assemble_elasticity(**d)
    rp0, ci0, v0 = tam.tam_matrix_export_bsr(K0)
    assert np.array_equal(rp0.cpu().numpy(), runs[0][0]) and np.array_equal(ci0.cpu().numpy(), runs[0][1])
    scale = np.abs(runs[0][2]).max()
    assert np.abs(v0.cpu().numpy() - runs[0][2]).max() <= 1e-13 * scale
    fs = np.abs(runs[0][3]).max()
    assert np.abs(rhs0.cpu().numpy() - runs[0][3]).max() <= 1e-13 * fs
    assert np.abs(runs[0][4] - runs[0][3]).max() <= 1e-13 * fs
    Ko, fo = fem.assemble_system(pb)
    assert sparse_rel(bsr_to_csr(*[torch.from_numpy(x) for x in runs[0][:3]], pb.n_nodes), Ko) <= 1e-12
    assert np.abs(runs[0][3].ravel() - fo).max() <= 1e-12 * np.abs(fo).max()
