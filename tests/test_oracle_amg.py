"""Pins for the oracle's smoothed-aggregation AMG-PCG (paper Sec. 2.1, Sec. 5.1).

Fixed by mathematics rather than by the oracle: SplitMix64 published outputs,
distance-2 independence and maximality of the aggregate roots, the exact range
property of the tentative prolongator, orthonormality, Galerkin product vs a
dense triple product, the Chebyshev error polynomial vs its closed form, the
Ritz bound on lambda_max, symmetry and positivity of the V-cycle, and the
paper's claim that omitting the rotational near-nullspace modes makes
iteration counts grow under refinement.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg, fem, linsolve
from paper_1804_10060_gb300 import meshgen


def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0 emits mix(g), mix(2g), mix(3g) with g = 0x9E3779B97F4A7C15.
    g = 0x9E3779B97F4A7C15
    assert amg.splitmix64(0) == 0xE220A8397B1DCDAF
    assert amg.splitmix64(g) == 0x6E789E6AA1B965F4
    assert amg.splitmix64(2 * g % (1 << 64)) == 0x06C45D188009454F
    arr = amg.splitmix64(np.array([0, g], dtype=np.uint64))
    assert int(arr[0]) == 0xE220A8397B1DCDAF and int(arr[1]) == 0x6E789E6AA1B965F4


def _cube_system(n=4, degree=1, twist=False):
    pb = meshgen.unit_cube_problem(n, degree)
    K, f = fem.assemble(pb.coords, pb.cells, pb.cell_material, pb.mat_props, pb.T, pb.T_ref)
    mask = pb.dirichlet_mask.astype(bool)
    ud = None
    if twist:
        far = pb.coords[:, 0] >= 1 - 1e-12
        mask = mask | far
        c = np.array([1.0, 0.5, 0.5])
        ud = np.zeros_like(pb.coords)
        d = pb.coords[far] - c
        ud[far] = 0.01 * np.stack([np.zeros(d.shape[0]), -d[:, 2], d[:, 1]], axis=1)
        f = np.zeros_like(f)
    Kd, fd = fem.apply_dirichlet(K, f, mask, ud)
    return pb, Kd, fd, mask


def _three_node_matrix():
    """Hand-built 3-node matrix of 3x3 blocks for the strength pin.

    Diagonal blocks 4I, 9I, I have Frobenius norms 4 sqrt3, 9 sqrt3, sqrt3, so
    sqrt(||A_ii|| ||A_jj||) is sqrt(108) = 10.392 for (0,1), sqrt(12) = 3.464
    for (0,2) and sqrt(27) = 5.196 for (1,2).  The off-diagonal blocks are
    constant blocks -0.1, 0.05 and 0.09 with Frobenius norms 0.3, 0.15 and
    0.27 (their largest entries, 0.1, 0.05 and 0.09, and their traces give
    other answers, as do the norms without the square root or squared).
    """
    A = np.zeros((9, 9))
    for i, d in enumerate((4.0, 9.0, 1.0)):
        A[3 * i:3 * i + 3, 3 * i:3 * i + 3] = d * np.eye(3)
    for (i, j), v in {(0, 1): -0.1, (0, 2): 0.05, (1, 2): 0.09}.items():
        A[3 * i:3 * i + 3, 3 * j:3 * j + 3] = v
        A[3 * j:3 * j + 3, 3 * i:3 * i + 3] = v
    return sp.csr_matrix(A)


@pytest.mark.parametrize("theta,expected", [
    # thresholds theta * sqrt(||A_ii|| ||A_jj||), hand-computed:
    #   theta = 0.02: (0,1) 0.2078, (0,2) 0.0693, (1,2) 0.1039 -> all three couplings strong
    #   theta = 0.05: (0,1) 0.5196 > 0.3, (0,2) 0.1732 > 0.15 weak; (1,2) 0.2598 < 0.27 strong
    (0.0, [[1, 2], [0, 2], [0, 1]]),
    (0.02, [[1, 2], [0, 2], [0, 1]]),
    (0.05, [[], [2], [1]]),
    (0.1, [[], [], []]),
])
def test_strength_graph_threshold_hand_computed(theta, expected):
    """Sec. 5.1 leaves the coupling threshold to the user; the strength rule
    ||A_ij||_F >= theta sqrt(||A_ii||_F ||A_jj||_F) on a 3-node matrix whose
    block norms straddle the thresholds."""
    nbrs = amg.strength_graph(_three_node_matrix(), 3, theta)
    assert [sorted(int(j) for j in nb) for nb in nbrs] == expected


def test_mis2_roots_independent_maximal_and_greedy():
    pb, K, f, mask = _cube_system(5)
    nbrs = amg.strength_graph(K, 3)
    agg, n_agg, roots = amg.mis2_aggregate(nbrs, 0)
    assert amg.check_aggregates(agg, n_agg, nbrs) == []
    n = len(nbrs)
    # Dirichlet nodes have no strong neighbour after elimination
    assert all(len(nbrs[i]) == 0 for i in np.nonzero(mask)[0])
    dist2 = [set() for _ in range(n)]
    for i in range(n):
        for j in nbrs[i]:
            dist2[i].add(int(j))
            dist2[i].update(int(k) for k in nbrs[j])
        dist2[i].discard(i)
    rs = set(int(r) for r in roots)
    prio = amg.node_priority(n, 0)
    key = lambda i: (int(prio[i]), i)
    for i in range(n):
        if not nbrs[i].size:
            continue
        near_roots = dist2[i] & rs
        if i in rs:
            assert not near_roots                      # distance-2 independent
            assert agg[i] == sorted(rs).index(i)       # numbered by increasing root id
        else:
            assert near_roots                          # maximal
            # greedy fixed point: some root within distance 2 outranks i
            assert max(key(r) for r in near_roots) > key(i)


def test_tentative_prolongator_exact_range_and_orthonormal():
    pb, K, f, mask = _cube_system(4)
    B = fem.rigid_body_modes(pb.coords, mask)
    nbrs = amg.strength_graph(K, 3)
    agg, n_agg, _ = amg.mis2_aggregate(nbrs, 0)
    P, Bc = amg.tentative_prolongator(agg, n_agg, B, 3)
    rows = np.repeat(agg >= 0, 3)
    np.testing.assert_allclose((P @ Bc)[rows], B[rows], atol=1e-13)
    assert np.abs((P @ Bc)[~rows]).max() == 0
    np.testing.assert_allclose((P.T @ P).toarray(), np.eye(6 * n_agg), atol=1e-13)
    for a in range(n_agg):
        R = Bc[6 * a:6 * a + 6]
        assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)


def test_rank_deficient_aggregate_drops_columns():
    # 2 nodes: translations + 1 rotation about their axis are zero on the line -> rank 5
    coords = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    B = fem.rigid_body_modes(coords)
    P, Bc = amg.tentative_prolongator(np.array([0, 0]), 1, B, 3)
    d = np.diag(Bc)
    assert (d == 0).sum() == 1 and np.all(d[d != 0] > 0)
    np.testing.assert_allclose(P @ Bc, B, atol=1e-13)
    Q = P.toarray()
    np.testing.assert_allclose(Q.T @ Q, np.diag((d != 0).astype(float)), atol=1e-13)


def test_galerkin_product_matches_dense_triple_product():
    pb, K, f, mask = _cube_system(4)
    H = amg.setup(K, fem.rigid_body_modes(pb.coords, mask), 3, coarse_max_dofs=50)
    L0, L1 = H.levels[0], H.levels[1]
    Pd, Ad = L0.P.toarray(), L0.A.toarray()
    np.testing.assert_allclose(L1.A.toarray(), Pd.T @ Ad @ Pd, atol=1e-13 * np.abs(Ad).max())
    Ac = L1.A.toarray()
    assert np.abs(Ac - Ac.T).max() <= 1e-13 * np.abs(Ac).max()
    # P = (I - 4/(3 lam) D^-1 A) P_tent, written with dense arrays
    Pt, _ = amg.tentative_prolongator(L0.agg, L0.n_agg, fem.rigid_body_modes(pb.coords, mask), 3)
    Dinv = np.diag(np.where(np.diag(Ad) != 0, 1 / np.diag(Ad), 0))
    P2 = (np.eye(Ad.shape[0]) - 4 / (3 * L0.lam) * Dinv @ Ad) @ Pt.toarray()
    np.testing.assert_allclose(Pd, P2, atol=1e-13)


def test_chebyshev_error_polynomial_closed_form():
    rng = np.random.default_rng(4)
    n = 40
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    dinv = 1.0 / np.diag(A)
    s = np.sqrt(dinv)
    lam_all, V = np.linalg.eigh(s[:, None] * A * s[None, :])
    lo, hi = 0.3 * lam_all[-1], 1.05 * lam_all[-1]
    theta, delta = (hi + lo) / 2, (hi - lo) / 2
    T = {1: lambda t: t, 2: lambda t: 2 * t * t - 1, 3: lambda t: 4 * t ** 3 - 3 * t}
    e0 = rng.standard_normal(n)
    for k in (1, 2, 3):
        # f = 0, exact solution 0: the iterate is the propagated error
        e = amg.chebyshev(sp.csr_matrix(A), dinv, np.zeros(n), e0, lo, hi, k)
        w0 = V.T @ (e0 / s)             # components of D^1/2 e in the eigenbasis
        g = T[k]((theta - lam_all) / delta) / T[k](theta / delta)
        expect = (V @ (g * w0)) * s
        np.testing.assert_allclose(e, expect, atol=1e-12 * np.abs(e0).max())


def test_lanczos_estimate_is_a_tight_lower_bound():
    pb, K, f, mask = _cube_system(5)
    d = K.diagonal()
    s = 1 / np.sqrt(d)
    lam_true = np.linalg.eigvalsh((s[:, None] * K.toarray() * s[None, :]))[-1]
    lam = amg.lanczos_lambda_max(K, 10, 0)
    assert lam <= lam_true * (1 + 1e-12)
    assert lam >= 0.85 * lam_true


def test_vcycle_is_symmetric_positive_definite():
    pb, K, f, mask = _cube_system(4)
    H = amg.setup(K, fem.rigid_body_modes(pb.coords, mask), 3, coarse_max_dofs=10)
    assert len(H.levels) >= 3
    n = K.shape[0]
    M = np.stack([amg.vcycle(H, e) for e in np.eye(n)], axis=1)
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() > 0
    # the preconditioned operator is well conditioned
    Kd = K.toarray()
    ew = np.sort(np.real(np.linalg.eigvals(M @ Kd)))
    assert ew[0] > 0 and ew[-1] / ew[0] < 50


@pytest.mark.parametrize("degree", [1, 2])
def test_amg_pcg_matches_direct_solve(degree):
    pb, K, f, mask = _cube_system(5 if degree == 1 else 3, degree)
    u = linsolve.direct_solve(K, f)
    x, it, rel, H = amg.solve(K, f, pb.coords, mask, rtol=1e-10, coarse_max_dofs=100)
    assert rel <= 1e-10
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-7
    assert it < 40


def test_rotational_modes_keep_iterations_flat_under_refinement():
    """Sec. 2.1: without the full rigid-body near-nullspace the iteration count
    grows with refinement, most visibly when the load induces rotation."""
    its6, its3 = [], []
    for n in (4, 8, 16):
        pb, K, f, mask = _cube_system(n, twist=True)
        _, it6, _, _ = amg.solve(K, f, pb.coords, mask, rotations=True, rtol=1e-8, coarse_max_dofs=200,
                                 small_level_dofs=0)
        _, it3, _, _ = amg.solve(K, f, pb.coords, mask, rotations=False, rtol=1e-8, coarse_max_dofs=200,
                                 small_level_dofs=0)
        its6.append(it6)
        its3.append(it3)
    assert its6[-1] <= 1.5 * its6[0] + 2, its6
    assert its3[-1] / its3[0] > its6[-1] / its6[0], (its3, its6)
    assert its3[-1] > its6[-1], (its3, its6)
