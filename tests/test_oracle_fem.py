"""Pins for the oracle's assembly (paper Sec. 3, Eqs. elasticity_bvp, u-dbc, wf_elastic).

Each check is fixed by the mathematics, not by the oracle itself: hand-derived
element matrices, the rigid-body kernel, symmetry, patch tests (exact linear /
quadratic / free-thermal-expansion solutions), load resultants and moments,
and manufactured-solution convergence rates (Sec. 2.1: error O(h^2) for P1).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, linsolve
from paper_1804_10060_gb300 import meshgen

UNIT_TET = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])


def _jittered_box(n, degree, seed=3, amount=0.2, two_mats=True):
    coords, cells = meshgen.box_kuhn(n, n, n)
    coords = meshgen.jitter_interior(coords, 1.0 / n, amount, seed)
    if degree == 2:
        coords, cells, _ = meshgen.p1_to_p2(coords, cells)
    xc = meshgen.cell_centroids(coords, cells)[:, 0]
    mat = (xc > 0.5).astype(np.int32) if two_mats else np.zeros(cells.shape[0], np.int32)
    props = np.array([[1.0, 0.3, 2e-3], [7.0, 0.21, 2e-3]])
    return coords, cells, mat, props


def _boundary_nodes(coords):
    lo, hi = coords.min(axis=0), coords.max(axis=0)
    return np.any(np.isclose(coords, lo) | np.isclose(coords, hi), axis=1)


@pytest.mark.parametrize("fname,E,nu", [("p1_unit_tet_nu0.txt", 1.0, 0.0),
                                        ("p1_unit_tet_lam1_mu1.txt", 2.5, 0.25)])
def test_single_p1_element_matches_hand_derivation(golden, fname, E, nu):
    Ke, _ = fem.element_matrices(UNIT_TET, np.array([[0, 1, 2, 3]]), np.array([0]),
                                 np.array([[E, nu, 0.0]]))
    np.testing.assert_allclose(Ke.reshape(12, 12), golden(fname), atol=1e-14)


def test_p2_mass_matrix_closed_form(golden):
    # body load of a unit body force in direction x on one P2 cell: f_a = sum_b M_ab
    X = UNIT_TET * np.array([2.0, 1.0, 0.5]) + np.array([0.3, -0.1, 0.7])
    coords, cells, _ = meshgen.p1_to_p2(X, np.array([[0, 1, 2, 3]]))
    vol = 2.0 * 1.0 * 0.5 / 6.0
    M = golden("p2_tet_mass_420.txt") * vol
    rng = np.random.default_rng(0)
    fb = rng.standard_normal((10, 3))
    _, fe = fem.element_matrices(coords, cells, np.array([0]), np.array([[1.0, 0.3, 0.0]]),
                                 body_force=fb)
    np.testing.assert_allclose(fe[0], M @ fb, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("degree", [1, 2])
def test_rigid_body_modes_in_kernel_and_symmetry(degree):
    coords, cells, mat, props = _jittered_box(3, degree)
    K, _ = fem.assemble(coords, cells, mat, props)
    B = fem.rigid_body_modes(coords)
    kn = abs(K).max()
    for k in range(6):
        assert np.abs(K @ B[:, k]).max() <= 1e-12 * kn * np.abs(B[:, k]).max()
    assert abs(K - K.T).max() <= 1e-14 * kn
    # positive definite once one face is clamped
    mask = coords[:, 0] <= 1e-12
    Kd, _ = fem.apply_dirichlet(K, np.zeros(K.shape[0]), mask)
    assert np.linalg.eigvalsh(Kd.toarray()).min() > 0


@pytest.mark.parametrize("degree", [1, 2])
def test_linear_patch_test(degree):
    # one material: a linear field has constant stress, hence no interface traction jump
    coords, cells, mat, props = _jittered_box(3, degree, two_mats=False)
    rng = np.random.default_rng(11)
    G, c = rng.standard_normal((3, 3)), rng.standard_normal(3)
    u_exact = coords @ G.T + c
    bnd = _boundary_nodes(coords)
    K, f = fem.assemble(coords, cells, mat, props)
    Kd, fd = fem.apply_dirichlet(K, f, bnd, u_exact)
    u = linsolve.direct_solve(Kd, fd).reshape(-1, 3)
    assert (~bnd).sum() > 0
    err = np.abs(u - u_exact).max() / np.abs(u_exact).max()
    assert err < 1e-10


def test_quadratic_patch_test_p2():
    # u quadratic -> sigma linear -> f = -div sigma constant; P2 reproduces u exactly.
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    E, nu = 3.0, 0.27
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    U = [x * x + 2 * y * z - z * z, x * y - 3 * z * z + x * z, y * y - x * z + 2 * x * x]
    X = [x, y, z]
    eps = [[(sympy.diff(U[i], X[j]) + sympy.diff(U[j], X[i])) / 2 for j in range(3)] for i in range(3)]
    tr = eps[0][0] + eps[1][1] + eps[2][2]
    sig = [[2 * mu * eps[i][j] + (lam * tr if i == j else 0) for j in range(3)] for i in range(3)]
    fvec = [-sum(sympy.diff(sig[i][j], X[j]) for j in range(3)) for i in range(3)]
    fconst = np.array([float(v) for v in fvec])
    coords, cells, _, _ = _jittered_box(2, 2, two_mats=False)
    ufun = sympy.lambdify((x, y, z), U, "numpy")
    u_exact = np.stack([np.broadcast_to(v, coords.shape[0]) for v in ufun(*coords.T)], axis=1)
    body = np.tile(fconst, (coords.shape[0], 1))
    K, f = fem.assemble(coords, cells, np.zeros(cells.shape[0], np.int32),
                        np.array([[E, nu, 0.0]]), body_force=body)
    bnd = _boundary_nodes(coords)
    Kd, fd = fem.apply_dirichlet(K, f, bnd, u_exact)
    u = linsolve.direct_solve(Kd, fd).reshape(-1, 3)
    assert np.abs(u - u_exact).max() / np.abs(u_exact).max() < 1e-10


@pytest.mark.parametrize("degree", [1, 2])
def test_free_thermal_expansion_is_stress_free(degree):
    # uniform alpha, uniform dT, any E field: u = alpha dT (x - x0) is exact.
    coords, cells, mat, props = _jittered_box(3, degree)
    T_ref, dT, x0 = 250.0, 40.0, np.array([0.2, 0.5, -0.1])
    T = np.full(coords.shape[0], T_ref + dT)
    alpha = props[0, 2]
    u_exact = alpha * dT * (coords - x0)
    K, f = fem.assemble(coords, cells, mat, props, T=T, T_ref=T_ref)
    bnd = _boundary_nodes(coords)
    Kd, fd = fem.apply_dirichlet(K, f, bnd, u_exact)
    u = linsolve.direct_solve(Kd, fd).reshape(-1, 3)
    assert np.abs(u - u_exact).max() / np.abs(u_exact).max() < 1e-10
    # the full (unconstrained) residual of the exact field vanishes: K u = f_T
    r = K @ u_exact.ravel() - f
    assert np.abs(r).max() < 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("degree", [1, 2])
def test_body_load_resultant_and_moment(degree):
    # f linear in x is reproduced by the nodal interpolant, so
    # sum_a f_a = int f dx and sum_a x_a x f_a = int x x f dx (both closed forms on a box).
    L = np.array([2.0, 1.0, 0.5])
    coords, cells = meshgen.box_kuhn(4, 3, 2, *L)
    if degree == 2:
        coords, cells, _ = meshgen.p1_to_p2(coords, cells)
    c0 = np.array([0.5, -1.0, 2.0])
    Gf = np.array([[1.0, 2.0, 0.0], [0.0, -1.0, 3.0], [0.5, 0.0, 1.0]])
    body = c0 + coords @ Gf.T
    _, f = fem.assemble(coords, cells, np.zeros(cells.shape[0], np.int32),
                        np.array([[1.0, 0.3, 0.0]]), body_force=body)
    f = f.reshape(-1, 3)
    vol = L.prod()
    m1 = vol * L / 2.0                                   # int x_i
    m2 = np.outer(m1, m1) / vol                          # int x_i x_j (i != j)
    np.fill_diagonal(m2, vol * L ** 2 / 3.0)
    F = vol * c0 + Gf @ m1
    np.testing.assert_allclose(f.sum(axis=0), F, rtol=1e-12)
    # int x cross f: (x cross f)_k = eps_kij x_i f_j, f_j = c0_j + G_jl x_l
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    Mom = np.einsum("kij,i,j->k", eps, m1, c0) + np.einsum("kij,jl,il->k", eps, Gf, m2)
    np.testing.assert_allclose(np.cross(coords, f).sum(axis=0), Mom, rtol=1e-12, atol=1e-12)


def _manufactured(degree, n):
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    E, nu, alpha, T_ref = 2.0, 0.3, 0.05, 1.0
    lam, mu = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    U = [sympy.sin(x + 2 * y) * sympy.cos(z), sympy.exp(x * z) * y, x * y * z + sympy.sin(3 * y)]
    T = 1.0 + sympy.cos(x) * sympy.exp(y) * (1 + z * z)
    X = [x, y, z]
    eps = [[(sympy.diff(U[i], X[j]) + sympy.diff(U[j], X[i])) / 2 for j in range(3)] for i in range(3)]
    tr = eps[0][0] + eps[1][1] + eps[2][2]
    sT = (3 * lam + 2 * mu) * alpha * (T - T_ref)
    sig = [[2 * mu * eps[i][j] + ((lam * tr - sT) if i == j else 0) for j in range(3)] for i in range(3)]
    fvec = [-sum(sympy.diff(sig[i][j], X[j]) for j in range(3)) for i in range(3)]
    coords, cells = meshgen.box_kuhn(n, n, n)
    if degree == 2:
        coords, cells, _ = meshgen.p1_to_p2(coords, cells)
    uf = sympy.lambdify((x, y, z), U, "numpy")
    ff = sympy.lambdify((x, y, z), fvec, "numpy")
    Tf = sympy.lambdify((x, y, z), T, "numpy")
    bc = lambda fn: np.stack([np.broadcast_to(v, coords.shape[0]) for v in fn(*coords.T)], axis=1)
    u_ex, body = bc(uf), bc(ff)
    Tn = np.broadcast_to(Tf(*coords.T), coords.shape[0]).astype(float)
    K, f = fem.assemble(coords, cells, np.zeros(cells.shape[0], np.int32),
                        np.array([[E, nu, alpha]]), T=Tn, T_ref=T_ref, body_force=body)
    bnd = _boundary_nodes(coords)
    Kd, fd = fem.apply_dirichlet(K, f, bnd, u_ex)
    u = linsolve.direct_solve(Kd, fd).reshape(-1, 3)
    return np.sqrt(np.mean((u - u_ex) ** 2))


@pytest.mark.parametrize("degree,ns,min_rate", [(1, (4, 8, 16), 1.8), (2, (2, 4, 8), 2.8)])
def test_manufactured_solution_convergence_rate(degree, ns, min_rate):
    errs = [_manufactured(degree, n) for n in ns]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] >= min_rate, (errs, rates)


def test_dirichlet_elimination_keeps_solution_and_symmetry():
    coords, cells, mat, props = _jittered_box(3, 1)
    T = meshgen.fourier_temperature(coords, 5, scale=(1, 1, 1))
    K, f = fem.assemble(coords, cells, mat, props, T=T)
    mask = coords[:, 0] <= 1e-12
    ud = np.zeros((coords.shape[0], 3))
    ud[mask] = [0.01, -0.02, 0.03]
    Kd, fd = fem.apply_dirichlet(K, f, mask, ud)
    assert abs(Kd - Kd.T).max() <= 1e-14 * abs(Kd).max()
    u = linsolve.dense_solve(Kd, fd)
    # same solution from the unsymmetric row-replacement form of the constraints
    dm = np.repeat(mask, 3)
    Kr = K.tolil()
    fr = f.copy()
    for r in np.nonzero(dm)[0]:
        Kr.rows[r] = [r]
        Kr.data[r] = [1.0]
        fr[r] = ud.ravel()[r]
    u2 = linsolve.direct_solve(sp.csr_matrix(Kr), fr)
    np.testing.assert_allclose(u, u2, rtol=1e-10, atol=1e-14)


def test_solvers_agree_on_unit_cube_config():
    pb = meshgen.unit_cube_problem(6)
    K, f = fem.assemble_system(pb)
    u_d = linsolve.dense_solve(K, f)
    u_s = linsolve.direct_solve(K, f)
    u_j, _ = linsolve.jacobi_pcg(K, f, rtol=1e-13)
    nrm = np.linalg.norm(u_d)
    assert np.linalg.norm(u_s - u_d) / nrm < 1e-12
    assert np.linalg.norm(u_j - u_d) / nrm < 1e-10


def test_planted_transposition_fails_the_patch_test(monkeypatch):
    """A plausible mistake (swapping the two shear strain terms) must be caught."""
    orig = fem.voigt_selector

    def wrong():
        B = orig()
        B[5] = 0.0
        B[5, 0, 0] = B[5, 1, 1] = 1.0   # 2 eps_xy taken as d_x u_x + d_y u_y
        return B

    monkeypatch.setattr(fem, "voigt_selector", wrong)
    coords, cells, mat, props = _jittered_box(2, 1)
    rng = np.random.default_rng(11)
    u_exact = coords @ rng.standard_normal((3, 3)).T
    K, f = fem.assemble(coords, cells, mat, props)
    bnd = _boundary_nodes(coords)
    Kd, fd = fem.apply_dirichlet(K, f, bnd, u_exact)
    u = np.linalg.lstsq(Kd.toarray(), fd, rcond=None)[0].reshape(-1, 3)
    assert np.abs(u - u_exact).max() / np.abs(u_exact).max() > 1e-6
