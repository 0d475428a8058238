"""Pins for the oracle's thermal problem (paper Sec. 3, Eq. wf_thermal, Eq. dt_spec).

Fixed by mathematics rather than by the oracle: a linear steady field that
the discrete problem must reproduce exactly (patch test with Robin faces and
with the theta-method's mass term), the Kirchhoff transform of the nonlinear
steady equation (kappa = k0 + k1 T: u = k0 T + k1 T^2 / 2 is harmonic) giving
a manufactured solution without a source term, the closed-form decay of a
sine mode under the theta-method (time order 1 for backward Euler, 2 for
Crank-Nicolson), the Jacobian against central differences of F, the Robin
face integrals of a single face by hand, and Eq. dt_spec's arithmetic.
"""
import numpy as np
import pytest

from oracle import thermal as oth
from paper_1804_10060_gb300 import meshgen


def _cube(n, degree=1, jitter=0.0, seed=3):
    coords, cells = meshgen.box_kuhn(n, n, n)
    if jitter:
        coords = meshgen.jitter_interior(coords, 1.0 / n, jitter, seed)
    if degree == 2:
        coords, cells, _ = meshgen.p1_to_p2(coords, cells)
    return coords, cells


def _tp(coords, cells, props, faces=None, beta=None, T_bc=None, mask=None, Td=None):
    n = coords.shape[0]
    if faces is None:
        faces = np.zeros((0, 3 if cells.shape[1] == 4 else 6), np.int32)
        beta = np.zeros(0)
    return meshgen.ThermalProblem(coords, cells, np.zeros(cells.shape[0], np.int32), np.asarray(props, float),
                                  faces, np.asarray(beta, float), np.zeros(n) if T_bc is None else T_bc, mask, Td)


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("transient", [False, True])
def test_linear_steady_field_is_reproduced_exactly(degree, transient):
    """T = 300 + 40 x on the jittered unit cube, Robin on x = 0 and x = 1
    (beta = -2, T_bc = T -+ kappa a / beta so that kappa dT/dn = beta (T - T_bc)),
    the other faces adiabatic: the discrete solution is T itself."""
    coords, cells = _cube(3, degree, jitter=0.2)
    kappa, a = 0.7, 40.0
    faces = meshgen.boundary_faces(cells)
    fx = coords[faces[:, :3], 0]
    on0, on1 = np.all(fx < 1e-12, axis=1), np.all(fx > 1 - 1e-12, axis=1)
    rob = faces[on0 | on1]
    beta = np.full(rob.shape[0], -2.0)
    T_lin = 300.0 + a * coords[:, 0]
    T_bc = T_lin.copy()
    x = coords[:, 0]
    T_bc[x < 1e-12] += kappa * a / -2.0          # n = -x:  -kappa a = beta (T - T_bc)
    T_bc[x > 1 - 1e-12] -= kappa * a / -2.0      # n = +x:   kappa a = beta (T - T_bc)
    tp = _tp(coords, cells, [[1.3, 0.9, 0.0, kappa, 0.0]], rob, beta, T_bc)
    kw = dict(T_old=T_lin, dt=0.05, theta=0.5) if transient else {}
    F, _ = oth.assemble_thermal(tp, T_lin, **kw)
    assert np.abs(F).max() <= 1e-11 * np.abs(T_lin).max()
    T, it, _ = oth.newton(tp, np.full(coords.shape[0], 400.0), **kw)
    assert np.abs(T - T_lin).max() <= 1e-9 * T_lin.max()


def _kirchhoff_error(degree, n, k0=1.0, k1=0.02):
    """Steady -div((k0 + k1 T) grad T) = 0 with u = k0 T + k1 T^2 / 2 = 5 + x^2 - y^2 + xz
    (harmonic), Dirichlet T on the whole boundary; RMS nodal error."""
    coords, cells = _cube(n, degree)
    x, y, z = coords.T
    u = 5.0 + x * x - y * y + x * z
    T_ex = (-k0 + np.sqrt(k0 * k0 + 2.0 * k1 * u)) / k1
    bnd = np.any((coords <= 1e-12) | (coords >= 1 - 1e-12), axis=1)
    tp = _tp(coords, cells, [[1.0, 1.0, 0.0, k0, k1]], mask=bnd.astype(np.uint8), Td=T_ex)
    T, it, hist = oth.newton(tp, np.full(coords.shape[0], 4.0))
    assert hist[-1] <= 1e-9 * hist[0]
    return np.sqrt(np.mean((T - T_ex) ** 2))


@pytest.mark.parametrize("degree,ns,min_rate", [(1, (4, 8, 16), 1.8), (2, (2, 4, 8), 2.8)])
def test_nonlinear_manufactured_solution_convergence_rate(degree, ns, min_rate):
    errs = [_kirchhoff_error(degree, n) for n in ns]
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert rates[-1] >= min_rate, (errs, rates)


def _decay_error(dt, theta, n=3, t_end=0.2):
    """rho c dT/dt = kappa T_xx, T = 300 + exp(-kappa pi^2 t / (rho c)) sin(pi x), T = 300 at
    x = 0, 1, adiabatic elsewhere; the error against a reference run with dt/8 of the
    same spatial discretisation isolates the time error."""
    coords, cells = _cube(n, 2)
    bnd = (coords[:, 0] <= 1e-12) | (coords[:, 0] >= 1 - 1e-12)
    T0 = 300.0 + np.sin(np.pi * coords[:, 0])
    tp = _tp(coords, cells, [[2.0, 1.5, 0.0, 0.8, 0.0]], mask=bnd.astype(np.uint8), Td=np.full(coords.shape[0], 300.0))

    def run(h):
        T = T0.copy()
        for _ in range(int(round(t_end / h))):
            T, _, _ = oth.newton(tp, T, T_old=T, dt=h, theta=theta, rtol=1e-10)
        return T
    return run(dt), run(dt / 8)


@pytest.mark.parametrize("theta,order", [(1.0, 1), (0.5, 2)])
def test_theta_method_time_order(theta, order):
    e = []
    for dt in (0.04, 0.02):
        T, T_ref = _decay_error(dt, theta)
        e.append(np.abs(T - T_ref).max())
    rate = np.log2(e[0] / e[1])
    assert rate >= order - 0.2, (e, rate)


@pytest.mark.parametrize("degree", [1, 2])
def test_jacobian_matches_central_differences(degree):
    coords, cells = _cube(2, degree, jitter=0.2)
    faces = meshgen.boundary_faces(cells)
    rng = np.random.default_rng(4)
    beta = -rng.uniform(0.5, 2.0, faces.shape[0])
    T_bc = 350.0 + 10.0 * rng.standard_normal(coords.shape[0])
    tp = _tp(coords, cells, [[1.2, 0.8, 3e-3, 0.4, 2e-3]], faces, beta, T_bc)
    T_old = 320.0 + 5.0 * rng.standard_normal(coords.shape[0])
    T = T_old + 3.0 * rng.standard_normal(coords.shape[0])
    kw = dict(T_old=T_old, dt=0.03, theta=0.6)
    _, J = oth.assemble_thermal(tp, T, **kw)
    v = rng.standard_normal(coords.shape[0])
    h = 1e-4
    Fp, _ = oth.assemble_thermal(tp, T + h * v, **kw)
    Fm, _ = oth.assemble_thermal(tp, T - h * v, **kw)
    fd = (Fp - Fm) / (2 * h)
    assert np.abs(J @ v - fd).max() <= 1e-7 * np.abs(fd).max()
    # the conductivity's dependence on T makes J non-symmetric; without it, symmetric
    assert abs(J - J.T).max() > 1e-6 * abs(J).max()
    tp.thermal_props[:, 4] = 0.0
    _, Js = oth.assemble_thermal(tp, T, **kw)
    assert abs(Js - Js.T).max() <= 1e-13 * abs(Js).max()


@pytest.mark.parametrize("degree", [1, 2])
def test_robin_face_integrals_by_hand(degree):
    """One tet, one Robin face (x3 = 0 plane), T - T_bc = 1 everywhere, no conduction:
    F_i = -beta int_F psi_i = -beta |F| / 3 on the face's P1 nodes; for P2 the vertex
    functions integrate to 0 and the edge functions to |F| / 3."""
    coords = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [0.0, 1.5, 0.0], [0.3, 0.2, 1.0]])
    cells = np.array([[0, 1, 2, 3]], np.int32)
    if degree == 2:
        coords, cells, _ = meshgen.p1_to_p2(coords, cells)
    faces = meshgen.boundary_faces(cells)
    base = faces[np.all(coords[faces[:, :3], 2] == 0.0, axis=1)]
    assert base.shape[0] == 1
    n = coords.shape[0]
    tp = _tp(coords, cells, [[1.0, 1.0, 0.0, 0.0, 0.0]], base, [-2.0], np.full(n, 10.0))
    F, _ = oth.assemble_thermal(tp, np.full(n, 11.0))
    area = 0.5 * 2.0 * 1.5
    expect = np.zeros(n)
    if degree == 1:
        expect[base[0]] = 2.0 * area / 3.0
    else:
        expect[base[0, 3:]] = 2.0 * area / 3.0
    np.testing.assert_allclose(F, expect, atol=1e-14)


def test_time_step_rule():
    """Eq. dt_spec: dt_{m+1} = eps dT_max / max|T_{m+1} - T_m| dt_m; rejected (halved)
    when the change exceeds dT_max."""
    T0 = np.array([300.0, 310.0, 320.0])
    dt, ok, ch = oth.next_dt(0.5, T0 + np.array([1.0, -4.0, 2.0]), T0, dT_max=10.0, eps=0.8)
    assert ok and ch == 4.0 and dt == pytest.approx(0.8 * 10.0 / 4.0 * 0.5)
    dt, ok, ch = oth.next_dt(0.5, T0 + np.array([0.0, 12.0, 0.0]), T0, dT_max=10.0, eps=0.8)
    assert not ok and dt == 0.25
