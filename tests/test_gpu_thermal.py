"""GPU thermal problem vs the CPU oracle (paper Sec. 3, Eq. wf_thermal, Eq. dt_spec).

The residual and the Newton Jacobian of the theta-method are compared entry
by entry with the oracle's exact-integral assembly (P1 and P2, temperature
dependent c_v and kappa, Robin faces, Dirichlet nodes, steady and transient);
Newton's solution with the oracle's Newton (direct solves) -- the discrete
problem has one solution, whatever the linear solver; a sequence of adaptive
time steps (Eq. dt_spec) with the oracle's sequence; and the one-way coupled
transient (thermal step, then the elastic solve with the new temperature,
the elastic hierarchy and the previous displacement reused) with the oracle's
direct elastic solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from gpu_util import need_gpu, torch
from oracle import fem, linsolve
from oracle import thermal as oth
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12        # assembly: FP64, different integration order only
SOL_TOL = 1e-8     # Newton solutions, both to ||F|| <= 1e-11 ||F_0||


def _disc(degree, n_r=6, blades=12):
    return meshgen.bladed_disc_problem(n_r=n_r, n_theta_per_blade=4, n_z=2, n_blades=blades, n_r_blade=3,
                                       degree=degree, seed=3)


def _thermal(degree, t=0.3, dirichlet=False, nonlinear=True):
    pb = _disc(degree)
    tp = meshgen.disc_thermal_problem(pb, t=t)
    if not nonlinear:
        tp.thermal_props = tp.thermal_props.copy()
        tp.thermal_props[:, [2, 4]] = 0.0
    if dirichlet:  # hold the bore at 280 K
        rad = np.hypot(pb.coords[:, 0], pb.coords[:, 1])
        tp.dirichlet_mask = (rad <= 0.2 + 1e-9).astype(np.uint8)
        tp.T_dirichlet = np.full(pb.n_nodes, 280.0)
    return pb, tp


def _handle(tam, tp, **prm):
    d = tam.thermal_to_device(tp)
    th = tam.Thermal(d["coords"], d["cells"], d["cell_material"], tp.thermal_props, d["faces"],
                     d["dirichlet_mask"], tam.amg_params_default(**prm) if prm else None)
    return th, d


def _jac_csr(th, n):
    rp, ci, v = th.jacobian()
    return sp.csr_matrix((v.cpu().numpy(), ci.cpu().numpy(), rp.cpu().numpy()), shape=(n, n))


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("transient", [False, True])
def test_residual_and_jacobian_match_oracle(degree, transient):
    tam = need_gpu()
    pb, tp = _thermal(degree, dirichlet=True)
    th, d = _handle(tam, tp)
    rng = np.random.default_rng(5)
    n = pb.n_nodes
    T = 300.0 + 400.0 * rng.random(n)
    T[tp.dirichlet_mask.astype(bool)] = 280.0
    T_old = T - 20.0 * rng.random(n) if transient else None
    kw = dict(T_old=T_old, dt=0.05, theta=0.6) if transient else {}
    Tg = torch.from_numpy(T).cuda()
    Tog = torch.from_numpy(T_old).cuda() if transient else None
    F = th.residual(Tg, Tog, kw.get("dt", 0.0), kw.get("theta", 1.0), d["beta"], d["T_bc"]).cpu().numpy()
    Fo, Jo = oth.assemble_thermal(tp, T, **kw)
    Fo, Jo = oth.apply_dirichlet(Fo, Jo, tp.dirichlet_mask)
    assert np.abs(F - Fo).max() <= TOL * np.abs(Fo).max()
    Jg = _jac_csr(th, n)
    D = (Jg - Jo).tocsr()
    assert (abs(D).max() if D.nnz else 0.0) <= TOL * abs(Jo).max()
    if degree == 1 and not transient:
        # the full linearisation is non-symmetric (kappa depends on T)
        assert abs(Jg - Jg.T).max() > 1e-8 * abs(Jg).max()
    th.destroy()


@pytest.mark.parametrize("degree", [1, 2])
@pytest.mark.parametrize("reuse", [0, 1])
def test_steady_newton_matches_oracle(degree, reuse):
    tam = need_gpu()
    pb, tp = _thermal(degree)
    th, d = _handle(tam, tp)
    n = pb.n_nodes
    T = torch.full((n,), 400.0, dtype=torch.float64, device="cuda")   # the paper's initial guess
    st = th.newton(T, beta=d["beta"], T_bc=d["T_bc"], rtol=1e-11, lin_rtol=1e-10, reuse=reuse)
    assert st["status"] == 0 and st["rel"] <= 1e-11
    assert 2 <= st["newton"] <= 12, st
    To, it_o, hist = oth.newton(tp, np.full(n, 400.0), rtol=1e-11)
    err = np.abs(T.cpu().numpy() - To).max() / np.abs(To).max()
    assert err <= SOL_TOL, (st, err)
    if reuse:
        assert st["setups"] < st["newton"], st
    th.destroy()


def test_transient_steps_with_adaptive_dt_match_oracle():
    """Backward Euler (the paper's transient choice) from 300 K under the rising
    hot-gas temperature, Eq. dt_spec with dT_max = 10 K, eps = 0.8; the GPU and
    the oracle take the same accepted / rejected steps."""
    tam = need_gpu()
    pb, _ = _thermal(1, dirichlet=True)
    n = pb.n_nodes
    th = None
    T = torch.full((n,), 300.0, dtype=torch.float64, device="cuda")
    To = np.full(n, 300.0)
    t, dt = 0.0, 0.02
    steps = rejected = 0
    while steps < 6:
        tp = meshgen.disc_thermal_problem(pb, t=t + dt)     # boundary data at t_{m+1} (theta = 1)
        tp.dirichlet_mask = (np.hypot(pb.coords[:, 0], pb.coords[:, 1]) <= 0.2 + 1e-9).astype(np.uint8)
        tp.T_dirichlet = np.full(n, 300.0)
        if th is None:
            th, d = _handle(tam, tp)
        dd = tam.thermal_to_device(tp)
        Tn = T.clone()
        st = th.newton(Tn, T_old=T, dt=dt, theta=1.0, beta=dd["beta"], T_bc=dd["T_bc"],
                       T_dirichlet=dd["T_dirichlet"], rtol=1e-11, lin_rtol=1e-10, reuse=1)
        assert st["status"] == 0
        Ton, _, _ = oth.newton(tp, To, T_old=To, dt=dt, theta=1.0, rtol=1e-11)
        ch = tam.tam_thermal_max_change(Tn, T)
        ch_o = float(np.max(np.abs(Ton - To)))
        assert abs(ch - ch_o) <= 1e-8 * ch_o
        dt_next, ok = tam.tam_thermal_next_dt(dt, ch, 10.0, 0.8)
        dt_o, ok_o, _ = oth.next_dt(dt, Ton, To, 10.0, 0.8)
        assert ok == ok_o and dt_next == pytest.approx(dt_o, rel=1e-9)
        if ok:
            T, To, t = Tn, Ton, t + dt
            steps += 1
        else:
            rejected += 1
        dt = dt_next
        err = np.abs(T.cpu().numpy() - To).max() / np.abs(To).max()
        assert err <= SOL_TOL, (steps, err)
    assert t > 0.0
    th.destroy()


def test_coupled_step_reuses_elastic_hierarchy():
    """One-way coupling (Sec. 3 "Solution strategy"): per step the thermal
    Newton, then K u = f(T) with the elastic K and hierarchy of the first step
    and the previous displacement as initial guess (Sec. 5.3); every
    displacement matches the oracle's direct solve with the oracle's T."""
    tam = need_gpu()
    pb = _disc(1)
    pb.mat_props = np.array([[1.0, 0.3, 1e-5]])
    n = pb.n_nodes
    dev = tam.problem_to_device(pb)
    K, rhs = tam.fem_assemble_elasticity(**dict(dev, T=torch.full((n,), 300.0, dtype=torch.float64, device="cuda")))
    H = tam.amg_setup(K, dev["coords"])
    u = torch.zeros_like(rhs)
    T = torch.full((n,), 300.0, dtype=torch.float64, device="cuda")
    th = None
    Ko, _ = fem.assemble_system(pb)
    its = []
    for k in range(3):
        tp = meshgen.disc_thermal_problem(pb, t=0.1 * (k + 1))
        if th is None:
            th, _ = _handle(tam, tp)
        dd = tam.thermal_to_device(tp)
        Tn = T.clone()
        st = th.newton(Tn, T_old=T, dt=0.1, theta=1.0, beta=dd["beta"], T_bc=dd["T_bc"], rtol=1e-11,
                       lin_rtol=1e-10, reuse=1)
        assert st["status"] == 0
        T = Tn
        b = tam.fem_assemble_load(K, **dict(dev, T=T), stream=None)
        it, rel, s = tam.amg_pcg_solve(H, b, u, rtol=1e-8)
        assert s == 0
        its.append(it)
        q = meshgen.Problem(pb.name, pb.coords, pb.cells, pb.cell_material, pb.mat_props, T.cpu().numpy(),
                            pb.T_ref, pb.body_force, pb.dirichlet_mask, None)
        _, fo = fem.assemble_system(q)
        uo = linsolve.direct_solve(Ko, fo)
        assert np.linalg.norm(u.cpu().numpy().ravel() - uo) <= 1e-6 * np.linalg.norm(uo)
    assert its[-1] <= its[0], its     # warm start from the previous displacement
    th.destroy()
    H.destroy()
    K.destroy()
