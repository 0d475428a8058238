"""Oracle: the paper's thermal problem (TEST INFRASTRUCTURE ONLY).

Plain FP64 NumPy/SciPy restatement of the temperature half of the model
(paper Sec. 3, "Thermomechanical model and numerical formulation"):

    rho c_v dT/dt - div(kappa grad T) = 0             in Omega,
    kappa grad T . n = beta (T - T_bc)                 on Gamma_N^T,

discretised in time by the theta-method (Eq. wf_thermal): given T_m, find
T = T_{m+1} in V_h with, for every basis function s,

    F(T; s) = int rho c_v,theta (T - T_m) / dt s
            + int kappa_theta grad T_theta . grad s
            - int_{Gamma_N^T} beta_theta (T_theta - T_bc,theta) s  = 0,

w_theta = (1 - theta) w_m + theta w_{m+1}.  The steady problem drops the
first term and takes theta = 1.  Newton's method on F (Sec. 3 "Solution
strategy": full linearisation, a non-symmetric Jacobian when kappa depends on
T), and the adaptive time step of Eq. dt_spec.

Readings where the paper gives no formula (the same on both sides):
* c_v(T) = c0 + c1 T and kappa(T) = k0 + k1 T per material (the paper's
  material curves are plots of proprietary data).  Both are affine, so the
  theta-weighted coefficients equal the coefficients of T_theta:
  c_v,theta = c_v(T_theta), kappa_theta = kappa(T_theta).
* T, T_m and T_bc are fields of V_h (nodal interpolants); beta is constant on
  each Robin face; the caller supplies beta_theta and T_bc,theta directly.
* The boundary condition is taken with the paper's sign: a cooling film has
  beta <= 0 (then the Robin term adds -beta int T s >= 0 to the operator).
* Optional nodal Dirichlet temperatures (not in the paper's model; used by the
  pins) are imposed like the elastic ones: rows and columns eliminated, unit
  diagonal, F = 0 there once T holds the prescribed value.

Every integral is exact (barycentric monomial integration on the tet,
int_F m0^a m1^b m2^c = 2 |F| a! b! c! / (a+b+c+2)! on a face).

Parity status: pinned (a linear steady field reproduced exactly, the
Kirchhoff-transformed manufactured solution of the nonlinear steady problem
converging at rates 2 / 3 in L2 for P1 / P2, the transient theta-method's
time order 1 / 2 against a closed-form decay, the Jacobian against finite
differences of F, the Robin face integral by hand, the steady heat balance,
and Eq. dt_spec).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import _pdiff, _pint, _pmul, barycentric_gradients, basis_polys

# ----------------------------------------------------------------------------
# Reference integrals
# ----------------------------------------------------------------------------


@lru_cache(maxsize=None)
def cell_integrals(degree):
    """Exact element integrals (each divided by |K|) of the thermal forms.

    M2[a, b]          = int phi_a phi_b
    M3[a, b, c]       = int phi_a phi_b phi_c
    S2[a, k, b, l]    = int dphi_a/dl_k dphi_b/dl_l
    S3[c, a, k, b, l] = int phi_c dphi_a/dl_k dphi_b/dl_l
    """
    phi = basis_polys(degree)
    n = len(phi)
    dphi = [[_pdiff(p, k) for k in range(4)] for p in phi]
    M2 = np.zeros((n, n))
    M3 = np.zeros((n, n, n))
    S2 = np.zeros((n, 4, n, 4))
    S3 = np.zeros((n, n, 4, n, 4))
    for a in range(n):
        for b in range(n):
            ab = _pmul(phi[a], phi[b])
            M2[a, b] = float(_pint(ab))
            for c in range(n):
                M3[a, b, c] = float(_pint(_pmul(ab, phi[c])))
    for a in range(n):
        for k in range(4):
            for b in range(n):
                for l in range(4):
                    g = _pmul(dphi[a][k], dphi[b][l])
                    S2[a, k, b, l] = float(_pint(g))
                    for c in range(n):
                        S3[c, a, k, b, l] = float(_pint(_pmul(phi[c], g)))
    return M2, M3, S2, S3


def _face_basis(degree):
    """Lagrange basis on a triangle (vertices, then edges 01, 12, 20) in barycentrics."""
    def unit(k):
        e = [0, 0, 0]
        e[k] = 1
        return tuple(e)
    if degree == 1:
        return [{unit(a): Fraction(1)} for a in range(3)]
    out = []
    for a in range(3):
        sq = [0, 0, 0]
        sq[a] = 2
        out.append({tuple(sq): Fraction(2), unit(a): Fraction(-1)})
    for a, b in ((0, 1), (1, 2), (2, 0)):
        e = [0, 0, 0]
        e[a] = 1
        e[b] = 1
        out.append({tuple(e): Fraction(4)})
    return out


def _face_int(p):
    """Integral over a triangle divided by its area: sum c * 2 a!b!c! / (|e|+2)!."""
    tot = Fraction(0)
    for e, c in p.items():
        tot += Fraction(c) * Fraction(2 * math.prod(math.factorial(x) for x in e), math.factorial(sum(e) + 2))
    return tot


@lru_cache(maxsize=None)
def face_integrals(degree):
    """F2[a, b] = int_F psi_a psi_b / |F| on a triangle."""
    psi = _face_basis(degree)
    n = len(psi)
    F2 = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            F2[a, b] = float(_face_int(_pmul(psi[a], psi[b])))
    return F2


def face_areas(coords, faces):
    x = coords[faces[:, :3]]
    return 0.5 * np.linalg.norm(np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), axis=1)


# ----------------------------------------------------------------------------
# Residual and Jacobian of Eq. wf_thermal
# ----------------------------------------------------------------------------


def assemble_thermal(tp, T, T_old=None, dt=0.0, theta=1.0, chunk=100_000):
    """(F[n], J) of Eq. wf_thermal at the iterate T (= T_{m+1}); J = dF/dT (CSR).

    T_old = None (or dt <= 0) is the steady problem (no mass term, theta = 1).
    No Dirichlet rows are applied here (see apply_dirichlet).
    """
    coords, cells = tp.coords, tp.cells
    degree = 1 if cells.shape[1] == 4 else 2
    M2, M3, S2, S3 = cell_integrals(degree)
    n = coords.shape[0]
    nl = cells.shape[1]
    steady = T_old is None or dt <= 0.0
    th = 1.0 if steady else float(theta)
    Tth_n = T if steady else (1.0 - th) * T_old + th * T
    F = np.zeros(n)
    rows, cols, vals = [], [], []
    for s in range(0, cells.shape[0], chunk):
        c = cells[s:s + chunk]
        G, vol = barycentric_gradients(coords[c[:, :4]])
        if np.any(vol <= 0):
            raise ValueError("non-positive cell volume")
        pr = tp.thermal_props[tp.cell_material[s:s + chunk]]
        rho, c0, c1, k0, k1 = (pr[:, i] for i in range(5))
        Tth = Tth_n[c]                                            # [e, a]
        # grad structure: H[e, a, b] = int grad phi_a . grad phi_b / |K|,
        # H3[e, c, a, b] = int phi_c grad phi_a . grad phi_b / |K|
        GG = np.einsum("ekp,elp->ekl", G, G)
        H = np.einsum("akbl,ekl->eab", S2, GG)
        H3 = np.einsum("cakbl,ekl->ecab", S3, GG)
        # kappa(T_theta) grad T_theta . grad s:  k0 H Tth + k1 (sum_c Tth_c H3_c) Tth
        KH = k0[:, None, None] * H + k1[:, None, None] * np.einsum("ec,ecab->eab", Tth, H3)
        Fe = vol[:, None] * np.einsum("eab,ea->eb", KH, Tth)
        # dF_b / dT_j (j a local node): theta [KH[j, b] + k1 sum_a Tth_a H3[j, a, b]]
        Je = th * (KH + k1[:, None, None] * np.einsum("ea,ejab->ejb", Tth, H3))
        if not steady:
            dT = (T[c] - T_old[c]) / dt                            # [e, a]
            # int rho (c0 + c1 T_theta) (T - T_old)/dt s
            Fe += vol[:, None] * rho[:, None] * (c0[:, None] * dT @ M2
                                                + c1[:, None] * np.einsum("ea,eb,abc->ec", Tth, dT, M3))
            # d/dT_j: rho [c1 theta phi_j (T - T_old)/dt + c_v(T_theta) phi_j / dt] s
            Je += rho[:, None, None] * (c1[:, None, None] * th * np.einsum("eb,jbc->ejc", dT, M3)
                                        + (c0[:, None, None] * M2[None] + c1[:, None, None]
                                           * np.einsum("ea,ajc->ejc", Tth, M3)) / dt)
        Je = vol[:, None, None] * Je                               # [e, j, b] = dF_b / dT_j
        np.add.at(F, c.ravel(), Fe.ravel())
        rows.append(np.repeat(c, nl, axis=1).ravel())              # row b? build (b, j) below
        cols.append(np.tile(c, (1, nl)).ravel())
        vals.append(np.transpose(Je, (0, 2, 1)).ravel())           # [e, b, j]
    # Robin faces: - int beta (T_theta - T_bc) s  and  d/dT_j: - beta theta int phi_j s
    if tp.faces is not None and len(tp.faces):
        fdeg = 1 if tp.faces.shape[1] == 3 else 2
        F2 = face_integrals(fdeg)
        area = face_areas(coords, tp.faces)
        w = tp.beta * area                                         # [f]
        d = Tth_n[tp.faces] - tp.T_bc[tp.faces]                    # [f, a]
        np.add.at(F, tp.faces.ravel(), (-w[:, None] * (d @ F2)).ravel())
        Jf = -th * w[:, None, None] * F2[None]
        nf = tp.faces.shape[1]
        rows.append(np.repeat(tp.faces, nf, axis=1).ravel())
        cols.append(np.tile(tp.faces, (1, nf)).ravel())
        vals.append(Jf.ravel())
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    J.sum_duplicates()
    return F, J


def apply_dirichlet(F, J, mask):
    """Dirichlet rows/columns of the Newton system eliminated: J_DD = I, F_D = 0."""
    if mask is None:
        return F, J
    dm = np.asarray(mask).astype(bool)
    keep = sp.diags((~dm).astype(np.float64))
    J2 = (keep @ J @ keep + sp.diags(dm.astype(np.float64))).tocsr()
    J2.eliminate_zeros()
    F2 = F.copy()
    F2[dm] = 0.0
    return F2, J2


def newton(tp, T0, T_old=None, dt=0.0, theta=1.0, rtol=1e-9, max_iter=30):
    """Newton on F(T) = 0 with a direct solve of each step.

    Returns (T, iterations, history of ||F||_2).  Dirichlet nodes take
    T_dirichlet first and stay fixed.  Stops when ||F|| <= rtol ||F(T0)||.
    """
    T = np.array(T0, dtype=np.float64)
    if tp.dirichlet_mask is not None:
        dm = np.asarray(tp.dirichlet_mask).astype(bool)
        T[dm] = tp.T_dirichlet[dm]
    hist = []
    for it in range(max_iter + 1):
        F, J = assemble_thermal(tp, T, T_old, dt, theta)
        F, J = apply_dirichlet(F, J, tp.dirichlet_mask)
        hist.append(float(np.linalg.norm(F)))
        if hist[-1] <= rtol * hist[0] or it == max_iter:
            return T, it, hist
        T = T - spla.spsolve(J.tocsc(), F)
    return T, max_iter, hist


def next_dt(dt, T_new, T_old, dT_max, eps):
    """Eq. dt_spec: dt_{m+1} = eps dT_max / max |T_{m+1} - T_m| * dt_m, and
    whether the step is accepted (max change <= dT_max; else repeat with dt/2)."""
    change = float(np.max(np.abs(T_new - T_old)))
    if change > dT_max:
        return 0.5 * dt, False, change
    return (eps * dT_max / change) * dt if change > 0 else 2.0 * dt, True, change
