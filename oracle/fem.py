"""Oracle: thermoelastic element integrals, assembly and Dirichlet elimination.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Plain FP64 NumPy/SciPy.

What is computed (paper Sec. 3, "Thermomechanical model and numerical
formulation"):

* Eq. (elasticity_bvp)/(u-dbc): -div sigma = f in Omega, u = u_bc on Gamma_D,
  traction free elsewhere (the pressure term of Eq. (wf_elastic) is zero).
* sigma = C : (eps - eps_T), eps = sym grad u, eps_T = alpha (T - T_ref) I,
  isotropic C from Young's modulus E and Poisson ratio nu.
* Eq. (wf_elastic), steady: find u_h in [V_h]^3 with
  int C:eps(u_h) : eps(v) = int f_h . v + int C:eps_T(T_h) : eps(v)
  for all v in [V_h]^3, V_h = P1 or P2 Lagrange on affine tetrahedra; T_h and
  f_h are the nodal interpolants in V_h.

Every integral is evaluated EXACTLY: each basis function is a polynomial in
the barycentric coordinates and
    int_K l0^a l1^b l2^c l3^d dx = 6 |K| a! b! c! d! / (a+b+c+d+3)!,
so the element matrix is the textbook B^T D B (Voigt notation, engineering
shear strains) with exact polynomial integration -- no quadrature.

Parity status: pinned (hand-derived single-element matrices, rigid-body
kernel, symmetry, P1/P2 patch tests, free thermal expansion, body-force
resultant and moment identities, manufactured-solution convergence rates).
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np
import scipy.sparse as sp

P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def lame(E, nu):
    """Lame parameters of isotropic C: mu = E/(2(1+nu)), lambda = E nu/((1+nu)(1-2nu))."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return lam, mu


def voigt_D(E, nu):
    """6x6 isotropic elasticity matrix for strains (xx, yy, zz, 2yz, 2xz, 2xy)."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2.0 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


# Voigt strain of the field phi * e_i: component s picks d(phi)/dx_p.
# (s, i, p) triples: eps_xx = d_x u_x, ..., 2 eps_yz = d_z u_y + d_y u_z, ...
_VOIGT = (
    (0, 0, 0), (1, 1, 1), (2, 2, 2),
    (3, 1, 2), (3, 2, 1),
    (4, 0, 2), (4, 2, 0),
    (5, 0, 1), (5, 1, 0),
)


def voigt_selector():
    """Bsel[s, i, p] = 1 when Voigt strain s of (phi e_i) contains d phi / d x_p."""
    B = np.zeros((6, 3, 3))
    for s, i, p in _VOIGT:
        B[s, i, p] = 1.0
    return B


# ----------------------------------------------------------------------------
# Polynomials in barycentric coordinates (exact rational coefficients)
# ----------------------------------------------------------------------------

def _pmul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return {e: c for e, c in out.items() if c != 0}


def _pdiff(p, k):
    out = {}
    for e, c in p.items():
        if e[k] > 0:
            f = list(e)
            f[k] -= 1
            out[tuple(f)] = out.get(tuple(f), 0) + c * e[k]
    return out


def _pint(p):
    """Integral over K divided by |K|: sum c * 6 a!b!c!d!/(|e|+3)!."""
    tot = Fraction(0)
    for e, c in p.items():
        num = 6 * math.prod(math.factorial(x) for x in e)
        tot += Fraction(c) * Fraction(num, math.factorial(sum(e) + 3))
    return tot


def _unit(k):
    e = [0, 0, 0, 0]
    e[k] = 1
    return tuple(e)


def basis_polys(degree):
    """Lagrange basis on the tet as barycentric polynomials (local node order)."""
    if degree == 1:
        return [{_unit(a): Fraction(1)} for a in range(4)]
    if degree == 2:
        out = []
        for a in range(4):
            sq = [0, 0, 0, 0]
            sq[a] = 2
            out.append({tuple(sq): Fraction(2), _unit(a): Fraction(-1)})
        for a, b in P2_EDGES:
            e = [0, 0, 0, 0]
            e[a] = 1
            e[b] = 1
            out.append({tuple(e): Fraction(4)})
        return out
    raise ValueError("degree must be 1 or 2")


@lru_cache(maxsize=None)
def reference_integrals(degree):
    """Element-independent exact integrals (each divided by |K|).

    S[a,k,b,l] = int dphi_a/dl_k * dphi_b/dl_l     (stiffness structure)
    Tm[c,a,k]  = int phi_c * dphi_a/dl_k           (thermal-load structure)
    M[a,b]     = int phi_a * phi_b                 (mass, body-force load)
    By the chain rule grad phi = sum_k (d phi/d l_k) grad l_k.
    """
    phi = basis_polys(degree)
    n = len(phi)
    dphi = [[_pdiff(p, k) for k in range(4)] for p in phi]
    S = np.zeros((n, 4, n, 4))
    for a in range(n):
        for k in range(4):
            for b in range(n):
                for l in range(4):
                    S[a, k, b, l] = float(_pint(_pmul(dphi[a][k], dphi[b][l])))
    Tm = np.zeros((n, n, 4))
    for c in range(n):
        for a in range(n):
            for k in range(4):
                Tm[c, a, k] = float(_pint(_pmul(phi[c], dphi[a][k])))
    M = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            M[a, b] = float(_pint(_pmul(phi[a], phi[b])))
    return S, Tm, M


def barycentric_gradients(X):
    """For vertex coords X[m,4,3]: (G[m,4,3] = grad l_k, vol[m] signed volume)."""
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)  # columns
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)              # rows are grad l_1..l_3
    G = np.empty((X.shape[0], 4, 3))
    G[:, 1:] = Jinv
    G[:, 0] = -Jinv.sum(axis=1)
    return G, det / 6.0


# ----------------------------------------------------------------------------
# Element matrices and load vectors
# ----------------------------------------------------------------------------

def element_matrices(coords, cells, cell_material, mat_props, T=None, T_ref=0.0,
                     body_force=None):
    """Element stiffness Ke[m, n_loc, 3, n_loc, 3] and load fe[m, n_loc, 3].

    Ke[e, a, i, b, j] = int (B^T D B) for DOF (node a, comp i) x (node b, comp j).
    fe = thermal load int B^T D eps_T + body load int f_h phi_a.
    """
    degree = 1 if cells.shape[1] == 4 else 2
    S, Tm, M = reference_integrals(degree)
    X = coords[cells[:, :4]]
    G, vol = barycentric_gradients(X)
    if np.any(vol <= 0):
        raise ValueError("non-positive cell volume")
    E = mat_props[cell_material, 0]
    nu = mat_props[cell_material, 1]
    alpha = mat_props[cell_material, 2]
    lam, mu = lame(E, nu)
    D = np.zeros((cells.shape[0], 6, 6))
    D[:, :3, :3] = lam[:, None, None]
    for s in range(3):
        D[:, s, s] = lam + 2.0 * mu
    for s in range(3, 6):
        D[:, s, s] = mu
    Bsel = voigt_selector()
    # H[e,a,b,p,q] = int d_p phi_a d_q phi_b
    H = vol[:, None, None, None, None] * np.einsum("akbl,ekp,elq->eabpq", S, G, G, optimize=True)
    # Ke[e,a,i,b,j] = sum_{s,t,p,q} Bsel[s,i,p] D[e,s,t] Bsel[t,j,q] H[e,a,b,p,q]
    DD = np.einsum("sip,est,tjq->eijpq", Bsel, D, Bsel, optimize=True)
    Ke = np.einsum("eijpq,eabpq->eaibj", DD, H, optimize=True)
    n_loc = cells.shape[1]
    fe = np.zeros((cells.shape[0], n_loc, 3))
    if T is not None:
        # eps_T = alpha (T_h - T_ref) (1,1,1,0,0,0);  sigma_T = D eps_T
        dT = T[cells] - T_ref                                  # [e, c]
        # int (T_h - T_ref) d_p phi_a = vol * sum_c dT_c sum_k Tm[c,a,k] G[k,p]
        Wt = vol[:, None, None] * np.einsum("ec,cak,ekp->eap", dT, Tm, G, optimize=True)
        sig_unit = D[:, :, :3].sum(axis=2) * alpha[:, None]    # D (1,1,1,0,0,0)^T alpha
        fe += np.einsum("sip,es,eap->eai", Bsel, sig_unit, Wt, optimize=True)
    if body_force is not None:
        fb = body_force[cells]                                 # [e, b, 3]
        fe += vol[:, None, None] * np.einsum("ab,ebi->eai", M, fb)
    return Ke, fe


def assemble(coords, cells, cell_material, mat_props, T=None, T_ref=0.0,
             body_force=None, chunk=200_000):
    """Global K (scipy CSR, 3n x 3n, DOF 3*node+comp) and load f[3n] (no BCs)."""
    n = coords.shape[0]
    n_loc = cells.shape[1]
    rows, cols, vals = [], [], []
    f = np.zeros(3 * n)
    for s in range(0, cells.shape[0], chunk):
        c = cells[s:s + chunk]
        Ke, fe = element_matrices(coords, c, cell_material[s:s + chunk], mat_props,
                                  T, T_ref, body_force)
        dof = (3 * c[:, :, None] + np.arange(3)[None, None, :]).reshape(c.shape[0], 3 * n_loc)
        Kf = Ke.reshape(c.shape[0], 3 * n_loc, 3 * n_loc)
        rows.append(np.repeat(dof, 3 * n_loc, axis=1).ravel())
        cols.append(np.tile(dof, (1, 3 * n_loc)).ravel())
        vals.append(Kf.ravel())
        np.add.at(f, dof.ravel(), fe.reshape(-1))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(3 * n, 3 * n)).tocsr()
    K.sum_duplicates()
    return K, f


def apply_dirichlet(K, f, dirichlet_mask, u_dirichlet=None):
    """Symmetric elimination (Eq. u-dbc): lift the load, zero rows/cols, unit diagonal.

    f_free -= K_{free,D} u_D;  K_{D,:} = K_{:,D} = 0;  K_{DD} = I;  f_D = u_D.
    """
    dm = np.repeat(np.asarray(dirichlet_mask).astype(bool), 3)
    ud = np.zeros(K.shape[0]) if u_dirichlet is None else np.asarray(u_dirichlet, float).ravel().copy()
    ud[~dm] = 0.0
    f2 = f - K @ ud
    keep = sp.diags((~dm).astype(np.float64))
    K2 = (keep @ K @ keep + sp.diags(dm.astype(np.float64))).tocsr()
    K2.eliminate_zeros()
    f2[dm] = ud[dm]
    return K2, f2


def assemble_system(problem):
    """K, f of a meshgen.Problem with Dirichlet conditions applied."""
    K, f = assemble(problem.coords, problem.cells, problem.cell_material, problem.mat_props,
                    problem.T, problem.T_ref, problem.body_force)
    return apply_dirichlet(K, f, problem.dirichlet_mask, problem.u_dirichlet)


def rigid_body_modes(coords, dirichlet_mask=None, rotations=True):
    """Near-nullspace B[3n, 6] of 3D elasticity (paper Sec. 2, smoothed aggregation).

    Columns: translations along x, y, z, then rotations about the x, y, z
    axes through the node centroid c:  rot_x = (0, -(z-cz), y-cy),
    rot_y = (z-cz, 0, -(x-cx)), rot_z = (-(y-cy), x-cx, 0).  Rows of Dirichlet
    nodes are zero.  With rotations=False only the 3 translations are kept.
    """
    n = coords.shape[0]
    d = coords - coords.mean(axis=0)
    B = np.zeros((n, 3, 6))
    B[:, 0, 0] = B[:, 1, 1] = B[:, 2, 2] = 1.0
    B[:, 1, 3], B[:, 2, 3] = -d[:, 2], d[:, 1]
    B[:, 0, 4], B[:, 2, 4] = d[:, 2], -d[:, 0]
    B[:, 0, 5], B[:, 1, 5] = -d[:, 1], d[:, 0]
    if dirichlet_mask is not None:
        B[np.asarray(dirichlet_mask).astype(bool)] = 0.0
    B = B.reshape(3 * n, 6)
    return B if rotations else B[:, :3].copy()


def block_rows(K, nodes):
    """Dense 3x3 blocks of the block rows `nodes`: dict node -> {col_node: 3x3}."""
    out = {}
    for i in nodes:
        blk = {}
        for r in range(3):
            row = K.getrow(3 * i + r)
            for c, v in zip(row.indices, row.data):
                blk.setdefault(c // 3, np.zeros((3, 3)))[r, c % 3] = v
        out[int(i)] = blk
    return out
