"""Oracle: reference linear solves for K u = f (TEST INFRASTRUCTURE ONLY).

The method's result is the exact solution of the assembled system; CG and
AMG (paper Sec. 2.1, "Iterative solvers" and "Multigrid preconditioned
iterative solvers") only reach it faster.  These routines reach it by other
means so that the GPU solve can be checked against them:

* ``dense_solve``   -- dense Cholesky (NumPy/LAPACK), tiny systems only.
* ``direct_solve``  -- sparse LU (SciPy SuperLU), small systems.
* ``jacobi_pcg``    -- plain Jacobi-preconditioned CG, written out.

Parity status: pinned (the three agree with one another and with closed-form
patch-test solutions).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def dense_solve(K, f):
    A = K.toarray() if hasattr(K, "toarray") else np.asarray(K)
    L = np.linalg.cholesky(A)
    y = sla.solve_triangular(L, f, lower=True)
    return sla.solve_triangular(L.T, y, lower=False)


def direct_solve(K, f):
    return spla.splu(K.tocsc(), permc_spec="COLAMD").solve(np.asarray(f, dtype=np.float64))


def jacobi_pcg(K, f, rtol=1e-12, max_iter=100_000, x0=None):
    """CG preconditioned by the point diagonal; stops on ||f - Kx|| <= rtol ||f||."""
    d = K.diagonal()
    dinv = np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - K @ x
    z = dinv * r
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(f)
    it = 0
    while np.linalg.norm(r) > rtol * nb and it < max_iter:
        q = K @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it
