"""Oracle: smoothed-aggregation AMG preconditioned CG (TEST INFRASTRUCTURE ONLY).

Plain FP64 restatement of the paper's elastic solver: CG preconditioned by a
smoothed-aggregation AMG V-cycle whose near-nullspace is the six rigid-body
modes (Sec. 2.1 "Multigrid preconditioned iterative solvers"; Sec. 5.1
"Solver configuration": Chebyshev smoothing with adequate lambda_max
estimates, fast coarsening, a sizeable coarsest grid).  The paper names the
method (Vanek-Mandel-Brezina smoothed aggregation) but not its details; the
readings taken here are:

* strength: block (i,j), i != j, is strong when ||A_ij||_F > 0 and
  ||A_ij||_F >= theta sqrt(||A_ii||_F ||A_jj||_F); a node with no strong
  neighbour (e.g. a Dirichlet node) is isolated and joins no aggregate.
* aggregation: roots form the distance-2 maximal independent set of the
  strength graph chosen greedily by decreasing priority (top 30 bits of
  SplitMix64(level << 32 | node), ties broken by the larger node id); a
  non-root joins the adjacent root
  of largest priority; a node left over joins the aggregate of its
  already-attached neighbour of largest priority.  Aggregates are numbered by
  increasing root id.
* tentative prolongator: per aggregate, modified Gram-Schmidt of the
  near-nullspace rows (node order increasing) gives Q (prolongator rows) and
  R (coarse near-nullspace); a column whose remainder is <= 1e-10 of its
  original norm is dropped (zero Q column, zero R row).
* smoothing: P = (I - 4/(3 lam) D^-1 A) P_tent with D the point diagonal and
  lam a k-step Lanczos estimate of lambda_max(D^-1 A) from a SplitMix64 start
  vector; A_c = P^T A P.
* smoother: Chebyshev on D^-1 A over [lo*lam, hi*lam], same polynomial before
  and after the coarse correction; coarsest level solved exactly (dense
  Cholesky; a zero row/column gets a unit pivot).
* CG stops when the recursively updated residual satisfies
  ||r|| <= max(rtol ||b||, atol).

Parity status: pinned (exact range of P_tent, orthonormal Q, Galerkin product
vs dense triple product, Chebyshev error polynomial vs its closed form,
symmetric positive-definite V-cycle, Ritz bound on lambda_max, aggregation
validity and distance-2 independence, AMG-PCG vs direct solve).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

U64 = np.uint64
MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 finaliser (Steele, Lea & Flood 2014) on Python ints or uint64 arrays."""
    if isinstance(x, (int, np.integer)):
        z = (int(x) + 0x9E3779B97F4A7C15) & MASK64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)
    x = np.asarray(x, dtype=U64)
    with np.errstate(over="ignore"):
        z = x + U64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
    return z ^ (z >> U64(31))


def node_priority(n, level):
    """30-bit node priority: top 30 bits of SplitMix64(level << 32 | node)."""
    return splitmix64((U64(level) << U64(32)) | np.arange(n, dtype=U64)) >> U64(34)


def lanczos_start(n_dof, level):
    """Start vector: v_k = U(splitmix64((level+1) << 40 | k)) - 1/2, U = top 53 bits / 2^53."""
    z = splitmix64((U64(level + 1) << U64(40)) | np.arange(n_dof, dtype=U64))
    return (z >> U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) - 0.5


# ----------------------------------------------------------------------------
# Strength and aggregation
# ----------------------------------------------------------------------------

def block_view(A, bs):
    B = sp.bsr_matrix(A, blocksize=(bs, bs))
    B.sort_indices()
    return B


def strength_graph(A, bs, theta=0.0):
    """List of strong neighbour arrays per node (self excluded)."""
    B = block_view(A, bs)
    n = B.shape[0] // bs
    nrm = np.sqrt((B.data ** 2).sum(axis=(1, 2)))
    diag = np.zeros(n)
    rows = np.repeat(np.arange(n), np.diff(B.indptr))
    on_diag = rows == B.indices
    diag[rows[on_diag]] = nrm[on_diag]
    strong = (rows != B.indices) & (nrm > 0) & (nrm >= theta * np.sqrt(diag[rows] * diag[B.indices]))
    nbrs = []
    for i in range(n):
        s, e = B.indptr[i], B.indptr[i + 1]
        m = strong[s:e]
        nbrs.append(B.indices[s:e][m].astype(np.int64))
    return nbrs


def mis2_aggregate(nbrs, level, distance=2):
    """Aggregates from the greedy distance-`distance` MIS (see module header).

    distance=2 is the default (aggressive) rule; distance=1 gives roots that
    are only pairwise non-adjacent (smaller aggregates).  Returns (agg, n_agg, roots).
    """
    n = len(nbrs)
    prio = node_priority(n, level)
    isolated = np.array([len(x) == 0 for x in nbrs])
    # decreasing (priority, id): sort ascending on (prio, id) and reverse
    order = np.lexsort((np.arange(n), prio))[::-1]
    excluded = isolated.copy()
    is_root = np.zeros(n, bool)
    for i in order:
        if excluded[i]:
            continue
        is_root[i] = True
        excluded[i] = True
        for j in nbrs[i]:
            excluded[j] = True
            if distance == 2:
                for k in nbrs[j]:
                    excluded[k] = True
    roots = np.nonzero(is_root)[0]
    agg = -np.ones(n, np.int64)
    agg[roots] = np.arange(roots.size)
    key = [(int(prio[j]), int(j)) for j in range(n)]
    # phase 2: attach to the adjacent root of largest priority
    agg2 = agg.copy()
    for i in range(n):
        if is_root[i] or isolated[i]:
            continue
        best = None
        for j in nbrs[i]:
            if is_root[j] and (best is None or key[j] > key[best]):
                best = j
        if best is not None:
            agg2[i] = agg[best]
    # phase 3: attach to the already-attached neighbour of largest priority
    agg3 = agg2.copy()
    for i in range(n):
        if agg2[i] >= 0 or isolated[i]:
            continue
        best = None
        for j in nbrs[i]:
            if agg2[j] >= 0 and (best is None or key[j] > key[best]):
                best = j
        if best is None:
            raise RuntimeError("aggregation left a node unassigned (MIS-2 not maximal)")
        agg3[i] = agg2[best]
    return agg3, int(roots.size), roots


def check_aggregates(agg, n_agg, nbrs):
    """Validity of an aggregation: returns a list of violations (empty = valid)."""
    bad = []
    n = len(nbrs)
    for i in range(n):
        if len(nbrs[i]) == 0 and agg[i] != -1:
            bad.append(f"isolated node {i} aggregated")
        if len(nbrs[i]) > 0 and not (0 <= agg[i] < n_agg):
            bad.append(f"node {i} unassigned")
    members = [[] for _ in range(n_agg)]
    for i in range(n):
        if agg[i] >= 0:
            members[agg[i]].append(i)
    for a, mem in enumerate(members):
        if not mem:
            bad.append(f"aggregate {a} empty")
            continue
        seen = {mem[0]}
        stack = [mem[0]]
        ms = set(mem)
        while stack:
            u = stack.pop()
            for v in nbrs[u]:
                if v in ms and v not in seen:
                    seen.add(int(v))
                    stack.append(int(v))
        if len(seen) != len(mem):
            bad.append(f"aggregate {a} not connected")
    return bad


# ----------------------------------------------------------------------------
# Tentative prolongator, smoothing, Galerkin product
# ----------------------------------------------------------------------------

def tentative_prolongator(agg, n_agg, B, bs, droptol=1e-10):
    """P_tent (CSR, n*bs x n_agg*k) and coarse near-nullspace Bc (n_agg*k x k) by MGS."""
    n = agg.size
    k = B.shape[1]
    rows, cols, vals = [], [], []
    Bc = np.zeros((n_agg * k, k))
    members = [[] for _ in range(n_agg)]
    for i in range(n):
        if agg[i] >= 0:
            members[agg[i]].append(i)
    for a in range(n_agg):
        dofs = np.array([bs * i + r for i in members[a] for r in range(bs)])
        V = B[dofs].copy()
        Q = np.zeros_like(V)
        R = np.zeros((k, k))
        for c in range(k):
            v = V[:, c].copy()
            norm0 = np.linalg.norm(v)
            for j in range(c):
                R[j, c] = Q[:, j] @ v
                v -= R[j, c] * Q[:, j]
            nv = np.linalg.norm(v)
            if norm0 > 0 and nv > droptol * norm0:
                R[c, c] = nv
                Q[:, c] = v / nv
        Bc[a * k:(a + 1) * k] = R
        for li, d in enumerate(dofs):
            for c in range(k):
                rows.append(d)
                cols.append(a * k + c)
                vals.append(Q[li, c])
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n * bs, n_agg * k))
    return P, Bc


def point_dinv(A):
    d = A.diagonal()
    return np.where(d != 0, 1.0 / np.where(d != 0, d, 1.0), 0.0)


def lanczos_lambda_max(A, steps, level):
    """Largest Ritz value of `steps` Lanczos steps on D^-1/2 A D^-1/2."""
    d = A.diagonal()
    s = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    v = lanczos_start(A.shape[0], level) * (s > 0)
    v /= np.linalg.norm(v)
    v_prev = np.zeros_like(v)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(steps):
        w = s * (A @ (s * v))
        a = w @ v
        w = w - a * v - beta * v_prev
        alphas.append(a)
        beta = np.linalg.norm(w)
        if beta <= 1e-14 * abs(a):
            break
        betas.append(beta)
        v_prev, v = v, w / beta
    m = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:m - 1], 1) + np.diag(betas[:m - 1], -1)
    return float(np.linalg.eigvalsh(T)[-1])


def smooth_prolongator(A, Pt, lam):
    dinv = point_dinv(A)
    return (Pt - (4.0 / (3.0 * lam)) * sp.diags(dinv) @ (A @ Pt)).tocsr()


def galerkin(A, P):
    R = P.T.tocsr()
    return (R @ (A @ P)).tocsr(), R


# ----------------------------------------------------------------------------
# Smoother, coarse solve, V-cycle, PCG
# ----------------------------------------------------------------------------

def chebyshev(A, dinv, f, x, lo, hi, degree):
    """Chebyshev iteration on D^-1 A over [lo, hi] from x (Saad, Alg. 12.1 form)."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = x.copy()
    r = dinv * (f - A @ x)
    d = r / theta
    for i in range(degree):
        x = x + d
        if i == degree - 1:
            break
        r = dinv * (f - A @ x)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x


def coarse_inverse(A):
    M = A.toarray() if hasattr(A, "toarray") else np.array(A, dtype=float)
    inactive = ~np.any(M != 0, axis=1)
    M[inactive, inactive] = 1.0
    L = np.linalg.cholesky(M)
    Linv = np.linalg.inv(L)
    Minv = Linv.T @ Linv
    Minv[inactive, :] = 0.0
    Minv[:, inactive] = 0.0
    return Minv


@dataclass
class Level:
    A: sp.csr_matrix
    bs: int
    dinv: np.ndarray = None
    lam: float = 0.0
    P: sp.csr_matrix = None
    R: sp.csr_matrix = None
    agg: np.ndarray = None
    n_agg: int = 0
    degree: int = 2


@dataclass
class Hierarchy:
    levels: list
    coarse_inv: np.ndarray
    params: dict = field(default_factory=dict)


DEFAULTS = dict(theta=0.02, theta_scale=0.5, degree=2, cheb_lo=0.1, cheb_hi=1.1, eig_steps=10,
                coarse_max_dofs=2000, coarse_min_dofs=500, aggressive_levels=1, small_level_dofs=0,
                small_level_degree=16, max_levels=10, droptol=1e-10)


def aggregate_level(nbrs, level, k, coarse_min_dofs, aggressive_levels=99):
    """Distance-2 aggregation on the first `aggressive_levels` levels (distance-1
    after), redone with distance-1 roots when it would leave fewer than
    coarse_min_dofs coarse DOFs (k per aggregate): the paper asks for fast
    coarsening but also finds a larger coarsest grid more robust."""
    if level >= aggressive_levels:
        agg, n_agg, _ = mis2_aggregate(nbrs, level, distance=1)
        return agg, n_agg
    agg, n_agg, _ = mis2_aggregate(nbrs, level)
    if coarse_min_dofs and n_agg * k < coarse_min_dofs:
        agg, n_agg, _ = mis2_aggregate(nbrs, level, distance=1)
    return agg, n_agg


def setup(A, B, bs=3, **kw):
    """Build the SA-AMG hierarchy from A (CSR, n*bs square) and near-nullspace B."""
    prm = dict(DEFAULTS)
    prm.update(kw)
    levels = []
    A = A.tocsr()
    for lev in range(prm["max_levels"]):
        L = Level(A=A, bs=bs, dinv=point_dinv(A))
        L.lam = lanczos_lambda_max(A, prm["eig_steps"], lev)
        levels.append(L)
        if A.shape[0] <= prm["coarse_max_dofs"] or lev == prm["max_levels"] - 1:
            break
        nbrs = strength_graph(A, bs, prm["theta"] * prm["theta_scale"] ** lev)
        agg, n_agg = aggregate_level(nbrs, lev, B.shape[1], prm["coarse_min_dofs"],
                                     prm["aggressive_levels"])
        if n_agg == 0 or n_agg >= A.shape[0] // bs:
            break
        Pt, Bc = tentative_prolongator(agg, n_agg, B, bs, prm["droptol"])
        P = smooth_prolongator(A, Pt, L.lam)
        Ac, R = galerkin(A, P)
        L.P, L.R, L.agg, L.n_agg = P, R, agg, n_agg
        A, B, bs = Ac, Bc, B.shape[1]
    # small (cheap) smoothed levels get a higher-degree Chebyshev: with an
    # aggressively coarsened coarsest grid they must nearly solve their own problem
    for L in levels[:-1]:
        small = L.A.shape[0] <= prm["small_level_dofs"]
        L.degree = prm["small_level_degree"] if small else prm["degree"]
    return Hierarchy(levels=levels, coarse_inv=coarse_inverse(levels[-1].A), params=prm)


def vcycle(H, b, lev=0):
    L = H.levels[lev]
    if lev == len(H.levels) - 1:
        return H.coarse_inv @ b
    p = H.params
    lo, hi = p["cheb_lo"] * L.lam, p["cheb_hi"] * L.lam
    x = chebyshev(L.A, L.dinv, b, np.zeros_like(b), lo, hi, L.degree)
    r = b - L.A @ x
    x = x + L.P @ vcycle(H, L.R @ r, lev + 1)
    return chebyshev(L.A, L.dinv, b, x, lo, hi, L.degree)


def pcg(A, b, H, rtol=1e-8, atol=0.0, max_iter=1000, x0=None):
    """AMG-preconditioned CG; returns (x, iterations, ||b - Ax|| / ||b||)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    nb = np.linalg.norm(b)
    tol = max(rtol * nb, atol)
    it = 0
    if np.linalg.norm(r) > tol:
        z = vcycle(H, r)
        p = z.copy()
        rz = r @ z
        while it < max_iter:
            q = A @ p
            a = rz / (p @ q)
            x += a * p
            r -= a * q
            it += 1
            if np.linalg.norm(r) <= tol:
                break
            z = vcycle(H, r)
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
    return x, it, float(np.linalg.norm(b - A @ x) / (nb if nb > 0 else 1.0))


def solve(problem_K, f, coords, dirichlet_mask, rotations=True, rtol=1e-8, **kw):
    """Convenience: setup with rigid-body modes and run PCG."""
    from .fem import rigid_body_modes
    B = rigid_body_modes(coords, dirichlet_mask, rotations)
    H = setup(problem_K, B, 3, **kw)
    x, it, rel = pcg(problem_K, f, H, rtol=rtol)
    return x, it, rel, H
