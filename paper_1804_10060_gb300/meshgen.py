"""Seeded synthetic inputs for the thermoelastic solve (meshes, fields, masks).

This module builds *inputs* only: node coordinates, tetrahedral cells, per-cell
material ids, nodal temperatures, nodal body forces and Dirichlet masks.  It
holds none of the method's arithmetic (no element integrals, no near-nullspace,
no solver), so both the CUDA path and the CPU oracle may consume what it makes.

The paper's turbocharger and steam-turbine meshes are proprietary; these
generators stand in for them with the same structure: multi-material bodies,
a thermal-strain load, rotating bladed parts, P1 and P2 Lagrange tetrahedra
and clamped boundaries (Sec. 4-5 of the paper).

Conventions
-----------
* ``coords``: float64 ``[n_nodes, 3]``.
* ``cells``: int32 ``[n_cells, 4]`` (P1) or ``[n_cells, 10]`` (P2).  P2 local
  order: vertices 0-3, then mid-edge nodes of edges (01, 02, 03, 12, 13, 23).
* All cells are positively oriented: det[x1-x0, x2-x0, x3-x0] > 0.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


@dataclass
class Problem:
    """One thermoelastic load case on one mesh (all host arrays)."""

    name: str
    coords: np.ndarray            # [n,3] f64
    cells: np.ndarray             # [m,4|10] i32
    cell_material: np.ndarray     # [m] i32
    mat_props: np.ndarray         # [n_mat,3] f64: E, nu, alpha
    T: np.ndarray | None          # [n] f64 nodal temperature
    T_ref: float
    body_force: np.ndarray | None  # [n,3] f64 nodal body force density
    dirichlet_mask: np.ndarray    # [n] u8
    u_dirichlet: np.ndarray | None  # [n,3] f64
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    @property
    def nodes_per_cell(self) -> int:
        return int(self.cells.shape[1])


# ----------------------------------------------------------------------------
# Structured boxes split into Kuhn (Freudenthal) tetrahedra
# ----------------------------------------------------------------------------

def box_kuhn(nx: int, ny: int, nz: int, lx: float = 1.0, ly: float = 1.0,
             lz: float = 1.0, origin=(0.0, 0.0, 0.0)):
    """Box [0,lx]x[0,ly]x[0,lz] with nx*ny*nz hexes, each split into 6 tets.

    Every hex is cut along its main diagonal into the 6 Kuhn tetrahedra (one
    per permutation of the axes), which conform across neighbouring hexes.
    Nodes are numbered lexicographically (x fastest), which keeps matrix
    bandwidth small.  Returns (coords [n,3] f64, cells [6*nx*ny*nz, 4] i32).
    """
    xs = origin[0] + np.linspace(0.0, lx, nx + 1)
    ys = origin[1] + np.linspace(0.0, ly, ny + 1)
    zs = origin[2] + np.linspace(0.0, lz, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)

    sx, sy, sz = 1, nx + 1, (nx + 1) * (ny + 1)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    v0 = (i * sx + j * sy + k * sz).ravel().astype(np.int64)
    step = (sx, sy, sz)
    tets = []
    for perm in itertools.permutations(range(3)):
        a, b, c = perm
        p1 = v0 + step[a]
        p2 = p1 + step[b]
        p3 = p2 + step[c]
        # sign of the permutation decides the orientation; swap to keep det > 0
        inversions = sum(1 for s in range(3) for t in range(s + 1, 3) if perm[s] > perm[t])
        if inversions % 2 == 0:
            tets.append(np.stack([v0, p1, p2, p3], axis=1))
        else:
            tets.append(np.stack([v0, p1, p3, p2], axis=1))
    # hex-major cell order (the 6 tets of one hex are adjacent in memory)
    cells = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return coords, cells


def jitter_interior(coords: np.ndarray, h: float, amount: float, seed: int,
                    fixed_mask: np.ndarray | None = None) -> np.ndarray:
    """Move interior nodes by a seeded uniform offset of at most amount*h per axis."""
    rng = np.random.default_rng(seed)
    lo, hi = coords.min(axis=0), coords.max(axis=0)
    on_bnd = np.any(np.isclose(coords, lo) | np.isclose(coords, hi), axis=1)
    if fixed_mask is not None:
        on_bnd |= fixed_mask.astype(bool)
    d = rng.uniform(-amount * h, amount * h, size=coords.shape)
    out = coords.copy()
    out[~on_bnd] += d[~on_bnd]
    return out


# ----------------------------------------------------------------------------
# P2 meshes: add one node at the midpoint of every edge
# ----------------------------------------------------------------------------

def p1_to_p2(coords: np.ndarray, cells: np.ndarray):
    """Quadratic (10-node) tets from linear ones by adding mid-edge nodes.

    Returns (coords2, cells2, n_vertices).  Edge nodes are numbered after the
    vertex nodes in order of their (sorted) vertex pair.
    """
    n = coords.shape[0]
    c = cells.astype(np.int64)
    pairs = np.stack([np.stack([c[:, a], c[:, b]], axis=1) for a, b in P2_EDGES], axis=1)
    pairs = np.sort(pairs, axis=2).reshape(-1, 2)
    keys = pairs[:, 0] * n + pairs[:, 1]
    uniq, inv = np.unique(keys, return_inverse=True)
    ea, eb = uniq // n, uniq % n
    mid = 0.5 * (coords[ea] + coords[eb])
    coords2 = np.concatenate([coords, mid], axis=0)
    edge_nodes = (n + inv).reshape(-1, 6)
    cells2 = np.concatenate([c, edge_nodes], axis=1).astype(np.int32)
    return coords2, cells2, n


def renumber_nodes(coords: np.ndarray, cells: np.ndarray, order: np.ndarray):
    """Apply a node permutation: new node k is old node order[k]."""
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size, dtype=order.dtype)
    return coords[order], inv[cells].astype(np.int32), inv


def spatial_order(coords: np.ndarray, h: float) -> np.ndarray:
    """Lexicographic (z, y, x) order on a lattice of spacing h/2.

    Used to interleave P2 edge nodes with vertices so that a block row's
    neighbours stay close in memory.
    """
    q = np.round((coords - coords.min(axis=0)) / (0.5 * h)).astype(np.int64)
    return np.lexsort((q[:, 0], q[:, 1], q[:, 2]))


# ----------------------------------------------------------------------------
# Fields
# ----------------------------------------------------------------------------

def fourier_temperature(coords: np.ndarray, seed: int, n_modes: int = 8,
                        scale=(4.0, 1.0, 1.0)) -> np.ndarray:
    """Smooth random field: mean of n_modes cosines, so max |T| <= 1.

    T(x) = (1/n_modes) * sum_m cos(pi * k_m . (x/scale) + phi_m), with integer
    wave vectors k_m drawn from {0..3}^3 without the zero vector and phases
    uniform on [0, 2pi), all from numpy default_rng(seed): first the n_modes
    wave vectors (redrawing a zero vector), then the n_modes phases.
    """
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(0, 4, size=3)
        if np.any(k != 0):
            ks.append(k)
    phis = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    xt = coords / np.asarray(scale, dtype=np.float64)
    T = np.zeros(coords.shape[0])
    for k, ph in zip(ks, phis):
        T += np.cos(np.pi * (xt @ k.astype(np.float64)) + ph)
    return T / n_modes


def cell_centroids(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    return coords[cells[:, :4]].mean(axis=1)


# ----------------------------------------------------------------------------
# The named workloads
# ----------------------------------------------------------------------------

def unit_cube_problem(n: int = 10, degree: int = 1) -> Problem:
    """Unit cube, n^3 hexes -> 6 tets each; E=1, nu=0.3, alpha=1e-3.

    T = sin(pi x) cos(pi y) (1 + z), T_ref = 0, clamped on x = 0, traction
    free elsewhere, no body force.  n=10, degree=1 gives 6,000 tets, 1,331
    nodes and 3,993 DOF.
    """
    coords, cells = box_kuhn(n, n, n)
    if degree == 2:
        coords, cells, _ = p1_to_p2(coords, cells)
        coords, cells, _ = renumber_nodes(coords, cells, spatial_order(coords, 1.0 / n))
    x, y, z = coords.T
    T = np.sin(np.pi * x) * np.cos(np.pi * y) * (1.0 + z)
    mask = (x <= 1e-12).astype(np.uint8)
    return Problem(
        name=f"cube{n}_p{degree}", coords=coords, cells=cells,
        cell_material=np.zeros(cells.shape[0], np.int32),
        mat_props=np.array([[1.0, 0.3, 1e-3]]), T=T, T_ref=0.0, body_force=None,
        dirichlet_mask=mask, u_dirichlet=None,
        meta={"hexes": (n, n, n), "degree": degree})


def slab_box_problem(nx: int = 256, ny: int = 64, nz: int = 64, seed: int = 2024,
                     degree: int = 1, slab_width: float = 0.5) -> Problem:
    """Box [0,4]x[0,1]^2, two materials in alternating x-slabs, random T.

    Slab index floor(x_c / slab_width) mod 2 of the cell centroid selects E=1
    (even) or E=10 (odd); nu=0.3, alpha=1e-3 for both.  T is the seeded
    8-mode Fourier field of amplitude 1 on x~=(x/4, y, z), T_ref = 0.
    Clamped on x=0.  256x64x64 gives 6,291,456 tets, 1,085,825 nodes and
    3,257,475 DOF.
    """
    coords, cells = box_kuhn(nx, ny, nz, 4.0, 1.0, 1.0)
    if degree == 2:
        coords, cells, _ = p1_to_p2(coords, cells)
        coords, cells, _ = renumber_nodes(coords, cells,
                                          spatial_order(coords, min(4.0 / nx, 1.0 / ny, 1.0 / nz)))
    xc = cell_centroids(coords, cells)[:, 0]
    mat = (np.floor(xc / slab_width).astype(np.int64) % 2).astype(np.int32)
    T = fourier_temperature(coords, seed)
    mask = (coords[:, 0] <= 1e-12).astype(np.uint8)
    return Problem(
        name=f"slabbox{nx}x{ny}x{nz}_p{degree}", coords=coords, cells=cells,
        cell_material=mat, mat_props=np.array([[1.0, 0.3, 1e-3], [10.0, 0.3, 1e-3]]),
        T=T, T_ref=0.0, body_force=None, dirichlet_mask=mask, u_dirichlet=None,
        meta={"hexes": (nx, ny, nz), "degree": degree, "seed": seed})


def bladed_disc_problem(n_r: int = 16, n_theta_per_blade: int = 8, n_z: int = 2,
                        n_blades: int = 48, n_r_blade: int = 6, degree: int = 2,
                        seed: int = 7, omega: float = 1.0, rho: float = 1.0,
                        jitter: float = 0.15, blade_fraction: float = 0.375) -> Problem:
    """Synthetic turbine disc: annulus r in [0.2, 1], thickness 0.1, plus blades.

    A structured polar hex grid (n_r radial, n_blades*n_theta_per_blade
    angular, n_z axial layers) covers the annulus.  In every blade pitch the
    first round(blade_fraction * n_theta_per_blade) (at least 1) angular
    cells are extruded radially from r=1 to r=1.3 with n_r_blade layers
    (straight-sided blades; 3/8 of the pitch, about 0.05 wide at r=1, for
    48 blades and 8 cells per pitch).  Meshes of one geometry at several
    resolutions need blade_fraction * n_theta_per_blade to be an integer for
    each of them.  Hexes are split into
    Kuhn tets, interior nodes jittered by up to jitter*h (seeded), then made
    P2 if degree == 2.  T = 300 + 500 r^2 + 10 F(x), F the 8-mode Fourier
    field of fourier_temperature with seed + 1 on the box [-1.3, 1.3]^2 x
    [-0.05, 0.05] (scale (2.6, 2.6, 0.1)): a seeded perturbation that does
    not depend on the mesh, so refined meshes discretise the same problem.
    T_ref = 300.  Centrifugal body force
    rho omega^2 (x, y, 0) about z.  Clamped at the bore r = 0.2.
    Material: E=1, nu=0.3, alpha=1e-5.
    """
    n_t = n_blades * n_theta_per_blade
    r_in, r_out, r_tip, thick = 0.2, 1.0, 1.3, 0.1
    # geometric radial spacing: dr / (r dtheta) = ln(r_out / r_in) n_t / (2 pi n_r)
    # is the same for every ring, and 1 (square cells in plan view) for the
    # n_r that isotropic_disc_kwargs picks
    r_nodes = np.concatenate([np.geomspace(r_in, r_out, n_r + 1),
                              np.geomspace(r_out, r_tip, n_r_blade + 1)[1:]])
    n_rr = r_nodes.size
    z_nodes = np.linspace(-0.5 * thick, 0.5 * thick, n_z + 1)
    t_nodes = np.arange(n_t) * (2.0 * np.pi / n_t)
    # node lattice (z, theta, r) -> id; theta periodic
    idx = -np.ones((n_z + 1, n_t, n_rr), np.int64)
    # which hexes exist: annulus all; blade layers only for blade columns
    blade_cols = min(n_theta_per_blade, max(1, int(round(blade_fraction * n_theta_per_blade))))
    in_blade_col = (np.arange(n_t) % n_theta_per_blade) < blade_cols
    hex_exists = np.zeros((n_z, n_t, n_rr - 1), bool)
    hex_exists[:, :, :n_r] = True
    hex_exists[:, in_blade_col, n_r:] = True
    node_used = np.zeros((n_z + 1, n_t, n_rr), bool)
    for dz in (0, 1):
        for dt in (0, 1):
            for dr in (0, 1):
                sl = hex_exists
                zz, tt, rr = np.nonzero(sl)
                node_used[zz + dz, (tt + dt) % n_t, rr + dr] = True
    idx[node_used] = np.arange(node_used.sum())
    zz, tt, rr = np.nonzero(node_used)
    R = r_nodes[rr]
    coords = np.stack([R * np.cos(t_nodes[tt]), R * np.sin(t_nodes[tt]), z_nodes[zz]], axis=1)
    # hexes -> Kuhn tets in local (r, theta, z) lattice axes
    hz, ht, hr = np.nonzero(hex_exists)

    def corner(dr, dt, dz):
        return idx[hz + dz, (ht + dt) % n_t, hr + dr]

    tets = []
    for perm in itertools.permutations(range(3)):
        off = [0, 0, 0]
        verts = [corner(*off)]
        for ax in perm:
            off[ax] += 1
            verts.append(corner(*off))
        tets.append(np.stack(verts, axis=1))
    cells = np.stack(tets, axis=1).reshape(-1, 4)
    # orient positively
    x = coords[cells]
    det = np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])
    neg = det < 0
    cells[neg] = cells[neg][:, [0, 1, 3, 2]]
    # seeded jitter of interior nodes (not on the bore, rim faces or blade surfaces)
    rng = np.random.default_rng(seed)
    h = min(thick / n_z, r_nodes[1] - r_nodes[0], 2 * np.pi * r_in / n_t)
    cnt = np.zeros(coords.shape[0], np.int64)
    np.add.at(cnt, cells.ravel(), 1)
    # interior nodes of a Kuhn lattice touch 24 tets
    interior = cnt == 24
    d = rng.uniform(-jitter * h, jitter * h, size=coords.shape)
    coords = coords.copy()
    coords[interior] += d[interior]
    cells = cells.astype(np.int32)
    if degree == 2:
        coords, cells, _ = p1_to_p2(coords, cells)
    # locality: order by (theta sector, z, r)
    th = np.mod(np.arctan2(coords[:, 1], coords[:, 0]), 2 * np.pi)
    rad = np.hypot(coords[:, 0], coords[:, 1])
    qt = np.floor(th / (2 * np.pi / n_t) * 2 + 0.25).astype(np.int64)
    qr = np.round(rad / (0.5 * h)).astype(np.int64)
    qz = np.round((coords[:, 2] + 0.5 * thick) / (0.25 * h)).astype(np.int64)
    order = np.lexsort((qr, qz, qt))
    coords, cells, _ = renumber_nodes(coords, cells, order)
    rad = np.hypot(coords[:, 0], coords[:, 1])
    # temperature: radial profile plus a smooth seeded perturbation
    T = 300.0 + 500.0 * rad ** 2 + 10.0 * fourier_temperature(coords, seed + 1, scale=(2.6, 2.6, 0.1))
    body = rho * omega ** 2 * np.stack([coords[:, 0], coords[:, 1], np.zeros(coords.shape[0])], axis=1)
    mask = (rad <= r_in + 1e-9).astype(np.uint8)
    return Problem(
        name=f"disc{n_blades}b_p{degree}", coords=coords, cells=cells,
        cell_material=np.zeros(cells.shape[0], np.int32),
        mat_props=np.array([[1.0, 0.3, 1e-5]]), T=T, T_ref=300.0, body_force=body,
        dirichlet_mask=mask, u_dirichlet=None,
        meta={"n_r": n_r, "n_theta": n_t, "n_z": n_z, "degree": degree, "seed": seed,
              "omega": omega})


def isotropic_disc_kwargs(n_blades: int = 48, n_theta_per_blade: int = 8, degree: int = 2, **extra) -> dict:
    """bladed_disc_problem arguments whose cells are near-isotropic.

    With dtheta = 2 pi / (n_blades n_theta_per_blade): n_r = ln(1 / 0.2) / dtheta
    rings on the annulus and n_r_blade = ln(1.3) / dtheta on the blades make
    dr = r dtheta everywhere; n_z = 0.1 / (0.6 dtheta) layers make dz equal
    to r dtheta at the mid radius r = 0.6 (at least 2 layers).
    """
    dth = 2.0 * np.pi / (n_blades * n_theta_per_blade)
    return dict(n_r=max(1, int(round(np.log(5.0) / dth))), n_theta_per_blade=n_theta_per_blade,
                n_z=max(2, int(round(0.1 / (0.6 * dth)))), n_blades=n_blades,
                n_r_blade=max(1, int(round(np.log(1.3) / dth))), degree=degree, **extra)


def load_case(pb: Problem, seed: int) -> tuple[np.ndarray, np.ndarray, float]:
    """One more load case on pb's mesh: (T[n], body force [n,3], omega).

    omega ~ U[0, 2] from numpy default_rng(seed); body force rho omega^2 (x, y, 0)
    with rho = 1 (rotation about z).  Temperature: for the boxes the 8-mode
    Fourier field of amplitude 1 with this seed (T_ref = 0); for the discs
    the mesh's radial profile plus 100 times that field on coordinates scaled
    by the disc's extent.
    """
    rng = np.random.default_rng(seed)
    omega = float(rng.uniform(0.0, 2.0))
    body = omega * omega * np.stack([pb.coords[:, 0], pb.coords[:, 1], np.zeros(pb.n_nodes)], axis=1)
    if pb.name.startswith("disc"):
        ext = np.ptp(pb.coords, axis=0)
        T = pb.T + 100.0 * fourier_temperature(pb.coords, seed, scale=np.where(ext > 0, ext, 1.0))
    else:
        T = fourier_temperature(pb.coords, seed)
    return T, body, omega


# 64 load cases on 8 meshes of uneven size (45k to 2M DOF), P1 and P2, boxes and
# bladed discs (near-isotropic cells, see isotropic_disc_kwargs; blades half a pitch wide)
BATCH_MESHES = (
    ("slab_box", dict(nx=64, ny=16, nz=16, degree=1)),                  # 56,355 DOF
    ("slab_box", dict(nx=32, ny=8, nz=8, degree=2)),                    # 56,355
    ("disc", dict(n_r=29, n_theta_per_blade=4, n_z=3, n_blades=28, n_r_blade=5, degree=1,
                  blade_fraction=0.5)),                                 # 45,360
    ("disc", dict(n_r=25, n_theta_per_blade=4, n_z=3, n_blades=24, n_r_blade=4, degree=2,
                  blade_fraction=0.5)),                                 # 225,792
    ("slab_box", dict(nx=128, ny=32, nz=32, degree=1)),                 # 421,443
    ("slab_box", dict(nx=96, ny=24, nz=24, degree=2)),                  # 1,390,179
    ("disc", dict(n_r=49, n_theta_per_blade=4, n_z=5, n_blades=48, n_r_blade=8, degree=2,
                  blade_fraction=0.5)),                                 # 1,381,248
    ("slab_box", dict(nx=216, ny=54, nz=54, degree=1)),                 # 1,969,275
)


def batch_problems(meshes=BATCH_MESHES, cases_per_mesh: int = 8, seed0: int = 100):
    """[(problem, [(T, body, omega) per case])]: case k of mesh i uses seed seed0 + i*cases_per_mesh + k."""
    out = []
    for i, (kind, kw) in enumerate(meshes):
        pb = slab_box_problem(**kw) if kind == "slab_box" else bladed_disc_problem(**kw)
        cases = [load_case(pb, seed0 + i * cases_per_mesh + k) for k in range(cases_per_mesh)]
        out.append((pb, cases))
    return out


def clamp_distance(pb: Problem) -> np.ndarray:
    """Distance of every node to the clamped boundary of a named workload.

    Geometry known to the generator: the disc is clamped at the bore r = 0.2,
    the boxes at x = 0.  Used as an input feature of the learned guess.
    """
    if pb.name.startswith("disc"):
        return np.hypot(pb.coords[:, 0], pb.coords[:, 1]) - 0.2
    return pb.coords[:, 0] - pb.coords[:, 0].min()


def mesh_quality(coords: np.ndarray, cells: np.ndarray):
    """Minimum volume and minimum dihedral angle (degrees) over the vertex tets."""
    x = coords[cells[:, :4]]
    e1, e2, e3 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]
    vol = np.einsum("ij,ij->i", np.cross(e1, e2), e3) / 6.0
    faces = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))
    normals = []
    for f in faces:
        p = x[:, list(f)]
        nrm = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
        # point the normal outward (away from the opposite vertex)
        opp = x[:, [k for k in range(4) if k not in f][0]]
        s = np.sign(np.einsum("ij,ij->i", nrm, p[:, 0] - opp))
        normals.append(nrm * s[:, None] / np.linalg.norm(nrm, axis=1)[:, None])
    ang = []
    for a in range(4):
        for b in range(a + 1, 4):
            c = -np.einsum("ij,ij->i", normals[a], normals[b])
            ang.append(np.degrees(np.arccos(np.clip(c, -1, 1))))
    return float(vol.min()), float(np.min(ang))


# ----------------------------------------------------------------------------
# Boundary faces and thermal inputs
# ----------------------------------------------------------------------------

# Local vertices of the four faces of a tet (face k is opposite vertex k).
TET_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


def boundary_faces(cells: np.ndarray) -> np.ndarray:
    """Faces that belong to exactly one cell, as node ids.

    P1 cells give [n_f, 3] (three vertices); P2 cells give [n_f, 6]: the three
    vertices (v0, v1, v2) then the mid-edge nodes of edges v0v1, v1v2, v2v0.
    Faces come out in the order of their sorted vertex triples (deterministic).
    """
    cells = np.asarray(cells)
    p2 = cells.shape[1] == 10
    edge_slot = {e: 4 + k for k, e in enumerate(P2_EDGES)}
    tri, full = [], []
    for f in TET_FACES:
        v = cells[:, list(f)]
        tri.append(v)
        if p2:
            def mid(a, b):
                return cells[:, edge_slot[(min(a, b), max(a, b))]]
            full.append(np.stack([v[:, 0], v[:, 1], v[:, 2], mid(f[0], f[1]), mid(f[1], f[2]),
                                  mid(f[2], f[0])], axis=1))
        else:
            full.append(v)
    tri = np.concatenate(tri)
    full = np.concatenate(full)
    key = np.sort(tri, axis=1)
    _, first, counts = np.unique(key, axis=0, return_index=True, return_counts=True)
    keep = first[counts == 1]
    return full[np.sort(keep)].astype(np.int32)


@dataclass
class ThermalProblem:
    """Thermal data on a mesh (host arrays): materials, Robin faces, fields.

    thermal_props[n_mat, 5] = (rho, c0, c1, k0, k1): density, specific heat
    c_v(T) = c0 + c1 T and conductivity kappa(T) = k0 + k1 T.  faces are the
    Robin faces (boundary_faces layout) with beta[n_f] per face and the
    exterior temperature T_bc[n] given at the nodes.  dirichlet_mask / T_dirichlet
    optionally fix nodal temperatures.
    """

    coords: np.ndarray
    cells: np.ndarray
    cell_material: np.ndarray
    thermal_props: np.ndarray
    faces: np.ndarray
    beta: np.ndarray
    T_bc: np.ndarray
    dirichlet_mask: np.ndarray | None = None
    T_dirichlet: np.ndarray | None = None

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])


def disc_thermal_problem(pb: Problem, t: float = 0.0, seed: int = 11) -> ThermalProblem:
    """Heating of a bladed disc (inputs for the transient thermal solve).

    One material (rho 1, c_v = 1 + 5e-4 T, kappa = 0.05 (1 + 1e-3 T)); Robin
    faces: the blade and rim faces (r > 0.995) see hot gas, T_bc = 300 + 600
    (1 - exp(-t / 0.5)) + 20 F(x) with a seeded smooth field F, coefficient
    beta = -5; the bore faces (r < 0.2005) are cooled, T_bc = 300,
    beta = -1; the other faces are adiabatic (not listed).  beta < 0 is the
    sign of a cooling film in the paper's boundary condition
    kappa grad T . n = beta (T - T_bc).
    """
    faces = boundary_faces(pb.cells)
    xc = pb.coords[faces[:, :3]].mean(axis=1)
    r = np.hypot(xc[:, 0], xc[:, 1])
    hot = r > 0.995
    bore = r < 0.2005
    sel = hot | bore
    beta = np.where(hot[sel], -5.0, -1.0)
    rad = np.hypot(pb.coords[:, 0], pb.coords[:, 1])
    ext = np.ptp(pb.coords, axis=0)
    F = fourier_temperature(pb.coords, seed, scale=np.where(ext > 0, ext, 1.0))
    T_bc = np.where(rad > 0.5, 300.0 + 600.0 * (1.0 - np.exp(-t / 0.5)) + 20.0 * F, 300.0)
    props = np.array([[1.0, 1.0, 5e-4, 0.05, 5e-5]])
    return ThermalProblem(pb.coords, pb.cells, np.zeros(pb.n_cells, np.int32), props, faces[sel],
                          beta, T_bc)


# ----------------------------------------------------------------------------
# Unstructured meshes: Delaunay tetrahedralisations of seeded point sets
# ----------------------------------------------------------------------------

def delaunay_box(n: int = 12, lx: float = 2.0, ly: float = 1.0, lz: float = 1.0, seed: int = 1,
                 jitter: float = 0.35, hub: int = 0):
    """Unstructured tets of the box [0,lx]x[0,ly]x[0,lz] (Delaunay of seeded points).

    Points: a lattice of spacing h = ly / n, every point moved by a seeded
    uniform offset of up to jitter*h along the box directions it is free in
    (points on a face stay on it, edge and corner points stay put), so the
    valences and cell shapes are irregular.  hub > 0 adds, around the box
    centre, a point ringed by `hub` points on a sphere of radius h/2 (seeded,
    quasi-uniform): the centre touches about 2 hub cells, a node of very high
    valence.  Cells of (near) zero volume from co-planar hull points are
    dropped; every cell is oriented positively.  Returns (coords, cells,
    quality) with quality = dict(min_volume, min_dihedral_deg, max_valence).
    """
    from scipy.spatial import Delaunay
    h = ly / n
    nx, ny, nz = max(1, round(lx / h)), n, max(1, round(lz / h))
    g = np.stack(np.meshgrid(np.linspace(0, lx, nx + 1), np.linspace(0, ly, ny + 1), np.linspace(0, lz, nz + 1),
                             indexing="ij"), axis=-1).reshape(-1, 3)
    rng = np.random.default_rng(seed)
    L = np.array([lx, ly, lz])
    free = (g > 1e-12) & (g < L - 1e-12)
    g = g + free * rng.uniform(-jitter * h, jitter * h, g.shape)
    pts = [g]
    if hub:
        c = L / 2.0
        far = np.linalg.norm(g - c, axis=1) > 0.75 * h
        pts = [g[far], c[None]]
        k = np.arange(hub) + 0.5                                 # Fibonacci sphere
        phi = np.arccos(1.0 - 2.0 * k / hub)
        th = np.pi * (1.0 + 5 ** 0.5) * k + rng.uniform(0, 2 * np.pi)
        pts.append(c + 0.5 * h * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1))
    coords = np.concatenate(pts)
    cells = Delaunay(coords, qhull_options="Qbb Qc Qz Q12").simplices.astype(np.int64)
    x = coords[cells]
    vol = np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0]) / 6.0
    keep = np.abs(vol) > 1e-10 * h ** 3
    cells, vol = cells[keep], vol[keep]
    neg = vol < 0
    cells[neg] = cells[neg][:, [0, 1, 3, 2]]
    used = np.unique(cells)
    remap = -np.ones(coords.shape[0], np.int64)
    remap[used] = np.arange(used.size)
    coords, cells = coords[used], remap[cells]
    order = spatial_order(coords, h)
    coords, cells, _ = renumber_nodes(coords, cells.astype(np.int32), order)
    mv, md = mesh_quality(coords, cells)
    val = np.bincount(cells.ravel(), minlength=coords.shape[0])
    q = dict(min_volume=mv, min_dihedral_deg=md, max_valence=int(val.max()))
    return coords, cells.astype(np.int32), q


def delaunay_box_problem(n: int = 12, degree: int = 1, seed: int = 1, hub: int = 0) -> Problem:
    """The two-material box load case (slab_box_problem's materials, temperature
    recipe and clamp at x = 0) on an unstructured Delaunay mesh of [0,2]x[0,1]^2."""
    coords, cells, q = delaunay_box(n, seed=seed, hub=hub)
    if degree == 2:
        coords, cells, _ = p1_to_p2(coords, cells)
    xc = cell_centroids(coords, cells)
    mat = (np.floor(xc[:, 0] / 0.5).astype(np.int64) % 2).astype(np.int32)
    T = fourier_temperature(coords, 2024, scale=(2.0, 1.0, 1.0))
    mask = (coords[:, 0] <= 1e-12).astype(np.uint8)
    return Problem(name=f"delaunay_p{degree}", coords=coords, cells=cells, cell_material=mat,
                   mat_props=np.array([[1.0, 0.3, 1e-3], [10.0, 0.3, 1e-3]]), T=T, T_ref=0.0, body_force=None,
                   dirichlet_mask=mask, u_dirichlet=None, meta=dict(q, n=n, seed=seed, hub=hub))
