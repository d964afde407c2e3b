"""Seeded synthetic inputs for the Lagrangian ADER-MOOD step (meshes, initial fields, BC tags).

This module is shared by the CPU oracle and the CUDA path and therefore holds none of the
scheme's arithmetic: it only places points, connects them into simplices, tags boundary
faces and evaluates the prescribed initial velocity / shear-modulus fields at the t=0
vertex average of each cell (the initial data of the problem, cf. the initialisation of the
test problems in Sect. "2D and 3D test problems").

The paper's meshes come from GMSH (Sect. "2D and 3D test problems") and are not available;
these generators stand in for them with the same element types and sizes:

* 2D: a jittered n x n point lattice on a rectangle, Delaunay-triangulated (Qhull through
  scipy), boundary points sliding along their side, corners fixed.
* 3D: a jittered box lattice split into Kuhn (Freudenthal) tetrahedra, 6 per cube.

Cells and nodes are renumbered along a Morton curve so that mesh neighbours are close in
memory (the caller orders; the library renumbers nothing).

Boundary-condition tags per boundary face: 0 free traction, 1 slip wall (symmetry plane),
2 clamped (symmetry point), following Appendix B of the paper.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

FREE, SLIP, CLAMPED, TRACTION, PRESSURE, VELOCITY, CONTACT = 0, 1, 2, 3, 4, 5, 6


@dataclass
class Mesh:
    dim: int
    x: np.ndarray          # [dim, n_nodes] float64 (SoA)
    c2n: np.ndarray        # [dim+1, n_cells] int32, positively oriented (SoA)
    bface: np.ndarray      # [dim, n_bfaces] int32 node ids of tagged boundary faces
    btag: np.ndarray       # [n_bfaces] int32 in {FREE, SLIP, CLAMPED, TRACTION, PRESSURE, VELOCITY}

    @property
    def n_nodes(self) -> int:
        return int(self.x.shape[1])

    @property
    def n_cells(self) -> int:
        return int(self.c2n.shape[1])


@dataclass
class Problem:
    """A mesh plus material and initial data: everything the step needs at t=0."""
    name: str
    mesh: Mesh
    rho0: float
    lam: float
    mu: np.ndarray          # [n_cells] shear modulus per cell
    v: np.ndarray           # [dim, n_cells] initial cell velocity
    cfl: float
    steps: int
    F: np.ndarray | None = None   # [dim*dim, n_cells] or None for F = I
    meta: dict = field(default_factory=dict)
    bcval: np.ndarray | None = None  # [dim, n_bfaces] boundary-face values (traction vector,
                                     # pressure in row 0, prescribed velocity) or None
    shear_a: float = -1.0            # a of the shear energy family; -1 neo-Hookean
    contact: tuple | None = None     # (planes [n][2 dim]: point, unit normal into the body; eps)
                                     # contact walls for faces tagged CONTACT
    stiffened_gas: tuple | None = None  # (gamma, p_inf, p0): stiffened-gas volumetric law


# ----------------------------------------------------------------------------- ordering
def _morton_keys(pts: np.ndarray, bits: int = 20) -> np.ndarray:
    """Morton (Z-order) key of each point (rows of pts, 2 or 3 columns)."""
    d = pts.shape[1]
    lo = pts.min(axis=0)
    span = np.maximum(pts.max(axis=0) - lo, 1e-300)
    q = np.floor((pts - lo) / span * ((1 << bits) - 1)).astype(np.uint64)
    key = np.zeros(pts.shape[0], dtype=np.uint64)
    for b in range(bits):
        for a in range(d):
            key |= ((q[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(b * d + a)
    return key


def _renumber(x_rows: np.ndarray, cells: np.ndarray):
    """Morton-order nodes and cells. x_rows [np, d], cells [nc, d+1]."""
    node_perm = np.argsort(_morton_keys(x_rows), kind="stable")
    inv = np.empty_like(node_perm)
    inv[node_perm] = np.arange(node_perm.size)
    x_rows = x_rows[node_perm]
    cells = inv[cells]
    cent = x_rows[cells].mean(axis=1)
    cell_perm = np.argsort(_morton_keys(cent), kind="stable")
    return x_rows, cells[cell_perm]


def _orient(x_rows: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """Swap two vertices of negatively oriented simplices (pure connectivity fix-up)."""
    d = x_rows.shape[1]
    e = x_rows[cells[:, 1:]] - x_rows[cells[:, :1]]
    s = np.linalg.det(e) if d == 3 else e[:, 0, 0] * e[:, 1, 1] - e[:, 0, 1] * e[:, 1, 0]
    cells = cells.copy()
    neg = s < 0
    cells[neg, 1], cells[neg, 2] = cells[neg, 2].copy(), cells[neg, 1].copy()
    if np.any(np.abs(s) < 1e-14 * np.abs(s).max()):
        raise ValueError("degenerate simplex in generated mesh")
    return cells


def _boundary_faces(cells: np.ndarray) -> np.ndarray:
    """Faces (sorted node tuples) that belong to exactly one simplex."""
    nv = cells.shape[1]
    faces = np.concatenate([np.delete(cells, k, axis=1) for k in range(nv)], axis=0)
    faces = np.sort(faces, axis=1).astype(np.int64)
    n = int(cells.max()) + 1
    key = faces[:, 0]
    for a in range(1, faces.shape[1]):
        key = key * n + faces[:, a]   # n^3 < 2^63 for n < 2^21 nodes
    if n ** faces.shape[1] >= 2 ** 63:
        uniq, cnt = np.unique(faces, axis=0, return_counts=True)
        return uniq[cnt == 1]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    first = np.ones(ks.size, dtype=bool)
    first[1:] = ks[1:] != ks[:-1]
    last = np.ones(ks.size, dtype=bool)
    last[:-1] = ks[:-1] != ks[1:]
    single = order[first & last]
    out = faces[single]
    return out[np.lexsort(out.T[::-1])]


def _tag_faces(x_rows: np.ndarray, faces: np.ndarray, lo, hi, bc: dict) -> tuple[np.ndarray, np.ndarray]:
    """Tag each boundary face by the box side it lies on. bc maps side names
    ('x0','x1','y0','y1','z0','z1') to a face tag (missing = FREE)."""
    d = x_rows.shape[1]
    tags = np.full(faces.shape[0], FREE, dtype=np.int32)
    names = "xyz"
    fx = x_rows[faces]  # [nb, d, d]
    for a in range(d):
        for side, val in ((0, lo[a]), (1, hi[a])):
            on = np.all(fx[:, :, a] == val, axis=1)
            tags[on] = bc.get(f"{names[a]}{side}", FREE)
    keep = tags != FREE
    return faces[keep].astype(np.int32), tags[keep]


# ----------------------------------------------------------------------------- 2D
def tri_mesh(n: int, seed: int, lx: float = 1.0, ly: float = 1.0, jitter: float = 0.25,
             bc: dict | None = None, ny: int | None = None) -> Mesh:
    """Seeded jittered Delaunay triangulation of an n x ny lattice (ny = n by default) on
    [0,lx]x[0,ly].

    Interior points move by U(-jitter, jitter)*h per axis, side points only along their side,
    corners stay. 2(n-1)(ny-1) triangles (Euler's formula for a convex point set with
    2(n-1) + 2(ny-1) hull points), checked.
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    ny = n if ny is None else ny
    hx, hy = lx / (n - 1), ly / (ny - 1)
    i, j = np.meshgrid(np.arange(n), np.arange(ny), indexing="ij")
    x = i * hx
    y = j * hy
    jx = rng.uniform(-jitter, jitter, (n, ny)) * hx
    jy = rng.uniform(-jitter, jitter, (n, ny)) * hy
    jx[0, :] = 0.0
    jx[-1, :] = 0.0
    jy[:, 0] = 0.0
    jy[:, -1] = 0.0
    x = x + jx
    y = y + jy
    x[0, :] = 0.0
    x[-1, :] = lx
    y[:, 0] = 0.0
    y[:, -1] = ly
    pts = np.stack([x.ravel(), y.ravel()], axis=1)
    tri = Delaunay(pts)
    cells = tri.simplices.astype(np.int64)
    if cells.shape[0] != 2 * (n - 1) * (ny - 1) or len(tri.coplanar):
        raise ValueError("unexpected triangulation size")
    cells = _orient(pts, cells)
    pts, cells = _renumber(pts, cells)
    faces = _boundary_faces(cells)
    bf, tags = _tag_faces(pts, faces, (0.0, 0.0), (lx, ly), bc or {})
    return Mesh(2, np.ascontiguousarray(pts.T), np.ascontiguousarray(cells.T.astype(np.int32)),
                np.ascontiguousarray(bf.T), tags)


# ----------------------------------------------------------------------------- 3D
def tet_mesh(nx: int, ny: int, nz: int, seed: int, lx: float = 1.0, ly: float = 1.0,
             lz: float = 1.0, jitter: float = 0.1, bc: dict | None = None) -> Mesh:
    """Seeded jittered box lattice of nx*ny*nz cubes, each split into 6 Kuhn tetrahedra
    (all sharing the cube's (0,0,0)-(1,1,1) diagonal, so the split is conforming).
    Points on a side move only within that side; edge points along the edge; corners stay.
    """
    rng = np.random.default_rng(seed)
    L = np.array([lx, ly, lz])
    nn = np.array([nx, ny, nz])
    h = L / nn
    idx = np.stack(np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    pts = idx * h
    jit = rng.uniform(-jitter, jitter, pts.shape) * h
    for a in range(3):
        onb = (idx[:, a] == 0) | (idx[:, a] == nn[a])
        jit[onb, a] = 0.0
    pts = pts + jit
    for a in range(3):
        pts[idx[:, a] == 0, a] = 0.0
        pts[idx[:, a] == nn[a], a] = L[a]

    def nid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        path = [np.zeros(3, dtype=np.int64)]
        for a in perm:
            nxt = path[-1].copy()
            nxt[a] = 1
            path.append(nxt)
        tets.append(np.stack([nid(ci + p[0], cj + p[1], ck + p[2]) for p in path], axis=1))
    cells = np.concatenate(tets, axis=0).astype(np.int64)
    cells = _orient(pts, cells)
    pts, cells = _renumber(pts, cells)
    faces = _boundary_faces(cells)
    bf, tags = _tag_faces(pts, faces, (0.0, 0.0, 0.0), tuple(L), bc or {})
    return Mesh(3, np.ascontiguousarray(pts.T), np.ascontiguousarray(cells.T.astype(np.int32)),
                np.ascontiguousarray(bf.T), tags)


# ----------------------------------------------------------------------------- fields
def cell_points(mesh: Mesh) -> np.ndarray:
    """t=0 vertex average of each cell, [n_cells, dim]: where initial fields are sampled."""
    return mesh.x.T[mesh.c2n.T].mean(axis=1)


def gaussian_random_field(pts: np.ndarray, seed: int, n_modes: int = 64, corr: float = 0.15) -> np.ndarray:
    """Unit-variance stationary Gaussian random field from random Fourier modes."""
    rng = np.random.default_rng(seed)
    d = pts.shape[1]
    k = rng.normal(0.0, 1.0 / corr, (n_modes, d))
    ph = rng.uniform(0.0, 2 * math.pi, n_modes)
    return math.sqrt(2.0 / n_modes) * np.cos(pts @ k.T + ph).sum(axis=1)


# ----------------------------------------------------------------------------- named workloads
def plain2d(n: int = 40, seed: int = 1, steps: int = 200) -> Problem:
    """Unit square, jittered Delaunay of an n x n lattice, slip walls on all sides;
    rho0=1, mu=1, lambda=2; v0 = 1e-3 (sin(pi x) sin(pi y), cos(pi x) cos(pi y)); CFL 0.4."""
    m = tri_mesh(n, seed, bc={"x0": SLIP, "x1": SLIP, "y0": SLIP, "y1": SLIP})
    p = cell_points(m)
    v = 1e-3 * np.stack([np.sin(np.pi * p[:, 0]) * np.sin(np.pi * p[:, 1]),
                         np.cos(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1])])
    return Problem(f"plain2d_n{n}", m, 1.0, 2.0, np.full(m.n_cells, 1.0), v, 0.4, steps)


def side_values(m: Mesh, tag: int, value) -> np.ndarray:
    """[dim, n_bfaces] boundary-face values: value (a vector of dim entries; a pressure goes
    in entry 0) on the faces tagged tag, zero elsewhere."""
    out = np.zeros((m.dim, m.btag.size))
    out[:, m.btag == tag] = np.asarray(value, dtype=float)[:, None]
    return out


def piston2d(n: int = 40, seed: int = 6, V: float = 0.02, steps: int = 200) -> Problem:
    """Unit square at rest (rho0=1, mu=1, lambda=2) pushed by a piston: the side x = 0 has the
    prescribed normal velocity V e_x (Appendix B, velocity condition), y = 0 and y = 1 are slip
    walls, x = 1 is free; CFL 0.4."""
    m = tri_mesh(n, seed, bc={"x0": VELOCITY, "y0": SLIP, "y1": SLIP})
    return Problem(f"piston2d_n{n}", m, 1.0, 2.0, np.full(m.n_cells, 1.0), np.zeros((2, m.n_cells)), 0.4, steps,
                   bcval=side_values(m, VELOCITY, (V, 0.0)))


def rebound2d(n: int = 21, seed: int = 8, V: float = 0.1, gap: float = 0.02, steps: int = 400) -> Problem:
    """Unit square (rho0=1, mu=1, lambda=2) flying at v = (-V, 0) toward a rigid wall at
    x = -gap (Sect. "Boundary condition treatments": a boundary condition that changes type
    with a distance function): its x = 0 side is a contact face, which becomes a slip wall
    while within eps = h/2 of the wall and moving into it; the other sides are free."""
    m = tri_mesh(n, seed, bc={"x0": CONTACT})
    h = 1.0 / (n - 1)
    v = np.zeros((2, m.n_cells))
    v[0] = -V
    planes = np.array([[-gap, 0.0, 1.0, 0.0]])
    return Problem(f"rebound2d_n{n}", m, 1.0, 2.0, np.full(m.n_cells, 1.0), v, 0.4, steps,
                   contact=(planes, 0.5 * h))


def jellydrop3d(n: int = 12, seed: int = 10, v: float = 2.0, shear_a: float = -1.0, steps: int = 200) -> Problem:
    """A jelly-like block dropped on a rigid floor (Sect. "Impact of a jelly-like droplet",
    on a box instead of the paper's cylinder): a quarter of a 12 mm x 12 mm x 8 mm block
    (symmetry walls x = 0, y = 0), stiffened gas gamma = 2.2, p_inf = 1e6 Pa, p0 = 0,
    mu = 85 Pa, rho0 = 1020 kg/m^3, moving at (0, 0, -v) m/s; its bottom is a contact face
    with the floor 0.2 mm below (capture distance 0.1 mm); n^3 cubes of Kuhn tetrahedra."""
    L0, H, gap = 6e-3, 8e-3, 2e-4
    m = tet_mesh(n, n, n, seed, lx=L0, ly=L0, lz=H, bc={"x0": SLIP, "y0": SLIP, "z0": CONTACT})
    vel = np.zeros((3, m.n_cells))
    vel[2] = -v
    planes = np.array([[0.0, 0.0, -gap, 0.0, 0.0, 1.0]])
    return Problem(f"jellydrop3d_n{n}", m, 1020.0, 0.0, np.full(m.n_cells, 85.0), vel, 0.25, steps,
                   shear_a=shear_a, contact=(planes, 0.5 * gap), stiffened_gas=(2.2, 1e6, 0.0))


def impact2d(n: int = 708, seed: int = 2, steps: int = 2000) -> Problem:
    """Unit square of jittered Delaunay triangles (n=708 gives 999,698 cells) moving at
    v = (-0.1, 0) against a rigid slip wall at x = 0, other sides free;
    rho0=8.93, mu=0.46, lambda=1.06; CFL 0.4."""
    m = tri_mesh(n, seed, bc={"x0": SLIP})
    v = np.zeros((2, m.n_cells))
    v[0] = -0.1
    return Problem(f"impact2d_n{n}", m, 8.93, 1.06, np.full(m.n_cells, 0.46), v, 0.4, steps)


def column3d(nxy: int = 55, nz: int = 330, seed: int = 3, steps: int = 500) -> Problem:
    """Box [0,1]x[0,1]x[0,6] of Kuhn tetrahedra (55x55x330 cubes give 5,989,500 cells),
    base z=0 clamped, rest free; rho0=1.1, mu=0.5, lambda=2.5; v = (0.1 (z/6)^2, 0, 0); CFL 0.25."""
    m = tet_mesh(nxy, nxy, nz, seed, 1.0, 1.0, 6.0, bc={"z0": CLAMPED})
    p = cell_points(m)
    v = np.zeros((3, m.n_cells))
    v[0] = 0.1 * (p[:, 2] / 6.0) ** 2
    return Problem(f"column3d_{nxy}x{nxy}x{nz}", m, 1.1, 2.5, np.full(m.n_cells, 0.5), v, 0.25, steps)


def cube3d(n: int = 44, seed: int = 5, steps: int = 400) -> Problem:
    """Unit cube of Kuhn tetrahedra (44^3 cubes give 511,104 cells), slip walls; rho0=1,
    lambda=2; per-cell mu = 1 + 0.2 g(x) with g a seeded unit-variance Gaussian random field
    (64 Fourier modes, correlation length 0.15); v0 a smooth divergence-free Taylor-Green field
    with zero normal component on the walls, 0.05 (sin(pi x) cos(pi y) cos(pi z),
    cos(pi x) sin(pi y) cos(pi z), -2 cos(pi x) cos(pi y) sin(pi z))."""
    bc = {s: SLIP for s in ("x0", "x1", "y0", "y1", "z0", "z1")}
    m = tet_mesh(n, n, n, seed, bc=bc)
    p = cell_points(m)
    mu = 1.0 + 0.2 * gaussian_random_field(p, seed + 10_000)
    sx, sy, sz = (np.sin(np.pi * p[:, a]) for a in range(3))
    cx, cy, cz = (np.cos(np.pi * p[:, a]) for a in range(3))
    v = 0.05 * np.stack([sx * cy * cz, cx * sy * cz, -2.0 * cx * cy * sz])
    return Problem(f"cube3d_n{n}", m, 1.0, 2.0, mu, v, 0.25, steps)


def swinging_plate(n: int, jitter: float = 0.0, seed: int = 7, u0: float = 5e-4) -> Problem:
    """2D swinging plate (Sect. "2D swinging plate", Eq. (SwingIni)): [0,2]^2, slip walls,
    rho0 = 1100, E = 1.7e7, nu = 0.45, v(x,0) = omega U0 (-sin(pi x/2) cos(pi y/2),
    cos(pi x/2) sin(pi y/2)), omega = (pi/2) sqrt(2 mu / rho0)."""
    E, nu, rho0 = 1.7e7, 0.45, 1100.0
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    omega = 0.5 * math.pi * math.sqrt(2 * mu / rho0)
    m = tri_mesh(n, seed, 2.0, 2.0, jitter=jitter,
                 bc={"x0": SLIP, "x1": SLIP, "y0": SLIP, "y1": SLIP})
    p = cell_points(m)
    a = omega * u0
    v = a * np.stack([-np.sin(0.5 * np.pi * p[:, 0]) * np.cos(0.5 * np.pi * p[:, 1]),
                      np.cos(0.5 * np.pi * p[:, 0]) * np.sin(0.5 * np.pi * p[:, 1])])
    return Problem(f"swing_n{n}", m, rho0, lam, np.full(m.n_cells, mu), v, 0.4, 0,
                   meta={"omega": omega, "u0": u0, "t_final": math.pi / omega, "amp": a})


def be_plate(nx: int = 61, ny: int = 11, seed: int = 11, amp: float = 1.0) -> Problem:
    """Elastic vibration of a beryllium plate (Sect. "Elastic vibration of a beryllium plate"):
    [-0.03, 0.03] x [-0.005, 0.005] m, free boundaries, rho0 = 1845, E = 3.1827e11, nu = 0.0539,
    v0 = (0, A omega [a1 (sinh x' + sin x') - a2 (cosh x' + cos x')]), x' = alpha (x + L/2),
    alpha = 78.834, A = 4.3369e-5 (times amp), omega = 2.3597e5, a1 = 56.6368, a2 = 57.6455
    (the first free-free bending mode of an Euler-Bernoulli plate); t_final = 3e-5; a jittered
    nx x ny lattice (the paper uses 5,344 GMSH triangles). CFL 0.4."""
    L, H = 0.06, 0.01
    rho0, E, nu = 1845.0, 3.1827e11, 0.0539
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    m = tri_mesh(nx, seed, L, H, ny=ny)
    m.x[0] -= 0.5 * L
    m.x[1] -= 0.5 * H
    p = cell_points(m)
    alpha, A, omega, a1, a2 = 78.834, 4.3369e-5 * amp, 2.3597e5, 56.6368, 57.6455
    xp = alpha * (p[:, 0] + 0.5 * L)
    vy = A * omega * (a1 * (np.sinh(xp) + np.sin(xp)) - a2 * (np.cosh(xp) + np.cos(xp)))
    return Problem(f"be_plate_{nx}x{ny}", m, rho0, lam, np.full(m.n_cells, mu), np.stack([np.zeros_like(vy), vy]),
                   0.4, 0, meta={"L": L, "H": H, "E": E, "nu": nu, "omega": omega, "alpha": alpha,
                                 "t_final": 3e-5})


def blake3d(nr: int = 100, nlat: int = 2, aperture_deg: float = 4.0, seed: int = 12) -> Problem:
    """Blake's problem (Sect. "Blake's problem"): a shell 0.1 m <= r <= 1 m, rho0 = 3000,
    E = 62.5e9, nu = 0.25, at rest, the inner face driven by a pressure 1e6 Pa from t = 0, the
    outer face free; t_final = 1.6e-4 (the front then reaches r = 0.9). As in the paper, a
    needle of the shell stands in for it, its lateral faces slip walls (planes through the
    centre: symmetry planes of the radial solution): the jittered Kuhn lattice of the unit cube
    (nr radial x nlat x nlat cubes) mapped by (xi, eta, zeta) -> r(xi) d(eta, zeta), r = 0.1 +
    0.9 xi, d the unit vector along (1, tan(A (eta - 1/2)), tan(A (zeta - 1/2))), A the aperture
    (the paper's is 1 degree; any aperture gives the same radial solution), so that each
    lateral face lies in one plane through the centre. CFL 0.25."""
    r_in, r_out, p0 = 0.1, 1.0, 1.0e6
    rho0, E, nu = 3000.0, 62.5e9, 0.25
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    m = tet_mesh(nr, nlat, nlat, seed, bc={"x0": PRESSURE, "y0": SLIP, "y1": SLIP, "z0": SLIP, "z1": SLIP})
    A = math.radians(aperture_deg)
    xi, eta, zeta = m.x
    d = np.stack([np.ones_like(xi), np.tan(A * (eta - 0.5)), np.tan(A * (zeta - 0.5))])
    d /= np.sqrt((d * d).sum(axis=0))
    m.x = np.ascontiguousarray((r_in + (r_out - r_in) * xi) * d)
    return Problem(f"blake3d_{nr}x{nlat}", m, rho0, lam, np.full(m.n_cells, mu), np.zeros((3, m.n_cells)), 0.25, 0,
                   bcval=side_values(m, PRESSURE, (p0, 0.0, 0.0)),
                   meta={"r_in": r_in, "p0": p0, "E": E, "nu": nu, "t_final": 1.6e-4})


def swinging_cube(n: int, jitter: float = 0.1, seed: int = 13, u0: float = 5e-4) -> Problem:
    """A 3D counterpart of the swinging plate (Sect. "2D swinging plate"): [0,2]^3, slip walls,
    rho0 = 1100, E = 1.7e7, nu = 0.45, v(x,0) = omega U0 (sin(k x) cos(k y) cos(k z),
    -cos(k x) sin(k y) cos(k z), 0), k = pi/2: a divergence-free standing shear wave whose normal
    velocity and shear tractions vanish on the walls, omega = k sqrt(3 mu / rho0)."""
    E, nu, rho0 = 1.7e7, 0.45, 1100.0
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    k = 0.5 * math.pi
    omega = k * math.sqrt(3.0 * mu / rho0)
    m = tet_mesh(n, n, n, seed, 2.0, 2.0, 2.0, jitter=jitter,
                 bc={s: SLIP for s in ("x0", "x1", "y0", "y1", "z0", "z1")})
    p = cell_points(m)
    a = omega * u0
    s, c = np.sin(k * p), np.cos(k * p)
    v = a * np.stack([s[:, 0] * c[:, 1] * c[:, 2], -c[:, 0] * s[:, 1] * c[:, 2], np.zeros(len(p))])
    return Problem(f"swing_cube_n{n}", m, rho0, lam, np.full(m.n_cells, mu), v, 0.25, 0,
                   meta={"omega": omega, "u0": u0, "t_final": math.pi / omega, "amp": a, "k": k})


def _batch_instance(args) -> Problem:
    i, n, mu, amp, steps = args
    m = tri_mesh(n, 1000 + i, bc={"x0": SLIP, "x1": SLIP, "y0": SLIP, "y1": SLIP})
    p = cell_points(m)
    v = amp * np.stack([np.sin(np.pi * p[:, 0]) * np.sin(np.pi * p[:, 1]),
                        np.cos(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1])])
    return Problem(f"batch{i}_n{n}", m, 1.0, 2.0, np.full(m.n_cells, mu), v, 0.4, steps, meta={"amp": amp})


def batched2d(n_inst: int = 256, seed: int = 4, lo: float = 1e3, hi: float = 2e5,
              steps: int = 500, workers: int = 1) -> list[Problem]:
    """Independent unit-square instances: cell counts log-uniform in [lo, hi], per-instance
    mu ~ U[0.5, 2] and velocity amplitude A ~ U[1e-3, 0.2] applied to the plain2d field;
    lambda=2, rho0=1, slip walls, CFL 0.4. Instance i meshes with seed 1000+i. workers > 1
    generates the meshes in spawned processes (same result)."""
    rng = np.random.default_rng(seed)
    ncell = np.exp(rng.uniform(math.log(lo), math.log(hi), n_inst))
    mus = rng.uniform(0.5, 2.0, n_inst)
    amps = rng.uniform(1e-3, 0.2, n_inst)
    jobs = [(i, int(math.ceil(1 + math.sqrt(ncell[i] / 2))), float(mus[i]), float(amps[i]), steps)
            for i in range(n_inst)]
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_batch_instance, jobs, chunksize=4))
    return [_batch_instance(j) for j in jobs]


def concat(problems: list[Problem], name: str = "batch") -> tuple[Problem, np.ndarray]:
    """Concatenate independent problems into one mesh (node and cell ids offset, no shared
    nodes) and return it with the instance id of every cell. All must share dim, rho0, lam
    and CFL; mu and v are per cell already."""
    d = problems[0].mesh.dim
    xs, c2ns, bfs, bts, mus, vs, inst = [], [], [], [], [], [], []
    off = 0
    for i, pb in enumerate(problems):
        assert pb.mesh.dim == d and pb.rho0 == problems[0].rho0 and pb.lam == problems[0].lam
        xs.append(pb.mesh.x)
        c2ns.append(pb.mesh.c2n + off)
        bfs.append(pb.mesh.bface + off)
        bts.append(pb.mesh.btag)
        mus.append(pb.mu)
        vs.append(pb.v)
        inst.append(np.full(pb.mesh.n_cells, i, dtype=np.int32))
        off += pb.mesh.n_nodes
    m = Mesh(d, np.ascontiguousarray(np.concatenate(xs, axis=1)), np.ascontiguousarray(np.concatenate(c2ns, axis=1)),
             np.ascontiguousarray(np.concatenate(bfs, axis=1)), np.concatenate(bts))
    pb = Problem(name, m, problems[0].rho0, problems[0].lam, np.concatenate(mus),
                 np.ascontiguousarray(np.concatenate(vs, axis=1)), problems[0].cfl, problems[0].steps,
                 meta={"n_inst": len(problems), "cells": [q.mesh.n_cells for q in problems],
                       "nodes": [q.mesh.n_nodes for q in problems]})
    return pb, np.concatenate(inst)


def translate_rotate(pb: Problem, R: np.ndarray, shift: np.ndarray) -> Problem:
    """Rigidly move a problem's whole configuration: x -> R x + shift, v -> R v, F -> R F R^T.
    (An input transformation used by objectivity tests.)"""
    d = pb.mesh.dim
    x = R @ pb.mesh.x + shift[:, None]
    m = Mesh(d, np.ascontiguousarray(x), pb.mesh.c2n, pb.mesh.bface, pb.mesh.btag)
    v = np.ascontiguousarray(R @ pb.v)
    F = None
    if pb.F is not None:
        Fm = pb.F.T.reshape(-1, d, d)
        F = np.ascontiguousarray((R @ Fm @ R.T).reshape(-1, d * d).T)
    return Problem(pb.name + "_rot", m, pb.rho0, pb.lam, pb.mu.copy(), v, pb.cfl, pb.steps, F, dict(pb.meta))
