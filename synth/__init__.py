"""Seeded synthetic scene generators.

This module builds the inputs that both the CUDA path and the FP64 oracle consume:
tetrahedral meshes of hex lattices (5-tet split with alternating parity), material
draws, initial velocities, targets, and vertex-plane and vertex-sphere contact sets with their frames.
It holds geometry and random draws only -- none of the adjoint method's arithmetic --
so that the oracle and the GPU library can share inputs without sharing any code.

All randomness goes through ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GRAVITY = 9.81  # m/s^2, along -z of the world frame


# --------------------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------------------

# Corners of a unit cell, index = x + 2y + 4z.  Even cells put the tet made of the four
# odd corners in the middle; odd cells the four even corners.  Neighbouring cells then
# agree on every face diagonal (conforming mesh).
_EVEN_SPLIT = ((1, 2, 4, 7), (0, 1, 2, 4), (3, 1, 2, 7), (5, 1, 4, 7), (6, 2, 4, 7))
_ODD_SPLIT = ((0, 3, 5, 6), (1, 0, 3, 5), (2, 0, 3, 6), (4, 0, 5, 6), (7, 3, 5, 6))


def hex_tet_mesh(nx: int, ny: int, nz: int, cell: float, origin=(0.0, 0.0, 0.0)):
    """Lattice of nx*ny*nz cubic cells of edge ``cell``, each split into 5 tets.

    Returns (X, tets): X float64 [n_v, 3] (vertex index = i + (nx+1)(j + (ny+1)k)),
    tets int32 [n_t, 4], every tet positively oriented.
    """
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)  # noqa: E731
    X = np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3))
    X[vid(ii, jj, kk).ravel(), 0] = ii.ravel() * cell + origin[0]
    X[vid(ii, jj, kk).ravel(), 1] = jj.ravel() * cell + origin[1]
    X[vid(ii, jj, kk).ravel(), 2] = kk.ravel() * cell + origin[2]
    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                corner = [vid(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1)) for c in range(8)]
                split = _EVEN_SPLIT if (i + j + k) % 2 == 0 else _ODD_SPLIT
                for t in split:
                    tets.append([corner[c] for c in t])
    tets = np.asarray(tets, dtype=np.int64)
    # orientation: swap two vertices where the signed volume is negative (mesh hygiene)
    e = X[tets[:, 1:]] - X[tets[:, [0]]]
    neg = np.linalg.det(e) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    return X, tets.astype(np.int32)


def voxel_tet_mesh(occ: np.ndarray, cell: float, origin=(0.0, 0.0, 0.0)):
    """Tet mesh of the occupied cells of a voxel grid ``occ`` [nx, ny, nz] (bool), each cell split
    into 5 tets with the parity-alternating pattern of ``hex_tet_mesh`` (so the mesh is conforming
    for any set of cells).  Unused lattice vertices are dropped.  Returns (X, tets int32)."""
    occ = np.asarray(occ, bool)
    nx, ny, nz = occ.shape
    ci, cj, ck = np.nonzero(occ)
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)  # noqa: E731
    corners = np.stack([vid(ci + (c & 1), cj + ((c >> 1) & 1), ck + ((c >> 2) & 1)) for c in range(8)], 1)
    even = ((ci + cj + ck) % 2 == 0)
    tets = np.concatenate([np.where(even[:, None], corners[:, list(te)], corners[:, list(to)])
                           for te, to in zip(_EVEN_SPLIT, _ODD_SPLIT)], 0).astype(np.int64)
    used, inv = np.unique(tets, return_inverse=True)
    tets = inv.reshape(tets.shape)
    i = used % (nx + 1)
    j = (used // (nx + 1)) % (ny + 1)
    k = used // ((nx + 1) * (ny + 1))
    X = np.stack([i * cell + origin[0], j * cell + origin[1], k * cell + origin[2]], 1).astype(np.float64)
    e = X[tets[:, 1:]] - X[tets[:, [0]]]
    neg = np.linalg.det(e) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    return X, tets.astype(np.int32)


# --------------------------------------------------------------------------------------
# contacts
# --------------------------------------------------------------------------------------

@dataclass
class Plane:
    """Rigid plane {x : n.x = offset} with friction coefficient mu; frame rows n, t1, t2.

    ``regions`` (optional) splits the plane into a grid of friction regions in its (t1, t2)
    coordinates: (n1, n2, lo1, hi1, lo2, hi2, mu_values [n1*n2]); a contact then takes the
    friction coefficient of its cell, and contacts are listed cell by cell."""
    normal: np.ndarray
    offset: float
    mu: float
    t1: np.ndarray = None
    t2: np.ndarray = None
    regions: tuple = None

    def __post_init__(self):
        self.normal = np.asarray(self.normal, float)
        if self.t1 is None:
            a = np.array([1.0, 0.0, 0.0]) if abs(self.normal[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
            t1 = a - self.normal * (a @ self.normal)
            self.t1 = t1 / np.linalg.norm(t1)
        self.t1 = np.asarray(self.t1, float)
        if self.t2 is None:
            self.t2 = np.cross(self.normal, self.t1)
        self.t2 = np.asarray(self.t2, float)

    @property
    def frame(self):
        return np.stack([self.normal, self.t1, self.t2])


@dataclass
class Contacts:
    """Vertex-plane contact set, frozen for one step.

    vertex int32 [n_c]; frame float64 [n_c, 3, 3] (rows n, t1, t2); d_n float64 [n_c]
    (normal gap delta_n = n.x - d_n); d_f float64 [n_c, 2] (tangential offset, zero here);
    mu float64 [n_c]; region int32 [n_c] (friction region id), n_regions.
    """
    vertex: np.ndarray
    frame: np.ndarray
    d_n: np.ndarray
    d_f: np.ndarray
    mu: np.ndarray
    region: np.ndarray
    n_regions: int

    @property
    def n(self):
        return int(self.vertex.shape[0])

    @staticmethod
    def empty():
        return Contacts(np.zeros(0, np.int32), np.zeros((0, 3, 3)), np.zeros(0), np.zeros((0, 2)),
                        np.zeros(0), np.zeros(0, np.int32), 1)


@dataclass
class Sphere:
    """Rigid sphere collider (center, radius) with friction coefficient mu.  A contact's frame is
    frozen at the previous positions: n = (x_prev - c)/|x_prev - c| with an orthonormal completion
    t1, t2, and d_n = n . c + radius, so delta_n = n . x - d_n is the gap along that normal."""
    center: np.ndarray
    radius: float
    mu: float = 0.0

    def contacts(self, x_prev: np.ndarray, margin: float, verts, region: int):
        c = np.asarray(self.center, float)
        d = x_prev[verts] - c
        dist = np.linalg.norm(d, axis=1)
        sel = verts[dist - self.radius < margin]
        n = (x_prev[sel] - c) / np.linalg.norm(x_prev[sel] - c, axis=1)[:, None]
        a = np.where((np.abs(n[:, 0]) < 0.9)[:, None], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0])
        t1 = a - n * np.sum(a * n, axis=1)[:, None]
        t1 /= np.linalg.norm(t1, axis=1)[:, None]
        frames = np.stack([n, t1, np.cross(n, t1)], axis=1).reshape(-1, 3, 3)
        return sel, frames, n @ c + self.radius, np.full(len(sel), self.mu), np.full(len(sel), region)


def detect_contacts(x_prev: np.ndarray, planes, margin: float, candidates=None, spheres=()) -> Contacts:
    """Vertices whose gap to a plane or a sphere at the previous positions is below ``margin``.

    ``candidates`` restricts the search to a vertex subset (e.g. a bottom face).  Each sphere is one
    more friction region, after the planes'.
    Friction regions: one region per plane, or the plane's grid of regions (listed in order,
    contacts grouped by region and ordered by position inside it).
    """
    verts = np.arange(x_prev.shape[0]) if candidates is None else np.asarray(candidates)
    vs, frames, dn, mus, reg = [], [], [], [], []
    base = 0
    for pl in planes:
        gap = x_prev[verts] @ pl.normal - pl.offset
        sel = verts[gap < margin]
        if pl.regions is None:
            vs.append(sel)
            mus.append(np.full(len(sel), pl.mu))
            reg.append(np.full(len(sel), base))
            base += 1
        else:
            n1, n2, lo1, hi1, lo2, hi2, mu_vals = pl.regions
            u = x_prev[sel] @ pl.t1
            v = x_prev[sel] @ pl.t2
            i1 = np.clip(((u - lo1) / (hi1 - lo1) * n1).astype(int), 0, n1 - 1)
            i2 = np.clip(((v - lo2) / (hi2 - lo2) * n2).astype(int), 0, n2 - 1)
            cell = i1 + n1 * i2
            order = np.lexsort((u, v, cell))
            sel, cell = sel[order], cell[order]
            vs.append(sel)
            mus.append(np.asarray(mu_vals, float)[cell])
            reg.append(base + cell)
            base += n1 * n2
        frames.append(np.repeat(pl.frame[None], len(sel), 0))
        dn.append(np.full(len(sel), pl.offset))
    for sph in spheres:
        sel, fr, d, m, r = sph.contacts(x_prev, margin, verts, base)
        vs.append(sel)
        frames.append(fr)
        dn.append(d)
        mus.append(m)
        reg.append(r)
        base += 1
    if not vs:
        return Contacts.empty()
    v = np.concatenate(vs).astype(np.int32)
    return Contacts(v, np.concatenate(frames).reshape(-1, 3, 3), np.concatenate(dn),
                    np.zeros((len(v), 2)), np.concatenate(mus), np.concatenate(reg).astype(np.int32),
                    max(1, base))


# --------------------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------------------

@dataclass
class Scene:
    """Mesh + material + step size.  E, nu are per tet (float64 [n_t])."""
    X: np.ndarray
    tets: np.ndarray
    E: np.ndarray
    nu: np.ndarray
    density: float
    h: float
    gravity: np.ndarray
    planes: list = field(default_factory=list)
    contact_candidates: np.ndarray = None
    margin: float = 2e-3
    eps: float = 1e-4
    name: str = ""
    spheres: list = field(default_factory=list)
    thickness: float = None  # triangle meshes (shells): thickness tau (m); None for tet meshes
    bend: float = 0.0        # shells: isometric bending stiffness k_b

    @property
    def n_verts(self):
        return int(self.X.shape[0])

    @property
    def n_tets(self):
        return int(self.tets.shape[0])

    def contacts(self, x_prev):
        if not self.planes and not self.spheres:
            return Contacts.empty()
        return detect_contacts(x_prev, self.planes, self.margin, self.contact_candidates, self.spheres)


@dataclass
class Problem:
    """A scene plus the start state (q0, v0), per-vertex external forces besides gravity
    (zeros unless stated), and a target for the loss."""
    scene: Scene
    q0: np.ndarray
    v0: np.ndarray
    f_ctrl: np.ndarray
    q_target: np.ndarray


def tri_grid(nx: int, ny: int, size_x: float, size_y: float, origin=(0.0, 0.0, 0.0)):
    """Flat (nx+1) x (ny+1) vertex grid in the z = origin[2] plane, two triangles per cell with
    alternating diagonals, counter-clockwise seen from +z.  Returns (X [n_v, 3], tris [n_t, 3])."""
    xs = origin[0] + np.linspace(0.0, size_x, nx + 1)
    ys = origin[1] + np.linspace(0.0, size_y, ny + 1)
    X = np.array([[x, y, origin[2]] for y in ys for x in xs])
    vid = lambda i, j: i + (nx + 1) * j  # noqa: E731
    tris = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    return X, np.asarray(tris, np.int32)


def cloth_drape(seed: int = 0, n: int = 31, size: float = 0.3, height: float = 0.005, radius: float = 0.08,
                E: float = 1e5, nu: float = 0.3, density: float = 1000.0, thickness: float = 1e-3,
                bend: float = 1e-4, h: float = 0.01, mu: float = 0.0, eps: float = 1e-4,
                margin: float = 2e-3, sag: float = 0.0) -> Problem:
    """A square cloth patch of n x n cells (2 triangles each) centred above a sphere collider of the
    given radius at the origin, its lowest point ``height`` above the sphere's top (sag > 0 bends it
    over the sphere first: z -= sag r^2 / R^2 at distance r from the axis, R the patch half-width),
    falling under gravity: the draping cloth of the paper's batched experiment (Sec. 5), with
    isometric bending.  Default 32 x 32 vertices (1,024), 1,922 triangles, frictionless sphere."""
    rng = np.random.default_rng(seed)
    X, tris = tri_grid(n, n, size, size, origin=(-size / 2, -size / 2, radius + height))
    r2 = X[:, 0] ** 2 + X[:, 1] ** 2
    X[:, 2] -= sag * r2 / (size / 2) ** 2
    ntri = len(tris)
    scene = Scene(X, tris, np.full(ntri, E), np.full(ntri, nu), density, h, np.array([0.0, 0.0, -GRAVITY]), [],
                  None, margin, eps, f"cloth{n}", spheres=[Sphere(np.zeros(3), radius, mu)], thickness=thickness,
                  bend=bend)
    v0 = rng.normal(0.0, 1e-3, X.shape)
    return Problem(scene, X.copy(), v0, np.zeros_like(X), X + rng.normal(0.0, 1e-3, X.shape))


def cube_drop(seed: int = 0, cells: int = 4, edge: float = 0.1, drop: float = 0.01,
              E: float = 1e5, nu: float = 0.4, density: float = 1000.0, h: float = 1.0 / 60.0,
              mu: float = 0.5, eps: float = 1e-4, v_sigma: float = 0.01, tgt_sigma: float = 1e-3,
              margin: float = 2e-3) -> Problem:
    """Neo-Hookean cube of cells^3 hex cells x 5 tets, bottom ``drop`` above the ground z=0.

    Default: 4x4x4 cells (125 vertices, 320 tets), edge 0.1 m, dropped 1 cm, E=1e5, nu=0.4,
    rho=1000, h=1/60, ground mu=0.5, eps=1e-4, v0 ~ N(0, 0.01^2), target = rest + N(0, 1e-3^2).
    """
    rng = np.random.default_rng(seed)
    X, tets = hex_tet_mesh(cells, cells, cells, edge / cells, origin=(-edge / 2, -edge / 2, drop))
    bottom = np.nonzero(np.isclose(X[:, 2], drop))[0]
    scene = Scene(X, tets, np.full(len(tets), E), np.full(len(tets), nu), density, h,
                  np.array([0.0, 0.0, -GRAVITY]), [Plane([0.0, 0.0, 1.0], 0.0, mu, [1.0, 0, 0], [0, 1.0, 0])],
                  bottom, margin, eps, f"cube{cells}")
    v0 = rng.normal(0.0, v_sigma, X.shape)
    q_tgt = X + rng.normal(0.0, tgt_sigma, X.shape)
    return Problem(scene, X.copy(), v0, np.zeros_like(X), q_tgt)


def beam_incline(seed: int = 0, nx: int = 40, ny: int = 10, nz: int = 10, cell: float = 0.01,
                 angle_deg: float = 20.0, E: float = 5e5, nu: float = 0.45, density: float = 1000.0,
                 h: float = 1.0 / 100.0, mu: float = 0.3, eps: float = 1e-4, gap0: float = 1e-7,
                 margin: float = 2e-3) -> Problem:
    """Beam of nx*ny*nz cells x 5 tets lying on a plane inclined by ``angle_deg`` about y.

    Default: 40x10x10 cells of 1 cm (4,961 vertices, 20,000 tets), 20 deg incline, mu=0.3
    (below tan 20 deg, so it slides), E=5e5, nu=0.45, h=1/100, starting at rest with its
    bottom face ``gap0`` above the plane.  Target: the start positions (the loss used with it
    is a centre-of-mass error, which the caller defines).
    """
    del seed  # deterministic geometry; kept for a uniform signature
    th = np.deg2rad(angle_deg)
    Xl, tets = hex_tet_mesh(nx, ny, nz, cell, origin=(0.0, -ny * cell / 2, gap0))
    rot = np.array([[np.cos(th), 0.0, -np.sin(th)], [0.0, 1.0, 0.0], [np.sin(th), 0.0, np.cos(th)]])
    X = Xl @ rot.T
    n = rot @ np.array([0.0, 0.0, 1.0])
    t1 = rot @ np.array([1.0, 0.0, 0.0])
    bottom = np.nonzero(np.isclose(Xl[:, 2], gap0))[0]
    scene = Scene(X, tets, np.full(len(tets), E), np.full(len(tets), nu), density, h,
                  np.array([0.0, 0.0, -GRAVITY]), [Plane(n, 0.0, mu, t1, [0.0, 1.0, 0.0])], bottom,
                  margin, eps, f"beam{nx}x{ny}x{nz}")
    return Problem(scene, X.copy(), np.zeros_like(X), np.zeros_like(X), X.copy())


def jittered_delaunay_ball(r: float = 0.1, cap: float = 0.05, cell: float = 4.5e-3, jitter: float = 0.2,
                           seed: int = 0, min_quality: float = 1e-2):
    """Tet mesh of the ball |x| <= r cut flat at |z| <= cap: points on a lattice of spacing ``cell``
    in x, y and of nz = round(2 cap / cell) layers exactly spanning [-cap, cap] in z, jittered by
    +-jitter*spacing (uniform, seeded; the two cut layers are not moved in z, so they stay on the
    planes and the tets next to them are lattice-shaped), Delaunay-tetrahedralised
    (scipy.spatial).  Tets below ``min_quality`` times the lattice tet volume (slivers) are dropped
    and vertices left without a tet removed.  Returns (X [n_v, 3], tets int32 [n_t, 4], positively
    oriented)."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    n = int(np.ceil(r / cell)) + 1
    nz = max(2, int(round(2 * cap / cell)))
    dz = 2 * cap / nz
    gx = np.arange(-n, n + 1) * cell
    gz = -cap + np.arange(nz + 1) * dz
    P = np.stack(np.meshgrid(gx, gx, gz, indexing="ij"), -1).reshape(-1, 3)
    P[:, :2] += rng.uniform(-jitter, jitter, (len(P), 2)) * cell
    inner = (P[:, 2] > -cap + 0.5 * dz) & (P[:, 2] < cap - 0.5 * dz)
    P[inner, 2] += rng.uniform(-jitter, jitter, int(inner.sum())) * dz
    P = P[np.linalg.norm(P, axis=1) <= r]
    T = Delaunay(P).simplices.astype(np.int64)
    e = P[T[:, 1:]] - P[T[:, [0]]]
    vol = np.einsum("ij,ij->i", np.cross(e[:, 0], e[:, 1]), e[:, 2]) / 6.0
    T[vol < 0] = T[vol < 0][:, [0, 2, 1, 3]]
    keep = np.abs(vol) >= min_quality * cell * cell * dz / 6.0
    # also drop slivers with a tiny altitude (nearly flat tets of large faces)
    Pt = P[T]
    alt = np.full(len(T), np.inf)
    for a in range(4):
        o = [k for k in range(4) if k != a]
        area = 0.5 * np.linalg.norm(np.cross(Pt[:, o[1]] - Pt[:, o[0]], Pt[:, o[2]] - Pt[:, o[0]]), axis=1)
        alt = np.minimum(alt, 3.0 * np.abs(vol) / np.maximum(area, 1e-300))
    keep &= alt >= 5.0 * min_quality * min(cell, dz)
    T = T[keep]
    used = np.unique(T)
    remap = -np.ones(len(P), np.int64)
    remap[used] = np.arange(len(used))
    return P[used], remap[T].astype(np.int32)


def sphere_press(seed: int = 0, r: float = 0.1, cap: float = 0.05, cell: float = 4.5e-3, E: float = 1e5,
                 nu: float = 0.4, density: float = 1000.0, h: float = 1.0 / 60.0, eps: float = 1e-4,
                 press: float = 2e-3, gap0: float = 1e-7, margin: float = 2e-3, grid: int = 4,
                 mu_range=(0.2, 1.0), tgt_sigma: float = 1e-3) -> Problem:
    """Large contact-heavy scene: a Neo-Hookean ball (r = 0.1 m, flattened at |z| <= cap: the contact
    patches of a pressed ball) between the ground z = -cap and a kinematic plate that has pressed it
    by ``press``: the start state is the rest shape compressed affinely in z so that its top disc
    sits at cap - press, touching the plate (both planes ``gap0`` away), at rest.  Each plane carries
    a grid x grid of friction regions over the cap disc with mu ~ U(mu_range) (seeded).  Default
    cell 4.5 mm: about 32k vertices, 210k tets, ~2,300 contacts (both discs).  Target X + N(0,
    tgt_sigma^2)."""
    X, tets = jittered_delaunay_ball(r, cap, cell, 0.2, seed)
    rng = np.random.default_rng(seed + 1)
    rc = np.sqrt(r * r - cap * cap)
    planes = []
    for nrm, off in (([0.0, 0.0, 1.0], -cap - gap0), ([0.0, 0.0, -1.0], -(cap - press + gap0))):
        t1 = np.array([1.0, 0.0, 0.0])
        t2 = np.cross(nrm, t1)
        mu_vals = rng.uniform(mu_range[0], mu_range[1], grid * grid)
        planes.append(Plane(nrm, off, float(mu_vals.mean()), t1, t2, (grid, grid, -rc, rc, -rc, rc, mu_vals)))
    on_disc = np.nonzero(np.abs(np.abs(X[:, 2]) - cap) < 1e-12)[0]
    scene = Scene(X, tets, np.full(len(tets), E), np.full(len(tets), nu), density, h,
                  np.array([0.0, 0.0, -GRAVITY]), planes, on_disc, margin, eps, f"sphere{len(X)}")
    q0 = X.copy()
    q0[:, 2] = -cap + (X[:, 2] + cap) * (1.0 - press / (2.0 * cap))
    q_tgt = X + rng.normal(0.0, tgt_sigma, X.shape)
    return Problem(scene, q0, np.zeros_like(X), np.zeros_like(X), q_tgt)


def quadruped(seed: int = 0, torso=(120, 80, 5), leg_r: float = 8.0, leg_h: int = 12, leg_c=(50, 32),
              pad=(78, 62, 2), cell: float = 5e-3, E: float = 2e5, nu: float = 0.45, density: float = 1000.0,
              h: float = 1.0 / 200.0, mu: float = 0.8, eps: float = 1e-4, gap0: float = 1e-7,
              margin: float = 2e-3, act_scale: float = 1e3) -> Problem:
    """Soft quadruped of voxel cells (``cell`` edge, 5 tets each) standing on the ground z = 0:
    foot pads (pad[0] x pad[1] x pad[2] cells, centred under the legs), cylindrical legs (radius
    leg_r cells, leg_h cells high, centred at (+-leg_c[0], +-leg_c[1]) cells from the torso centre)
    and a torso of torso[0] x torso[1] x torso[2] cells on top.  Defaults: ~96k cells, ~482k tets,
    ~100k vertices, ~19.9k pad-bottom contacts, E=2e5, nu=0.45, mu=0.8, h=1/200.  The problem also
    carries seeded per-tet activations a ~ N(0, act_scale^2) Pa and unit fibres (``act``, ``fibre``).
    """
    tx, ty, tz = torso
    px, py, pz = pad
    half_x = max(tx // 2, leg_c[0] + px // 2 + 1)
    half_y = max(ty // 2, leg_c[1] + py // 2 + 1)
    nx, ny, nz = 2 * half_x, 2 * half_y, pz + leg_h + tz
    occ = np.zeros((nx, ny, nz), bool)
    ci = np.arange(nx)[:, None] - half_x + 0.5   # cell centres, torso centre at 0
    cj = np.arange(ny)[None, :] - half_y + 0.5
    occ[half_x - tx // 2:half_x - tx // 2 + tx, half_y - ty // 2:half_y - ty // 2 + ty, pz + leg_h:] = True
    for sx in (-1, 1):
        for sy in (-1, 1):
            cx, cy = sx * leg_c[0], sy * leg_c[1]
            disc = (ci - cx) ** 2 + (cj - cy) ** 2 <= leg_r ** 2
            occ[:, :, pz:pz + leg_h] |= disc[:, :, None]
            x0 = half_x + cx - px // 2
            y0 = half_y + cy - py // 2
            occ[x0:x0 + px, y0:y0 + py, :pz] = True
    X, tets = voxel_tet_mesh(occ, cell, origin=(-half_x * cell, -half_y * cell, gap0))
    bottom = np.nonzero(np.isclose(X[:, 2], gap0))[0]
    scene = Scene(X, tets, np.full(len(tets), E), np.full(len(tets), nu), density, h,
                  np.array([0.0, 0.0, -GRAVITY]), [Plane([0.0, 0.0, 1.0], 0.0, mu, [1.0, 0, 0], [0, 1.0, 0])],
                  bottom, margin, eps, f"quadruped{len(tets)}")
    pb = Problem(scene, X.copy(), np.zeros_like(X), np.zeros_like(X), X.copy())
    pb.act, pb.fibre = random_actuation(len(tets), seed, act_scale)
    return pb


def two_tet(seed: int = 0, E: float = 1e5, nu: float = 0.4, h: float = 1.0 / 60.0, mu: float = 0.5,
            eps: float = 1e-4, jitter: float = 0.1) -> Problem:
    """Tiny jittered mesh (one cell, 5 tets, 8 vertices) resting on the ground, 4 contacts."""
    rng = np.random.default_rng(seed)
    X, tets = hex_tet_mesh(1, 1, 1, 0.05, origin=(0.0, 0.0, 1e-6))
    X[4:] += rng.normal(0, jitter * 0.05, (4, 3))
    bottom = np.arange(4)
    scene = Scene(X, tets, np.full(len(tets), E), np.full(len(tets), nu), 1000.0, h,
                  np.array([0.0, 0.0, -GRAVITY]), [Plane([0.0, 0.0, 1.0], 0.0, mu, [1.0, 0, 0], [0, 1.0, 0])],
                  bottom, 2e-3, eps, "twotet")
    v0 = rng.normal(0.0, 0.01, X.shape)
    return Problem(scene, X.copy(), v0, np.zeros_like(X), X + rng.normal(0, 1e-3, X.shape))


def random_deformation_gradients(n: int, seed: int = 0, strain: float = 0.05) -> np.ndarray:
    """n random F = R (I + S): R a random rotation, S ~ strain * N(0,1) (float64 [n, 3, 3])."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, 3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diagonal(Rr, axis1=1, axis2=2))[:, None, :]
    Q[np.linalg.det(Q) < 0, :, 0] *= -1
    S = strain * rng.normal(size=(n, 3, 3))
    return Q @ (np.eye(3) + S)


def random_actuation(n_tets: int, seed: int = 0, scale: float = 1e3):
    """Per-tet activations a ~ N(0, scale^2) Pa (float32, [n_t]) and unit fibre directions d_i
    uniform on the sphere (float64, [n_t, 3]), both seeded."""
    rng = np.random.default_rng(seed)
    act = (scale * rng.standard_normal(n_tets)).astype(np.float32)
    d = rng.standard_normal((n_tets, 3))
    return act, d / np.linalg.norm(d, axis=1, keepdims=True)


def random_seed_vectors(n_verts: int, seed: int = 0, scale: float = 1.0):
    """Seeded dL/dq, dL/dv seeds (float64 [n_v, 3] each)."""
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=(n_verts, 3)), scale * rng.normal(size=(n_verts, 3))


def block_batch(n_blocks: int = 64, seed: int = 0, tets_range=(2000, 50000), cell: float = 0.01,
                h: float = 1.0 / 60.0, eps: float = 1e-4, margin: float = 2e-3, height_range=(0.0, 0.02),
                v_sigma: float = 0.05):
    """Independent Neo-Hookean blocks for the batched adjoint.

    Tet counts log-uniform in ``tets_range``; each block has a x b x c cells of edge ``cell`` with
    n_cells = round(n_t / 5) and aspect (r_x, r_y, r_z) ~ U(0.5, 2)^3; E log-uniform in [1e4, 1e6],
    nu ~ U(0.3, 0.48), ground friction mu ~ U(0.1, 1.0), bottom at a height ~ U(0, 2 cm) above its
    own ground plane z = 0, initial velocity N(0, 0.05^2) per vertex component, h = 1/60.
    Returns a list of Problems (one per block; loss target = rest positions + N(0, 1e-3^2)).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_blocks):
        nt = np.exp(rng.uniform(np.log(tets_range[0]), np.log(tets_range[1])))
        ncell = max(1, int(round(nt / 5)))
        r = rng.uniform(0.5, 2.0, 3)
        s = (ncell / np.prod(r)) ** (1.0 / 3.0)
        a = max(1, int(round(r[0] * s)))
        b = max(1, int(round(r[1] * s)))
        c = max(1, int(round(ncell / (a * b))))
        height = rng.uniform(*height_range)
        X, tets = hex_tet_mesh(a, b, c, cell, origin=(0.0, 0.0, max(height, 1e-7)))
        E = np.exp(rng.uniform(np.log(1e4), np.log(1e6)))
        nu = rng.uniform(0.3, 0.48)
        mu = rng.uniform(0.1, 1.0)
        bottom = np.nonzero(np.isclose(X[:, 2], max(height, 1e-7)))[0]
        scene = Scene(X, tets, np.full(len(tets), E), np.full(len(tets), nu), 1000.0, h,
                      np.array([0.0, 0.0, -GRAVITY]), [Plane([0.0, 0.0, 1.0], 0.0, mu, [1.0, 0, 0], [0, 1.0, 0])],
                      bottom, margin, eps, f"block{a}x{b}x{c}")
        v0 = rng.normal(0.0, v_sigma, X.shape)
        out.append(Problem(scene, X.copy(), v0, np.zeros_like(X), X + rng.normal(0.0, 1e-3, X.shape)))
    return out
