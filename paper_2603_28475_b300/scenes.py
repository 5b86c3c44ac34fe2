"""Seeded synthetic inputs for the gel-pad contact solve.

This module only builds geometry and motion: tetrahedral gel pads, rigid
indenter triangle meshes, marker grids and per-frame indenter poses. It holds
none of the solver's arithmetic (no deformation gradients, energies, masses,
contact distances or marker weights); both the CUDA library and the FP64
oracle take its arrays as plain inputs.

Units are SI (metres, kilograms, seconds, pascals). A pad occupies the box
[0, Lx] x [0, Ly] x [0, Lz]; its bottom face z = 0 is the Dirichlet face and
its top face z = Lz carries the markers. An indenter pose is a rotation vector
(3) followed by a translation (3), mapping the indenter's local vertices into
the pad frame.

Workloads (each seeded with numpy PCG64):
  * ``config_single_pad``  -- 20x16x4 mm pad, 10x8x2 hex cells x 6 tets
    (297 verts, 960 tets), icosphere r = 4 mm (320 tris) pressed 10 frames x
    0.05 mm at the centre, 7x9 markers.
  * ``config_realistic``   -- 18.6x14.3x4 mm pad with jittered, renumbered
    connectivity (~20k verts), cylinder / box-edge / ridged-thread indenter,
    press then slide, 11x9 markers.
  * ``config_batched``     -- many environments x 2 pads; pad size classes of
    ~2k / 5k / 10k verts; per-pad cylinder peg poses.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

MM = 1e-3

# ---------------------------------------------------------------------------
# pads


@dataclasses.dataclass
class Pad:
    rest: np.ndarray          # float32 [V, 3]
    tets: np.ndarray          # int32 [T, 4], positive orientation
    fixed: np.ndarray         # int32 [F] Dirichlet vertices (bottom face)
    markers: np.ndarray       # float32 [M, 2] marker (x, y) on the top face
    size: tuple               # (Lx, Ly, Lz) metres

    @property
    def n_verts(self):
        return int(self.rest.shape[0])

    @property
    def n_tets(self):
        return int(self.tets.shape[0])


def _freudenthal_cells(nx, ny, nz):
    """Tets of the 6-tet Kuhn (Freudenthal) split of an nx x ny x nz grid.

    Every cell is split along its (0,0,0)-(1,1,1) diagonal into the six
    monotone lattice paths, which makes the split conforming across cells.
    Returns vertex-index tets in lattice order (x fastest) and the lattice
    coordinate of every vertex.
    """
    def vid(i, j, k):
        return (k * (ny + 1) + j) * (nx + 1) + i

    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for perm in itertools.permutations(range(3)):
                    c = [0, 0, 0]
                    path = [vid(i, j, k)]
                    for ax in perm:
                        c[ax] += 1
                        path.append(vid(i + c[0], j + c[1], k + c[2]))
                    tets.append(path)
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    lat = np.stack([ii.transpose(2, 1, 0).ravel(), jj.transpose(2, 1, 0).ravel(),
                    kk.transpose(2, 1, 0).ravel()], axis=1)
    return np.asarray(tets, dtype=np.int64), lat


def _orient(rest, tets):
    """Swap two corners of every tet whose signed volume is negative."""
    x = rest.astype(np.float64)
    d = np.linalg.det(np.stack([x[tets[:, 1]] - x[tets[:, 0]], x[tets[:, 2]] - x[tets[:, 0]],
                                x[tets[:, 3]] - x[tets[:, 0]]], axis=2))
    tets = tets.copy()
    neg = d < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def marker_grid(lx, ly, cols, rows, dtype=np.float32):
    """Centred uniform grid: ``cols`` markers along x, ``rows`` along y,
    pitch = side / (n + 1)."""
    xs = lx * (np.arange(cols) + 1) / (cols + 1)
    ys = ly * (np.arange(rows) + 1) / (rows + 1)
    gx, gy = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([gx.ravel(), gy.ravel()], axis=1).astype(dtype)


def hex_pad(size, cells, marker_shape=(9, 7), jitter=0.0, renumber=False, rng=None):
    """Box pad split into 6 tets per hex cell.

    ``jitter`` moves every vertex by U(-jitter, jitter) cell sizes along each
    axis that keeps it on its boundary faces (interior vertices move along all
    three axes); ``renumber`` applies random vertex and tet permutations so
    the index order carries no spatial structure.
    """
    lx, ly, lz = size
    nx, ny, nz = cells
    tets, lat = _freudenthal_cells(nx, ny, nz)
    h = np.array([lx / nx, ly / ny, lz / nz])
    rest = lat * h
    if jitter > 0.0:
        rng = rng if rng is not None else np.random.default_rng(0)
        n = np.array([nx, ny, nz])
        movable = (lat > 0) & (lat < n)            # per axis: not on a face normal to it
        for _ in range(50):
            d = rng.uniform(-jitter, jitter, size=rest.shape) * h * movable
            cand = rest + d
            t2 = _orient(cand, tets)
            x = cand
            vol = np.linalg.det(np.stack([x[t2[:, 1]] - x[t2[:, 0]], x[t2[:, 2]] - x[t2[:, 0]],
                                          x[t2[:, 3]] - x[t2[:, 0]]], axis=2))
            if np.all(vol > 0.05 * h.prod() / 6.0) and np.array_equal(t2, _orient(rest, tets)):
                rest = cand
                break
        else:
            raise RuntimeError("could not jitter the pad without inverting a tet")
    tets = _orient(rest, tets)
    fixed = np.nonzero(lat[:, 2] == 0)[0]
    if renumber:
        rng = rng if rng is not None else np.random.default_rng(0)
        perm = rng.permutation(rest.shape[0])       # new index of old vertex i is inv[i]
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        rest = rest[perm]
        tets = inv[tets]
        fixed = np.sort(inv[fixed])
        tets = tets[rng.permutation(tets.shape[0])]
    mk = marker_grid(lx, ly, marker_shape[0], marker_shape[1])
    return Pad(rest=rest.astype(np.float32), tets=tets.astype(np.int32), fixed=fixed.astype(np.int32),
               markers=mk, size=(lx, ly, lz))


# Hex-split pads sized to the 2k / 5k / 10k vertex classes on an
# 18.6 x 14.3 x 4 mm sensor gel (near-cubic cells).
SIZE_CLASSES = {
    2000: (22, 17, 4),     # 23*18*5  = 2070 verts,  8976 tets
    5000: (29, 22, 6),     # 30*23*7  = 4830 verts, 22968 tets
    10000: (37, 28, 8),    # 38*29*9  = 9918 verts, 49728 tets
}
SENSOR_SIZE = (18.6 * MM, 14.3 * MM, 4.0 * MM)

# ---------------------------------------------------------------------------
# indenters (rigid triangle meshes, outward winding)


@dataclasses.dataclass
class Indenter:
    verts: np.ndarray   # float32 [N, 3] local frame
    tris: np.ndarray    # int32 [K, 3]


def icosphere(radius, subdiv):
    """Icosahedron subdivided ``subdiv`` times and projected to the sphere,
    rotated so that one vertex is the lowest point (local -z pole)."""
    p = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p),
         (0, -1, -p), (0, 1, -p), (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = list(f)
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    # rotate vertex 6's direction onto -z so that a vertex is the lowest point
    a = V[6] / np.linalg.norm(V[6])
    b = np.array([0.0, 0.0, -1.0])
    ax = np.cross(a, b)
    s, c = np.linalg.norm(ax), float(a @ b)
    if s > 1e-12:
        k = ax / s
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        R = np.eye(3) + s * K + (1 - c) * K @ K
        V = V @ R.T
    F = np.array(faces, dtype=np.int64)
    # outward winding
    cen = V[F].mean(axis=1)
    nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return Indenter(verts=(V * radius).astype(np.float32), tris=F.astype(np.int32))


def cylinder(radius, length, n_around=64, n_along=8):
    """Closed cylinder with its axis along local x, centred at the origin."""
    xs = np.linspace(-length / 2, length / 2, n_along + 1)
    th = 2 * np.pi * np.arange(n_around) / n_around
    verts = [(x, radius * np.cos(t), radius * np.sin(t)) for x in xs for t in th]
    tris = []
    for i in range(n_along):
        for j in range(n_around):
            a = i * n_around + j
            b = i * n_around + (j + 1) % n_around
            c = (i + 1) * n_around + j
            d = (i + 1) * n_around + (j + 1) % n_around
            tris += [(a, b, d), (a, d, c)]
    c0 = len(verts)
    verts.append((xs[0], 0.0, 0.0))
    c1 = len(verts)
    verts.append((xs[-1], 0.0, 0.0))
    last = n_along * n_around
    for j in range(n_around):
        tris.append((c0, (j + 1) % n_around, j))
        tris.append((c1, last + j, last + (j + 1) % n_around))
    V = np.array(verts)
    F = np.array(tris, dtype=np.int64)
    cen = V[F].mean(axis=1) - np.array([1, 0, 0]) * 0.0
    nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    # outward: compare against the direction from the axis (or along x for caps)
    out = cen.copy()
    side = np.abs(np.abs(cen[:, 0]) - length / 2) > 1e-12
    out[side, 0] = 0.0
    out[~side, 1:] = 0.0
    flip = np.einsum("ij,ij->i", nrm, out) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return Indenter(verts=V.astype(np.float32), tris=F.astype(np.int32))


def box_edge(size=(24 * MM, 6 * MM, 6 * MM), n=(24, 6, 6)):
    """Rectangular bar (a box edge presses into the gel when rotated 45
    degrees about x); every face is a regular grid of quads split in two."""
    sx, sy, sz = size
    verts, tris, index = [], [], {}

    def v(p):
        key = tuple(np.round(np.asarray(p) / 1e-9).astype(np.int64))
        if key not in index:
            index[key] = len(verts)
            verts.append(p)
        return index[key]
    half = np.array(size) / 2
    for ax in range(3):
        u_ax, w_ax = [a for a in range(3) if a != ax]
        for sgn in (-1.0, 1.0):
            nu, nw = n[u_ax], n[w_ax]
            for i in range(nu):
                for j in range(nw):
                    q = []
                    for di, dj in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        p = np.zeros(3)
                        p[ax] = sgn * half[ax]
                        p[u_ax] = -half[u_ax] + (i + di) * size[u_ax] / nu
                        p[w_ax] = -half[w_ax] + (j + dj) * size[w_ax] / nw
                        q.append(v(p))
                    tris += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
    V = np.array(verts)
    F = np.array(tris, dtype=np.int64)
    cen = V[F].mean(axis=1)
    nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return Indenter(verts=V.astype(np.float32), tris=F.astype(np.int32))


def ridged_thread(radius=3 * MM, length=20 * MM, pitch=1.5 * MM, depth=0.4 * MM,
                  n_around=48, n_along=80):
    """Cylinder along x whose radius follows a triangular thread profile."""
    ind = cylinder(radius, length, n_around, n_along)
    V = ind.verts.astype(np.float64)
    ph = (V[:, 0] / pitch) % 1.0
    prof = depth * (1.0 - 2.0 * np.abs(ph - 0.5))
    rr = np.hypot(V[:, 1], V[:, 2])
    scale = np.where(rr > 0, (radius - depth + prof) / np.maximum(rr, 1e-30), 1.0)
    V[:, 1] *= scale
    V[:, 2] *= scale
    return Indenter(verts=V.astype(np.float32), tris=ind.tris)


def chamfered_peg(radius=2.5 * MM, length=12 * MM, chamfer=0.6 * MM, n_around=96, n_along=40, n_cap=12):
    """Closed peg with its axis along local z, centred at the origin, whose
    lower end is chamfered at 45 degrees by ``chamfer``: a surface of
    revolution (side rings down the straight part and the chamfer, then
    concentric rings across the lower face, a fan at each end). Convex, so
    each face is oriented away from the centroid."""
    zb, zt = -length / 2, length / 2
    # profile (r, z) from the top rim down the side and chamfer, then in to the axis
    n_ch = max(2, n_along // 8)
    zs = np.linspace(zt, zb + chamfer, n_along - n_ch + 1)
    prof = [(radius, z) for z in zs]
    prof += [(radius - chamfer * k / n_ch, zb + chamfer * (1 - k / n_ch)) for k in range(1, n_ch + 1)]
    r_end = radius - chamfer
    prof += [(r_end * (1 - k / n_cap), zb) for k in range(1, n_cap)]
    th = 2 * np.pi * np.arange(n_around) / n_around
    verts = [(r * np.cos(t), r * np.sin(t), z) for r, z in prof for t in th]
    tris = []
    for i in range(len(prof) - 1):
        for j in range(n_around):
            a = i * n_around + j
            b = i * n_around + (j + 1) % n_around
            c = (i + 1) * n_around + j
            d = (i + 1) * n_around + (j + 1) % n_around
            tris += [(a, b, d), (a, d, c)]
    top = len(verts)
    verts.append((0.0, 0.0, zt))
    bot = len(verts)
    verts.append((0.0, 0.0, zb))
    last = (len(prof) - 1) * n_around
    for j in range(n_around):
        tris.append((top, j, (j + 1) % n_around))
        tris.append((bot, last + j, last + (j + 1) % n_around))
    V = np.array(verts)
    F = np.array(tris, dtype=np.int64)
    cen = V[F].mean(axis=1) - V.mean(axis=0)
    nrm = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2].copy(), F[flip, 1].copy()
    return Indenter(verts=V.astype(np.float32), tris=F.astype(np.int32))


def nut_flank(radius=3 * MM, length=16 * MM, pitch=1.0 * MM, depth=0.35 * MM):
    """A threaded flank of about 10k triangles: the ridged thread profile
    on a cylinder along local x (64 around x 80 along)."""
    return ridged_thread(radius=radius, length=length, pitch=pitch, depth=depth, n_around=64, n_along=80)


def lowest_z(verts, rotvec):
    """Lowest local-frame-rotated z of an indenter (pose helper for placing
    the indenter above the gel; plain rotation, no solver arithmetic)."""
    R = _rotation(np.asarray(rotvec, dtype=np.float64))
    return float((verts.astype(np.float64) @ R.T)[:, 2].min())


def _box_dist(P, size):
    d = np.maximum(np.maximum(-P, P - np.asarray(size, dtype=np.float64)), 0.0)
    return np.sqrt(np.einsum("...c,...c->...", d, d))


def place_above_box(verts, rotvec, xy, size, gap, tris=None, n=4):
    """Height z of the translation (xy[0], xy[1], z) that puts the rotated
    indenter at minimum distance ``gap`` from the solid pad box
    [0, Lx] x [0, Ly] x [0, Lz] (scene placement only).

    Vertices alone fix a first height by bisection. With ``tris`` given,
    points sampled on the triangles that can reach the box (a triangle's
    points are within its diameter of its vertices) then raise it until the
    sampled surface is ``gap`` away."""
    R = _rotation(np.asarray(rotvec, dtype=np.float64))
    V = np.asarray(verts, dtype=np.float64) @ R.T
    V[:, 0] += xy[0]
    V[:, 1] += xy[1]
    over = (V[:, 0] > 0) & (V[:, 0] < size[0]) & (V[:, 1] > 0) & (V[:, 1] < size[1])
    if not np.any(over):
        raise ValueError("no indenter vertex lies over the pad")
    lo = 0.5 * size[2] - V[over, 2].min()   # a vertex inside the box: distance 0
    hi = size[2] - V[:, 2].min() + gap      # every vertex above the top: distance >= gap
    for _ in range(44):
        mid = 0.5 * (lo + hi)
        if _box_dist(V + np.array([0.0, 0.0, mid]), size).min() < gap:
            lo = mid
        else:
            hi = mid
    z = hi
    if tris is None:
        return z
    T = np.asarray(tris, dtype=np.int64)
    dv = _box_dist(V + np.array([0.0, 0.0, z]), size)[T]              # [K, 3]
    e = V[T]
    diam = np.max(np.linalg.norm(e[:, [1, 2, 0]] - e, axis=2), axis=1)
    near = dv.min(axis=1) < gap + diam
    ij = [(i, j) for i in range(n + 1) for j in range(n + 1 - i)]
    w = np.array([(1 - (i + j) / n, i / n, j / n) for i, j in ij])
    Ps = np.einsum("sk,tkc->tsc", w, e[near]).reshape(-1, 3)
    for _ in range(50):
        dm = _box_dist(Ps + np.array([0.0, 0.0, z]), size).min()
        if dm >= gap * (1.0 - 1e-6):
            break
        z += gap - dm            # the distance grows at most as fast as z
    return z


def _rotation(rv):
    th = float(np.linalg.norm(rv))
    if th < 1e-300:
        return np.eye(3)
    k = rv / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


# ---------------------------------------------------------------------------
# workloads

DHAT = 0.05 * MM


@dataclasses.dataclass
class Material:
    E: float = 0.3e6
    nu: float = 0.45
    rho: float = 1100.0
    h: float = 1.0 / 60.0
    dhat: float = DHAT
    mu_f: float = 0.0


@dataclasses.dataclass
class Workload:
    name: str
    pads: list                # [Pad] one per pad (pads may share arrays)
    materials: list           # [Material] one per pad
    indenters: list           # [Indenter] one per env
    pads_per_env: int
    poses: np.ndarray         # float32 [frames + 1, n_pads, 6]; row 0 = initial pose

    @property
    def n_pads(self):
        return len(self.pads)

    @property
    def n_envs(self):
        return len(self.indenters)

    @property
    def n_frames(self):
        return int(self.poses.shape[0]) - 1


def config_single_pad(frames=10, step=0.05 * MM):
    """20x16x4 mm pad, 10x8x2 hexes, icosphere r = 4 mm pressed at the pad
    centre in ``frames`` steps of ``step``; frictionless."""
    pad = hex_pad((20 * MM, 16 * MM, 4 * MM), (10, 8, 2), marker_shape=(9, 7))
    ind = icosphere(4 * MM, 2)
    lx, ly, lz = pad.size
    z0 = lz + DHAT - lowest_z(ind.verts, np.zeros(3))
    poses = np.zeros((frames + 1, 1, 6), dtype=np.float64)
    poses[:, 0, 3] = lx / 2
    poses[:, 0, 4] = ly / 2
    poses[:, 0, 5] = z0 - step * np.arange(frames + 1)
    return Workload("single_pad_297v_icosphere", [pad], [Material()], [ind], 1, poses.astype(np.float32))


def config_realistic(seed=0, frames=30, n_verts_target=20000, indenter_kind=None):
    """Jittered, renumbered pad on the 18.6x14.3x4 mm gel; press then slide
    with friction 0.5; E ~ U[0.1, 0.5] MPa."""
    rng = np.random.default_rng(np.random.PCG64(20260 + 2000 + seed))
    # cells scaled so that (nx+1)(ny+1)(nz+1) ~ n_verts_target
    k = (n_verts_target / (4.65 * 3.575)) ** (1 / 3)
    cells = (max(2, round(4.65 * k)), max(2, round(3.575 * k)), max(2, round(k)))
    pad = hex_pad(SENSOR_SIZE, cells, marker_shape=(11, 9), jitter=0.15, renumber=True, rng=rng)
    kind = indenter_kind or ["cylinder", "box_edge", "thread"][int(rng.integers(3))]
    if kind == "cylinder":
        ind = cylinder(3 * MM, 24 * MM, 64, 16)
    elif kind == "box_edge":
        ind = box_edge()
    else:
        ind = ridged_thread()
    rot = np.deg2rad(rng.uniform(-15, 15, size=3))
    if kind == "box_edge":
        rot[0] += np.pi / 4
    press = rng.uniform(0, 1.5 * MM)
    slide = rng.uniform(0, 1.0 * MM)
    lx, ly, lz = pad.size
    z0 = lz + DHAT - lowest_z(ind.verts, rot)
    n_press = frames // 2
    poses = np.zeros((frames + 1, 1, 6))
    poses[:, 0, :3] = rot
    poses[:, 0, 3] = lx / 2
    poses[:, 0, 4] = ly / 2
    for f in range(frames + 1):
        dz = press * min(f, n_press) / n_press
        dy = slide * max(0, f - n_press) / max(1, frames - n_press)
        poses[f, 0, 4] += dy
        poses[f, 0, 5] = z0 - dz
    mat = Material(E=float(rng.uniform(0.1e6, 0.5e6)), mu_f=0.5)
    return Workload(f"realistic_{pad.n_verts}v_{kind}", [pad], [mat], [ind], 1, poses.astype(np.float32))


_CLASS_CACHE = {}


def size_class_pad(cls):
    """Hex-split sensor pad of one size class (cached: pads of a class share
    their host arrays). Classes outside SIZE_CLASSES get cells in the
    sensor's aspect with about ``cls`` vertices."""
    if cls not in _CLASS_CACHE:
        if cls in SIZE_CLASSES:
            cells = SIZE_CLASSES[cls]
        else:
            k = (cls / (4.65 * 3.575)) ** (1 / 3)
            cells = (max(2, round(4.65 * k)), max(2, round(3.575 * k)), max(2, round(k)))
        _CLASS_CACHE[cls] = hex_pad(SENSOR_SIZE, cells, marker_shape=(9, 7))
    return _CLASS_CACHE[cls]


def config_batched(n_envs=4096, frames=12, seed=0, step=0.05 * MM, classes=(2000, 5000, 10000),
                   mu_f=0.5):
    """``n_envs`` environments x 2 pads. Per env: size class drawn uniformly,
    cylinder peg r ~ U[2, 4] mm (64 x 8 side quads). Per pad: rotation vector
    components ~ U(+-15 deg), xy offset ~ U(+-1 mm), press depth
    ~ U[0, 1.2] mm reached at ``step`` per frame from a d-hat gap to the pad
    (the indenter surface starts dhat from the solid pad box), then held."""
    rng = np.random.default_rng(np.random.PCG64(20260 + 3000 + seed))
    pads, mats, inds = [], [], []
    n_pads = 2 * n_envs
    poses = np.zeros((frames + 1, n_pads, 6))
    cyl_cache = {}
    for e in range(n_envs):
        cls = classes[int(rng.integers(len(classes)))]
        r = float(rng.uniform(2 * MM, 4 * MM))
        key = round(r / (0.05 * MM))          # quantise radii so meshes can be shared
        if key not in cyl_cache:
            cyl_cache[key] = cylinder(key * 0.05 * MM, 24 * MM, 64, 8)
        ind = cyl_cache[key]
        inds.append(ind)
        for q in range(2):
            pad = size_class_pad(cls)
            pads.append(pad)
            mats.append(Material(mu_f=mu_f))
            i = 2 * e + q
            rot = np.deg2rad(rng.uniform(-15, 15, size=3))
            off = rng.uniform(-1 * MM, 1 * MM, size=2)
            depth = float(rng.uniform(0, 1.2 * MM))
            lx, ly, lz = pad.size
            cx, cy = lx / 2 + off[0], ly / 2 + off[1]
            z0 = place_above_box(ind.verts, rot, (cx, cy), pad.size, DHAT, ind.tris)
            poses[:, i, :3] = rot
            poses[:, i, 3] = cx
            poses[:, i, 4] = cy
            poses[:, i, 5] = z0 - np.minimum(step * np.arange(frames + 1), depth + DHAT)
    return Workload(f"batched_{n_envs}env_x2pads", pads, mats, inds, 2, poses.astype(np.float32))


def config_calibration(n_envs=256, frames=16, seed=0, step=0.05 * MM, mu_f=0.5, pad_verts=5000):
    """Adjoint calibration workload: ``n_envs`` environments of one
    ``pad_verts``-vertex-class pad (default 5k) and a cylinder peg (r ~ U[2, 4] mm, rotation vector
    components ~ U(+-15 deg), xy offset ~ U(+-1 mm)). Each runs a
    press-and-slide sequence: ``frames // 2`` frames pressing ``step`` per
    frame from a d-hat gap, then ``frames - frames // 2`` frames sliding
    ``step`` per frame along a random in-plane direction at constant depth.
    Returns (workload at the nominal material, hidden per-env materials with
    E ~ U[0.1, 0.5] MPa, nu ~ U[0.40, 0.49], mu_f ~ U[0.3, 0.9])."""
    rng = np.random.default_rng(np.random.PCG64(20260 + 4000 + seed))
    pads, mats, inds, hidden = [], [], [], []
    poses = np.zeros((frames + 1, n_envs, 6))
    cyl_cache = {}
    n_press = frames // 2
    for e in range(n_envs):
        r = float(rng.uniform(2 * MM, 4 * MM))
        key = round(r / (0.05 * MM))
        if key not in cyl_cache:
            cyl_cache[key] = cylinder(key * 0.05 * MM, 24 * MM, 64, 8)
        ind = cyl_cache[key]
        pad = size_class_pad(pad_verts)
        pads.append(pad)
        mats.append(Material(mu_f=mu_f))
        inds.append(ind)
        hidden.append(Material(E=float(rng.uniform(0.1e6, 0.5e6)), nu=float(rng.uniform(0.40, 0.49)),
                               mu_f=float(rng.uniform(0.3, 0.9))))
        rot = np.deg2rad(rng.uniform(-15, 15, size=3))
        off = rng.uniform(-1 * MM, 1 * MM, size=2)
        ang = float(rng.uniform(0, 2 * np.pi))
        lx, ly, lz = pad.size
        cx, cy = lx / 2 + off[0], ly / 2 + off[1]
        z0 = place_above_box(ind.verts, rot, (cx, cy), pad.size, DHAT, ind.tris)
        k = np.arange(frames + 1)
        press = step * np.minimum(k, n_press)
        slide = step * np.maximum(k - n_press, 0)
        poses[:, e, :3] = rot
        poses[:, e, 3] = cx + np.cos(ang) * slide
        poses[:, e, 4] = cy + np.sin(ang) * slide
        poses[:, e, 5] = z0 - press
    w = Workload(f"calibration_{n_envs}env", pads, mats, inds, 1, poses.astype(np.float32))
    return w, hidden


def config_trajectory(n_envs=64, n_verts=50000, frames=60, seed=0, step=0.05 * MM, slide_step=0.02 * MM,
                      mu_f=0.5):
    """Long trajectories on fine pads (the large-scale sweep's configuration):
    ``n_envs`` environments of one hex-split pad of about ``n_verts``
    vertices and an indenter of about 10k triangles, alternately a
    chamfered peg pressing its end (axis near vertical) and a threaded nut
    flank pressing its thread (axis near horizontal). Per env: rotation
    vector components ~ U(+-15 deg) about the indenter's nominal
    orientation, xy offset ~ U(+-1 mm); the indenter presses ``step`` per
    frame from a d-hat gap to a depth ~ U[0.2, 1.0] mm and holds until half
    the frames, then slides ``slide_step`` per frame along a random
    in-plane direction at that depth; friction ``mu_f``."""
    rng = np.random.default_rng(np.random.PCG64(20260 + 6000 + seed))
    pad = size_class_pad(n_verts)
    peg, flank = chamfered_peg(), nut_flank()
    pads, mats, inds = [], [], []
    poses = np.zeros((frames + 1, n_envs, 6))
    half = frames // 2
    for e in range(n_envs):
        ind = peg if e % 2 == 0 else flank
        pads.append(pad)
        mats.append(Material(mu_f=mu_f))
        inds.append(ind)
        rot = np.deg2rad(rng.uniform(-15, 15, size=3))
        off = rng.uniform(-1 * MM, 1 * MM, size=2)
        depth = float(rng.uniform(0.2 * MM, 1.0 * MM))
        ang = float(rng.uniform(0, 2 * np.pi))
        lx, ly, lz = pad.size
        cx, cy = lx / 2 + off[0], ly / 2 + off[1]
        z0 = place_above_box(ind.verts, rot, (cx, cy), pad.size, DHAT, ind.tris)
        k = np.arange(frames + 1)
        press = np.minimum(step * np.minimum(k, half), depth + DHAT)
        slide = slide_step * np.maximum(k - half, 0)
        poses[:, e, :3] = rot
        poses[:, e, 3] = cx + np.cos(ang) * slide
        poses[:, e, 4] = cy + np.sin(ang) * slide
        poses[:, e, 5] = z0 - press
    return Workload(f"trajectory_{n_envs}env_{pad.n_verts}v", pads, mats, inds, 1, poses.astype(np.float32))


def config_sweep(n_envs, n_verts, frames=8, seed=0, step=0.05 * MM, mu_f=0.5):
    """Throughput sweep workload: ``n_envs`` environments of one pad of about
    ``n_verts`` vertices (hex-split sensor pad) and a cylinder peg
    (r ~ U[2, 4] mm, rotation vector components ~ U(+-15 deg), xy offset
    ~ U(+-1 mm)), pressed ``step`` per frame from a d-hat gap to a depth
    ~ U[0, 1.2] mm, then held; friction ``mu_f``."""
    rng = np.random.default_rng(np.random.PCG64(20260 + 5000 + seed))
    pads, mats, inds = [], [], []
    poses = np.zeros((frames + 1, n_envs, 6))
    cyl_cache = {}
    pad = size_class_pad(n_verts)
    for e in range(n_envs):
        r = float(rng.uniform(2 * MM, 4 * MM))
        key = round(r / (0.05 * MM))
        if key not in cyl_cache:
            cyl_cache[key] = cylinder(key * 0.05 * MM, 24 * MM, 64, 8)
        ind = cyl_cache[key]
        pads.append(pad)
        mats.append(Material(mu_f=mu_f))
        inds.append(ind)
        rot = np.deg2rad(rng.uniform(-15, 15, size=3))
        off = rng.uniform(-1 * MM, 1 * MM, size=2)
        depth = float(rng.uniform(0, 1.2 * MM))
        lx, ly, lz = pad.size
        cx, cy = lx / 2 + off[0], ly / 2 + off[1]
        z0 = place_above_box(ind.verts, rot, (cx, cy), pad.size, DHAT, ind.tris)
        poses[:, e, :3] = rot
        poses[:, e, 3] = cx
        poses[:, e, 4] = cy
        poses[:, e, 5] = z0 - np.minimum(step * np.arange(frames + 1), depth + DHAT)
    return Workload(f"sweep_{n_envs}env_{pad.n_verts}v", pads, mats, inds, 1, poses.astype(np.float32))
