"""Rest-shape quantities, surface primitives, markers, indenter placement
(oracle, FP64).

Canonical orderings (shared by definition with the library, so that pair
sets can be compared index by index):
  * surface triangles: boundary faces of the tet mesh (faces that belong to
    exactly one tet), each stored with its vertex ids sorted ascending, the
    list sorted lexicographically;
  * surface edges: the distinct edges of the surface triangles, (lo, hi),
    sorted lexicographically;
  * surface vertices: the distinct vertices of the surface triangles, sorted;
  * indenter edges: the distinct edges of the indenter triangles, (lo, hi),
    sorted; indenter triangles keep their input order.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial.transform import Rotation


def lame(E, nu):
    """Lame parameters (mu, lambda) of Young's modulus E and Poisson ratio nu."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def rest_shape(rest, tets):
    """Dm^-1 and rest volume per tet: Dm = [X1-X0, X2-X0, X3-X0] (columns),
    volume = det(Dm) / 6 (linear tetrahedra, Supp. A)."""
    X = np.asarray(rest, dtype=np.float64)
    t = np.asarray(tets)
    Dm = np.stack([X[t[:, 1]] - X[t[:, 0]], X[t[:, 2]] - X[t[:, 0]], X[t[:, 3]] - X[t[:, 0]]], axis=2)
    vol = np.linalg.det(Dm) / 6.0
    return np.linalg.inv(Dm), vol


def lumped_mass(n_verts, tets, vol, rho):
    """Lumped mass: each tet gives rho * V / 4 to each of its corners."""
    m = np.zeros(n_verts)
    np.add.at(m, np.asarray(tets).ravel(), np.repeat(rho * vol / 4.0, 4))
    return m


def surface(tets):
    """Canonical surface triangles, edges and vertices of a tet mesh."""
    t = np.asarray(tets, dtype=np.int64)
    faces = np.concatenate([t[:, [0, 1, 2]], t[:, [0, 1, 3]], t[:, [0, 2, 3]], t[:, [1, 2, 3]]])
    faces = np.sort(faces, axis=1)
    uniq, counts = np.unique(faces, axis=0, return_counts=True)
    tris = uniq[counts == 1]                         # np.unique sorts lexicographically
    edges = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [0, 2]]])
    edges = np.unique(np.sort(edges, axis=1), axis=0)
    verts = np.unique(tris.ravel())
    return tris, edges, verts


def mesh_edges(tris):
    """Canonical distinct edges of a triangle mesh."""
    t = np.asarray(tris, dtype=np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [0, 2]]])
    return np.unique(np.sort(e, axis=1), axis=0)


def marker_map(rest, surf_tris, markers_xy):
    """Barycentric mapping of markers onto the rest top face.

    Top-face triangles are surface triangles whose three rest vertices lie at
    the maximum rest z. Each marker takes the top triangle that maximises its
    smallest 2-D barycentric coordinate (the containing triangle; ties at
    shared edges resolve to the first in canonical order). Returns
    (tri vertex ids [M, 3], weights [M, 3])."""
    X = np.asarray(rest, dtype=np.float64)
    ztop = X[:, 2].max()
    top = surf_tris[np.all(X[surf_tris][:, :, 2] == ztop, axis=1)]
    a, b, c = X[top[:, 0], :2], X[top[:, 1], :2], X[top[:, 2], :2]
    ids = np.zeros((len(markers_xy), 3), dtype=np.int64)
    w = np.zeros((len(markers_xy), 3))
    for m, q in enumerate(np.asarray(markers_xy, dtype=np.float64)):
        v0, v1, v2 = b - a, c - a, q[None, :] - a
        den = v0[:, 0] * v1[:, 1] - v1[:, 0] * v0[:, 1]
        l1 = (v2[:, 0] * v1[:, 1] - v1[:, 0] * v2[:, 1]) / den
        l2 = (v0[:, 0] * v2[:, 1] - v2[:, 0] * v0[:, 1]) / den
        l0 = 1.0 - l1 - l2
        score = np.minimum(np.minimum(l0, l1), l2)
        k = int(np.argmax(score))
        ids[m] = top[k]
        w[m] = (l0[k], l1[k], l2[k])
    return ids, w


def marker_map_knn(rest, markers_xy, k=4):
    """kNN inverse-distance mapping of markers onto rest mesh nodes (Sec. 3.2:
    the k nearest initial nodes, the marker displacement interpolated from
    them with weights). Readings: the candidate nodes are those of the rest
    top face (rest z equal to the maximum rest z, the face the markers lie
    on); distance is the 2-D distance in that face, ranked by the squared
    distance dx^2 + dy^2 with ties to the smaller node id; the k nearest take
    weights w_i proportional to 1/d_i, normalised to sum to 1 (summed in
    rank order); a marker at zero distance from its nearest node takes that
    node alone. Returns (node ids [M, k], weights [M, k])."""
    X = np.asarray(rest, dtype=np.float64)
    top = np.flatnonzero(X[:, 2] == X[:, 2].max())
    if top.size < k:
        raise ValueError("fewer top-face nodes than marker neighbours")
    nm = len(markers_xy)
    ids = np.zeros((nm, k), dtype=np.int64)
    w = np.zeros((nm, k))
    for m, q in enumerate(np.asarray(markers_xy, dtype=np.float64)):
        dx, dy = X[top, 0] - q[0], X[top, 1] - q[1]
        d2 = dx * dx + dy * dy
        order = np.lexsort((top, d2))[:k]
        ids[m] = top[order]
        d = np.sqrt(d2[order])
        if d[0] == 0.0:
            w[m, 0] = 1.0
        else:
            inv = 1.0 / d
            w[m] = inv / inv.sum()
    return ids, w


def indenter_world(verts, pose):
    """World (pad-frame) indenter vertices y = R(rotvec) Y + t for a pose
    (rotvec[3], t[3])."""
    pose = np.asarray(pose, dtype=np.float64)
    R = Rotation.from_rotvec(pose[:3]).as_matrix()
    return np.asarray(verts, dtype=np.float64) @ R.T + pose[3:]


def mean_surface_edge(rest, surf_edges):
    """Mean rest length of the surface edges (the length scale l-bar)."""
    X = np.asarray(rest, dtype=np.float64)
    return float(np.linalg.norm(X[surf_edges[:, 1]] - X[surf_edges[:, 0]], axis=1).mean())


@dataclasses.dataclass
class PadModel:
    """Everything the oracle precomputes for one pad."""
    rest: np.ndarray
    tets: np.ndarray
    Dm_inv: np.ndarray
    vol: np.ndarray
    mass: np.ndarray
    free: np.ndarray          # bool [V]: not Dirichlet
    surf_tris: np.ndarray
    surf_edges: np.ndarray
    surf_verts: np.ndarray
    marker_ids: np.ndarray
    marker_w: np.ndarray
    mu: float
    lam: float
    rho: float
    h: float
    dhat: float
    kappa: float
    mu_f: float
    eps_v: float
    g_ref: float
    lbar: float


@dataclasses.dataclass
class IndenterModel:
    verts: np.ndarray         # local frame
    tris: np.ndarray
    edges: np.ndarray


def build_pad(rest, tets, fixed, markers_xy, E, nu, rho, h, dhat, mu_f, kappa=None, eps_v=None,
              marker_mode="bary"):
    """Precompute a pad. Conventions: kappa (barrier stiffness) defaults to
    KAPPA_SCALE * h^2 E l-bar, eps_v (friction mollifier width, a
    displacement) to 1e-3 m/s * h, and the gradient scale of the stopping
    rule is g_ref = h^2 E l-bar dhat (the elastic gradient of a dhat-sized
    displacement over one element). marker_mode "bary" maps each marker to
    its rest top-face triangle (marker_map), "knn" to its 4 nearest rest
    nodes with inverse-distance weights (marker_map_knn)."""
    rest = np.asarray(rest, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    Dm_inv, vol = rest_shape(rest, tets)
    if np.any(vol <= 0):
        raise ValueError("tet with non-positive rest volume")
    mass = lumped_mass(rest.shape[0], tets, vol, rho)
    free = np.ones(rest.shape[0], dtype=bool)
    free[np.asarray(fixed, dtype=np.int64)] = False
    st, se, sv = surface(tets)
    if marker_mode == "bary":
        mids, mw = marker_map(rest, st, markers_xy)
    elif marker_mode == "knn":
        mids, mw = marker_map_knn(rest, markers_xy)
    else:
        raise ValueError(f"unknown marker_mode {marker_mode!r}")
    mu, lam = lame(E, nu)
    lbar = mean_surface_edge(rest, se)
    if kappa is None or kappa <= 0:
        kappa = KAPPA_SCALE * h * h * E * lbar
    if eps_v is None or eps_v <= 0:
        eps_v = 1e-3 * h
    return PadModel(rest=rest, tets=tets, Dm_inv=Dm_inv, vol=vol, mass=mass, free=free,
                    surf_tris=st, surf_edges=se, surf_verts=sv, marker_ids=mids, marker_w=mw,
                    mu=mu, lam=lam, rho=rho, h=h, dhat=dhat, kappa=kappa, mu_f=mu_f,
                    eps_v=eps_v, g_ref=h * h * E * lbar * dhat, lbar=lbar)


KAPPA_SCALE = 1.0


def build_indenter(verts, tris):
    return IndenterModel(verts=np.asarray(verts, dtype=np.float64), tris=np.asarray(tris, dtype=np.int64),
                         edges=mesh_edges(tris))
