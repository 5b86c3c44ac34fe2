"""Contact candidate set (oracle, FP64).

The set C of Eq. (ipc_energy) is taken as every (gel-surface primitive,
indenter primitive) pair of the three types whose axis-aligned bounding
boxes overlap once the gel primitive's box is inflated by r = dhat + margin.
It is evaluated here by its definition, over the full Cartesian product, in
float64 on the float32 input coordinates:

    overlap  <=>  for every axis:  (gel_lo - r) <= ind_hi  and  ind_lo <= (gel_hi + r)

The result is a list of (type, i, j) triples sorted lexicographically
(type 0: gel vertex id x indenter triangle; type 1: gel surface triangle x
indenter vertex; type 2: gel surface edge x indenter edge). Any pair whose
distance is below r is in the set; pairs outside it are farther than r.
"""
from __future__ import annotations

import numpy as np

from . import energy as En


def _boxes(pos, prims):
    P = pos[prims]                      # [n, k, 3]
    return P.min(axis=1), P.max(axis=1)


def _overlap_pairs(glo, ghi, ilo, ihi, r, chunk=4096):
    out_i, out_j = [], []
    for s in range(0, glo.shape[0], chunk):
        a_lo = glo[s:s + chunk, None, :] - r
        a_hi = ghi[s:s + chunk, None, :] + r
        ok = np.all((a_lo <= ihi[None]) & (ilo[None] <= a_hi), axis=2)
        ii, jj = np.nonzero(ok)
        out_i.append(ii + s)
        out_j.append(jj)
    if not out_i:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(out_i), np.concatenate(out_j)


def candidates(x, y, pad, ind, r):
    """Sorted candidate triples [n, 3] for gel positions x and indenter world
    vertices y (both float64 arrays holding float32 values)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = []
    # type 0: gel surface vertex x indenter triangle
    sv = pad.surf_verts
    ilo, ihi = _boxes(y, ind.tris)
    i, j = _overlap_pairs(x[sv], x[sv], ilo, ihi, r)
    out.append(np.stack([np.zeros_like(i), sv[i], j], 1))
    # type 1: gel surface triangle x indenter vertex
    glo, ghi = _boxes(x, pad.surf_tris)
    i, j = _overlap_pairs(glo, ghi, y, y, r)
    out.append(np.stack([np.ones_like(i), i, j], 1))
    # type 2: gel surface edge x indenter edge
    glo, ghi = _boxes(x, pad.surf_edges)
    ilo, ihi = _boxes(y, ind.edges)
    i, j = _overlap_pairs(glo, ghi, ilo, ihi, r)
    out.append(np.stack([np.full_like(i, 2), i, j], 1))
    allp = np.concatenate(out).astype(np.int64)
    order = np.lexsort((allp[:, 2], allp[:, 1], allp[:, 0]))
    return allp[order]


def all_pairs(pad, ind):
    """Every (type, i, j) triple of the three types (the brute-force domain)."""
    nsv, nst, nse = pad.surf_verts.size, pad.surf_tris.shape[0], pad.surf_edges.shape[0]
    nit, niv, nie = ind.tris.shape[0], ind.verts.shape[0], ind.edges.shape[0]
    a = np.stack(np.meshgrid(pad.surf_verts, np.arange(nit), indexing="ij"), -1).reshape(-1, 2)
    b = np.stack(np.meshgrid(np.arange(nst), np.arange(niv), indexing="ij"), -1).reshape(-1, 2)
    c = np.stack(np.meshgrid(np.arange(nse), np.arange(nie), indexing="ij"), -1).reshape(-1, 2)
    return np.concatenate([np.c_[np.zeros(len(a), np.int64), a], np.c_[np.ones(len(b), np.int64), b],
                           np.c_[np.full(len(c), 2, np.int64), c]])


def brute_force_close(x, y, pad, ind, dist):
    """Every triple whose exact distance is below ``dist`` (all-pairs search;
    tiny meshes only)."""
    ap = all_pairs(pad, ind)
    d, _, _ = En.distances(ap, np.asarray(x, np.float64), np.asarray(y, np.float64), pad, ind)
    return ap[d < dist]
