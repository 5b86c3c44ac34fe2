"""The library's marker map (host preprocessing, no device work) against the
oracle's, bit for bit: neighbour ids exactly, weights as float32 of the
oracle's FP64 weights (the library rounds once, from the same FP64 values).

Both readings of Sec. 3.2 are covered: the barycentric map on the rest
top-face triangle and the kNN inverse-distance map over the rest top-face
nodes, on a regular pad, a jittered and renumbered pad (no structure in the
ids) and a pad whose markers sit on nodes, edges and cell centres (exact
distance ties, settled by the smaller id on both sides).
"""
import ctypes

import numpy as np
import pytest

from oracle import geometry as G
from paper_2603_28475_b300 import scenes as S

from _cases import MM


@pytest.fixture(scope="module")
def tac():
    from paper_2603_28475_b300 import build, tac as T
    build.build()
    return T


def _pads():
    rng = np.random.default_rng(11)
    reg = S.hex_pad((18.6 * MM, 14.3 * MM, 4 * MM), (12, 9, 3), marker_shape=(9, 7))
    jit = S.hex_pad((18.6 * MM, 14.3 * MM, 4 * MM), (14, 11, 3), marker_shape=(11, 9), jitter=0.25,
                    renumber=True, rng=rng)
    sp = 2.0 ** -9
    tie = S.hex_pad((6 * sp, 4 * sp, 2 * sp), (6, 4, 2), marker_shape=(3, 3))
    tie.markers = (np.stack(np.meshgrid(np.arange(13), np.arange(9), indexing="ij"), -1).reshape(-1, 2)
                   * (sp / 2)).astype(np.float32)
    return {"regular": reg, "jittered_renumbered": jit, "ties": tie}


def _oracle_map(pd, mode):
    X = pd.rest.astype(np.float64)
    mk = pd.markers.astype(np.float32).astype(np.float64)
    if mode == 1:
        return G.marker_map_knn(X, mk)
    st, _, _ = G.surface(pd.tets)
    return G.marker_map(X, st, mk)


@pytest.mark.parametrize("mode", [0, 1], ids=["barycentric", "knn_idw"])
@pytest.mark.parametrize("name", ["regular", "jittered_renumbered", "ties"])
def test_library_marker_map_is_the_oracle_map(tac, name, mode):
    pd = _pads()[name]
    ids, w = tac.marker_map(pd, mode)
    oid, ow = _oracle_map(pd, mode)
    k = oid.shape[1]
    assert np.array_equal(ids[:, :k], oid)
    assert np.array_equal(w[:, :k], ow.astype(np.float32))
    if k == 3:                                   # the unused fourth slot
        assert np.all(w[:, 3] == 0) and np.array_equal(ids[:, 3], ids[:, 0])


def test_marker_map_rejects_bad_mode_and_bad_mesh(tac):
    pd = _pads()["regular"]
    with pytest.raises(tac.TacError):
        tac.marker_map(pd, 2)
    pd.markers = pd.markers.copy()
    pd.markers[0] = (-1.0, -1.0)                 # off the top face
    with pytest.raises(tac.TacError):
        tac.marker_map(pd, 0)
