"""Host-side mesh layout of the library (no device work): the colour
classes of the tet patches and the rest-shape table of structured meshes.

Colour classes: no two patches of one class share a vertex (the scatter
passes write a class's vertices without synchronisation), and the balanced
classes take no more warp rounds than the greedy colouring did, within a
few rounds of the bound ceil(patches / 8).

A regular hex-split grid has one rest shape per tet of the cell split (6).
Its float32 coordinates are exact multiples of the cell size only up to
rounding, so the tets of one kind differ in the last bits and the library
groups them within a relative tolerance. Checked here: the number of
classes; the recorded deviation against one computed independently from
the oracle's FP64 rest shapes; exact grids (dyadic coordinates) give zero
deviation; irregular meshes fall back to per-tet Dm^-1.
"""
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


def _class_spread(pd):
    """Largest entry deviation of a tet's float32 Dm^-1 from the first tet of
    its kind, relative to that tet's largest entry, with kinds found by
    rounding the entries to 1e-3 of the largest entry."""
    Dm, _ = G.rest_shape(pd.rest.astype(np.float32).astype(np.float64), pd.tets)
    B = Dm.reshape(-1, 9).astype(np.float32).astype(np.float64)
    q = np.round(B / np.abs(B).max() * 1e3).astype(np.int64)
    _, first, inv = np.unique(q, axis=0, return_index=True, return_inverse=True)
    rep = B[first][inv.ravel()]
    return len(first), float((np.abs(B - rep).max(axis=1) / np.abs(rep).max(axis=1)).max())


@pytest.mark.parametrize("cls", [2000, 5000, 10000])
def test_regular_pads_have_six_rest_shapes(tac, cls):
    pd = S.size_class_pad(cls)
    info = tac.mesh_info(pd)
    kinds, spread = _class_spread(pd)
    assert kinds == 6 and info["dm_types"] == 6
    assert 0 < info["dm_dev"] <= 1e-5
    # the library's representatives are some member of each kind: its
    # deviation is at most twice the spread about the first member
    assert info["dm_dev"] <= 2 * spread + 1e-12
    assert info["patches"] * 32 >= pd.n_tets


def test_exact_grid_has_zero_deviation(tac):
    sp = 2.0 ** -9
    pd = S.hex_pad((6 * sp, 4 * sp, 2 * sp), (6, 4, 2), marker_shape=(3, 3))
    info = tac.mesh_info(pd)
    assert info["dm_types"] == 6 and info["dm_dev"] == 0.0


def test_irregular_mesh_streams_per_tet_rest_shapes(tac):
    pd = S.hex_pad((18.6 * MM, 14.3 * MM, 4 * MM), (14, 11, 3), jitter=0.25, renumber=True,
                   rng=np.random.default_rng(5))
    assert tac.mesh_info(pd)["dm_types"] == 0


@pytest.mark.parametrize("pd", [S.size_class_pad(2000), S.size_class_pad(5000), S.size_class_pad(10000),
                                S.hex_pad((18.6 * MM, 14.3 * MM, 4 * MM), (14, 11, 3), jitter=0.25, renumber=True,
                                          rng=np.random.default_rng(9))],
                         ids=["2k", "5k", "10k", "jittered_renumbered"])
def test_colour_classes_share_no_vertex_and_are_balanced(tac, pd):
    info = tac.mesh_info(pd)
    assert info["conflicts"] == 0
    bound = -(-info["patches"] // 8)
    assert bound <= info["rounds"] <= bound + info["colours"] // 4


def test_degenerate_meshes_lay_out(tac):
    """The smallest mesh (one tet) and a pad without markers."""
    import types
    one = types.SimpleNamespace(rest=np.array([[0, 0, 0], [1e-3, 0, 0], [0, 1e-3, 0], [0, 0, 1e-3]], np.float32),
                                tets=np.array([[0, 1, 2, 3]], np.int32), fixed=np.array([0, 1, 2], np.int32),
                                markers=np.zeros((0, 2), np.float32))
    info = tac.mesh_info(one)
    assert (info["patches"], info["colours"], info["rounds"], info["conflicts"], info["dm_types"]) == (1, 1, 1, 0, 1)
    assert info["dm_dev"] == 0.0
    for mode in (0, 1):
        ids, w = tac.marker_map(one, mode)
        assert ids.shape == (0, 4) and w.shape == (0, 4)
    pd = S.size_class_pad(2000)
    bare = types.SimpleNamespace(rest=pd.rest, tets=pd.tets, fixed=pd.fixed, markers=np.zeros((0, 2), np.float32))
    assert tac.mesh_info(bare)["conflicts"] == 0
