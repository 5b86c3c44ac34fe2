"""The rest-shape table of structured meshes on the GPU (through the C ABI).

* On an exact grid (dyadic coordinates: every tet of a kind has the same
  float32 Dm^-1) the table path and the per-tet path are bit-identical.
* On the regular single-pad press, whose float32 coordinates make tets of
  one kind differ in the last bits, the two paths agree within the parity
  tolerance, and the table path matches the FP64 oracle (which always uses
  the exact per-tet rest shapes) within it.
* With friction and the three size classes of the batched press, both paths
  converge and agree within the parity tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM, c1

pytestmark = pytest.mark.gpu
TOL = 1e-4 * 4 * MM


@pytest.fixture(scope="module")
def tac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac as T
    return T


def _run(tac, w, dm_table, frames):
    b = tac.batch_from_workload(w, dm_table=dm_table, pair_capacity=8192)
    poses = torch.tensor(w.poses, dtype=torch.float32, device=b.device)
    b.reset(poses[0])
    xs, mks, sts, its = [], [], [], []
    for f in range(1, frames + 1):
        b.set_indenter(poses[f])
        st, it = b.step()
        x, _ = b.get_state()
        xs.append(x.cpu().numpy())
        mks.append(b.markers().cpu().numpy())
        sts.append(st.cpu().numpy())
        its.append(it.cpu().numpy())
    b.close()
    return xs, mks, sts, its


def _dyadic_press(frames=4):
    sp = 2.0 ** -9                                  # 1.95 mm cells, exact in binary
    pad = S.hex_pad((10 * sp, 8 * sp, 2 * sp), (10, 8, 2), marker_shape=(9, 7))
    ind = S.icosphere(4 * MM, 2)
    lx, ly, lz = pad.size
    z0 = lz + S.DHAT - S.lowest_z(ind.verts, np.zeros(3))
    poses = np.zeros((frames + 1, 1, 6))
    poses[:, 0, 3], poses[:, 0, 4] = lx / 2, ly / 2
    poses[:, 0, 5] = z0 - 0.05 * MM * np.arange(frames + 1)
    return S.Workload("dyadic_single_pad", [pad], [S.Material()], [ind], 1, poses.astype(np.float32))


def test_exact_grid_table_is_bitwise_the_per_tet_path(tac):
    w = _dyadic_press()
    assert tac.mesh_info(w.pads[0])["dm_dev"] == 0.0
    a = _run(tac, w, True, 4)
    b = _run(tac, w, False, 4)
    for f in range(4):
        for k in range(4):
            assert np.array_equal(a[k][f], b[k][f]), (f, k)
    assert np.abs(a[0][-1] - w.pads[0].rest).max() > 1e-5       # the pad was pressed


def test_regular_pad_table_path_matches_oracle_and_per_tet_path(tac):
    w, pad, ind = c1()
    assert tac.mesh_info(w.pads[0])["dm_types"] == 6
    frames = 10
    xt, mt, st, _ = _run(tac, w, True, frames)
    xp, mp, sp_, _ = _run(tac, w, False, frames)
    poses = w.poses[:, 0].astype(np.float64)
    states, infos = SV.run(pad, ind, poses)
    worst = 0.0
    for f in range(frames):
        assert st[f][0] == 0 and sp_[f][0] == 0
        worst = max(worst, np.abs(xt[f] - xp[f]).max())
        assert np.abs(xt[f] - states[f + 1].x).max() <= TOL
        assert np.abs(mt[f] - SV.markers(pad, states[f + 1].x)).max() <= TOL
    print(f"table vs per-tet Dm^-1: max |dx| {worst:.2e} m over {frames} frames")
    assert worst <= TOL


def test_batched_press_table_and_per_tet_paths_agree(tac):
    w = S.config_batched(n_envs=6, frames=5, seed=2)
    xt, mt, st, _ = _run(tac, w, True, 5)
    xp, mp, sp_, _ = _run(tac, w, False, 5)
    for f in range(5):
        assert np.all(st[f] == 0) and np.all(sp_[f] == 0), (f, st[f], sp_[f])
        assert np.abs(xt[f] - xp[f]).max() <= TOL
        assert np.abs(mt[f] - mp[f]).max() <= TOL
