"""Parity of the CUDA path with the FP64 oracle on the same seeded inputs.

All calls go through the C ABI (libtac.so via the ctypes binding).
Tolerances: positions and markers within 1e-4 of the gel thickness (max
abs error); per-iteration pieces within float32-derived relative bounds;
candidate pair sets bit-exact on identical float32 inputs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import broadphase as BP
from oracle import energy as En
from oracle import geometry as G
from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM, c1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac as T
    return T


@pytest.fixture(scope="module")
def c1_oracle():
    w, pad, ind = c1()
    poses = w.poses[:, 0].astype(np.float64)
    states, infos = SV.run(pad, ind, poses)
    return w, pad, ind, poses, states, infos


def _world32(ind, pose):
    return G.indenter_world(ind.verts, pose).astype(np.float32)


def _oracle_eval(pad, ind, u32, p, alpha, pose):
    rest32 = pad.rest.astype(np.float32)
    x = pad.rest + u32.astype(np.float64)
    x32 = (rest32 + u32).astype(np.float64)
    y = _world32(ind, pose).astype(np.float64)
    pairs = BP.candidates(x32, y, pad, ind, 2 * pad.dhat)
    empty = En.friction_lag(np.zeros((0, 3), np.int64), x, y, pad, ind)
    fr = En.Frame(pad, ind, x, x, y, y, empty)
    xa = x + alpha * p
    E0 = En.energy_only(fr, x, 1.0, pairs)
    E1 = En.energy_only(fr, xa, 1.0, pairs)
    _, g1, blk1 = En.total(fr, xa, 1.0, pairs)
    php_e = float(En.elastic_line(x, p, pad).dd)
    php_c = float(En.contact_line(pairs, x, p, y, pad, ind).dd)
    php_m = float(En.inertia_line(x, p, x, pad).dd)
    accd = SV.ccd_bound(fr, x, p, 1.0, pairs, 0.9)
    dmin = SV.min_distance(fr, x, 1.0, pairs)
    return dict(g=g1, blk=blk1, php_e=php_e, php_c=php_c, php_m=php_m, dE=E1 - E0, accd=accd, dmin=dmin,
                npairs=len(pairs))


def _smooth_field(pad, scale, seed):
    rng = np.random.default_rng(seed)
    X = pad.rest
    k = rng.normal(size=(3, 3)) * 400.0
    ph = rng.uniform(0, 6.28, size=3)
    p = np.stack([np.sin(X @ k[c] + ph[c]) for c in range(3)], axis=1) * scale
    p[~pad.free] = 0.0
    return p


def _blk6(blk):
    return np.stack([blk[:, 0, 0], blk[:, 1, 1], blk[:, 2, 2], blk[:, 0, 1], blk[:, 0, 2], blk[:, 1, 2]], axis=1)


@pytest.mark.parametrize("frame", [0, 3, 9])
def test_iteration_pieces_match_oracle(tac, c1_oracle, frame):
    """Gradient, diagonal blocks, p^T H p (elastic / contact / inertia), the
    line energy change, the per-pair step bound and the minimum distance of
    one PNCG iteration, GPU vs oracle, at oracle states of the single-pad
    workload."""
    w, pad, ind, poses, states, infos = c1_oracle
    pose = poses[frame]
    u32 = (states[frame].x - pad.rest).astype(np.float32)
    p = _smooth_field(pad, 2e-6, frame)
    y = _world32(ind, pose).astype(np.float64)
    x = pad.rest + u32.astype(np.float64)
    x32 = (pad.rest.astype(np.float32) + u32).astype(np.float64)
    pairs = BP.candidates(x32, y, pad, ind, 2 * pad.dhat)
    fr = En.Frame(pad, ind, x, x, y, y, En.friction_lag(np.zeros((0, 3), np.int64), x, y, pad, ind))
    alpha = 0.5 * min(1.0, SV.ccd_bound(fr, x, p, 1.0, pairs, 0.9))
    ref = _oracle_eval(pad, ind, u32, p, alpha, pose)
    b = tac.batch_from_workload(w)
    b.reset(torch.tensor(pose, dtype=torch.float32).reshape(1, 6))
    g, k, sc = b.debug_eval(torch.tensor(u32), torch.tensor(p, dtype=torch.float32), alpha)
    torch.cuda.synchronize()
    g, k, sc = g.cpu().numpy().astype(np.float64), k.cpu().numpy().astype(np.float64), sc.cpu().numpy()[0]
    gs = np.abs(ref["g"]).max()
    assert np.abs(g - ref["g"]).max() <= 2e-4 * gs
    kref = _blk6(ref["blk"])
    free = pad.free
    assert np.abs(k[free] - kref[free]).max() <= 1e-4 * np.abs(kref[free]).max()
    assert sc[0] == pytest.approx(ref["php_e"], rel=1e-4)
    assert sc[1] == pytest.approx(ref["php_c"], rel=1e-6, abs=1e-12 * abs(ref["php_e"]))
    assert sc[2] == pytest.approx(ref["php_m"], rel=1e-5)
    assert sc[3] == pytest.approx(ref["dE"], rel=2e-3, abs=1e-6 * abs(ref["dE"]) + 1e-22)
    if np.isfinite(ref["accd"]):
        assert sc[4] == pytest.approx(ref["accd"], rel=1e-5)
    if np.isfinite(ref["dmin"]):
        assert sc[5] == pytest.approx(ref["dmin"], rel=1e-6)
    assert abs(int(sc[6]) - ref["npairs"]) <= max(2, ref["npairs"] // 200)
    b.close()


def _bp_cases():
    w, pad, ind = c1()
    pd = w.pads[0]
    out = []
    rng = np.random.default_rng(11)
    for k in range(4):
        pose = w.poses[0, 0].astype(np.float64).copy()
        pose[:3] = rng.uniform(-0.3, 0.3, 3)
        pose[3:5] += rng.uniform(-2e-3, 2e-3, 2)
        pose[5] -= rng.uniform(0.0, 0.3e-3)
        u = (rng.normal(size=pd.rest.shape) * 2e-5).astype(np.float32)
        u[pd.fixed] = 0
        out.append((pose, u, [2 * pad.dhat, 0.4e-3][k % 2]))
    return out


@pytest.mark.parametrize("case", range(4))
def test_candidate_set_bit_exact(tac, case):
    w, pad, ind = c1()
    pose, u, r = _bp_cases()[case]
    x32 = (w.pads[0].rest + u).astype(np.float32)
    y32 = _world32(ind, pose)
    ref = BP.candidates(x32.astype(np.float64), y32.astype(np.float64), pad, ind, r)
    b = tac.batch_from_workload(w)
    got, n = b.broadphase(0, torch.tensor(x32), torch.tensor(y32), r, capacity=1 << 17)
    got = got.cpu().numpy().astype(np.int64)
    assert n == len(ref) and len(ref) > 0
    assert np.array_equal(got, ref)
    assert set(np.unique(ref[:, 0])) == {0, 1, 2} or r < 1e-3
    b.close()


def test_candidate_set_bit_exact_unstructured(tac):
    """Renumbered, jittered pad and a cylinder (C2-like, small)."""
    rng = np.random.default_rng(5)
    pd = S.hex_pad(S.SENSOR_SIZE, (12, 9, 3), marker_shape=(3, 3), jitter=0.15, renumber=True, rng=rng)
    ind_s = S.cylinder(3 * MM, 24 * MM, 64, 8)
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, 0.3e6, 0.45, 1100, 1 / 60, 0.05 * MM, 0.0)
    ind = G.build_indenter(ind_s.verts, ind_s.tris)
    pose = np.array([0.1, -0.2, 0.15, 9e-3, 7e-3, 4e-3 + 3 * MM - 0.2e-3])
    x32 = pd.rest
    y32 = _world32(ind, pose)
    r = 3 * 0.05 * MM
    ref = BP.candidates(x32.astype(np.float64), y32.astype(np.float64), pad, ind, r)
    w = S.Workload("bp", [pd], [S.Material()], [ind_s], 1, np.zeros((1, 1, 6), np.float32))
    b = tac.batch_from_workload(w)
    got, n = b.broadphase(0, torch.tensor(x32), torch.tensor(y32), r, capacity=1 << 18)
    assert n == len(ref) and len(ref) > 100
    assert np.array_equal(got.cpu().numpy().astype(np.int64), ref)
    b.close()


@pytest.fixture(scope="module")
def c1_gpu(tac, c1_oracle):
    w, pad, ind, poses, states, infos = c1_oracle
    b = tac.batch_from_workload(w)
    b.reset(torch.tensor(poses[0], dtype=torch.float32).reshape(1, 6))
    xs, mks, sts, its = [], [], [], []
    for f in range(1, len(poses)):
        b.set_indenter(torch.tensor(poses[f], dtype=torch.float32).reshape(1, 6))
        st, it = b.step()
        x, v = b.get_state()
        m = b.markers()
        torch.cuda.synchronize()
        xs.append(x.cpu().numpy().astype(np.float64))
        mks.append(m.cpu().numpy().astype(np.float64))
        sts.append(int(st.item()))
        its.append(int(it.item()))
    stats = b.stats().cpu().numpy()
    b.close()
    return xs, mks, sts, its, stats


def test_single_pad_frames_converge(c1_gpu):
    xs, mks, sts, its, stats = c1_gpu
    assert sts == [0] * len(sts), (sts, its)


def test_single_pad_positions_match_oracle(c1_gpu, c1_oracle):
    xs, mks, sts, its, stats = c1_gpu
    w, pad, ind, poses, states, infos = c1_oracle
    thickness = 4 * MM
    for f, x in enumerate(xs):
        err = np.abs(x - states[f + 1].x).max()
        assert err <= 1e-4 * thickness, (f, err)


def test_single_pad_markers_match_oracle(c1_gpu, c1_oracle):
    xs, mks, sts, its, stats = c1_gpu
    w, pad, ind, poses, states, infos = c1_oracle
    thickness = 4 * MM
    for f, m in enumerate(mks):
        ref = SV.markers(pad, states[f + 1].x)
        assert np.abs(m - ref).max() <= 1e-4 * thickness, f
    assert np.abs(mks[-1]).max() > 1e-6                     # the field is not trivially zero


def test_single_pad_no_interpenetration(c1_gpu, c1_oracle):
    xs, mks, sts, its, stats = c1_gpu
    w, pad, ind, poses, states, infos = c1_oracle
    ap = BP.all_pairs(pad, ind)
    for f in (0, 4, 9):
        d, _, _ = En.distances(ap, xs[f], G.indenter_world(ind.verts, poses[f + 1]), pad, ind)
        assert d.min() > 0


def test_no_contact_stays_at_rest(tac):
    w = S.config_single_pad(frames=2)
    poses = w.poses.copy()
    poses[:, 0, 5] += 5 * MM                          # indenter well above the gel
    b = tac.batch_from_workload(w)
    b.reset(torch.tensor(poses[0]))
    b.set_indenter(torch.tensor(poses[1]))
    st, it = b.step()
    x, v = b.get_state()
    assert int(st.item()) == 0 and int(it.item()) == 0
    assert np.array_equal(x.cpu().numpy(), w.pads[0].rest)
    assert np.abs(b.markers().cpu().numpy()).max() == 0.0
    b.close()


def test_ragged_batch_is_bitwise_equal_to_single_pads(tac):
    """Pads of different sizes in one batch give exactly the results of the
    same pads solved alone (each CTA's work depends only on its pad)."""
    w1 = S.config_single_pad(frames=2)
    small = S.hex_pad((12 * MM, 10 * MM, 4 * MM), (6, 5, 2), marker_shape=(5, 4))
    pose_s = w1.poses.copy()
    pose_s[:, 0, 3] = 6 * MM
    pose_s[:, 0, 4] = 5 * MM
    wb = S.Workload("ragged", [w1.pads[0], small, w1.pads[0]], [S.Material()] * 3, [w1.indenters[0]] * 3, 1,
                    np.concatenate([w1.poses, pose_s, w1.poses], axis=1))
    b = tac.batch_from_workload(wb)
    b.reset(torch.tensor(wb.poses[0]))
    for f in (1, 2):
        b.set_indenter(torch.tensor(wb.poses[f]))
        st, _ = b.step()
    mb = b.markers().cpu().numpy()
    assert st.cpu().numpy().tolist() == [0, 0, 0]
    b.close()
    singles = []
    for k in range(3):
        ws = S.Workload("one", [wb.pads[k]], [S.Material()], [wb.indenters[k]], 1, wb.poses[:, k:k + 1])
        bs = tac.batch_from_workload(ws)
        bs.reset(torch.tensor(ws.poses[0]))
        for f in (1, 2):
            bs.set_indenter(torch.tensor(ws.poses[f]))
            bs.step()
        singles.append(bs.markers().cpu().numpy())
        bs.close()
    assert np.array_equal(mb, np.concatenate(singles))


def test_pair_overflow_is_reported(tac):
    w = S.config_single_pad(frames=3)
    b = tac.batch_from_workload(w, pair_capacity=4)
    b.reset(torch.tensor(w.poses[0]))
    st = None
    for f in (1, 2, 3):
        b.set_indenter(torch.tensor(w.poses[f]))
        st, _ = b.step()
    assert int(st.item()) == 4
    b.close()
