"""The 512-thread block shape of the solve launch and its autotuner.

The 512-thread shape (one CTA of 16 warps per pad, one per SM) runs the same
method with each phase spread over twice the threads. It is compared with the
FP64 oracle on the single-pad press (10 frames) at the parity tolerance
(1e-4 of the gel thickness); a ragged batch in this shape must give, bit for
bit, what its pads give alone in it; and the autotuner must leave the state
as it found it and make the following frame exactly what an explicit
tac_set_block_shape of its choice makes.
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


def test_wide_shape_matches_oracle(tac):
    w, pad, ind = c1()
    poses = w.poses[:, 0].astype(np.float64)
    states, infos = SV.run(pad, ind, poses)
    b = tac.batch_from_workload(w)
    b.set_block_shape(512)
    b.reset(torch.tensor(poses[0], dtype=torch.float32).reshape(1, 6))
    worst_x = worst_m = 0.0
    for f in range(1, len(poses)):
        b.set_indenter(torch.tensor(poses[f], dtype=torch.float32).reshape(1, 6))
        st, it = b.step()
        assert int(st.item()) == 0, (f, int(it.item()))
        x, _ = b.get_state()
        mk = b.markers().cpu().numpy().astype(np.float64)
        worst_x = max(worst_x, np.abs(x.cpu().numpy().astype(np.float64) - states[f].x).max())
        worst_m = max(worst_m, np.abs(mk - SV.markers(pad, states[f].x)).max())
    b.close()
    print(f"512-thread shape: max |dx| {worst_x:.2e} m, markers {worst_m:.2e} m (tolerance {TOL:.1e} m)")
    assert worst_x <= TOL and worst_m <= TOL


def _ragged():
    w1 = S.config_single_pad(frames=2)
    small = S.hex_pad((12 * MM, 10 * MM, 4 * MM), (6, 5, 2), marker_shape=(5, 4))
    pose_s = w1.poses.copy()
    pose_s[:, 0, 3] = 6 * MM
    pose_s[:, 0, 4] = 5 * MM
    return S.Workload("ragged", [w1.pads[0], small, w1.pads[0]], [S.Material()] * 3, [w1.indenters[0]] * 3, 1,
                      np.concatenate([w1.poses, pose_s, w1.poses], axis=1))


def _run(tac, w, shape, frames=(1, 2)):
    b = tac.batch_from_workload(w)
    b.set_block_shape(shape)
    b.reset(torch.tensor(w.poses[0]))
    for f in frames:
        b.set_indenter(torch.tensor(w.poses[f]))
        st, _ = b.step()
    out = b.markers().cpu().numpy(), st.cpu().numpy()
    b.close()
    return out


def test_wide_shape_ragged_batch_is_bitwise_single_pads(tac):
    wb = _ragged()
    mb, st = _run(tac, wb, 512)
    assert st.tolist() == [0, 0, 0]
    singles = []
    for k in range(3):
        ws = S.Workload("one", [wb.pads[k]], [S.Material()], [wb.indenters[k]], 1, wb.poses[:, k:k + 1])
        singles.append(_run(tac, ws, 512)[0])
    assert np.array_equal(mb, np.concatenate(singles))


def test_autotuner_leaves_the_state_and_picks_a_shape(tac):
    wb = _ragged()
    b = tac.batch_from_workload(wb)
    b.reset(torch.tensor(wb.poses[0]))
    b.set_indenter(torch.tensor(wb.poses[1]))
    b.step()
    x0, v0 = b.get_state()
    x0, v0 = x0.clone(), v0.clone()
    shape, ms = b.autotune_block_shape(torch.tensor(wb.poses[2]), reps=2)
    assert shape in (256, 512) and all(m > 0 for m in ms)
    x1, v1 = b.get_state()
    assert torch.equal(x0, x1) and torch.equal(v0, v1)
    b.set_indenter(torch.tensor(wb.poses[2]))
    st, _ = b.step()
    tuned = b.markers().cpu().numpy()
    b.close()
    # the same two frames with the shape set by hand before the second one
    b = tac.batch_from_workload(wb)
    b.reset(torch.tensor(wb.poses[0]))
    b.set_indenter(torch.tensor(wb.poses[1]))
    b.step()
    b.set_block_shape(shape)
    b.set_indenter(torch.tensor(wb.poses[2]))
    b.step()
    explicit = b.markers().cpu().numpy()
    b.close()
    print(f"autotuner: {shape} threads (256: {ms[0]:.2f} ms, 512: {ms[1]:.2f} ms)")
    assert st.cpu().numpy().tolist() == [0, 0, 0]
    assert np.array_equal(tuned, explicit)
