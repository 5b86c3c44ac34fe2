"""The plain FP32 form (precision_mode 1) against the FP64 oracle.

The plain form is the same method with single-float displacements and the
pair distance, barrier, step bounds and every sum in float32: the form the
precision split is measured against. It is compared on the single-pad press
(10 frames) with the oracle solving each frame to the same tolerance. The
plain form cannot resolve the line search's energy test near the tolerance
(float32 sums of the element remainders are noise there), so many of its
pad-frames end on a failed line search or the iteration cap short of the
tolerance; its positions and markers still stay within 2.5e-4 of the gel
thickness of the oracle's. The chosen form meets 1e-4 on the same frames
(tests/test_gpu_parity.py). A batch that mixes the two forms pad by pad
gives, bit for bit, what single-form batches give.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM, c1

pytestmark = pytest.mark.gpu
TOL_FP32 = 2.5e-4 * 4 * MM


@pytest.fixture(scope="module")
def tac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac as T
    return T


def _run(tac, w, poses, precision, max_iter=2000):
    b = tac.batch_from_workload(w, precision=precision, max_iter=max_iter)
    b.reset(torch.tensor(poses[0], dtype=torch.float32).reshape(1, 6))
    out = []
    for f in range(1, len(poses)):
        b.set_indenter(torch.tensor(poses[f], dtype=torch.float32).reshape(1, 6))
        st, it = b.step()
        x, _ = b.get_state()
        out.append((int(st.item()), int(it.item()), x.cpu().numpy().astype(np.float64),
                    b.markers().cpu().numpy().astype(np.float64)))
    b.close()
    return out


def test_plain_fp32_form_against_oracle(tac):
    w, pad, ind = c1()
    poses = w.poses[:, 0].astype(np.float64)
    states, infos = SV.run(pad, ind, poses)
    assert all(i.status == SV.CONVERGED for i in infos)
    res = _run(tac, w, poses, precision=1)
    worst_x = worst_m = 0.0
    for f, (st, it, x, mk) in enumerate(res):
        assert st in (0, 1, 3), (f, st)            # converged, iteration cap or line search
        assert np.isfinite(x).all() and np.isfinite(mk).all()
        worst_x = max(worst_x, np.abs(x - states[f + 1].x).max())
        worst_m = max(worst_m, np.abs(mk - SV.markers(pad, states[f + 1].x)).max())
    n_conv = sum(r[0] == 0 for r in res)
    print(f"plain FP32: {n_conv}/{len(res)} frames converged; max |dx| {worst_x:.2e} m, markers {worst_m:.2e} m "
          f"(stated tolerance {TOL_FP32:.1e} m)")
    assert worst_x <= TOL_FP32 and worst_m <= TOL_FP32
    assert np.abs(res[-1][3]).max() > 1e-6


def test_mixed_precision_batch_is_bitwise_single_form(tac):
    w = S.config_single_pad()
    poses = w.poses[:4, 0].astype(np.float32)
    pad, mat, ind = w.pads[0], w.materials[0], w.indenters[0]
    params = [tac.make_params(mat, precision=p, max_iter=2000) for p in (0, 1)]
    b = tac.TacBatch([pad] * 2, params, [ind] * 2, pads_per_env=1)
    b.reset(torch.tensor(np.repeat(poses[:1], 2, 0)))
    for f in range(1, len(poses)):
        b.set_indenter(torch.tensor(np.repeat(poses[f:f + 1], 2, 0)))
        b.step()
    x_all, _ = b.get_state()
    x_all = x_all.cpu().numpy()
    b.close()
    nv = pad.rest.shape[0]
    for k in (0, 1):
        res = _run(tac, S.config_single_pad(frames=3), poses.astype(np.float64), precision=k)
        assert np.array_equal(x_all[k * nv:(k + 1) * nv], res[-1][2].astype(np.float32)), k
