"""Parity on the realistic recipe: a jittered, renumbered pad of the sensor's
18.6 x 14.3 x 4 mm gel (reduced to ~5k vertices so that the oracle re-solves
a frame in under a minute), sharp indenters (a box edge and a ridged
thread), friction 0.5 and a press-then-slide motion. The GPU runs the
sequence into the slide phase; the FP64 oracle then solves the last frame
from the GPU's own start state, and end positions and markers must agree
within 1e-4 of the gel thickness. The GPU's own end state is checked for
interpenetration: every candidate pair (r = 2 dhat; the pairs outside the
set are farther than r) has a positive distance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import broadphase as BP
from oracle import energy as En
from oracle import geometry as G
from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM, oracle_pad

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FRAMES, LAST = 30, 18      # the last frame compared lies in the slide phase
TOL_X = 1e-4 * 4 * MM


@pytest.fixture(scope="module")
def tac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac as T
    return T


@pytest.mark.parametrize("kind", ["box_edge", "thread"])
def test_realistic_frame_matches_oracle(tac, kind):
    w = S.config_realistic(seed=0, frames=FRAMES, n_verts_target=5000, indenter_kind=kind)
    b = tac.batch_from_workload(w)
    poses = torch.tensor(w.poses, dtype=torch.float32, device=b.device)
    b.reset(poses[0])
    for f in range(1, LAST):
        b.set_indenter(poses[f])
        st, _ = b.step()
        assert int(st.item()) == 0, (kind, f)
    x0, v0 = b.get_state()
    b.set_indenter(poses[LAST])
    st, it = b.step()
    assert int(st.item()) == 0
    x1, _ = b.get_state()
    mk = b.markers().cpu().numpy().astype(np.float64)
    b.close()
    pd, mat, ind_s = w.pads[0], w.materials[0], w.indenters[0]
    pad = oracle_pad(pd, mat)
    ind = G.build_indenter(ind_s.verts, ind_s.tris)
    state = SV.State(x=x0.cpu().numpy().astype(np.float64), v=v0.cpu().numpy().astype(np.float64),
                     pose=w.poses[LAST - 1, 0].astype(np.float64))
    new, info = SV.solve_frame(pad, ind, state, w.poses[LAST, 0].astype(np.float64), SV.Params(tol=1e-6))
    assert info.status == SV.CONVERGED
    x1 = x1.cpu().numpy().astype(np.float64)
    err = np.abs(x1 - new.x).max()
    merr = np.abs(mk - SV.markers(pad, new.x)).max()
    y = G.indenter_world(ind.verts, w.poses[LAST, 0].astype(np.float64))
    cand = BP.candidates(x1, y, pad, ind, 2 * pad.dhat)
    assert len(cand) > 0
    dmin = float(En.distances(cand, x1, y, pad, ind)[0].min())
    print(f"{kind}: {pd.n_verts} vertices, GPU {int(it.item())} / oracle {info.iters} iterations, "
          f"max |dx| {err:.2e} m, markers {merr:.2e} m (tolerance {TOL_X:.1e} m); GPU min gap {dmin:.2e} m")
    assert err <= TOL_X, (kind, err)
    assert merr <= TOL_X, (kind, merr)
    assert dmin > 0.0, (kind, dmin)
