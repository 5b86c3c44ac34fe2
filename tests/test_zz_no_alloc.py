"""The allocation-free candidate search (tac_broadphase_static) against the
batch entry point tac_broadphase.

The static variant exists for callers that cannot allocate device memory
(work captured into a CUDA graph, fixed-memory real-time loops, hosts that
give the library no allocator): its scratch is a fixed array inside the
library. Two calls in a row on different inputs must each give exactly the
candidate set the batch entry point gives (pair sets are compared bit-exact),
so no state leaks from one call into the next through the shared array.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as G
from paper_2603_28475_b300 import scenes as S

pytestmark = pytest.mark.gpu


def _inputs(seed):
    w = S.config_single_pad()
    pd = w.pads[0]
    ind = w.indenters[0]
    rng = np.random.default_rng(seed)
    pose = w.poses[0, 0].astype(np.float64).copy()
    pose[:3] = rng.uniform(-0.3, 0.3, 3)
    pose[3:5] += rng.uniform(-2e-3, 2e-3, 2)
    pose[5] -= rng.uniform(0.0, 0.3e-3)
    u = (rng.normal(size=pd.rest.shape) * 2e-5).astype(np.float32)
    u[pd.fixed] = 0
    x = (pd.rest + u).astype(np.float32)
    y = G.indenter_world(ind.verts, pose).astype(np.float32)
    st, se, sv = G.surface(pd.tets)
    ie = G.mesh_edges(ind.tris)
    return w, x, y, sv, st, se, ind.tris, ie


def test_static_broadphase_matches_batch_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac
    r = 0.4e-3
    for call, seed in enumerate((3, 4)):
        w, x, y, sv, st, se, it, ie = _inputs(seed)
        b = tac.batch_from_workload(w)
        ref, n_ref = b.broadphase(0, torch.tensor(x), torch.tensor(y), r, capacity=1 << 14)
        b.close()
        got, n = tac.broadphase_static(torch.tensor(x, device="cuda"), sv, st, se, torch.tensor(y, device="cuda"),
                                       it, ie, r, capacity=1 << 14)
        torch.cuda.synchronize()
        assert n_ref > 0, call
        assert n == n_ref, call
        assert torch.equal(got.cpu(), ref.cpu()), call


def test_static_broadphase_rejects_requests_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import tac
    w, x, y, sv, st, se, it, ie = _inputs(5)
    with pytest.raises(tac.TacError, match="fixed scratch"):
        tac.broadphase_static(torch.tensor(x, device="cuda"), sv, st, se, torch.tensor(y, device="cuda"), it, ie,
                              1e-4, capacity=1 << 17)
