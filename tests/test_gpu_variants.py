"""Parity of the paper-literal variants with the FP64 oracle (through the C ABI).

* step_mode 1 (Eq. step_size as printed: no CCD bound, no energy test)
  read out through marker_mode 1 (kNN inverse-distance markers, Sec. 3.2);
* precond_mode 1 (scalar Jacobi, Supp. A) with barycentric markers.

Each runs the single-pad press (10 frames) on the GPU and in the oracle
with the same variant; positions and markers must agree within 1e-4 of
the gel thickness in every frame. A batch that mixes the modes pad by pad
must give, bit for bit, what single-mode batches give.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geometry as G
from oracle import solver as SV
from paper_2603_28475_b300 import scenes as S

from _cases import MM, c1, f32

pytestmark = pytest.mark.gpu
TOL = 1e-4 * 4 * MM

VARIANTS = {
    "literal_step_knn_markers": (dict(step=1, marker=1), SV.Params(step="literal"), "knn"),
    "scalar_jacobi": (dict(precond=1), SV.Params(precond="scalar"), "bary"),
}


@pytest.fixture(scope="module")
def tac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_28475_b300 import build
    build.build()
    from paper_2603_28475_b300 import tac as T
    return T


def _run_gpu(tac, w, poses, **modes):
    b = tac.batch_from_workload(w, **modes)
    b.reset(torch.tensor(poses[0], dtype=torch.float32).reshape(1, 6))
    xs, mks, sts = [], [], []
    for f in range(1, len(poses)):
        b.set_indenter(torch.tensor(poses[f], dtype=torch.float32).reshape(1, 6))
        st, it = b.step()
        x, _ = b.get_state()
        xs.append(x.cpu().numpy().astype(np.float64))
        mks.append(b.markers().cpu().numpy().astype(np.float64))
        sts.append(int(st.item()))
    b.close()
    return xs, mks, sts


@pytest.mark.parametrize("name", list(VARIANTS))
def test_variant_matches_oracle(tac, name):
    modes, prm, mmode = VARIANTS[name]
    w, _, ind = c1()
    pd, mat = w.pads[0], w.materials[0]
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, f32(mat.E), f32(mat.nu), f32(mat.rho), f32(mat.h),
                      f32(mat.dhat), f32(mat.mu_f), marker_mode=mmode)
    poses = w.poses[:, 0].astype(np.float64)
    states, infos = SV.run(pad, ind, poses, prm)
    assert all(i.status == SV.CONVERGED for i in infos)
    xs, mks, sts = _run_gpu(tac, w, poses, **modes)
    assert sts == [0] * len(sts)
    for f in range(len(xs)):
        ex = np.abs(xs[f] - states[f + 1].x).max()
        em = np.abs(mks[f] - SV.markers(pad, states[f + 1].x)).max()
        assert ex <= TOL and em <= TOL, (f, ex, em)
    assert np.abs(mks[-1]).max() > 1e-6


def test_mixed_modes_in_one_batch_are_bitwise_single_mode(tac):
    w = S.config_single_pad()
    poses = w.poses[:4, 0].astype(np.float32)
    combos = [dict(), dict(step=1), dict(precond=1), dict(step=1, precond=1, marker=1)]
    pad, mat, ind = w.pads[0], w.materials[0], w.indenters[0]
    params = [tac.make_params(mat, **c) for c in combos]
    b = tac.TacBatch([pad] * 4, params, [ind] * 4, pads_per_env=1)
    b.reset(torch.tensor(np.repeat(poses[:1], 4, 0)))
    for f in range(1, len(poses)):
        b.set_indenter(torch.tensor(np.repeat(poses[f:f + 1], 4, 0)))
        st, _ = b.step()
    x_all, _ = b.get_state()
    m_all = b.markers()
    x_all, m_all = x_all.cpu().numpy(), m_all.cpu().numpy()
    b.close()
    nv, nm = pad.rest.shape[0], pad.markers.shape[0]
    for k, c in enumerate(combos):
        xs, mks, sts = _run_gpu(tac, S.config_single_pad(frames=3), poses.astype(np.float64), **c)
        assert np.array_equal(x_all[k * nv:(k + 1) * nv], xs[-1].astype(np.float32)), c
        assert np.array_equal(m_all[k * nm:(k + 1) * nm], mks[-1].astype(np.float32)), c


def test_marker_mode_is_fixed_at_creation(tac):
    w = S.config_single_pad(frames=2)
    b = tac.batch_from_workload(w)
    p = tac.make_params(w.materials[0], marker=1)
    with pytest.raises(tac.TacError):
        b.set_params([p])
    b.close()
