"""Writes the calibration targets that the GPU calibration runs fit: the
marker fields of the calibration workload's first environments, solved by
the FP64 oracle at the environments' hidden materials.

The workload is the adjoint-calibration recipe (256 environments of a 5k
pad, a 16-frame press-and-slide, hidden per-env E ~ U[0.1, 0.5] MPa,
nu ~ U[0.40, 0.49], mu_f ~ U[0.3, 0.9]; seeded generator in
paper_2603_28475_b300/scenes.py). The barrier stiffness and the friction
mollifier width are those of the nominal material (E = 0.3 MPa), as in a
calibration, where every candidate shares them, so the fields are a
function of (E, nu, mu_f) alone.

  python tests/golden/make_calibration_targets.py [n_envs]

Only oracle/ and the scene generator are called. One process per
environment (spawned); about ten minutes of host time per environment.
"""
import multiprocessing
import os
import sys

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "calibration_targets.npz")
FRAMES = 16


def f32(v):
    return float(np.float32(v))


def run_env(e):
    from oracle import geometry as G
    from oracle import solver as SV
    from paper_2603_28475_b300 import scenes as S
    w, hidden = S.config_calibration(n_envs=256, frames=FRAMES, seed=0)
    pd, m, hm = w.pads[e], w.materials[e], hidden[e]
    # the nominal material's barrier stiffness and mollifier width, as the
    # library resolves them (float32 values of h^2 E l-bar and 1e-3 m/s h)
    nominal = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, f32(m.E), f32(m.nu), f32(m.rho), f32(m.h),
                          f32(m.dhat), f32(m.mu_f))
    kappa, eps_v = f32(nominal.kappa), f32(nominal.eps_v)
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, f32(hm.E), f32(hm.nu), f32(m.rho), f32(m.h),
                      f32(m.dhat), f32(hm.mu_f), kappa=kappa, eps_v=eps_v)
    ind = G.build_indenter(w.indenters[e].verts, w.indenters[e].tris)
    states, infos = SV.run(pad, ind, w.poses[:, e].astype(np.float64))
    status = [i.status for i in infos]
    markers = np.stack([SV.markers(pad, s.x) for s in states[1:]])
    return e, markers, status, (hm.E, hm.nu, hm.mu_f), kappa, eps_v, [i.iters for i in infos]


def main(n_envs):
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(min(n_envs, os.cpu_count() or 1)) as pool:
        res = sorted(pool.map(run_env, range(n_envs)))
    for e, _, st, _, _, _, its in res:
        print(f"env {e}: statuses {st}, iterations {its}")
        assert all(s == 0 for s in st), (e, st)
    np.savez(OUT, envs=np.array([r[0] for r in res]), markers=np.stack([r[1] for r in res]),
             hidden=np.array([r[3] for r in res]), kappa=np.array([r[4] for r in res]),
             eps_v=np.array([r[5] for r in res]), frames=FRAMES)
    print("wrote", OUT)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 4)
