"""Writes central differences of the calibration misfit that the GPU's
sequence adjoint is checked against: for the first environment of the
calibration workload (5k pad, 16-frame press-and-slide, friction), the loss
L = sum over frames of |markers(theta) - targets|^2 at the nominal material
(E = 0.3 MPa, nu = 0.45, mu_f = 0.5; the nominal barrier stiffness and
mollifier width), against the oracle targets of calibration_targets.npz.
Each frame lags itself from its own start (the run the forward solve
makes), so the differences are the total derivative the relagged adjoint
computes. Steps of 1e-4 and 3e-5 of each parameter.

  python tests/golden/make_calibration_gradient.py

Only oracle/ and the scene generator are called; one spawned process per
loss evaluation (13 of them), about 25 minutes on 8 host cores.
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

OUT = os.path.join(HERE, "calibration_gradient.npz")
NAMES = ("E", "nu", "mu_f")
STEPS = (1e-4, 3e-5)


def f32(v):
    return float(np.float32(v))


def loss(task):
    name, rel = task
    from oracle import geometry as G
    from oracle import solver as SV
    from paper_2603_28475_b300 import scenes as S
    g = np.load(os.path.join(HERE, "calibration_targets.npz"))
    F = int(g["frames"])
    w, _ = S.config_calibration(n_envs=256, frames=F, seed=0)
    pd, m = w.pads[0], w.materials[0]
    th = {"E": f32(m.E), "nu": f32(m.nu), "mu_f": f32(m.mu_f)}
    if name is not None:
        th[name] = th[name] * (1.0 + rel)
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, th["E"], th["nu"], f32(m.rho), f32(m.h),
                      f32(m.dhat), th["mu_f"], kappa=float(g["kappa"][0]), eps_v=float(g["eps_v"][0]))
    ind = G.build_indenter(w.indenters[0].verts, w.indenters[0].tris)
    states, infos = SV.run(pad, ind, w.poses[:, 0].astype(np.float64))
    assert all(i.status == SV.CONVERGED for i in infos)
    mk = np.stack([SV.markers(pad, s.x) for s in states[1:]])
    return name, rel, float(np.sum((mk - g["markers"][0]) ** 2)), th


def main():
    tasks = [(None, 0.0)] + [(n, sg * h) for n in NAMES for h in STEPS for sg in (1.0, -1.0)]
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(min(len(tasks), os.cpu_count() or 1)) as pool:
        res = pool.map(loss, tasks)
    base = [r for r in res if r[0] is None][0]
    out = {"L0": base[2], "theta0": np.array([base[3][n] for n in NAMES]), "names": np.array(NAMES),
           "steps": np.array(STEPS)}
    fd = np.zeros((len(NAMES), len(STEPS)))
    for i, n in enumerate(NAMES):
        for j, h in enumerate(STEPS):
            lp = [r for r in res if r[0] == n and r[1] == h][0]
            lm = [r for r in res if r[0] == n and r[1] == -h][0]
            dp = lp[3][n] - lm[3][n]
            fd[i, j] = (lp[2] - lm[2]) / dp
            print(f"dL/d{n} at step {h:g}: {fd[i, j]:.6e}")
    out["fd"] = fd
    np.savez(OUT, **out)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
