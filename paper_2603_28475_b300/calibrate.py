"""Material calibration on top of the batched solve: the baseline calibration of
TacAlign (Sec. 4.2, Eq. loss_function and Eq. optimization_problem; Supp. C:
the parameters normalised to [0, 1], population 12).

* ``CMAES``: the (mu/mu_w, lambda) covariance matrix adaptation evolution
  strategy (Hansen and Ostermeier; the formulation and default strategy
  parameters of Hansen's published CMA-ES tutorial). It combines weighted
  recombination, cumulative step-size adaptation, and rank-one plus rank-mu
  covariance updates. It runs on the unit cube: a sample outside it is
  reflected back in, and the reflected point is the one evaluated and used in
  the updates.
* ``Calibration``: the marker-field misfit of Eq. loss_function for
  parameter vectors theta = [E, nu, rho, mu_f] over N indenter scenes and K
  frames. It evaluates a whole population in one batch of popsize x N pads,
  so one frame of a generation is one tac_step launch.
* ``calibrate_cmaes``: the gradient-free driver.
* ``calibrate_adjoint``: the gradient-based comparison. It runs Adam on the
  normalised (E, nu, mu_f), with gradients from the implicit adjoint of
  every frame (autograd.TacStepFn).

Readings: the parameter ranges are the paper's table, in SI units with
rho's range 1e-3..5e-3 read as g/mm^3 (1000..5000 kg/m^3). The barrier
stiffness and the friction mollifier width are held at one fixed value for
every candidate, so that the misfit is a function of theta alone. Without
that, kappa would follow E through its default rule.
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np
import torch

from . import tac as T

PARAMS = ("E", "nu", "rho", "mu_f")
RANGES = {"E": (1e4, 2e5), "nu": (0.4, 0.497), "rho": (1e3, 5e3), "mu_f": (0.25, 2.5)}


def to_theta(x, names=PARAMS, ranges=None):
    """Physical parameters from normalised coordinates x in [0, 1]^n
    (ranges: the search box, RANGES by default)."""
    r = RANGES if ranges is None else ranges
    x = np.asarray(x, dtype=np.float64)
    lo = np.array([r[n][0] for n in names])
    hi = np.array([r[n][1] for n in names])
    return lo + x * (hi - lo)


def to_unit(theta, names=PARAMS, ranges=None):
    r = RANGES if ranges is None else ranges
    lo = np.array([r[n][0] for n in names])
    hi = np.array([r[n][1] for n in names])
    return (np.asarray(theta, dtype=np.float64) - lo) / (hi - lo)


def reflect_unit(x):
    """Reflect coordinates into [0, 1] (period 2 in each coordinate)."""
    r = np.mod(x, 2.0)
    return np.where(r > 1.0, 2.0 - r, r)


class CMAES:
    """(mu/mu_w, lambda)-CMA-ES minimising over [0, 1]^n."""

    def __init__(self, x0, sigma0, popsize=12, seed=0):
        self.n = n = len(x0)
        self.lam = lam = int(popsize)
        self.mu = mu = lam // 2
        w = np.log(mu + 0.5) - np.log(np.arange(1, mu + 1))
        self.w = w / w.sum()
        self.mueff = 1.0 / np.sum(self.w ** 2)
        me = self.mueff
        self.cs = (me + 2.0) / (n + me + 5.0)
        self.ds = 1.0 + 2.0 * max(0.0, np.sqrt((me - 1.0) / (n + 1.0)) - 1.0) + self.cs
        self.cc = (4.0 + me / n) / (n + 4.0 + 2.0 * me / n)
        self.c1 = 2.0 / ((n + 1.3) ** 2 + me)
        self.cmu = min(1.0 - self.c1, 2.0 * (me - 2.0 + 1.0 / me) / ((n + 2.0) ** 2 + me))
        self.chi_n = np.sqrt(n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n * n))
        self.m = reflect_unit(np.asarray(x0, dtype=np.float64))
        self.sigma = float(sigma0)
        self.C = np.eye(n)
        self.B = np.eye(n)
        self.D = np.ones(n)
        self.ps = np.zeros(n)
        self.pc = np.zeros(n)
        self.gen = 0
        self.rng = np.random.default_rng(seed)
        self.best_x, self.best_f = self.m.copy(), np.inf

    def ask(self):
        """lambda candidates [lam, n] inside the unit cube."""
        z = self.rng.standard_normal((self.lam, self.n))
        y = (z * self.D) @ self.B.T
        self._x = reflect_unit(self.m + self.sigma * y)
        return self._x.copy()

    def tell(self, f):
        """Update from the objective values of the last ``ask``."""
        f = np.asarray(f, dtype=np.float64)
        f = np.where(np.isfinite(f), f, np.inf)
        order = np.argsort(f, kind="stable")
        if f[order[0]] < self.best_f:
            self.best_f, self.best_x = float(f[order[0]]), self._x[order[0]].copy()
        xs = self._x[order[:self.mu]]
        y = (xs - self.m) / self.sigma                       # steps of the selected (reflected) points
        yw = self.w @ y
        self.m = self.m + self.sigma * yw
        Cm12 = self.B @ np.diag(1.0 / self.D) @ self.B.T     # C^(-1/2)
        self.ps = (1.0 - self.cs) * self.ps + np.sqrt(self.cs * (2.0 - self.cs) * self.mueff) * (Cm12 @ yw)
        self.gen += 1
        hs = float(np.linalg.norm(self.ps) / np.sqrt(1.0 - (1.0 - self.cs) ** (2 * self.gen))
                   < (1.4 + 2.0 / (self.n + 1.0)) * self.chi_n)
        self.pc = (1.0 - self.cc) * self.pc + hs * np.sqrt(self.cc * (2.0 - self.cc) * self.mueff) * yw
        rank_mu = (y.T * self.w) @ y
        dh = (1.0 - hs) * self.cc * (2.0 - self.cc)
        self.C = ((1.0 - self.c1 - self.cmu) * self.C + self.c1 * (np.outer(self.pc, self.pc) + dh * self.C)
                  + self.cmu * rank_mu)
        self.sigma *= np.exp((self.cs / self.ds) * (np.linalg.norm(self.ps) / self.chi_n - 1.0))
        self.C = 0.5 * (self.C + self.C.T)
        ev, self.B = np.linalg.eigh(self.C)
        self.D = np.sqrt(np.maximum(ev, 1e-300))
        return order


@dataclasses.dataclass
class History:
    best_loss: list            # best loss seen after each generation (or iteration)
    mean_loss: list            # loss at the distribution mean (CMA-ES) / current point (adjoint)
    theta: list                # parameters at the mean / current point
    frames_solved: list        # cumulative pad-frames solved
    seconds: list              # cumulative wall time


class Calibration:
    """Eq. loss_function over the scenes of a workload (one pad per env,
    the scenes' poses [F + 1, N, 6]) for ``popsize`` parameter vectors at
    once. Pad c * N + i is scene i under candidate c. ``names`` selects the
    calibrated parameters; the others stay at ``base`` (a Material)."""

    def __init__(self, scenes, popsize, base, names=PARAMS, kappa=None, pair_capacity=8192):
        self.N, self.P, self.names = scenes.n_pads, int(popsize), tuple(names)
        self.F = scenes.poses.shape[0] - 1
        self.base = base
        pads = [scenes.pads[i] for _ in range(self.P) for i in range(self.N)]
        inds = [scenes.indenters[i] for _ in range(self.P) for i in range(self.N)]
        # one fixed barrier stiffness for every candidate (h^2 E_ref l-bar at E_ref = base.E)
        self.kappa = kappa
        prm = [T.make_params(base) for _ in pads]
        self.batch = T.TacBatch(pads, prm, inds, pads_per_env=1, pair_capacity=pair_capacity)
        resolved = self.batch.get_params()
        if self.kappa is None:
            self.kappa = [q.kappa for q in resolved]
        self.eps_v = [q.eps_v for q in resolved]
        dev = self.batch.device
        self.poses = torch.tensor(np.tile(scenes.poses, (1, self.P, 1)), dtype=torch.float32, device=dev)
        self.n_mk = self.batch.total_markers // (self.P * self.N)

    def _params(self, thetas):
        """thetas [P, n]: one vector per candidate for all scenes; or
        [P, N, n]: one per candidate and scene."""
        thetas = np.asarray(thetas, dtype=np.float64)
        prm = []
        for c in range(self.P):
            for i in range(self.N):
                th = dict(zip(self.names, thetas[c, i] if thetas.ndim == 3 else thetas[c]))
                k = c * self.N + i
                m = copy.copy(self.base)
                for nme in PARAMS:
                    if nme in th:
                        setattr(m, nme, float(th[nme]))
                prm.append(T.make_params(m, kappa=self.kappa[k], eps_v=self.eps_v[k]))
        return prm

    def markers(self, thetas):
        """Marker fields [F, P, N * M, 2] and pad status [F, P * N] for the
        parameter vectors thetas [P, len(names)]."""
        b = self.batch
        b.set_params(self._params(np.asarray(thetas, dtype=np.float64)))
        b.reset(self.poses[0])
        out, sts = [], []
        for f in range(1, self.F + 1):
            b.set_indenter(self.poses[f])
            st, _ = b.step()
            out.append(b.markers().clone())
            sts.append(st.clone())
        m = torch.stack(out).reshape(self.F, self.P, self.N * self.n_mk, 2)
        return m, torch.stack(sts)

    def loss(self, thetas, targets):
        """Eq. loss_function per candidate [P] against targets [F, N * M, 2]:
        the mean over frames and scenes of the squared L2 norm of the field
        difference; +inf for a candidate with an unconverged frame."""
        m, st = self.markers(thetas)
        d = (m - targets[:, None]).double().reshape(self.F, self.P, self.N, self.n_mk * 2)
        L = (d * d).sum(dim=3).mean(dim=(0, 2))
        ok = (st.reshape(self.F, self.P, self.N) == 0).all(dim=2).all(dim=0)
        L = torch.where(ok, L, torch.full_like(L, float("inf")))
        return L.cpu().numpy()

    def loss_per_scene(self, thetas, targets):
        """Eq. loss_function per candidate and scene [P, N] (thetas [P, N, n]
        or [P, n]) against targets [F, N * M, 2]: the mean over frames of the
        squared L2 norm of the scene's field difference; +inf where a frame
        of that scene did not converge."""
        m, st = self.markers(thetas)
        d = (m - targets[:, None]).double().reshape(self.F, self.P, self.N, self.n_mk * 2)
        L = (d * d).sum(dim=3).mean(dim=0)
        ok = (st.reshape(self.F, self.P, self.N) == 0).all(dim=0)
        L = torch.where(ok, L, torch.full_like(L, float("inf")))
        return L.cpu().numpy()

    def targets(self, theta_true):
        """Marker fields [F, N * M, 2] at one parameter vector (the synthetic
        recordings)."""
        m, st = self.markers(np.repeat(np.asarray(theta_true, dtype=np.float64)[None], self.P, 0))
        if not bool((st == 0).all()):
            raise RuntimeError("a target frame did not converge")
        return m[:, 0].clone()

    def close(self):
        self.batch.close()


def calibrate_cmaes(cal, targets, generations=80, sigma0=0.3, x0=None, seed=0, callback=None):
    """CMA-ES on the normalised parameters (Supp. C: population = cal.P).
    Returns (best theta, History)."""
    import time
    n = len(cal.names)
    es = CMAES(np.full(n, 0.5) if x0 is None else x0, sigma0, popsize=cal.P, seed=seed)
    h = History([], [], [], [], [])
    t0, frames = time.perf_counter(), 0
    for g in range(generations):
        X = es.ask()
        f = cal.loss(to_theta(X, cal.names), targets)
        es.tell(f)
        frames += cal.F * cal.P * cal.N
        h.best_loss.append(es.best_f)
        h.mean_loss.append(float("nan"))
        h.theta.append(to_theta(es.m, cal.names).tolist())
        h.frames_solved.append(frames)
        h.seconds.append(time.perf_counter() - t0)
        if callback:
            callback(g, es, f)
    return to_theta(es.best_x, cal.names), h


def calibrate_cmaes_per_scene(cal, targets, generations=40, sigma0=0.3, x0=None, seed=0, ranges=None):
    """One CMA-ES per scene (each scene its own material), all scenes'
    populations solved in the same batches: a generation is one batch of
    popsize x N pads. Returns (best theta per scene [N, n], History of the
    mean over scenes of the best losses)."""
    import time
    n = len(cal.names)
    es = [CMAES(np.full(n, 0.5) if x0 is None else x0[i], sigma0, popsize=cal.P, seed=seed + i)
          for i in range(cal.N)]
    h = History([], [], [], [], [])
    t0, frames = time.perf_counter(), 0
    for g in range(generations):
        X = np.stack([e.ask() for e in es], axis=1)                 # [P, N, n]
        L = cal.loss_per_scene(to_theta(X.reshape(-1, n), cal.names, ranges).reshape(X.shape), targets)
        for i, e in enumerate(es):
            e.tell(L[:, i])
        frames += cal.F * cal.P * cal.N
        h.best_loss.append(float(np.mean([e.best_f for e in es])))
        h.mean_loss.append(float("nan"))
        h.theta.append([to_theta(e.m, cal.names, ranges).tolist() for e in es])
        h.frames_solved.append(frames)
        h.seconds.append(time.perf_counter() - t0)
    return np.stack([to_theta(e.best_x, cal.names, ranges) for e in es]), h


def calibrate_adjoint(scenes, base, targets, iterations=40, lr=0.05, x0=None, kappa=None, pair_capacity=8192,
                      relag=True, per_scene=False, ranges=None):
    """Adam on the normalised (E, nu, mu_f) with gradients of Eq.
    loss_function from the frames' implicit adjoints (rho stays at
    ``base.rho``; the adjoint gives no density gradient), each frame's
    friction lag differentiated unless ``relag`` is False. One iteration is
    the forward sequence plus its reverse sweep on the N scenes. With
    ``per_scene`` each scene has its own (E, nu, mu_f) and the loss is the
    sum of the scenes' losses (Adam acts per coordinate, so the scenes are
    calibrated independently). Returns (theta [3] or [N, 3], History)."""
    import time
    from . import autograd as A
    names = ("E", "nu", "mu_f")
    N, F = scenes.n_pads, scenes.poses.shape[0] - 1
    b = T.TacBatch(scenes.pads, [T.make_params(base) for _ in scenes.pads], scenes.indenters, pads_per_env=1,
                   pair_capacity=pair_capacity)
    resolved = b.get_params()
    if kappa is not None:
        for q, k in zip(resolved, kappa):
            q.kappa = k
    b.set_params(resolved)
    base_params = b.get_params()
    dev = b.device
    poses = torch.tensor(scenes.poses.astype(np.float64), device=dev)
    b.reset(poses[0].float())
    x0s, v0s = b.get_state()
    r = RANGES if ranges is None else ranges
    lo = torch.tensor([r[n][0] for n in names], dtype=torch.float64)
    hi = torch.tensor([r[n][1] for n in names], dtype=torch.float64)
    shape = (N, 3) if per_scene else (3,)
    x = torch.tensor(np.full(shape, 0.5) if x0 is None else np.asarray(x0, np.float64).reshape(shape),
                     dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([x], lr=lr)
    h = History([], [], [], [], [])
    t0, frames, best = time.perf_counter(), 0, np.inf
    n_mk = b.total_markers // N
    for it in range(iterations):
        opt.zero_grad()
        th = lo + x * (hi - lo)
        E, nu, muf = th[..., 0], th[..., 1], th[..., 2]
        lam = E * nu / ((1 + nu) * (1 - 2 * nu))
        mu = E / (2 * (1 + nu))
        lame = torch.stack([lam, mu], dim=-1).reshape(-1, 2).expand(N, 2)
        mu_f = muf.reshape(-1).expand(N)
        m = A.sequence_markers(b, x0s, v0s, lame, mu_f, poses, base_params=base_params, relag=relag)
        d = (m.double() - targets.double().to(m.device)).reshape(F, N, n_mk * 2)
        loss = (d * d).sum(dim=2).mean()
        loss.backward()
        frames += F * N                                    # PNCG solves; the reverse sweep solves none
        lv = float(loss.item())
        best = min(best, lv)
        h.best_loss.append(best)
        h.mean_loss.append(lv)
        h.theta.append(th.detach().tolist())
        opt.step()
        with torch.no_grad():
            x.clamp_(0.0, 1.0)
        h.frames_solved.append(frames)
        h.seconds.append(time.perf_counter() - t0)
    b.close()
    return (lo + x.detach() * (hi - lo)).numpy(), h
