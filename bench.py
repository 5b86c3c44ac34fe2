"""Benchmark: converged tactile env-frames per second of the batched PNCG-IPC
frame solve, with the roofline of the solve kernel and the FP64 oracle timed
on the host cores beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--envs E] [--impl ours|reference]

Workload (the batched RL step): E environments x 2 gel pads, each env's pads
drawn from the 2k / 5k / 10k-vertex size classes, a cylinder peg per env
(r ~ U[2, 4] mm) pressed into each pad at 0.05 mm per frame from a dhat gap
with a random pose (+-15 deg, +-1 mm) up to a depth ~ U[0, 1.2] mm, friction
0.5. One step = one frame for every pad: set the target poses, solve
(tac_step), read the markers. W warm-up frames, then K timed frames; the
defaults (W = 5, K = 20) time frames 6..25, which take every pad through
its deepest press into the hold.
Under torchrun every rank solves its own E environments (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing
import os
import subprocess
import sys
import threading
import time

# the oracle leg runs on one host thread: pin BLAS pools before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged tactile frames/s (PNCG-IPC) at 4096 envs; % of HBM roofline"
UNIT = "env-frames/s"

# algorithmic bytes per unit of work of the solve kernel:
# a tet pass reads each tet's Dm^-1 (36 B), local connectivity (4 B) and
# corner slots (8 B) once, and per patch vertex the displacement (hi, lo) and
# the direction (36 B); a gradient pass also writes the gradient and the
# diagonal block (36 B per vertex), the p^T H p pass writes none; a vertex
# pass moves ~120 B per vertex; a pair evaluation ~64 B per candidate pair.
# A mesh with a Dm^-1 table (the structured case) reads no per-tet Dm^-1.
B_TET = 48.0
B_DM = 36.0
B_TET_VERT_PHP = 36.0
B_TET_VERT_GRAD = 72.0
B_VERT_PASS = 120.0
B_PAIR = 64.0
# the per-iteration byte model of the workload's planning (both tet passes at
# 56 B per tet, 150 B per vertex of vector traffic)
B_ITER_TET = 112.0
B_ITER_VERT = 150.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pair-capacity", type=int, default=16384)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--adjoint", action="store_true",
                    help="time the calibration workload's 16-frame forward and reverse sweep instead")
    ap.add_argument("--adjoint-envs", type=int, default=256)
    ap.add_argument("--adjoint-frames", type=int, default=16)
    ap.add_argument("--sweep", action="store_true",
                    help="throughput over env counts and pad sizes (the large-scale sweep) instead")
    ap.add_argument("--no-dm-table", action="store_true",
                    help="stream one Dm^-1 per tet even for structured meshes (the unstructured form)")
    ap.add_argument("--calibrate", action="store_true",
                    help="CMA-ES (population 12, 80 generations) and adjoint-gradient calibration instead")
    ap.add_argument("--fp32-steps", type=int, default=1,
                    help="frames of the plain FP32 form timed beside the chosen form (0: skip)")
    ap.add_argument("--fp32-max-iter", type=int, default=500,
                    help="iteration cap of the plain FP32 form (it stalls short of the tolerance)")
    ap.add_argument("--per-frame", action="store_true",
                    help="add each timed frame's convergence record (statuses, iterations, substeps, queue use) "
                         "to the JSON line")
    ap.add_argument("--trajectory", action="store_true",
                    help="60-frame trajectories of fine pads under 10k-triangle indenters (the large-scale "
                         "configuration) instead")
    ap.add_argument("--trajectory-envs", type=int, default=64)
    ap.add_argument("--calibrate-oracle", action="store_true",
                    help="per-environment CMA-ES and adjoint calibration against the FP64 oracle's targets "
                         "(tests/golden/calibration_targets.npz) instead")
    ap.add_argument("--variants", action="store_true",
                    help="iterations and throughput of the paper-literal variants on the batched workload instead")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: the --envs environments partitioned over the ranks (balanced by tets) "
                         "with a per-frame all-gather of the marker fields, instead of one workload per rank")
    ap.add_argument("--sweep-points", default="",
                    help="with --sweep: the points to run, as envs x pad vertices, e.g. 64x50000,1024x2000 "
                         "(default: all of SWEEP_POINTS)")
    ap.add_argument("--block-shape", default="auto", choices=["auto", "256", "512"],
                    help="threads per pad's CTA in the solve launch: the library's autotuner on the first timed "
                         "frame (auto, before the timed region) or a fixed shape")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers


def choose_block_shape(b, poses_next, mode):
    """Block shape of the batch's solve launch: 'auto' runs the library's
    autotuner (tac_autotune_block_shape: the next frame solved in each shape
    from the same state, the state put back) on poses_next; otherwise the
    given thread count. Returns the bench line's record of the choice."""
    if mode == "auto":
        th, ms = b.autotune_block_shape(poses_next, reps=1)
        return {"threads": th, "chosen_by": "tac_autotune_block_shape on the first timed frame",
                "tuning_ms": {"256": ms[0], "512": ms[1]}}
    b.set_block_shape(int(mode))
    return {"threads": int(mode), "chosen_by": "--block-shape"}

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def rank_seed(seed, rank):
    """Workload seed of a rank: each rank solves its own envs (weak scaling,
    no data-path exchange)."""
    return seed + 1000 * rank


def job_totals(ms, conv, world, device=None):
    """Whole-job (time, converged count) of one timed region: the slowest
    rank's time and the sum of the ranks' converged envs (an all-reduce over
    the default process group when world > 1)."""
    if world <= 1:
        return float(ms), float(conv)
    import torch
    t = torch.tensor([float(ms), float(conv)], dtype=torch.float64, device=device)
    mx = t.clone()
    torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
    sm = t.clone()
    torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def workload(envs, frames, seed):
    from paper_2603_28475_b300 import scenes as S
    return S.config_batched(n_envs=envs, frames=frames, seed=seed)


_TABLED = {}


def tabled(pad, dm_table=True):
    """Whether the library reads this pad's rest shapes from a Dm^-1 table."""
    if not dm_table:
        return False
    key = id(pad.tets)
    if key not in _TABLED:
        from paper_2603_28475_b300 import tac
        _TABLED[key] = tac.mesh_info(pad)["dm_types"] > 0
    return _TABLED[key]


def phase_bytes(stats, w, dm_table=True):
    """Counted bytes of one solve launch from the per-pad counters, by phase:
    (p^T H p tet passes, gradient tet passes, vertex passes, pair passes).
    A pad runs one p^T H p tet pass per PNCG iteration; its other tet passes
    are gradient passes."""
    out = np.zeros(4)
    for k, pad in enumerate(w.pads):
        it, sub, reb, hal, tp, vp, pe, peak = [float(v) for v in stats[k][:8]]
        bt = B_TET - (B_DM if tabled(pad, dm_table) else 0.0)
        n_php = min(it, tp)
        out[0] += n_php * (bt * pad.n_tets + B_TET_VERT_PHP * pad.n_verts)
        out[1] += (tp - n_php) * (bt * pad.n_tets + B_TET_VERT_GRAD * pad.n_verts)
        out[2] += vp * B_VERT_PASS * pad.n_verts
        out[3] += pe * B_PAIR
    return out


def algorithmic_bytes(stats, w, dm_table=True):
    """Counted bytes of one solve launch from the per-pad counters."""
    return float(phase_bytes(stats, w, dm_table).sum())


def iteration_model_bytes(stats, w):
    """Bytes of one launch under the per-iteration model 112 T + 150 V (two
    tet passes of 56 B per tet and the vector traffic per PNCG iteration)."""
    return float(sum(float(stats[k][0]) * (B_ITER_TET * p.n_tets + B_ITER_VERT * p.n_verts)
                     for k, p in enumerate(w.pads)))


def kernel_hash():
    import hashlib
    h = hashlib.sha256()
    # the kernels and the mesh layout they stream (patches, colours, tables)
    for f in ("kernels.cu", "device_math.cuh", "solve.cuh", "layout.h", "mesh.cpp"):
        with open(os.path.join(ROOT, "paper_2603_28475_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(bytes_alg_per_launch):
    """DRAM bytes per launch from the committed ncu summary, scaled from the
    captured case by the counted bytes, or None when the kernel changed."""
    path = os.path.join(ROOT, "profiles", "solve_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("kernel_hash") != kernel_hash():
        return None
    ratio = float(rec["dram_bytes"]) / float(rec["algorithmic_bytes"])
    return ratio * bytes_alg_per_launch


# --------------------------------------------------------------------------- oracle sample

def sample_envs(w, n):
    """The oracle's sample of a workload: the first n environments whose pads
    are all of the smallest size class (so that a frame of the sample takes
    seconds on one core per pad), and the factor from one such env-frame to
    an average env-frame of the workload (the ratio of tet counts)."""
    small = min(p.n_verts for p in w.pads)
    envs = [e for e in range(w.n_envs)
            if all(w.pads[w.pads_per_env * e + q].n_verts == small for q in range(w.pads_per_env))][:n]
    mean_env = np.mean([sum(w.pads[w.pads_per_env * e + q].n_tets for q in range(w.pads_per_env))
                        for e in range(w.n_envs)])
    sample_env = sum(w.pads[w.pads_per_env * envs[0] + q].n_tets for q in range(w.pads_per_env))
    return envs, mean_env / sample_env


_ORACLE_MODELS = {}


def oracle_pad_frame(task):
    """One pad-frame of the FP64 oracle as it stands (runs in a spawned
    worker; the pad model is built once per worker and not timed). Returns
    (key, x, v, solve seconds, iterations, status)."""
    key, pad_arrays, material, ind_arrays, x, v, pose_t, pose_n = task
    from oracle import geometry as G
    from oracle import solver as SV
    if key not in _ORACLE_MODELS:
        rest, tets, fixed, markers = pad_arrays
        f32 = lambda a: float(np.float32(a))
        E, nu, rho, h, dhat, mu_f = material
        pad = G.build_pad(rest, tets, fixed, markers, f32(E), f32(nu), f32(rho), f32(h), f32(dhat), f32(mu_f))
        _ORACLE_MODELS[key] = (pad, G.build_indenter(*ind_arrays))
    pad, ind = _ORACLE_MODELS[key]
    st = SV.State(x=np.asarray(x, np.float64), v=np.asarray(v, np.float64), pose=np.asarray(pose_t, np.float64))
    t = time.perf_counter()
    new, info = SV.solve_frame(pad, ind, st, np.asarray(pose_n, np.float64))
    return key, new.x, new.v, time.perf_counter() - t, info.iters, info.status


def _oracle_task(w, k, x, v, f):
    pd, m = w.pads[k], w.materials[k]
    ind = w.indenters[k // w.pads_per_env]
    return (k, (pd.rest, pd.tets, pd.fixed, pd.markers), (m.E, m.nu, m.rho, m.h, m.dhat, m.mu_f),
            (ind.verts, ind.tris), x, v, w.poses[f - 1, k], w.poses[f, k])


def oracle_pool(n):
    """A pool of n spawned workers with single-threaded BLAS (spawn: a pool
    forked from a process that holds a CUDA context hangs)."""
    return multiprocessing.get_context("spawn").Pool(n)


def oracle_frame_step(pool, w, envs, states, f):
    """Frame f for every pad of the sample envs, the pads in parallel on the
    pool's cores. states: {pad: (x, v)} updated in place. Returns the
    step's time (its slowest pad: the pads run concurrently) and the pads'
    iterations."""
    pads = [w.pads_per_env * e + q for e in envs for q in range(w.pads_per_env)]
    res = pool.map(oracle_pad_frame, [_oracle_task(w, k, states[k][0], states[k][1], f) for k in pads])
    for k, x, v, dt, it, stt in res:
        states[k] = (x, v)
    return max(r[3] for r in res), [r[4] for r in res]


# --------------------------------------------------------------------------- arms

def oracle_cores():
    """Host cores the oracle sample uses: one per pad of the sample, at most
    8 pads (4 environments)."""
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return max(1, min(8, n))


def run_reference(args, rank, world):
    """The FP64 oracle as it stands on the host cores, on a sample of the
    same workload: the first environments whose pads are both of the 2k
    class (one pad per core), run from rest through the same frames as the
    GPU arm (W warm-up frames, then K timed frames), each frame's pads in
    parallel. A step's time is its slowest pad; the value is the sample's
    env-frames per second scaled by tet count to an average env-frame."""
    if rank != 0:
        return
    cores = oracle_cores()
    w = workload(args.envs, args.warmup + args.steps + 1, args.seed)
    envs, scale = sample_envs(w, max(1, cores // w.pads_per_env))
    states = {}
    for e in envs:
        for q in range(w.pads_per_env):
            k = w.pads_per_env * e + q
            states[k] = (w.pads[k].rest.astype(np.float64), np.zeros((w.pads[k].n_verts, 3)))
    n_pads = len(states)
    times, iters = [], []
    with oracle_pool(n_pads) as pool:
        for f in range(1, args.warmup + args.steps + 1):
            dt, its = oracle_frame_step(pool, w, envs, states, f)
            if f > args.warmup:
                times.append(dt)
                iters += its
    t_env = float(np.mean(times)) * scale / len(envs)
    value = 1.0 / t_env
    sample = (f"oracle (numpy FP64) on {len(envs)} env(s) x {w.pads_per_env} pads of the "
              f"{w.pads[2 * envs[0]].n_verts}-vertex class, one pad per core, from rest through frames "
              f"1..{args.warmup + args.steps} (frames {args.warmup + 1}..{args.warmup + args.steps} timed, "
              f"{np.mean(iters):.0f} iterations per pad-frame); a step is its slowest pad; scaled by {scale:.2f} "
              "(tet count) to an average env-frame of the workload (extrapolated)")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_env * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"batched_{args.envs}env_x2pads", "envs": args.envs,
                      "frames": f"{args.warmup + 1}..{args.warmup + args.steps} of a 0.05 mm/frame press"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_pads, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world):
    import torch
    from paper_2603_28475_b300 import tac
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    frames = args.warmup + args.steps
    w = workload(args.envs, 2 * frames + 1, rank_seed(args.seed, rank))
    n_pads = w.n_pads
    t0 = time.time()
    b = tac.batch_from_workload(w, pair_capacity=args.pair_capacity, dm_table=not args.no_dm_table)
    t_create = time.time() - t0
    stream = torch.cuda.current_stream()
    poses = torch.tensor(w.poses, dtype=torch.float32, device=dev)      # [F+1, n_pads, 6]
    b.reset(poses[0])
    status = torch.empty(n_pads, dtype=torch.int32, device=dev)
    iters = torch.empty(n_pads, dtype=torch.int32, device=dev)
    mk = torch.empty(b.total_markers, 2, dtype=torch.float32, device=dev)
    for f in range(1, args.warmup + 1):
        b.set_indenter(poses[f])
        b.step(status, iters)
        b.markers(mk)
    torch.cuda.synchronize()
    shape = choose_block_shape(b, poses[args.warmup + 1], args.block_shape)
    # the state after the warm-up: the end-to-end leg re-runs the same frames from it
    ck_x, ck_v = b.get_state()
    ck_x, ck_v = ck_x.clone(), ck_v.clone()
    # timed frames: inputs resident in HBM
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    conv, iter_hist, stats_all = 0, [], []
    bytes_alg = 0.0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for s in range(args.steps):
            f = args.warmup + 1 + s
            b.set_indenter(poses[f])
            ev[s][0].record(stream)
            b.step(status, iters)
            ev[s][1].record(stream)
            b.markers(mk)
            st = b.stats()
            stats_all.append((status.clone(), iters.clone(), st, b.norms()))
        stop.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = start.elapsed_time(stop)
    solve_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    phase = np.zeros(8)
    pbytes = np.zeros(4)
    bytes_iter_model = 0.0
    pad_ms = []
    floor_stops, pad_frames = 0, 0
    for stt, it, st, nr in stats_all:
        s_np = stt.cpu().numpy().reshape(-1, w.pads_per_env)
        conv += int(np.all(s_np == 0, axis=1).sum())
        iter_hist.append(it.cpu().numpy())
        st_np = st.cpu().numpy()
        pbytes += phase_bytes(st_np, w, not args.no_dm_table)
        bytes_iter_model += iteration_model_bytes(st_np, w)
        phase += st_np[:, 8:16].sum(axis=0)
        pad_ms.append(st_np[:, 15] / 1e6)
        # pads whose stopping target was the float32 resolution floor rather
        # than tol * g_ref (norms: final |g|, target, g_ref, force scale)
        nr_np = nr.cpu().numpy()
        floor_stops += int((nr_np[:, 1] > 1e-6 * nr_np[:, 2] * (1.0 + 1e-6)).sum())
        pad_frames += nr_np.shape[0]
    bytes_alg = float(pbytes.sum())
    per_frame = []
    if args.per_frame:
        for q, (stt, it, st, nr) in enumerate(stats_all):
            sn, st_np, nr_np = stt.cpu().numpy(), st.cpu().numpy(), nr.cpu().numpy()
            per_frame.append({
                "frame": args.warmup + 1 + q, "ms": solve_ms[q],
                "status": {str(int(a)): int(c) for a, c in zip(*np.unique(sn, return_counts=True))},
                "iters": [float(np.percentile(st_np[:, 0], 50)), float(np.percentile(st_np[:, 0], 99)),
                          int(st_np[:, 0].max())],
                "substeps": [float(np.percentile(st_np[:, 1], 99)), int(st_np[:, 1].max())],
                "halvings_per_pad": float(st_np[:, 3].mean()),
                "busy": float(st_np[:, 15].sum() / 1e6 / (b.grid_ctas * solve_ms[q])),
                "longest_pad_ms": float(st_np[:, 15].max() / 1e6),
                "float32_floor_stops": float((nr_np[:, 1] > 1e-6 * nr_np[:, 2] * (1.0 + 1e-6)).mean())})
    pad_ms = np.concatenate(pad_ms)
    names = ["tet_pHp", "tet_grad", "pair_pHp", "pair_grad", "vertex", "advance_rebuild", "setup"]
    phase_share = {n: float(phase[i] / phase[7]) for i, n in enumerate(names)} if phase[7] > 0 else None
    # CTA-time spent inside pads over the launch's CTA-time: below 1 the grid idles
    # behind the queue's last pads
    queue = {"ctas": b.grid_ctas, "busy": float(phase[7] / 1e6 / (b.grid_ctas * sum(solve_ms))),
             "longest_pad_ms": float(pad_ms.max())}
    total_ms_job, conv_job = job_totals(total_ms, conv, world, dev)
    value = conv_job / (total_ms_job / 1e3)
    its = np.concatenate(iter_hist)
    bytes_per_launch = bytes_alg / args.steps
    launch_ms = float(np.mean(solve_ms))
    peak, peak_kind = load_peaks()
    achieved = bytes_per_launch / (launch_ms / 1e3) / 1e9
    achieved_iter_model = bytes_iter_model / args.steps / (launch_ms / 1e3) / 1e9
    traffic = committed_traffic(bytes_per_launch)
    # per phase: its counted bytes over the CTA-seconds it took, spread over
    # the grid's resident CTAs (the bandwidth the phase draws while it runs)
    phase_gbs = {}
    for nm, by, cols in (("elastic_tet_passes", pbytes[0] + pbytes[1], (0, 1)), ("tet_pHp", pbytes[0], (0,)),
                         ("tet_grad", pbytes[1], (1,)), ("barrier_pair_passes", pbytes[3], (2, 3)),
                         ("vertex", pbytes[2], (4,))):
        ns = sum(phase[c] for c in cols)
        if ns > 0:
            gbs = by / (ns / 1e9 / b.grid_ctas) / 1e9
            phase_gbs[nm] = {"achieved_gbs": gbs, "frac": gbs / peak}
    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        host_poses = poses.cpu().pin_memory()
        host_mk = torch.empty(b.total_markers, 2, dtype=torch.float32).pin_memory()
        host_st = torch.empty(n_pads, dtype=torch.int32).pin_memory()
        dev_pose = torch.empty(n_pads, 6, dtype=torch.float32, device=dev)
        n_e2e = args.steps
        conv_e = 0
        b.reset(poses[args.warmup])
        b.set_state(ck_x, ck_v)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t1 = time.perf_counter()
        for s in range(n_e2e):
            f = args.warmup + 1 + s
            dev_pose.copy_(host_poses[f], non_blocking=True)
            b.set_indenter(dev_pose)
            b.step(status, iters)
            b.markers(mk)
            host_mk.copy_(mk, non_blocking=True)
            host_st.copy_(status, non_blocking=True)
            torch.cuda.synchronize()
            conv_e += int(np.all(host_st.numpy().reshape(-1, w.pads_per_env) == 0, axis=1).sum())
        dt_e = time.perf_counter() - t1
        ms_e, conv_e = job_totals(1e3 * dt_e, conv_e, world, dev)
        e2e = {"value": conv_e / (ms_e / 1e3), "unit": UNIT,
               "frames": "the device-timed frames again, from the state after the warm-up",
               "h2d_bytes_per_step": n_pads * 6 * 4,
               "d2h_bytes_per_step": b.total_markers * 2 * 4 + n_pads * 4}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            # the first timed frame of the same workload from the GPU's own
            # start state, for a sample of 2k-class environments, one pad per
            # host core
            cores = oracle_cores()
            envs, scale = sample_envs(w, max(1, cores // w.pads_per_env))
            xs, vs = ck_x.cpu().numpy(), ck_v.cpu().numpy()
            vo = b.vert_offsets
            states = {}
            for e in envs:
                for q in range(w.pads_per_env):
                    k = w.pads_per_env * e + q
                    states[k] = (xs[vo[k]:vo[k + 1]], vs[vo[k]:vo[k + 1]])
            f = args.warmup + 1
            with oracle_pool(len(states)) as pool:
                dt, o_its = oracle_frame_step(pool, w, envs, states, f)
            cpu = {"value": len(envs) / (dt * scale), "unit": UNIT, "cores": len(states), "kind": "oracle",
                   "sample": f"oracle (numpy FP64) on {len(envs)} env(s) x {w.pads_per_env} pads of the "
                             f"{w.pads[w.pads_per_env * envs[0]].n_verts}-vertex class, frame {f} from the GPU's "
                             f"start state, one pad per core ({np.mean(o_its):.0f} iterations per pad, slowest pad "
                             f"{dt:.1f} s), scaled by {scale:.2f} (tet count) to an average env-frame (extrapolated)"}
        except Exception as exc:             # the GPU line is still reported
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc!r}"}
    # the plain FP32 form on the same frames from the same start state (the
    # state after the warm-up): same tolerance, iteration cap bounded
    fp32 = None
    if args.fp32_steps > 0:
        k32 = min(args.steps, args.fp32_steps)
        b32 = tac.batch_from_workload(w, pair_capacity=args.pair_capacity, dm_table=not args.no_dm_table,
                                      precision=1, max_iter=args.fp32_max_iter)
        b32.set_block_shape(shape["threads"])
        b32.reset(poses[args.warmup])
        b32.set_state(ck_x, ck_v)
        ms32, conv32, st32, it32 = [], 0, [], []
        for q in range(k32):
            f = args.warmup + 1 + q
            b32.set_indenter(poses[f])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b32.step(status, iters)
            e1.record(stream)
            torch.cuda.synchronize()
            ms32.append(e0.elapsed_time(e1))
            sn = status.cpu().numpy()
            conv32 += int(np.all(sn.reshape(-1, w.pads_per_env) == 0, axis=1).sum())
            st32.append(sn)
            it32.append(iters.cpu().numpy())
        b32.close()
        del b32
        torch.cuda.empty_cache()
        st32, it32 = np.concatenate(st32), np.concatenate(it32)
        # the chosen form over the same frames
        ms_c = solve_ms[:k32]
        conv_c = sum(int(np.all(stt.cpu().numpy().reshape(-1, w.pads_per_env) == 0, axis=1).sum())
                     for stt, _, _, _ in stats_all[:k32])
        fp32 = {"form": "plain FP32 (precision_mode 1): single-float displacements; float32 pair distance, "
                        "barrier, step bounds and sums",
                "frames": f"{args.warmup + 1}..{args.warmup + k32}, from the chosen form's state after the warm-up",
                "tol_rel_grad": 1e-6, "max_iter": args.fp32_max_iter,
                "value": conv32 / (sum(ms32) / 1e3), "unit": UNIT, "ms_per_frame": float(np.mean(ms32)),
                "converged_fraction": conv32 / (k32 * args.envs),
                "status_counts": {str(int(a)): int(c) for a, c in zip(*np.unique(st32, return_counts=True))},
                "iters_per_pad_frame": {"p50": float(np.percentile(it32, 50)), "p99": float(np.percentile(it32, 99))},
                "chosen_form_same_frames": {"value": conv_c / (sum(ms_c) / 1e3), "ms_per_frame": float(np.mean(ms_c)),
                                            "converged_fraction": conv_c / (k32 * args.envs)}}
    if rank == 0:
        v_state = b.total_verts * 168 / 1e9
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": total_ms_job / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f32 (double-float displacements; f64 pair distance, barrier, CCD and reductions)",
               "data": "synthetic",
               "config": {"workload": f"batched_{args.envs}env_x2pads", "envs": args.envs, "pads": n_pads,
                          "pads_per_env": 2, "size_classes_verts": [2070, 4830, 9918],
                          "total_verts": b.total_verts, "total_tets": int(sum(p.n_tets for p in w.pads)),
                          "frames": f"{args.warmup + 1}..{args.warmup + args.steps} of a 0.05 mm/frame press",
                          "tol_rel_grad": 1e-6, "friction": 0.5, "pair_capacity": args.pair_capacity,
                          "rest_shapes": "per-tet Dm^-1" if args.no_dm_table else "Dm^-1 table (structured meshes)",
                          "l2": f"inputs larger than L2 (solver state {v_state:.1f} GB)",
                          "parallelism": f"{world} rank(s), env-sharded"},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                            "kernel": "tac::solve_kernel", "bytes_per_launch": bytes_per_launch,
                            "launch_ms": launch_ms,
                            "iteration_model": {"bytes_per_launch": bytes_iter_model / args.steps,
                                                "achieved": achieved_iter_model,
                                                "frac": achieved_iter_model / peak,
                                                "model": "112 B/tet + 150 B/vertex per PNCG iteration"},
                            "phases": phase_gbs},
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 3 * args.steps,
               "clocks": clk.summary(),
               "converged_fraction": conv_job / (args.steps * args.envs * world),
               "float32_floor_stops": floor_stops / max(1, pad_frames),
               "pad_frame_ms": {"p50": float(np.percentile(pad_ms, 50)), "p99": float(np.percentile(pad_ms, 99)),
                                "max": float(pad_ms.max())},
               "iters_per_pad_frame": {"p50": float(np.percentile(its, 50)), "p99": float(np.percentile(its, 99)),
                                       "max": int(its.max())},
               "frame_ms": {"p50": float(np.percentile(solve_ms, 50)), "p99": float(np.percentile(solve_ms, 99))},
               "setup_s": t_create, "phase_share": phase_share, "queue": queue, "block_shape": shape}
        if fp32 is not None:
            out["plain_fp32"] = fp32
        if per_frame:
            out["per_frame"] = per_frame
        print(json.dumps(out), flush=True)
    b.close()


def shard_workload(w, env_ids):
    """The environments env_ids (ascending) of workload w as a workload of
    their own: their pads, materials, indenters and poses."""
    from paper_2603_28475_b300 import scenes as S
    ppe = w.pads_per_env
    pads = [ppe * int(e) + q for e in env_ids for q in range(ppe)]
    return S.Workload(f"{w.name}_shard", [w.pads[k] for k in pads], [w.materials[k] for k in pads],
                      [w.indenters[int(e)] for e in env_ids], ppe, w.poses[:, pads])


def run_sharded(args, rank, world, make_batch=None, device=None):
    """The job's environments partitioned across the ranks (strong
    scaling). Every rank builds the same workload, takes its share of
    partition.balanced_partition (cost: the tets of each env's pads),
    solves that share with a batch of its own, and every frame all-gathers
    the marker fields of all environments (partition.gather_markers): the
    per-frame exchange of the paper's per-GPU simulation actors. W warm-up
    frames, then K timed frames between barriers; the time is the slowest
    rank's (CUDA events on the rank's stream, or the host clock for a batch
    on the host). Rank 0 prints one JSON line; every rank returns the
    gathered field of the last frame [envs, markers per env, 2]."""
    import torch
    import torch.distributed as dist
    from paper_2603_28475_b300 import partition as PT
    if device is None:
        device = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
        torch.cuda.set_device(device)
    if make_batch is None:
        from paper_2603_28475_b300 import tac

        def make_batch(ws):
            return tac.batch_from_workload(ws, pair_capacity=args.pair_capacity, dm_table=not args.no_dm_table)
    frames = args.warmup + args.steps
    w = workload(args.envs, frames + 1, args.seed)          # the job's workload, the same on every rank
    costs = PT.env_costs([p.n_tets for p in w.pads], w.pads_per_env)
    parts = PT.balanced_partition(costs, world)
    mine = parts[rank]
    n_mk = {int(np.asarray(p.markers).shape[0]) for p in w.pads}
    if len(n_mk) != 1:
        raise ValueError("the marker gather needs one marker count per pad")
    per_env = w.pads_per_env * n_mk.pop()
    ws = shard_workload(w, mine)
    b = make_batch(ws)
    poses = torch.tensor(ws.poses, dtype=torch.float32, device=device)
    st = torch.empty(ws.n_pads, dtype=torch.int32, device=device)
    it = torch.empty(ws.n_pads, dtype=torch.int32, device=device)
    on_gpu = device.type == "cuda"

    def frame(f):
        b.set_indenter(poses[f])
        b.step(st, it)
        mk = b.markers().reshape(len(mine), per_env, 2)
        full = PT.gather_markers(mk, mine, w.n_envs)
        conv = int((st.reshape(-1, w.pads_per_env) == 0).all(dim=1).sum().item())
        return full, conv

    b.reset(poses[0])
    for f in range(1, args.warmup + 1):
        frame(f)
    dist.barrier()
    if on_gpu:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
    t0 = time.perf_counter()
    conv = 0
    full = None
    for f in range(args.warmup + 1, frames + 1):
        full, c = frame(f)
        conv += c
    if on_gpu:
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    else:
        ms = (time.perf_counter() - t0) * 1e3
    dist.barrier()
    t = torch.tensor([ms, float(conv)], dtype=torch.float64, device=device)
    mx, tot = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    if rank == 0:
        loads = PT.rank_loads(costs, parts)
        out = {"metric": METRIC, "value": float(tot[1]) / (float(mx[0]) / 1e3), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(mx[0]) / args.steps,
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
               "dtype": "f32 (double-float displacements; f64 pair distance, barrier, CCD and reductions)",
               "data": "synthetic",
               "config": {"workload": w.name, "envs": w.n_envs, "pads": w.n_pads,
                          "parallelism": f"the {w.n_envs} envs partitioned over {world} ranks "
                                         "(balanced by tets), marker fields all-gathered every frame"},
               "partition": {"envs_per_rank": [int(len(p)) for p in parts],
                             "tets_per_rank": [float(v) for v in loads],
                             "imbalance": float(loads.max() / loads.mean())},
               "gather_bytes_per_frame": int(w.n_envs * per_env * 2 * 4),
               "converged_fraction": float(tot[1]) / (args.steps * w.n_envs)}
        print(json.dumps(out), flush=True)
    return full


def run_adjoint(args):
    """Calibration workload (256 envs x one 5k-class pad, 16-frame
    press-and-slide): targets are the marker fields at hidden per-env
    materials; the loss is the L2 misfit at the nominal material; one step is
    the forward sequence through TacStepFn plus loss.backward() (the reverse
    sweep, which re-solves each frame from its checkpoint and runs
    tac_adjoint_frame). Prints one JSON line (ms per frame)."""
    import copy
    import torch
    from paper_2603_28475_b300 import autograd as A
    from paper_2603_28475_b300 import scenes as S
    from paper_2603_28475_b300 import tac
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w, hidden = S.config_calibration(n_envs=args.adjoint_envs, frames=args.adjoint_frames, seed=args.seed)
    b = tac.batch_from_workload(w, pair_capacity=args.pair_capacity)
    base = b.get_params()
    poses = torch.tensor(w.poses.astype(np.float64), device=dev)
    F = w.n_frames
    # targets: forward at the hidden materials
    hp = []
    for k, q in enumerate(base):
        r = copy.copy(q)
        r.E, r.nu, r.mu_f = hidden[k].E, hidden[k].nu, hidden[k].mu_f
        hp.append(r)
    b.set_params(hp)
    b.reset(poses[0].float())
    targets = []
    for f in range(1, F + 1):
        b.set_indenter(poses[f].float())
        b.step()
        targets.append(b.markers().clone())
    targets = torch.stack(targets)
    b.set_params(base)
    b.reset(poses[0].float())
    x0, v0 = b.get_state()
    lam = np.array([q.E * q.nu / ((1 + q.nu) * (1 - 2 * q.nu)) for q in base])
    mu = np.array([q.E / (2 * (1 + q.nu)) for q in base])
    lame = torch.tensor(np.stack([lam, mu], 1), dtype=torch.float64, requires_grad=True)
    mu_f = torch.tensor([q.mu_f for q in base], dtype=torch.float64, requires_grad=True)
    stream = torch.cuda.current_stream()
    # warm-up: the first two frames forward and backward, untimed
    mw = A.sequence_markers(b, x0, v0, lame, mu_f, poses[:3], base_params=base)
    ((mw - targets[:2]) ** 2).sum().backward()
    lame.grad, mu_f.grad = None, None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        ev[0].record(stream)
        m = A.sequence_markers(b, x0, v0, lame, mu_f, poses, base_params=base)
        loss = ((m - targets) ** 2).sum()
        ev[1].record(stream)
        loss.backward()
        ev[2].record(stream)
        torch.cuda.synchronize()
    fwd, bwd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    out = {"metric": "adjoint calibration step: 16-frame forward + reverse sweep (calibration workload)",
           "value": (fwd + bwd) / F, "unit": "ms/frame", "higher_is_better": False, "n_gpus": 1,
           "forward_ms_per_frame": fwd / F, "backward_ms_per_frame": bwd / F,
           "note": "backward installs each frame from its saved start and end states (tac_set_frame, no re-solve), "
                   "then runs the frame adjoint",
           "dtype": "f32 (double-float displacements; f64 pair distance, barrier, CCD and reductions)",
           "data": "synthetic",
           "config": {"workload": w.name, "envs": w.n_envs, "pads": w.n_pads, "pad_verts": w.pads[0].n_verts,
                      "frames": F, "friction": 0.5, "targets": "GPU forward at hidden per-env (E, nu, mu_f)"},
           "clocks": clk.summary(), "warmup": "frames 1-2 forward and backward, untimed",
           "loss": float(loss.item()), "grad_norm_lame": float(lame.grad.norm().item()),
           "grad_norm_mu_f": float(mu_f.grad.norm().item())}
    print(json.dumps(out), flush=True)
    b.close()


SWEEP_POINTS = ((64, 2000), (256, 2000), (1024, 2000), (1024, 10000), (64, 50000), (256, 50000),
                (1024, 50000))


def sweep_points(args):
    """The sweep's (envs, pad vertices) points: --sweep-points "64x50000,..."
    or all of SWEEP_POINTS."""
    if not args.sweep_points:
        return SWEEP_POINTS
    return tuple(tuple(int(v) for v in q.split("x")) for q in args.sweep_points.split(","))


def run_sweep(args):
    """Throughput over environment counts and pad sizes: one pad of ~V
    vertices per env, a cylinder press with friction 0.5 (scenes.config_sweep).
    Per point: W warm-up frames, then K timed frames (CUDA events on the
    stream); converged env-frames/s, ms per frame and counted GB/s of the
    solve launch. Prints one JSON line with all points."""
    import torch
    from paper_2603_28475_b300 import scenes as S
    from paper_2603_28475_b300 import tac
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    W, K = 2, 2
    peak, peak_kind = load_peaks()
    pts = []
    for envs, nv in sweep_points(args):
        w = S.config_sweep(envs, nv, frames=W + K, seed=args.seed)
        cap = max(args.pair_capacity, int(args.pair_capacity * 1.5 * (nv / 10000.0) ** (2.0 / 3.0)))
        b = tac.batch_from_workload(w, pair_capacity=cap)
        poses = torch.tensor(w.poses, dtype=torch.float32, device=dev)
        st = torch.empty(w.n_pads, dtype=torch.int32, device=dev)
        it = torch.empty(w.n_pads, dtype=torch.int32, device=dev)
        b.reset(poses[0])
        for f in range(1, W + 1):
            b.set_indenter(poses[f])
            b.step(st, it)
        torch.cuda.synchronize()
        shape = choose_block_shape(b, poses[W + 1], args.block_shape)
        stream = torch.cuda.current_stream()
        ms, conv, nbytes, iters = 0.0, 0, 0.0, []
        for f in range(W + 1, W + K + 1):
            b.set_indenter(poses[f])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(st, it)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            conv += int((st == 0).sum().item())
            nbytes += algorithmic_bytes(b.stats().cpu().numpy(), w)
            iters.append(it.cpu().numpy())
        its = np.concatenate(iters)
        gbs = nbytes / (ms / 1e3) / 1e9
        pts.append({"envs": envs, "pad_verts": w.pads[0].n_verts, "pad_tets": w.pads[0].n_tets,
                    "pair_capacity": cap, "env_frames_per_s": conv / (ms / 1e3), "ms_per_frame": ms / K,
                    "converged_fraction": conv / (K * envs), "iters_p50": float(np.percentile(its, 50)),
                    "counted_gbs": gbs, "frac_of_peak": gbs / peak, "block_shape": shape})
        b.close()
        del b
        torch.cuda.empty_cache()
        print(json.dumps(pts[-1]), file=sys.stderr, flush=True)
    out = {"metric": "converged env-frames/s over env counts and pad sizes (large-scale sweep)",
           "unit": "env-frames/s", "higher_is_better": True, "n_gpus": 1, "warmup": W, "steps": K,
           "peak": peak, "peak_kind": peak_kind, "data": "synthetic",
           "dtype": "f32 (double-float displacements; f64 pair distance, barrier, CCD and reductions)",
           "config": {"workload": "sweep (scenes.config_sweep)", "friction": 0.5, "tol_rel_grad": 1e-6,
                      "frames": f"{W + 1}..{W + K} of a 0.05 mm/frame press"},
           "points": pts}
    print(json.dumps(out), flush=True)


VARIANTS = (("block_jacobi_bounded_step", dict()),
            ("scalar_jacobi", dict(precond=1)),
            ("literal_step", dict(step=1)),
            ("scalar_jacobi_literal_step", dict(precond=1, step=1)))


def run_variants(args):
    """The paper-literal variants (scalar Jacobi preconditioner; Eq.
    (step_size) as printed, without CCD bound or energy test) against the
    chosen forms on the batched workload: W warm-up frames, then K timed
    frames per variant (CUDA events on the stream). Per variant: converged
    env-frames/s, ms per frame, converged fraction, PNCG iterations per pad
    (mean, p50, p99) and step halvings per pad-frame. Prints one JSON line."""
    import torch
    from paper_2603_28475_b300 import tac
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    W, K = args.warmup, args.steps
    w = workload(args.envs, W + K + 1, args.seed)
    poses = torch.tensor(w.poses, dtype=torch.float32, device=dev)
    res = []
    for name, modes in VARIANTS:
        b = tac.batch_from_workload(w, pair_capacity=args.pair_capacity, **modes)
        st = torch.empty(w.n_pads, dtype=torch.int32, device=dev)
        it = torch.empty(w.n_pads, dtype=torch.int32, device=dev)
        b.reset(poses[0])
        for f in range(1, W + 1):
            b.set_indenter(poses[f])
            b.step(st, it)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        ms, conv, iters, halv, status = 0.0, 0, [], [], []
        for f in range(W + 1, W + K + 1):
            b.set_indenter(poses[f])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(st, it)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            conv += int(np.all(st.cpu().numpy().reshape(-1, w.pads_per_env) == 0, axis=1).sum())
            iters.append(it.cpu().numpy())
            halv.append(b.stats().cpu().numpy()[:, 3])
            status.append(st.cpu().numpy())
        its, hv, sts = np.concatenate(iters), np.concatenate(halv), np.concatenate(status)
        res.append({"variant": name, "modes": modes, "env_frames_per_s": conv / (ms / 1e3),
                    "ms_per_frame": ms / K, "converged_env_fraction": conv / (K * w.n_envs),
                    "status_counts": {str(k): int(v) for k, v in zip(*np.unique(sts, return_counts=True))},
                    "iters_mean": float(its.mean()), "iters_p50": float(np.percentile(its, 50)),
                    "iters_p99": float(np.percentile(its, 99)), "halvings_per_pad_frame": float(hv.mean())})
        b.close()
        del b
        torch.cuda.empty_cache()
        print(json.dumps(res[-1]), file=sys.stderr, flush=True)
    out = {"metric": "converged env-frames/s and PNCG iterations per variant (batched press)",
           "unit": "env-frames/s", "higher_is_better": True, "n_gpus": 1, "warmup": W, "steps": K,
           "data": "synthetic", "config": {"workload": f"batched press, {args.envs} envs x 2 pads (2k/5k/10k)",
                                           "tol_rel_grad": 1e-6, "pair_capacity": args.pair_capacity},
           "variants": res}
    print(json.dumps(out), flush=True)


def run_calibrate(args):
    """Baseline calibration (Eq. loss_function) on synthetic recordings: 3
    press-and-slide scenes (2k-class pad, cylinder pegs, 8 frames) at hidden
    theta* = (E, nu, rho, mu_f). CMA-ES with the paper's settings
    (normalised parameters, population 12, 80 generations; each generation
    one batch of 36 pads) over all four parameters and over (E, nu, mu_f)
    with rho at its nominal value; Adam on (E, nu, mu_f) with adjoint
    gradients (40 iterations, forward + reverse sweep each; the frames'
    friction lags differentiated, and held fixed) for comparison.
    Prints one JSON line with the loss curves and times."""
    import torch
    from paper_2603_28475_b300 import calibrate as C
    from paper_2603_28475_b300 import scenes as S
    torch.cuda.set_device(0)
    w, _ = S.config_calibration(n_envs=3, frames=8, seed=args.seed, pad_verts=2000)
    base = S.Material(E=1.05e5, nu=0.4485, rho=3000.0, mu_f=1.375)      # the centre of the ranges
    truth = {"E": 1.4e5, "nu": 0.46, "rho": 1100.0, "mu_f": 0.9}
    runs = {}
    for names, gens in ((C.PARAMS, 80), (("E", "nu", "mu_f"), 80)):
        cal = C.Calibration(w, 12, base if "rho" in names else S.Material(**{**base.__dict__, "rho": truth["rho"]}),
                            names=names)
        tgt = cal.targets([truth[n] for n in names])
        best, h = C.calibrate_cmaes(cal, tgt, generations=gens, sigma0=0.3, seed=args.seed)
        cal.close()
        runs["cmaes_" + "_".join(names)] = {
            "params": list(names), "generations": gens, "popsize": 12, "best": dict(zip(names, best.tolist())),
            "rel_error": {n: abs(b / truth[n] - 1) for n, b in zip(names, best)},
            "best_loss": h.best_loss[::max(1, gens // 20)] + [h.best_loss[-1]],
            "pad_frames_solved": h.frames_solved[-1], "seconds": h.seconds[-1],
            "ms_per_generation": 1e3 * h.seconds[-1] / gens}
    names = ("E", "nu", "mu_f")
    base_r = S.Material(**{**base.__dict__, "rho": truth["rho"]})
    cal = C.Calibration(w, 12, base_r, names=names)
    tgt = cal.targets([truth[n] for n in names])
    kappa = cal.kappa[:w.n_pads]
    cal.close()
    for relag in (True, False):
        th, h = C.calibrate_adjoint(w, base_r, tgt, iterations=40, lr=0.05, kappa=kappa, relag=relag)
        runs["adjoint_adam_E_nu_mu_f" + ("" if relag else "_frozen_lag")] = {
            "params": list(names), "iterations": 40, "lag": "differentiated" if relag else "frozen",
            "best": dict(zip(names, th.tolist())),
            "rel_error": {n: abs(b / truth[n] - 1) for n, b in zip(names, th)},
            "loss": h.mean_loss[::2] + [h.mean_loss[-1]], "pad_frames_solved": h.frames_solved[-1],
            "seconds": h.seconds[-1], "ms_per_iteration": 1e3 * h.seconds[-1] / 40}
    out = {"metric": "baseline calibration on synthetic recordings: loss curves and time (CMA-ES vs adjoint)",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "dtype": "f32 (double-float displacements; f64 pair distance, barrier, CCD and reductions)",
           "config": {"workload": w.name + " (2k-class pad, 3 scenes, 8 frames)", "truth": truth,
                      "start": "centre of the parameter ranges", "ranges": C.RANGES},
           "runs": runs}
    print(json.dumps(out), flush=True)


def run_trajectory(args, frames=60, n_verts=50000):
    """Long trajectories (scenes.config_trajectory): envs x one ~50k-vertex
    pad (54k), a chamfered peg or a threaded nut flank of ~10k triangles per
    env, press then hold then slide with friction 0.5, 60 frames from rest,
    every frame timed (CUDA events on the stream). Prints one JSON line:
    env-frames/s over the trajectory and per phase of it, statuses,
    iterations and the counted GB/s of the solve launches."""
    import torch
    from paper_2603_28475_b300 import scenes as S
    from paper_2603_28475_b300 import tac
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peak, peak_kind = load_peaks()
    w = S.config_trajectory(n_envs=args.trajectory_envs, n_verts=n_verts, frames=frames, seed=args.seed)
    nv = w.pads[0].n_verts
    cap = max(args.pair_capacity, int(args.pair_capacity * 1.5 * (nv / 10000.0) ** (2.0 / 3.0)))
    b = tac.batch_from_workload(w, pair_capacity=cap)
    poses = torch.tensor(w.poses, dtype=torch.float32, device=dev)
    st = torch.empty(w.n_pads, dtype=torch.int32, device=dev)
    it = torch.empty(w.n_pads, dtype=torch.int32, device=dev)
    # the block shape: tuned on frame 6 of an untimed first pass (the
    # press in contact), then the trajectory runs from rest in that shape
    tune_frame = 6
    b.reset(poses[0])
    if args.block_shape == "auto":
        for f in range(1, tune_frame):
            b.set_indenter(poses[f])
            b.step(st, it)
        torch.cuda.synchronize()
    shape = choose_block_shape(b, poses[tune_frame], args.block_shape)
    if args.block_shape == "auto":
        shape["chosen_by"] = f"tac_autotune_block_shape on frame {tune_frame} of an untimed first pass"
    b.reset(poses[0])
    stream = torch.cuda.current_stream()
    rec = []
    with ClockSampler(dev.index) as clk:
        for f in range(1, frames + 1):
            b.set_indenter(poses[f])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(st, it)
            e1.record(stream)
            torch.cuda.synchronize()
            sn, itn = st.cpu().numpy(), it.cpu().numpy()
            rec.append((f, e0.elapsed_time(e1), int((sn == 0).sum()), itn, algorithmic_bytes(b.stats().cpu().numpy(), w)))
    b.close()
    ms = np.array([r[1] for r in rec])
    conv = np.array([r[2] for r in rec])
    its = np.concatenate([r[3] for r in rec])
    half = frames // 2

    def span(a, z):
        sl = slice(a, z)
        return {"frames": f"{a + 1}..{z}", "env_frames_per_s": float(conv[sl].sum() / (ms[sl].sum() / 1e3)),
                "ms_per_frame": float(ms[sl].mean())}
    gbs = sum(r[4] for r in rec) / (ms.sum() / 1e3) / 1e9
    out = {"metric": "converged env-frames/s over 60-frame trajectories of fine pads (large-scale configuration)",
           "unit": "env-frames/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
           "value": float(conv.sum() / (ms.sum() / 1e3)),
           "dtype": "f32 (double-float displacements; f64 pair distance, barrier, CCD and reductions)",
           "config": {"workload": w.name, "envs": w.n_envs, "pad_verts": nv, "pad_tets": w.pads[0].n_tets,
                      "indenters": "chamfered peg (9984 tris) and threaded nut flank (10368 tris), alternating",
                      "frames": f"1..{frames} from rest: press 0.05 mm/frame to U[0.2, 1.0] mm, hold to frame "
                                f"{half}, slide 0.02 mm/frame", "friction": 0.5, "pair_capacity": cap,
                      "tol_rel_grad": 1e-6},
           "converged_fraction": float(conv.sum() / (frames * w.n_pads)),
           "not_converged_by_frame": {str(r[0]): int(w.n_pads - r[2]) for r in rec if r[2] < w.n_pads},
           "phases": {"press_hold": span(0, half), "slide": span(half, frames)},
           "frame_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                        "max": float(ms.max())},
           "iters_per_pad_frame": {"p50": float(np.percentile(its, 50)), "p99": float(np.percentile(its, 99)),
                                   "max": int(its.max())},
           "counted_gbs": gbs, "frac_of_peak": gbs / peak, "peak": peak, "peak_kind": peak_kind,
           "clocks": clk.summary(), "block_shape": shape}
    print(json.dumps(out), flush=True)


# the hidden materials' prior of the calibration workload: the search box
C4_RANGES = {"E": (1e5, 5e5), "nu": (0.40, 0.49), "mu_f": (0.3, 0.9), "rho": (1e3, 5e3)}


def run_calibrate_oracle(args, generations=30, iterations=20):
    """Calibration against targets the FP64 oracle solved (written by
    tests/golden/make_calibration_targets.py): the calibration workload's
    first environments (5k pad, 16-frame press-and-slide, friction), each
    at its own hidden (E, nu, mu_f). Per environment: CMA-ES (population 12,
    the populations of all environments solved in the same batches) and
    Adam on adjoint gradients (lags differentiated), both started at the
    nominal material, over the hidden materials' prior box. Prints one
    JSON line: per-environment relative errors, loss curves and times."""
    import torch
    from paper_2603_28475_b300 import calibrate as C
    from paper_2603_28475_b300 import scenes as S
    torch.cuda.set_device(0)
    g = np.load(os.path.join(ROOT, "tests", "golden", "calibration_targets.npz"))
    n, F = len(g["envs"]), int(g["frames"])
    w_all, hidden = S.config_calibration(n_envs=256, frames=F, seed=0)
    w = S.Workload("calibration_head", w_all.pads[:n], w_all.materials[:n], w_all.indenters[:n], 1,
                   w_all.poses[:, :n])
    names = ("E", "nu", "mu_f")
    truth = np.array(g["hidden"])
    base = w.materials[0]
    x0 = np.tile(C.to_unit([base.E, base.nu, base.mu_f], names, C4_RANGES), (n, 1))
    targets = torch.tensor(np.transpose(g["markers"], (1, 0, 2, 3)).reshape(F, -1, 2), dtype=torch.float32,
                           device="cuda")
    kappa = list(np.tile(g["kappa"], 12))
    cal = C.Calibration(w, 12, base, names=names, kappa=kappa)
    best, h = C.calibrate_cmaes_per_scene(cal, targets, generations=generations, sigma0=0.3, x0=x0,
                                          seed=args.seed, ranges=C4_RANGES)
    cal.close()
    runs = {"cmaes_per_env": {
        "generations": generations, "popsize": 12, "theta": best.tolist(),
        "rel_error": (np.abs(best / truth - 1.0)).tolist(),
        "best_loss_mean_over_envs": h.best_loss[::max(1, generations // 15)] + [h.best_loss[-1]],
        "pad_frames_solved": h.frames_solved[-1], "seconds": h.seconds[-1]}}
    th, ha = C.calibrate_adjoint(w, base, targets, iterations=iterations, lr=0.05, x0=x0, kappa=list(g["kappa"]),
                                 relag=True, per_scene=True, ranges=C4_RANGES)
    runs["adjoint_adam_per_env"] = {
        "iterations": iterations, "lag": "differentiated", "theta": np.asarray(th).tolist(),
        "rel_error": (np.abs(np.asarray(th) / truth - 1.0)).tolist(),
        "loss": ha.mean_loss[::2] + [ha.mean_loss[-1]], "pad_frames_solved": ha.frames_solved[-1],
        "seconds": ha.seconds[-1]}
    out = {"metric": "calibration against FP64-oracle targets: relative parameter errors, loss and time",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "dtype": "f32 (double-float displacements; f64 pair distance, barrier, CCD and reductions)",
           "config": {"workload": f"calibration workload, first {n} envs x {F} frames (5k pads, friction)",
                      "targets": "FP64 oracle at each env's hidden (E, nu, mu_f)",
                      "hidden": truth.tolist(), "start": "nominal material (0.3 MPa, 0.45, 0.5)",
                      "search_box": {k: C4_RANGES[k] for k in names}},
           "runs": runs}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.adjoint:
        if rank == 0:
            run_adjoint(args)
        return
    if args.sweep:
        if rank == 0:
            run_sweep(args)
        return
    if args.variants:
        if rank == 0:
            run_variants(args)
        return
    if args.calibrate:
        if rank == 0:
            run_calibrate(args)
        return
    if args.calibrate_oracle:
        if rank == 0:
            run_calibrate_oracle(args)
        return
    if args.trajectory:
        if rank == 0:
            run_trajectory(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.shard:
        import torch
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        torch.distributed.init_process_group("nccl", world_size=world, rank=rank)
        run_sharded(args, rank, world)
        torch.distributed.destroy_process_group()
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
