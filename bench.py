"""Benchmark: converged tactile env-frames per second of the batched PNCG-IPC
frame solve, with the roofline of the solve kernel and the FP64 oracle timed
on the host cores beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--envs E] [--impl ours|reference]

Workload (the batched RL step): E environments x 2 gel pads, each env's pads
drawn from the 2k / 5k / 10k-vertex size classes, a cylinder peg per env
(r ~ U[2, 4] mm) pressed into each pad at 0.05 mm per frame from a dhat gap
with a random pose (+-15 deg, +-1 mm) up to a depth ~ U[0, 1.2] mm, friction
0.5. One step = one frame for every pad: set the target poses, solve
(tac_step), read the markers. W warm-up frames, then K timed frames.
Under torchrun every rank solves its own E environments (weak scaling).
"""
from __future__ import annotations

import argparse
import json
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
# the direction (36 B) and, averaged over the two pass kinds, writes the
# gradient and diagonal block (36 B / 2); a vertex pass moves ~120 B per
# vertex; a pair evaluation ~64 B per candidate pair. A mesh with a Dm^-1
# table (the structured case) reads no per-tet Dm^-1.
B_TET = 48.0
B_DM = 36.0
B_TET_VERT = 36.0 + 18.0
B_VERT_PASS = 120.0
B_PAIR = 64.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
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
    ap.add_argument("--variants", action="store_true",
                    help="iterations and throughput of the paper-literal variants on the batched workload instead")
    return ap.parse_args()


# --------------------------------------------------------------------------- helpers

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


def algorithmic_bytes(stats, w, dm_table=True):
    """Counted bytes of one solve launch from the per-pad counters."""
    tot = 0.0
    for k, pad in enumerate(w.pads):
        it, sub, reb, hal, tp, vp, pe, peak = [float(v) for v in stats[k][:8]]
        bt = B_TET - (B_DM if tabled(pad, dm_table) else 0.0)
        tot += tp * (bt * pad.n_tets + B_TET_VERT * pad.n_verts) + vp * B_VERT_PASS * pad.n_verts + pe * B_PAIR
    return tot


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

def class_mean_tets():
    """Expected tet count of a pad when classes are drawn uniformly."""
    from paper_2603_28475_b300 import scenes as S
    return float(np.mean([6 * a * b * c for a, b, c in S.SIZE_CLASSES.values()]))


def oracle_sample(w, frame_pose_idx=1):
    """The oracle as it stands on one pad of the smallest size class for one
    frame (contact from rest). Returns (seconds, pad index, scale) where scale
    converts one such pad-frame into one average env-frame of the workload
    (2 pads, tet count averaged over the workload's pads)."""
    from oracle import geometry as G
    from oracle import solver as SV
    f32 = lambda v: float(np.float32(v))
    k = int(np.argmin([p.n_tets for p in w.pads]))
    pd, m = w.pads[k], w.materials[k]
    pad = G.build_pad(pd.rest, pd.tets, pd.fixed, pd.markers, f32(m.E), f32(m.nu), f32(m.rho), f32(m.h),
                      f32(m.dhat), f32(m.mu_f))
    e = k // w.pads_per_env
    ind = G.build_indenter(w.indenters[e].verts, w.indenters[e].tris)
    st = SV.rest_state(pad, w.poses[0, k].astype(np.float64))
    t = time.perf_counter()
    st, info = SV.solve_frame(pad, ind, st, w.poses[frame_pose_idx, k].astype(np.float64))
    dt = time.perf_counter() - t
    scale = w.pads_per_env * class_mean_tets() / pd.n_tets
    return dt, k, scale, info


# --------------------------------------------------------------------------- arms

def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(min(args.envs, 8), 2, args.seed)
    times = []
    info = None
    for i in range(args.warmup + args.steps):
        dt, k, scale, info = oracle_sample(w)
        if i >= args.warmup:
            times.append(dt * scale)
    t_env = float(np.mean(times))
    value = 1.0 / t_env
    sample = (f"oracle (numpy FP64, 1 thread) on one {w.pads[k].n_verts}-vert pad for its first contact frame "
              f"({info.iters} iterations), scaled by {scale:.2f} to one average env-frame of the workload "
              "(2 pads, mean tet count of the size classes)")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_env * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": f"batched_{args.envs}env_x2pads", "envs": args.envs},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
            stats_all.append((status.clone(), iters.clone(), st))
        stop.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = start.elapsed_time(stop)
    solve_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    phase = np.zeros(8)
    pad_ms_max = 0.0
    for stt, it, st in stats_all:
        s_np = stt.cpu().numpy().reshape(-1, w.pads_per_env)
        conv += int(np.all(s_np == 0, axis=1).sum())
        iter_hist.append(it.cpu().numpy())
        st_np = st.cpu().numpy()
        bytes_alg += algorithmic_bytes(st_np, w, not args.no_dm_table)
        phase += st_np[:, 8:16].sum(axis=0)
        pad_ms_max = max(pad_ms_max, float(st_np[:, 15].max()) / 1e6)
    names = ["tet_pHp", "tet_grad", "pair_pHp", "pair_grad", "vertex", "advance_rebuild", "setup"]
    phase_share = {n: float(phase[i] / phase[7]) for i, n in enumerate(names)} if phase[7] > 0 else None
    # CTA-time spent inside pads over the launch's CTA-time: below 1 the grid idles
    # behind the queue's last pads
    queue = {"ctas": b.grid_ctas, "busy": float(phase[7] / 1e6 / (b.grid_ctas * sum(solve_ms))),
             "longest_pad_ms": pad_ms_max}
    total_ms_job, conv_job = job_totals(total_ms, conv, world, dev)
    value = conv_job / (total_ms_job / 1e3)
    its = np.concatenate(iter_hist)
    bytes_per_launch = bytes_alg / args.steps
    launch_ms = float(np.mean(solve_ms))
    peak, peak_kind = load_peaks()
    achieved = bytes_per_launch / (launch_ms / 1e3) / 1e9
    traffic = committed_traffic(bytes_per_launch)
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
            dt, k, scale, info = oracle_sample(w)
            cpu = {"value": 1.0 / (dt * scale), "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"oracle (numpy FP64, 1 thread) on one {w.pads[k].n_verts}-vert pad, first contact "
                             f"frame ({info.iters} iterations, {dt:.1f} s), scaled by {scale:.2f} to an average "
                             "env-frame (2 pads, mean tet count of the size classes)"}
        except Exception as exc:             # the GPU line is still reported
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {exc!r}"}
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
                            "launch_ms": launch_ms},
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 3 * args.steps,
               "clocks": clk.summary(),
               "converged_fraction": conv_job / (args.steps * args.envs * world),
               "iters_per_pad_frame": {"p50": float(np.percentile(its, 50)), "p99": float(np.percentile(its, 99)),
                                       "max": int(its.max())},
               "frame_ms": {"p50": float(np.percentile(solve_ms, 50)), "p99": float(np.percentile(solve_ms, 99))},
               "setup_s": t_create, "phase_share": phase_share, "queue": queue}
        print(json.dumps(out), flush=True)
    b.close()


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
    for envs, nv in SWEEP_POINTS:
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
                    "counted_gbs": gbs, "frac_of_peak": gbs / peak})
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
    if args.impl == "reference":
        run_reference(args, rank, world)
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
