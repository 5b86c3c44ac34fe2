"""The multi-rank bench paths on the CPU (world size 2, gloo; no GPU).

Weak scaling: environments shard across ranks with no data-path exchange;
each rank builds its own workload from its own seed, and only the timed
region's totals are reduced: the slowest rank's time and the sum of
converged envs. The reference arm runs on rank 0 alone. Strong scaling
(--shard): one job's environments partitioned across the ranks and their
marker fields all-gathered every frame.
"""
import json
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r timed 100 + 50 r ms and converged 10 + r envs
    ms, conv = bench.job_totals(100.0 + 50.0 * rank, 10 + rank, world)
    out[rank] = (ms, conv)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_take_the_slowest_rank_and_sum_the_envs():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (150.0, 21.0)


def test_single_rank_totals_pass_through():
    import bench
    assert bench.job_totals(12.5, 7, 1) == (12.5, 7.0)


def test_ranks_solve_different_environments():
    import bench
    from paper_2603_28475_b300 import scenes as S
    ws = [S.config_batched(n_envs=3, frames=2, seed=bench.rank_seed(0, r)) for r in range(2)]
    assert not np.array_equal(ws[0].poses, ws[1].poses)
    assert bench.rank_seed(0, 0) == 0 and bench.rank_seed(0, 1) != 0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    import argparse
    args = argparse.Namespace(envs=4, warmup=0, steps=1, seed=0, gpus=2)
    bench.run_reference(args, 1, 2)
    assert capsys.readouterr().out == ""


# --------------------------------------------------------------------------
# environments partitioned across ranks and the per-frame marker gather


def test_balanced_partition_of_the_benchmark_workload():
    """Every environment lands on exactly one rank; the greedy bound holds
    (the largest rank load is at most the mean load plus the largest
    environment cost); the split is deterministic; with the size classes'
    tet counts the ranks come within 1% of each other."""
    from paper_2603_28475_b300 import partition as PT
    from paper_2603_28475_b300 import scenes as S
    w = S.config_batched(n_envs=4096, frames=1, seed=0)
    costs = PT.env_costs([p.n_tets for p in w.pads], w.pads_per_env)
    for n in (2, 3, 8):
        parts = PT.balanced_partition(costs, n)
        allids = np.sort(np.concatenate(parts))
        assert np.array_equal(allids, np.arange(w.n_envs))
        loads = PT.rank_loads(costs, parts)
        assert loads.max() <= costs.sum() / n + costs.max() + 1e-6
        assert loads.max() / loads.min() < 1.01
        again = PT.balanced_partition(costs, n)
        assert all(np.array_equal(a, b) for a, b in zip(parts, again))
    # iteration-weighted costs move environments towards the cheap ranks
    iters = np.where(np.arange(w.n_pads) % 7 == 0, 500, 50)
    c2 = PT.env_costs([p.n_tets for p in w.pads], w.pads_per_env, iters)
    loads = PT.rank_loads(c2, PT.balanced_partition(c2, 4))
    assert loads.max() <= c2.sum() / 4 + c2.max() + 1e-6


def _gather_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2603_28475_b300 import partition as PT
    n_envs, per_env = 11, 126
    rng = np.random.default_rng(3)
    full = rng.normal(size=(n_envs, per_env, 2)).astype(np.float32)
    costs = rng.uniform(1, 10, size=n_envs)
    parts = PT.balanced_partition(costs, world)
    mine = parts[rank]
    local = torch.tensor(full[mine])          # this rank's solved marker fields
    got = PT.gather_markers(local, mine, n_envs)
    out[rank] = bool(np.array_equal(got.numpy(), full)), [len(p) for p in parts]
    dist.barrier()
    dist.destroy_process_group()


def test_marker_gather_reassembles_the_global_field():
    """World size 2 on gloo: each rank holds the marker fields of its
    partition (unequal counts); the all-gather returns the full field in
    global environment order on both ranks."""
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_gather_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ok, counts = res[r]
        assert ok
        assert sum(counts) == 11 and counts[0] != counts[1]


class _FakeShardBatch:
    """Stands in for a rank's TacBatch on the host: every pad converges and
    its markers all read the (x, y) translation of its current pose, so the
    gathered field says which environment each entry came from."""

    def __init__(self, ws):
        self.ws = ws
        self.m = int(np.asarray(ws.pads[0].markers).shape[0])
        self.pose = None

    def reset(self, poses):
        self.pose = poses

    def set_indenter(self, poses):
        self.pose = poses

    def step(self, st, it):
        st.zero_()
        it.fill_(7)

    def markers(self):
        xy = self.pose[:, 3:5]
        return xy.repeat_interleave(self.m, dim=0).contiguous()


def _sharded_rank(rank, world, port, out):
    import argparse
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    args = argparse.Namespace(envs=5, warmup=1, steps=2, seed=0, pair_capacity=16384, no_dm_table=False)
    full = bench.run_sharded(args, rank, world, make_batch=_FakeShardBatch, device=torch.device("cpu"))
    w = bench.workload(5, 4, 0)
    m = int(np.asarray(w.pads[0].markers).shape[0])
    want = np.repeat(w.poses[3, :, 3:5], m, axis=0).reshape(w.n_envs, w.pads_per_env * m, 2)
    out[rank] = bool(np.array_equal(full.numpy(), want.astype(np.float32)))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_run_partitions_and_gathers_every_frame(capfd):
    """bench.run_sharded on 2 gloo ranks with host stand-ins for the
    batches: each rank solves its partition of the 5 environments, and the
    last frame's gathered field holds every environment's markers in global
    order on both ranks; rank 0 reports the partition and the converged
    fraction."""
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_sharded_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res == {0: True, 1: True}
    lines = [ln for ln in capfd.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["scaling"] == "strong" and rec["n_gpus"] == 2
    assert sum(rec["partition"]["envs_per_rank"]) == 5
    assert rec["converged_fraction"] == 1.0
