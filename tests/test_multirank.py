"""The multi-rank bench path on the CPU (world size 2, gloo; no GPU).

Environments shard across ranks with no data-path exchange: each rank
builds its own workload from its own seed, and only the timed region's
totals are reduced: the slowest rank's time and the sum of converged envs.
The reference arm runs on rank 0 alone.
"""
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
