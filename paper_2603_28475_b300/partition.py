"""Environments across GPUs: a balanced partition and the per-frame gather
of marker fields.

The paper runs one simulation actor per GPU and gathers every actor's
tactile observations for the policy each step (Sec. 3.3, "Multi-node
Multi-GPU parallelization"). Environments are independent solves, so the
only exchange is that gather. Here one process drives one GPU:

* ``balanced_partition`` splits the environments into per-rank sets of
  about equal predicted cost, the cost of an environment being the sum
  over its pads of tets x expected PNCG iterations (the previous frame's
  iterations when known, else one per pad). Longest processing time first:
  each environment, costliest first, goes to the rank with the least cost
  so far (ties to the lower rank), which keeps the largest rank cost within
  4/3 of the optimum.
* ``gather_markers`` all-gathers the ranks' marker fields into the full
  field in the global environment order, over whatever backend the default
  process group has (NCCL between GPUs, gloo on the host).

Host code only: the solve itself runs per rank on the rank's environments.
"""
from __future__ import annotations

import heapq

import numpy as np


def env_costs(pad_tets, pads_per_env, pad_iters=None):
    """Predicted cost per environment: sum over its pads of tets x
    iterations (pad_iters None: one iteration per pad)."""
    t = np.asarray(pad_tets, dtype=np.float64)
    it = np.ones_like(t) if pad_iters is None else np.maximum(np.asarray(pad_iters, dtype=np.float64), 1.0)
    return (t * it).reshape(-1, pads_per_env).sum(axis=1)


def balanced_partition(costs, n_ranks):
    """Environment ids per rank [n_ranks] (each sorted ascending): greedy
    longest-processing-time assignment of the environments by cost.
    Deterministic: ties between costs go to the lower environment id,
    ties between ranks to the lower rank."""
    costs = np.asarray(costs, dtype=np.float64)
    if n_ranks < 1:
        raise ValueError("n_ranks must be positive")
    order = sorted(range(len(costs)), key=lambda e: (-costs[e], e))
    heap = [(0.0, r) for r in range(n_ranks)]
    heapq.heapify(heap)
    parts = [[] for _ in range(n_ranks)]
    for e in order:
        load, r = heapq.heappop(heap)
        parts[r].append(e)
        heapq.heappush(heap, (load + costs[e], r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def rank_loads(costs, parts):
    """Summed cost per rank of a partition."""
    costs = np.asarray(costs, dtype=np.float64)
    return np.array([costs[p].sum() for p in parts])


def gather_markers(local, env_ids, n_envs, group=None):
    """All-gather the ranks' marker fields. ``local``: this rank's tensor
    [n_local_envs, per_env, 2] for the environments ``env_ids`` (its
    partition, ascending); returns the full [n_envs, per_env, 2] tensor in
    global environment order on every rank. Ranks may hold different
    numbers of environments: each pads to the largest count for the
    collective and the padding is dropped."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n_local = torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device)
    counts = [torch.zeros_like(n_local) for _ in range(world)]
    dist.all_gather(counts, n_local, group=group)
    counts = [int(c.item()) for c in counts]
    cap = max(counts)
    pad = torch.zeros((cap,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    ids = torch.full((cap,), -1, dtype=torch.int64, device=local.device)
    ids[:local.shape[0]] = torch.as_tensor(env_ids, dtype=torch.int64, device=local.device)
    bufs = [torch.empty_like(pad) for _ in range(world)]
    idbufs = [torch.empty_like(ids) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    dist.all_gather(idbufs, ids, group=group)
    out = torch.zeros((n_envs,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    for r in range(world):
        c = counts[r]
        if c:
            out[idbufs[r][:c]] = bufs[r][:c]
    return out
