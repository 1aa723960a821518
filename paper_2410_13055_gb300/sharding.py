"""Scenario sharding across ranks and the one collective of a plan step.

Scenarios are independent given the plan (Section 2.2: every scenario's dispatch and
Jacobian can be computed in parallel), so each rank solves its own shard and the only
exchange per plan step is the sum of the partial gradients sum_{s in shard} w_s dh_s /
deta (a K-vector) and of the partial objectives.  Shards are balanced by device-hours.
"""
from __future__ import annotations

import numpy as np

from . import synth


def shard(nets, scens, world: int):
    """Greedy longest-processing-time split of scenario indices into `world` shards
    balanced by device-hours; returns a list of index lists (each sorted)."""
    loads = [synth.device_hours(nets, [sc]) for sc in scens]
    order = np.argsort(loads, kind="stable")[::-1]
    bins = [[] for _ in range(world)]
    tot = np.zeros(world)
    for i in order:
        k = int(np.argmin(tot))
        bins[k].append(int(i))
        tot[k] += loads[i]
    return [sorted(b) for b in bins]


def local_problem(nets, scens, idx):
    """The networks and scenarios of one shard, with scenario weights unchanged (so the
    shard's weighted sum is its exact share of sum_s w_s h_s)."""
    used = sorted({scens[i]["net"] for i in idx})
    remap = {k: j for j, k in enumerate(used)}
    sub = []
    for i in idx:
        sc = dict(scens[i])
        sc["net"] = remap[sc["net"]]
        sub.append(sc)
    return [nets[k] for k in used], sub, used


def scatter_to_global(nets, used, local_grad):
    """Place a shard's gradient (over its networks) into the full plan vector."""
    offs = np.cumsum([0] + [int(n["K"]) for n in nets])
    out = np.zeros(offs[-1])
    o = 0
    for k in used:
        K = int(nets[k]["K"])
        out[offs[k]:offs[k] + K] = local_grad[o:o + K]
        o += K
    return out


def allreduce_sum(vec, group=None):
    """Sum a vector over all ranks (torch.distributed; NCCL for CUDA tensors, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    t = vec if isinstance(vec, torch.Tensor) else torch.as_tensor(vec)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
