"""Scenario sharding + gradient all-reduce on two CPU ranks (gloo): the reduced partial
gradients equal the full-batch gradient (computed here with the FP64 oracle)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2410_13055_gb300 import sharding, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _problem():
    nets, scens = [], []
    for k, (nb, nl, ng, nbt, T) in enumerate([(4, 5, 8, 1, 4), (5, 7, 10, 1, 3), (3, 3, 6, 1, 5)]):
        n, sc = synth.custom(nb, nl, ng, nbt, T, S=1, seed=60 + k, net_index=k)
        sc[0]["weight"] = 1.0 / 3
        nets.append(n)
        scens.append(sc[0])
    return nets, scens


def _partial(nets, scens, idx, kappa):
    from oracle import dispatch, grad
    ln, ls, used = sharding.local_problem(nets, scens, idx)
    eta = np.concatenate([n["eta_min"] for n in ln])
    sols = dispatch.solve_all(ln, ls, eta, synth.default_opts(kappa=kappa))
    offs = np.cumsum([0] + [int(n["K"]) for n in ln])
    g = np.zeros(offs[-1])
    for sc, sol in zip(ls, sols):
        k = sc["net"]
        g[offs[k]:offs[k + 1]] += sc["weight"] * grad.adjoint_grad(sol)
    return sharding.scatter_to_global(nets, used, g)


def _rank(rank, world, port, kappa, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nets, scens = _problem()
    parts = sharding.shard(nets, scens, world)
    g = torch.tensor(_partial(nets, scens, parts[rank], kappa))
    sharding.allreduce_sum(g)
    out[rank] = g.numpy().copy()
    dist.destroy_process_group()


def test_shards_balance_and_cover():
    nets, scens = synth.batching(S=12)
    parts = sharding.shard(nets, scens, 3)
    assert sorted(i for p in parts for i in p) == list(range(12))
    loads = [synth.device_hours(nets, [scens[i] for i in p]) for p in parts]
    assert max(loads) <= 1.6 * (sum(loads) / 3)


@pytest.mark.timeout(300)
def test_two_rank_gradient_allreduce_equals_full_batch():
    world, kappa = 2, 50.0
    ctx = mp.get_context("spawn")  # the manager and the ranks alike: no fork of a threaded process
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, kappa, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    nets, scens = _problem()
    full = _partial(nets, scens, list(range(len(scens))), kappa)
    for r in range(world):
        np.testing.assert_allclose(out[r], full, rtol=1e-9, atol=1e-9)
