"""Sampled kernel timing (gx_profile_enable): the device-timer stamps of the sampled launches
leave the iterates bitwise unchanged, cover every residual-check chunk of the whole-loop
graph, and the per-scenario active counts bound the work of those launches."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(profile):
    import torch
    nets, scens = synth.medium(S=4, T=48)
    net = gpu_net(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=20000, adj_max_iter=20000,
                  check_every=20, rho=0.2)
    if profile:
        net.profile(True)
    eta = eta_tensor(nets[0]["eta_min"])
    net.solve(eta)
    g = net.grad(eta).clone()
    torch.cuda.synchronize()
    its = (net.last_stats["iters_max"], net.last_grad_stats["iters_max"])
    out = dict(g=g.cpu().numpy(), its=its, x=net.state(False).cpu().numpy().copy(),
               a=net.state(True).cpu().numpy().copy())
    if profile:
        out["prof"] = net.profile_read()
        out["active"] = net.profile_active()
        out["iters_s"] = net.array("iters").cpu().numpy().copy()
        out["adj_iters_s"] = net.array("adj_iters").cpu().numpy().copy()
    return out


def test_stamps_leave_iterates_unchanged_and_cover_chunks():
    a = _run(False)
    b = _run(True)
    assert a["its"] == b["its"]
    assert np.array_equal(a["g"], b["g"]) and np.array_equal(a["x"], b["x"]) and np.array_equal(a["a"], b["a"])
    chunks = (b["its"][0] + b["its"][1]) // 20
    prof = b["prof"]
    for k in ("k_bus", "k_line", "k_bat"):
        assert prof[k]["samples"] == chunks, (k, prof[k], chunks)
        avg_us = 1e3 * prof[k]["ms"] / prof[k]["samples"]
        assert 0.5 < avg_us < 5e3, (k, avg_us)
    # a scenario iterates in the chunks up to its own stop, forward and adjoint
    act = b["active"]
    assert np.array_equal(act, (b["iters_s"] + b["adj_iters_s"]) // 20), (act, b["iters_s"], b["adj_iters_s"])
