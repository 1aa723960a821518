"""Kernel schedules (gx_network_set_schedule) change speed, not results.

The staged bus kernels (device rows brought into shared memory by bulk copies, or by
per-thread asynchronous copies) and the per-thread-load bus kernel compute the same
expressions in the same order: forward and
adjoint iterates, iteration counts and gradients agree bitwise, on networks that exercise
the stage's layout (several buses per block, ragged horizons, ramp-limited generators,
HVDC links) and blocks too large to stage.  One or two warps per battery sum their scans
in different orders, so those agree to the solver's tolerance."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu


def _cases():
    nets, scens = synth.medium(S=3, T=48)
    yield "medium-48h", nets, scens, 50.0
    # uneven networks and horizons (one block spans several short buses)
    nets, scens = synth.batching(seed=5, S=4)
    yield "uneven", nets, scens, 50.0
    n, sc = synth.custom(30, 45, 90, 9, 13, S=2, seed=7)
    n = synth.add_hvdc(synth.add_ramps(n, seed=1), 2, seed=2)
    yield "ramps-hvdc-13h", [n], sc, 50.0
    # T = 1: Tp = 4, one quad per bus; 128 buses per block, whose record is too large to stage
    n, sc = synth.custom(400, 600, 1200, 40, 1, S=1, seed=9)
    yield "one-hour", [n], sc, 0.0


def _run(nets, scens, kappa, **sched):
    import torch
    net = gpu_net(nets, scens, kappa=kappa, tol=1e-4, adj_tol=1e-4, max_iter=20000, adj_max_iter=20000,
                  check_every=20)
    net.set_schedule(**sched)
    eta = eta_tensor(np.concatenate([n["eta_min"] for n in nets]) * 1.05)
    rc = net.solve(eta)
    g = net.grad(eta).clone()
    torch.cuda.synchronize()
    return dict(rc=rc, its=(net.last_stats["iters_max"], net.last_grad_stats["iters_max"]),
                g=g.cpu().numpy(), x=net.state(False).cpu().numpy().copy(), a=net.state(True).cpu().numpy().copy(),
                cost=net.array("cost").cpu().numpy().copy())


@pytest.mark.parametrize("case", ["medium-48h", "uneven", "ramps-hvdc-13h", "one-hour"])
def test_staged_bus_kernels_are_bitwise_equal(case):
    nets, scens, kappa = next((n, s, k) for name, n, s, k in _cases() if name == case)
    a = _run(nets, scens, kappa, bus_staged=0)
    for staged in (1, 2):  # bulk copies (TMA), per-thread asynchronous copies
        b = _run(nets, scens, kappa, bus_staged=staged)
        assert a["its"] == b["its"], staged
        for k in ("g", "x", "a", "cost"):
            assert np.array_equal(a[k], b[k]), (case, staged, k)


def test_battery_warps_agree_to_tolerance():
    nets, scens = synth.medium(S=2, T=168)
    a = _run(nets, scens, 50.0, bat_warps=2)
    b = _run(nets, scens, 50.0, bat_warps=1)
    assert np.max(np.abs(a["cost"] - b["cost"]) / np.abs(a["cost"])) <= 1e-4
    assert np.linalg.norm(a["g"] - b["g"]) <= 5e-2 * np.linalg.norm(a["g"])  # both at 1e-4 residuals
