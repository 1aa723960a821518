"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs.

Tolerances (FP32 state, FP64 final reductions), for solves run to a 1e-6 residual:
objective relative error <= 1e-4, FP64 KKT residuals of the GPU (x, lambda) evaluated
by the oracle <= 1e-3 (relative), gradient relative error <= 1e-3."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net, pack_x, ref_groups, rel, solution
from oracle import dispatch, grad as ograd, kkt
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-6, max_iter=200000, adj_tol=1e-5, adj_max_iter=200000, check_every=50)
# FP32 solutions sit at their bounds to ~1e-4 relative; the KKT check treats a constraint
# within 1e-3 of its bound as possibly active.
ACT_TOL = 1e-3


def _solve_pair(nets, scens, eta, kappa=0.0, **kw):
    opts = synth.default_opts(kappa=kappa)
    net = gpu_net(nets, scens, kappa=kappa, **{**TIGHT, **kw})
    e = eta_tensor(eta)
    rc = net.solve(e)
    refs = dispatch.solve_all(nets, scens, np.asarray(eta, float), opts)
    return net, e, rc, refs


def test_tiny_dispatch_parity():
    nets, scens = synth.tiny()
    eta = nets[0]["eta_min"]
    net, e, rc, refs = _solve_pair(nets, scens, eta)
    assert rc == 0, net.last_stats
    ref = refs[0]
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    assert rel(g["price"], ref.price) <= 1e-3
    assert rel(g["p"], ref.p) <= 1e-3


@pytest.mark.parametrize("kappa", [0.0, 50.0])
def test_tiny_gradient_parity(kappa):
    nets, scens = synth.tiny()
    eta = nets[0]["eta_min"] * 1.1
    net, e, rc, refs = _solve_pair(nets, scens, eta, kappa=kappa)
    assert rc == 0
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0, net.last_grad_stats
    g_ref = ograd.adjoint_grad(refs[0])
    assert rel(gg, g_ref) <= 1e-3, (gg, g_ref)


def test_tiny_plan_trajectory_matches_golden():
    """Ten projected implicit-gradient steps (Section 2.2) on the GPU follow the oracle's."""
    import json
    import os

    import torch
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tiny_plan.json")))
    nets, scens = synth.tiny()
    net = gpu_net(nets, scens, kappa=gold["kappa"], **TIGHT)
    eta = eta_tensor(gold["eta"][0])
    gamma = eta_tensor(nets[0]["gamma"])
    lo, hi = eta_tensor(nets[0]["eta_min"]), eta_tensor(nets[0]["eta_max"])
    for k in range(len(gold["delta"])):
        assert net.solve(eta) == 0
        g = net.grad(eta)
        delta = (g + gamma).double().cpu().numpy()
        assert rel(delta, gold["delta"][k]) <= 1e-3, k
        net.plan_step(eta, g, gamma, lo, hi, gold["alpha"])
        e = eta.double().cpu().numpy()
        step = np.asarray(gold["eta"][k + 1]) - np.asarray(gold["eta"][0])
        assert np.max(np.abs(e - gold["eta"][k + 1])) <= 1e-3 * max(np.max(np.abs(step)), 1e-3), k
    torch.cuda.synchronize()


def test_medium_slice_parity():
    """100-bus network, one scenario, 24 hours: dispatch, prices and the adjoint gradient.

    The gradient is held to the 1e-3 of the tolerance table on the whole vector and on every
    entry (relative to the largest).  The adjoint runs to a 3e-6 residual: at the table's
    parity setting of 1e-5 the FP32 message passing leaves entries at up to 7e-4 of the
    largest, too close to the bound to be a stable test; at 3e-6 they fall below 1e-4."""
    nets, scens = synth.medium(S=1)
    nets, scens = synth.slice_hours(nets, scens, 0, 24)
    eta = nets[0]["eta_min"]
    # tight solves use the smaller phase penalty (faster to 1e-6; the default is tuned for 1e-3)
    net, e, rc, refs = _solve_pair(nets, scens, eta, kappa=50.0, tol=1e-6, adj_tol=3e-6, rho_theta_c=0.01,
                                   adj_max_iter=400000)
    ref = refs[0]
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0, net.last_grad_stats
    g_ref = ograd.adjoint_grad(ref)
    err = np.abs(gg - g_ref) / np.max(np.abs(g_ref))
    assert np.all(err <= 1e-3), np.sort(err)[-8:]
    assert rel(gg, g_ref) <= 1e-3, (net.last_grad_stats, rel(gg, g_ref))


def test_batching_full_size_sampled_parity():
    """The full batching workload (64 scenarios, each on its own network of 50-500 buses, 24, 72
    or 168 hours) solved and differentiated in one batch, in the launch configuration bench.py
    times (whole-loop graphs, the bind-time bus-kernel schedule), then checked on the sampled
    scenarios the oracle can solve one by one (the two smallest): objective, FP64 KKT residuals
    of the GPU dispatch, and the per-scenario gradient dh_s/deta (GX_ARR_GRAD_S).

    Tolerances sit above this batch's FP32 floor: the 135-bus scenario's forward residual
    levels off near 1.2e-6 and its adjoint near 5e-6, so the forward runs to 3e-6 and the
    adjoint to 1e-5 (the parity setting of the other tests); scenarios that have not reached
    them within the caps stop there without affecting the sampled ones."""
    import torch
    from oracle.dispatch import net_slices
    nets, scens = synth.batching()
    eta = np.concatenate([n["eta_min"] for n in nets]) * 1.05
    kappa = 50.0
    net = gpu_net(nets, scens, kappa=kappa, tol=3e-6, adj_tol=1e-5, rho_theta_c=0.01, max_iter=100000,
                  adj_max_iter=100000, check_every=50)
    e = eta_tensor(eta)
    size = [int(nets[sc["net"]]["n_bus"]) * sc["T"] for sc in scens]
    sampled = [int(s) for s in np.argsort(size)[:2]]
    assert net.solve(e) in (0, 1)
    torch.cuda.synchronize()
    fwd_status = net.array("status").cpu().numpy().copy()
    net.grad(e)
    torch.cuda.synchronize()
    adj_status = net.array("status").cpu().numpy().copy()
    offs = net_slices(nets)
    opts = synth.default_opts(kappa=kappa)
    for s in sampled:
        assert fwd_status[s] == 0 and adj_status[s] == 0, (s, fwd_status[s], adj_status[s])
        k = scens[s]["net"]
        ref = dispatch.solve(nets[k], scens[s], eta[offs[k]:offs[k + 1]], opts)
        g = solution(net, s, ref_groups(ref.qp))
        assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4, (s, g["cost"], ref.cost)
        res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
        assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, (s, res)
        gs = net.array("grad_s", s).cpu().numpy()
        g_ref = ograd.adjoint_grad(ref)
        assert gs.shape == g_ref.shape, (gs.shape, g_ref.shape)
        assert rel(gs, g_ref) <= 1e-3, (s, rel(gs, g_ref))
        assert np.max(np.abs(gs - g_ref)) <= 1e-3 * np.max(np.abs(g_ref)), s


def test_medium_full_size_sampled_parity():
    """The headline workload (100 buses, 16 scenarios of 168 h) solved and differentiated in one
    batch in bench.py's launch configuration, checked on a sampled scenario over its whole week
    (the oracle's interior point takes about a minute on it): objective, FP64 KKT residuals of
    the GPU dispatch, per-scenario gradient.  Forward to 3e-6 and adjoint to 1e-5, above the
    FP32 floor of the week-long scenarios.

    The sampled scenario is the first.  Scenarios at a degenerate vertex have no unique
    derivative: scenario 5 at this plan has generator 0 at zero in 67 hours with multipliers
    down to 0.017 $/MWh, the oracle's one-sided derivatives along eta_0 (+-0.01 MW) are 133.4
    and 129.8, and the GPU's active-set rule returns another element (104.5; 109.6 with a ten
    times larger threshold), so the per-entry comparison does not apply there."""
    import torch
    nets, scens = synth.medium()
    eta = nets[0]["eta_min"] * 1.05
    kappa = 50.0
    net = gpu_net(nets, scens, kappa=kappa, tol=3e-6, adj_tol=1e-5, rho_theta_c=0.01, max_iter=200000,
                  adj_max_iter=200000, check_every=50)
    e = eta_tensor(eta)
    s = 0
    assert net.solve(e) in (0, 1)
    torch.cuda.synchronize()
    fwd_status = int(net.array("status").cpu().numpy()[s])
    net.grad(e)
    torch.cuda.synchronize()
    adj_status = int(net.array("status").cpu().numpy()[s])
    assert fwd_status == 0 and adj_status == 0, (fwd_status, adj_status)
    ref = dispatch.solve(nets[0], scens[s], eta, synth.default_opts(kappa=kappa))
    g = solution(net, s, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4, (g["cost"], ref.cost)
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    gs = net.array("grad_s", s).cpu().numpy()
    g_ref = ograd.adjoint_grad(ref)
    assert rel(gs, g_ref) <= 1e-3, rel(gs, g_ref)
    assert np.max(np.abs(gs - g_ref)) <= 1e-3 * np.max(np.abs(g_ref)), np.sort(np.abs(gs - g_ref))[-5:]
