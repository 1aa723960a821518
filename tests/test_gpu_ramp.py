"""Ramp-limited generators on the CUDA path (their prox solved per warp by the ramp kernel)
against the FP64 oracle: dispatch, prices, and the capacity gradient through both the
capacity and the ramp bounds."""
import numpy as np
import pytest

from cases import network, scenario
from gpu_util import eta_tensor, gpu_net, pack_x, ref_groups, rel, solution
from oracle import dispatch, grad as ograd, kkt
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-6, max_iter=200000, adj_tol=1e-5, adj_max_iter=200000, check_every=50)
ACT_TOL = 1e-3


def _check(nets, scens, eta, kappa, grad_tol=1e-3):
    net = gpu_net(nets, scens, kappa=kappa, **TIGHT)
    e = eta_tensor(eta)
    assert net.solve(e) == 0, net.last_stats
    ref = dispatch.solve(nets[0], scens[0], eta, synth.default_opts(kappa=kappa))
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    assert rel(g["price"], ref.price) <= 1e-3
    assert rel(g["p"], ref.p) <= 1e-3
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0, net.last_grad_stats
    g_ref = ograd.adjoint_grad(ref)
    assert rel(gg, g_ref) <= grad_tol, (rel(gg, g_ref), gg, g_ref)
    return g, ref


def test_ramp_closed_form_on_gpu():
    """The oracle's two-hour closed form: the cheap unit ramps 100 -> 200 MW, the hour-0
    price is negative, and dc/deta of the ramping unit is -0.2 mu."""
    net, eta = network(1, gens=[(0, 10.0, 500.0), (0, 60.0, 500.0)], ramp={0: 0.2})
    sc = scenario([[100.0, 300.0]], G=2)
    g, ref = _check([net], [sc], eta, 0.0)
    np.testing.assert_allclose(g["p"][0], [100.0, 200.0], atol=0.05)
    assert g["price"][0, 0] < 0


@pytest.mark.parametrize("kappa", [0.0, 50.0])
def test_ramp_three_bus_parity(kappa):
    net, eta = network(3, gens=[(0, 12.0, 300.0, 0.5), (1, 25.0, 250.0, 0.4), (2, 70.0, 400.0, 0.3)],
                       lines=[(0, 1, 800.0, 400.0), (1, 2, 600.0, 400.0), (0, 2, 500.0, 400.0)],
                       ramp={0: 0.25, 1: 0.3})
    load = np.array([[30, 60, 120, 150, 90, 40], [40, 70, 110, 160, 80, 50], [20, 50, 90, 120, 70, 30]], float)
    g, ref = _check([net], [scenario(load, G=3)], eta, kappa)
    dp = np.abs(np.diff(g["p"][:2], axis=1))
    assert np.any(np.abs(dp[0] - 0.25 * eta[0]) < 0.05)  # the limits bind on the GPU too


def test_ramp_medium_slice_parity():
    """100-bus network, one scenario of 24 hours, gas units limited to 10-30 % of their
    capacity per hour; the phase penalty of the tight medium-slice solves."""
    nets, scens = synth.medium(S=1)
    nets, scens = synth.slice_hours(nets, scens, 0, 24)
    nets = [synth.add_ramps(nets[0], rate=(0.1, 0.3), seed=7)]
    eta = nets[0]["eta_min"]
    net = gpu_net(nets, scens, kappa=50.0, **{**TIGHT, "rho_theta_c": 0.01})
    e = eta_tensor(eta)
    assert net.solve(e) == 0, net.last_stats
    ref = dispatch.solve(nets[0], scens[0], eta, synth.default_opts(kappa=50.0))
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    ramping = np.where((nets[0]["gen_ramp"] > 0) & (nets[0]["gen_ramp"] < 1))[0]
    R = nets[0]["gen_ramp"][ramping] * eta[ramping]
    assert np.all(np.abs(np.diff(g["p"][ramping], axis=1)) <= R[:, None] * (1 + 1e-4) + 1e-2)
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0
    g_ref = ograd.adjoint_grad(ref)
    # the medium slice's criterion (a few entries sit at nearly degenerate active sets)
    err = np.abs(gg - g_ref) / np.max(np.abs(g_ref))
    assert np.mean(err <= 1e-3) >= 0.98, np.sort(err)[-8:]
    assert rel(gg, g_ref) <= 2e-3, rel(gg, g_ref)
