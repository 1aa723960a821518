"""Capacity-dependent line susceptance (beta = beta0 eta / ref, the A(eta) of Eq. 2) on the
CUDA path against the FP64 oracle: dispatch, prices, and the capacity gradient with its
constraint-matrix term, by the adjoint and by the envelope theorem, on the per-iteration
kernels and the cluster-resident path, and after the plan moves between calls."""
import numpy as np
import pytest

from cases import network, scenario
from gpu_util import eta_tensor, gpu_net, pack_x, ref_groups, rel, solution
from oracle import dispatch, grad as ograd, kkt
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-6, max_iter=200000, adj_tol=1e-5, adj_max_iter=200000, check_every=50)
ACT_TOL = 1e-3


def _triangle():
    """Meshed triangle whose line 0-2 scales; line 1-2 is congested, 0-2 below its limit."""
    net, eta = network(3, gens=[(0, 10.0, 600.0, 0.5), (1, 30.0, 300.0, 0.3), (2, 80.0, 300.0, 0.6)],
                       lines=[(0, 1, 1000.0, 500.0), (1, 2, 800.0, 70.0), (0, 2, 500.0, 400.0)])
    load = np.array([[20, 40, 30], [30, 50, 40], [200, 260, 230]], float)
    net["line_beta_ref"] = np.array([0.0, 0.0, eta[5]])
    return net, eta * 1.02, scenario(load, G=3)


def _dispatch_checks(net, nets, scens, eta, kappa):
    ref = dispatch.solve(nets[0], scens[0], eta, synth.default_opts(kappa=kappa))
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    assert rel(g["price"], ref.price) <= 1e-3
    assert rel(g["flow"], ref.flow) <= 1e-3
    return g, ref


@pytest.mark.parametrize("kappa", [0.0, 50.0])
@pytest.mark.parametrize("persistent", [False, True])
def test_scaling_triangle_parity(kappa, persistent):
    net0, eta, sc = _triangle()
    net = gpu_net([net0], [sc], kappa=kappa, **TIGHT)
    net.use_persistent(persistent)
    e = eta_tensor(eta)
    assert net.solve(e) == 0, net.last_stats
    g, ref = _dispatch_checks(net, [net0], [sc], eta, kappa)
    assert np.all(np.abs(g["flow"][2]) < eta[5] - 1.0)  # the scaling line is below its limit
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0, net.last_grad_stats
    g_ref = ograd.adjoint_grad(ref)
    assert rel(gg, g_ref) <= 1e-3, (gg, g_ref)
    # the scaling line's own entry: the A(eta) term alone (its flow limit is slack)
    assert abs(gg[5] - g_ref[5]) <= 2e-3 * np.max(np.abs(g_ref)), (gg[5], g_ref[5])
    assert gg[5] < -1.0


def test_scaling_triangle_envelope():
    """kappa = 0 with the envelope route: -D^T z plus y^T dA x from the forward prices."""
    net0, eta, sc = _triangle()
    net = gpu_net([net0], [sc], kappa=0.0, grad_envelope=1, **TIGHT)
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    _, ref = _dispatch_checks(net, [net0], [sc], eta, 0.0)
    gg = net.grad(e).double().cpu().numpy()
    g_env = ograd.envelope_grad(ref)
    assert rel(gg, g_env) <= 1e-3, (gg, g_env)
    assert abs(gg[5] - g_env[5]) <= 2e-3 * np.max(np.abs(g_env))


def test_scaling_radial_line_at_limit():
    """A radial line at its flow limit: the gradient equals that of the fixed-susceptance
    line (the limit row's two eta-derivatives cancel), here on the GPU."""
    net0, eta = network(2, gens=[(0, 10.0, 1000.0), (1, 60.0, 1000.0)], lines=[(0, 1, 1000.0, 150.0)])
    sc = scenario([[20.0, 30.0], [300.0, 260.0]], G=2)
    fixed = gpu_net([net0], [sc], **TIGHT)
    e = eta_tensor(eta)
    assert fixed.solve(e) == 0
    g_fixed = fixed.grad(e).double().cpu().numpy()
    net0["line_beta_ref"] = np.array([0.5 * eta[2]])
    net = gpu_net([net0], [sc], **TIGHT)
    assert net.solve(e) == 0
    g, ref = _dispatch_checks(net, [net0], [sc], eta, 0.0)
    np.testing.assert_allclose(g["flow"][0], [eta[2], eta[2]], rtol=1e-4)
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0
    assert rel(gg, ograd.adjoint_grad(ref)) <= 1e-3
    assert rel(gg, g_fixed) <= 1e-3


def test_scaling_follows_the_plan_between_calls():
    """The effective susceptances are rewritten per call: after the plan changes, a warm
    solve and gradient match the oracle at the new plan, and a network bound with the new
    susceptances fixed gives the same dispatch."""
    net0, eta, sc = _triangle()
    net = gpu_net([net0], [sc], kappa=50.0, **TIGHT)
    assert net.solve(eta_tensor(eta)) == 0
    eta2 = eta.copy()
    eta2[5] *= 1.6
    e2 = eta_tensor(eta2)
    assert net.solve(e2, warm="prev") == 0
    g, ref = _dispatch_checks(net, [net0], [sc], eta2, 50.0)
    gg = net.grad(e2, warm="prev").double().cpu().numpy()
    assert net.last_grad_status == 0
    assert rel(gg, ograd.adjoint_grad(ref)) <= 1e-3
    fixed0 = dict(net0)
    fixed0["line_beta"] = net0["line_beta"].copy()
    fixed0["line_beta"][2] = net0["line_beta"][2] * np.float32(eta2[5]) / net0["line_beta_ref"][2]
    fixed0["line_dtheta"] = net0["line_dtheta"].copy()
    del fixed0["line_beta_ref"]
    fx = gpu_net([fixed0], [sc], kappa=50.0, **TIGHT)
    assert fx.solve(e2) == 0
    gf = solution(fx, 0, ref_groups(ref.qp))
    assert rel(g["flow"], gf["flow"]) <= 1e-3 and rel(g["price"], gf["price"]) <= 1e-3


def test_scaling_medium_slice_parity():
    """100-bus network, one scenario of 24 hours, 30 % of its AC lines scaling with
    capacity, at a plan 20 % above the existing capacities."""
    nets, scens = synth.medium(S=1)
    nets, scens = synth.slice_hours(nets, scens, 0, 24)
    nets = [synth.add_scaling(nets[0], share=0.3, seed=5)]
    eta = nets[0]["eta_min"] * 1.2
    # FP32 iterates on this plan settle at a primal residual of about 1.1e-6 (the same with
    # every susceptance fixed), so the forward tolerance is 3e-6
    net = gpu_net(nets, scens, kappa=50.0, **{**TIGHT, "tol": 3e-6, "rho_theta_c": 0.01})
    e = eta_tensor(eta)
    assert net.solve(e) == 0, net.last_stats
    ref = dispatch.solve(nets[0], scens[0], eta, synth.default_opts(kappa=50.0))
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0
    g_ref = ograd.adjoint_grad(ref)
    err = np.abs(gg - g_ref) / np.max(np.abs(g_ref))
    assert np.mean(err <= 1e-3) >= 0.98, np.sort(err)[-8:]
    assert rel(gg, g_ref) <= 2e-3, rel(gg, g_ref)
    G = nets[0]["gen_bus"].size
    sc_lines = G + np.where(nets[0]["line_beta_ref"] > 0)[0]
    assert np.max(np.abs(gg[sc_lines] - g_ref[sc_lines])) <= 2e-3 * np.max(np.abs(g_ref))


def test_scaling_full_horizon_properties():
    """Four scenarios of 168 h on the 100-bus network with 30 % of the AC lines scaling, at
    the bench's 1e-3 tolerance: every scenario converges, reported flows respect |f| <=
    eta and balance every bus-hour within the residual tolerance, the scaling lines'
    flows follow the effective susceptance (closer to beta_eff dtheta than to beta0
    dtheta), and the gradient agrees with a GPU central difference of sum_s w_s h_s
    along a random direction (solves at 1e-6), the A(eta) entries included."""
    import torch
    nets, scens = synth.medium(S=4)
    nets = [synth.add_scaling(nets[0], share=0.3, seed=11)]
    n = nets[0]
    G, L = n["gen_bus"].size, n["line_from"].size
    eta = n["eta_min"] * 1.3
    net = gpu_net(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    e = eta_tensor(eta)
    assert net.solve(e) == 0 and net.last_stats["n_converged"] == 4
    ref = n["line_beta_ref"]
    sc_l = ref > 0
    beta_eff = np.where(sc_l, n["line_beta"] * eta[G:G + L] / np.where(sc_l, ref, 1.0), n["line_beta"])
    for s in (0, 3):
        sc = scens[s]
        f = net.array("flow", s).double().cpu().numpy()
        assert np.all(np.abs(f) <= eta[G:G + L][:, None] * (1 + 1e-5) + 1e-3)
        p = net.array("p", s).double().cpu().numpy()
        sh = net.array("shed", s).double().cpu().numpy()
        ch = net.array("ch", s).double().cpu().numpy()
        dis = net.array("dis", s).double().cpu().numpy()
        inj = np.zeros_like(sc["load"])
        np.add.at(inj, n["gen_bus"], p)
        np.add.at(inj, n["bat_bus"], dis - ch)
        inj += sh - sc["load"]
        np.add.at(inj, n["line_from"], -f)
        np.add.at(inj, n["line_to"], f)
        assert np.linalg.norm(inj) <= 5e-3 * np.linalg.norm(sc["load"])
        th = net.array("theta", s).double().cpu().numpy()
        dth = (th[n["line_from"]] - th[n["line_to"]])[sc_l]
        err_eff = np.linalg.norm(f[sc_l] - beta_eff[sc_l, None] * dth)
        err_0 = np.linalg.norm(f[sc_l] - n["line_beta"][sc_l, None] * dth)
        assert err_eff < 0.5 * err_0, (err_eff, err_0)
    g = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0
    tight = gpu_net(nets, scens, kappa=50.0, tol=1e-6, max_iter=200000, check_every=100)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(eta.size) * eta * 1e-3
    vals = []
    for sgn in (+1, -1):
        assert tight.solve(eta_tensor(eta + sgn * d)) in (0, 1)
        torch.cuda.synchronize()
        vals.append(float(np.sum(tight.array("h").cpu().numpy() * np.array([sc["weight"] for sc in scens]))))
    fd = (vals[0] - vals[1]) / 2.0
    lin = float(np.dot(g, d))
    assert abs(fd - lin) <= 2e-2 * abs(fd), (fd, lin)
