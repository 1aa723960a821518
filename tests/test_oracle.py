"""Pins of the FP64 oracle against closed forms, brute force, a library LP solver and
invariants (no GPU).  Each test names the part of the oracle that a plausible slip
(dropped term, wrong sign, wrong index) would break."""
import math

import numpy as np
import pytest

from cases import network, scenario
from oracle import closed, dispatch, grad, kkt, plan
from oracle.qp import DispatchQP
from paper_2410_13055_gb300 import synth

EPS = 1e-3
VOLL = 1000.0


def opts(**kw):
    o = dict(eps=EPS, voll=VOLL, kappa=0.0)
    o.update(kw)
    return o


# ---------------------------------------------------------------- single bus
@pytest.mark.parametrize("shortage", [False, True])
def test_single_bus_waterfill(shortage):
    """Generator cost, eps term, shed variable and price sign: water-filling closed form."""
    rng = np.random.default_rng(5)
    costs = rng.uniform(10, 90, 5)
    caps = rng.uniform(50, 200, 5)
    T = 3
    tot = caps.sum()
    load = np.array([0.3 * tot, 0.7 * tot, (1.3 if shortage else 0.95) * tot])
    net, eta = network(1, gens=[(0, c, u) for c, u in zip(costs, caps)])
    sol = dispatch.solve(net, scenario(load[None, :], G=5), eta, opts())
    assert sol.converged
    for t in range(T):
        p, sh, lam = closed.waterfill(costs, caps, load[t], EPS, VOLL)
        np.testing.assert_allclose(sol.p[:, t], p, atol=1e-6)
        assert abs(sol.sh[0, t] - sh) < 1e-6
        assert abs(sol.price[0, t] - lam) < 1e-6 * max(1, lam)
    if shortage:
        assert sol.sh[0, 2] > 1.0
        assert abs(sol.price[0, 2] - (VOLL + EPS * sol.sh[0, 2])) < 1e-6


def test_merit_order_limit():
    """eps -> 0: price equals the marginal generator's cost, cheapest units fill first."""
    costs = np.array([30.0, 10.0, 50.0, 20.0])
    caps = np.array([100.0, 80.0, 100.0, 60.0])
    load = 200.0
    net, eta = network(1, gens=[(0, c, u) for c, u in zip(costs, caps)])
    sol = dispatch.solve(net, scenario([[load]], G=4), eta, opts(eps=1e-7))
    p_mo, lam = closed.merit_order(costs, caps, load)
    np.testing.assert_allclose(sol.p[:, 0], p_mo, atol=1e-3)
    assert lam == 30.0
    assert abs(sol.price[0, 0] - lam) < 1e-3


def test_single_bus_envelope_gradient_closed_form():
    """Capacity derivative of a generator at its cap: -(lambda - c - eps p) per hour."""
    costs = np.array([10.0, 40.0])
    caps = np.array([100.0, 300.0])
    load = np.array([[150.0, 250.0]])
    net, eta = network(1, gens=[(0, c, u) for c, u in zip(costs, caps)])
    sol = dispatch.solve(net, scenario(load, G=2), eta, opts())
    lam = sol.price[0]
    expect0 = -np.sum(lam - costs[0] - EPS * sol.p[0])
    g_env = grad.envelope_grad(sol)
    g_adj = grad.adjoint_grad(sol)
    assert abs(g_env[0] - expect0) < 1e-6 * abs(expect0)
    assert abs(g_adj[0] - expect0) < 1e-6 * abs(expect0)
    assert abs(g_adj[1]) < 1e-6  # the dear unit is never at its cap


def test_zero_capacity_hours_gradient():
    """A generator with capacity factor 0 in some hours (0 <= p <= 0): the adjoint's
    active set must stay independent; FD, envelope and adjoint agree."""
    costs = np.array([0.0, 30.0, 60.0])
    caps = np.array([120.0, 150.0, 400.0])
    cf = np.array([[0.0, 0.5, 1.0, 0.0], [1.0, 1.0, 1.0, 1.0], [1.0, 1.0, 1.0, 1.0]])
    load = np.array([[100.0, 180.0, 300.0, 220.0]])
    net, eta = network(1, gens=[(0, c, u, e) for c, u, e in zip(costs, caps, [0.0, 0.4, 0.6])])
    for kappa in (0.0, 50.0):
        o = opts(kappa=kappa)
        sol = dispatch.solve(net, scenario(load, cf=cf), eta, o)
        g_adj = grad.adjoint_grad(sol)
        g_fd, _ = grad.fd_grad(net, scenario(load, cf=cf), eta, o)
        assert np.max(np.abs(g_adj - g_fd)) < 1e-5 * max(1.0, np.max(np.abs(g_fd)))
        if kappa == 0.0:
            assert np.max(np.abs(grad.envelope_grad(sol) - g_fd)) < 1e-5 * max(1.0, np.max(np.abs(g_fd)))


# ---------------------------------------------------------------- lines
def test_two_bus_congestion():
    """Line flow direction, beta, flow limit and the line-capacity gradient."""
    c0, c1, L0, L1, cap = 10.0, 60.0, 20.0, [200.0, 240.0, 150.0], 120.0
    net, eta = network(2, gens=[(0, c0, 1000.0), (1, c1, 1000.0)], lines=[(0, 1, 2000.0, cap)])
    sc = scenario([[L0] * 3, L1], G=2)
    sol = dispatch.solve(net, sc, eta, opts())
    g_expect = 0.0
    for t in range(3):
        p0, p1, lam0, lam1, dg = closed.two_bus_congested(c0, c1, L0, L1[t], cap, EPS)
        assert abs(sol.p[0, t] - p0) < 1e-6 and abs(sol.p[1, t] - p1) < 1e-6
        assert abs(sol.flow[0, t] - cap) < 1e-6
        assert abs(sol.price[0, t] - lam0) < 1e-6 and abs(sol.price[1, t] - lam1) < 1e-6
        g_expect += dg
    for g in (grad.envelope_grad(sol), grad.adjoint_grad(sol)):
        assert abs(g[2] - g_expect) < 1e-6 * abs(g_expect)


def test_angle_limit_binds():
    """Angle-difference limit: flow = beta * dtheta_max when that is below the flow limit."""
    beta, dth = 300.0, 0.2  # beta * dth = 60 MW < 200 MW flow limit
    net, eta = network(2, gens=[(0, 10.0, 1000.0), (1, 60.0, 1000.0)], lines=[(0, 1, beta, 200.0, dth)])
    sol = dispatch.solve(net, scenario([[5.0], [150.0]], G=2), eta, opts())
    assert abs(sol.flow[0, 0] - beta * dth) < 1e-6
    assert abs((sol.th[0, 0] - sol.th[1, 0]) - dth) < 1e-9
    assert abs(sol.th[0, 0]) < 1e-12  # bus 0 is the reference
    # the flow limit is slack, so its capacity derivative vanishes
    assert abs(grad.adjoint_grad(sol)[2]) < 1e-6


def test_kvl_loop_flows():
    """Meshed triangle: flows split by susceptance (Kirchhoff's voltage law)."""
    net, eta = network(3, gens=[(0, 10.0, 1000.0)],
                       lines=[(0, 1, 1000.0, 1e4), (1, 2, 1000.0, 1e4), (0, 2, 500.0, 1e4)])
    sol = dispatch.solve(net, scenario([[1.0], [1.0], [300.0]], G=1), eta, opts())
    f = sol.flow[:, 0]
    # loop 0-1-2-0: angle drops sum to zero, f01/1000 + f12/1000 = f02/500;
    # with bus 1 drawing 1 MW: f01 = f12 + 1, f12 + f02 = 300  =>  f12 = 149.75, f02 = 150.25
    np.testing.assert_allclose(f, [150.75, 149.75, 150.25], atol=1e-6)
    assert abs(f[0] / 1000.0 + f[1] / 1000.0 - f[2] / 500.0) < 1e-9


# ---------------------------------------------------------------- HVDC transport links
@pytest.mark.parametrize("F", [120.0, 1e4])
def test_hvdc_link_closed_form(F):
    """A transport link between a cheap and an expensive bus.  The KKT conditions of the
    link's flow (eps f = lambda_to - lambda_from - mu) give the closed form: congested,
    f = F, lambda_0 = c0 + eps F, lambda_1 = c1 + eps (L1 - F), d cost / dF = -mu;
    uncongested, the cheap bus serves the whole load and the link's flow sets the price
    difference, lambda_1 - lambda_0 = eps f."""
    c0, c1, L1 = 10.0, 50.0, 200.0
    net, eta = network(2, gens=[(0, c0, 1000.0), (1, c1, 1000.0)], lines=[(0, 1, 1.0, F)], dc=(0,))
    sol = dispatch.solve(net, scenario([[0.0], [L1]], G=2), eta, opts())
    if F < L1:
        lam0, lam1 = c0 + EPS * F, c1 + EPS * (L1 - F)
        assert abs(sol.flow[0, 0] - F) < 1e-6
        mu = lam1 - lam0 - EPS * F
        for g in (grad.envelope_grad(sol), grad.adjoint_grad(sol)):
            assert abs(g[2] + mu) < 1e-6 * mu
    else:
        lam0, lam1 = c0 + EPS * L1, c0 + 2 * EPS * L1
        assert abs(sol.flow[0, 0] - L1) < 1e-6 and abs(sol.p[1, 0]) < 1e-6
        assert abs(grad.adjoint_grad(sol)[2]) < 1e-9
    assert abs(sol.price[0, 0] - lam0) < 1e-6 and abs(sol.price[1, 0] - lam1) < 1e-6


@pytest.mark.parametrize("kappa", [0.0, 50.0])
def test_hvdc_joins_ac_islands(kappa):
    """Two AC islands joined only by an HVDC link: one reference angle per island, the
    link's flow decoupled from the angles, its capacity gradient equal to minus the sum
    of the hourly price gaps net of the eps term, and the adjoint equal to the central
    finite difference."""
    net, eta = network(4, gens=[(0, 20.0, 300.0, 0.4), (1, 35.0, 300.0, 0.3), (2, 60.0, 300.0, 0.5),
                                (3, 80.0, 300.0, 0.6)],
                       lines=[(0, 1, 1000.0, 250.0), (2, 3, 800.0, 250.0), (1, 2, 1.0, 90.0)], dc=(2,))
    sc = scenario([[20, 30], [40, 60], [120, 150], [90, 100]], G=4)
    o = opts(kappa=kappa)
    sol = dispatch.solve(net, sc, eta, o)
    assert list(sol.qp.ref_bus) == [0, 2]
    res = kkt.residuals(sol.qp, sol.x, sol.price)
    assert res["primal"] < 1e-9 and res["dual"] < 1e-9
    np.testing.assert_allclose(sol.flow[2], [90.0, 90.0], atol=1e-6)
    g = grad.adjoint_grad(sol)
    gf, ok = grad.fd_grad(net, sc, eta, o)
    assert ok.all()
    np.testing.assert_allclose(g, gf, atol=1e-6 * np.max(np.abs(gf)))
    if kappa == 0.0:
        mu = sol.price[2] - sol.price[1] - EPS * sol.flow[2]
        assert abs(g[6] + mu.sum()) < 1e-6 * mu.sum()


# ---------------------------------------------------------------- capacity-dependent susceptance
def _scaling_triangle():
    net, eta = network(3, gens=[(0, 10.0, 600.0, 0.5), (1, 30.0, 300.0, 0.3), (2, 80.0, 300.0, 0.6)],
                       lines=[(0, 1, 1000.0, 500.0), (1, 2, 800.0, 70.0), (0, 2, 500.0, 400.0)])
    load = np.array([[20, 40, 30], [30, 50, 40], [200, 260, 230]], float)
    return net, eta * 1.02, scenario(load, G=3)


@pytest.mark.parametrize("kappa", [0.0, 50.0])
def test_scaling_susceptance_gradient_routes(kappa):
    """A meshed triangle whose line 0-2 gains susceptance with capacity (beta eta / ref):
    below its own limit, more capacity still pays by drawing loop flow off the congested
    line 1-2 (the A(eta) term of Eq. 2).  Adjoint, envelope (kappa = 0) and central finite
    differences agree; with the susceptance fixed the same line's gradient is zero."""
    net, eta, sc = _scaling_triangle()
    o = opts(kappa=kappa)
    fixed = dispatch.solve(net, sc, eta, o)
    assert abs(grad.adjoint_grad(fixed)[5]) < 1e-9
    net["line_beta_ref"] = np.array([0.0, 0.0, eta[5]])
    sol = dispatch.solve(net, sc, eta, o)
    assert np.all(np.abs(sol.flow[2]) < eta[5] - 1.0)            # the scaling line is not at its limit
    g = grad.adjoint_grad(sol)
    gf, ok = grad.fd_grad(net, sc, eta, o)
    assert ok.all()
    np.testing.assert_allclose(g, gf, atol=1e-6 * np.max(np.abs(gf)))
    assert g[5] < -1.0
    if kappa == 0.0:
        np.testing.assert_allclose(grad.envelope_grad(sol), gf, atol=1e-6 * np.max(np.abs(gf)))


def test_scaling_susceptance_radial_line_at_limit():
    """A radial line at its flow limit: scaling its susceptance with capacity leaves the
    capacity gradient unchanged (the flow is fixed by balance and its MW limit is eta
    either way), which pins the cancellation between the limit row's eta-derivatives."""
    net, eta = network(2, gens=[(0, 10.0, 1000.0), (1, 60.0, 1000.0)], lines=[(0, 1, 1000.0, 150.0)])
    sc = scenario([[20.0, 30.0], [300.0, 260.0]], G=2)
    g_fixed = grad.adjoint_grad(dispatch.solve(net, sc, eta, opts()))
    assert g_fixed[2] < -1.0  # the flow limit binds (beta dtheta_max = 524 MW > 150 MW)
    net["line_beta_ref"] = np.array([0.5 * eta[2]])
    sol = dispatch.solve(net, sc, eta, opts())
    np.testing.assert_allclose(sol.flow[0], [eta[2], eta[2]], atol=1e-6)
    for g in (grad.adjoint_grad(sol), grad.envelope_grad(sol)):
        np.testing.assert_allclose(g, g_fixed, atol=1e-6 * np.max(np.abs(g_fixed)))


# ---------------------------------------------------------------- ramping generators
def test_ramp_limit_closed_form():
    """A cheap generator limited to ramping 0.2 of its 500 MW per hour while the load
    jumps from 100 to 300 MW: it serves 100 then 200 MW and the expensive unit covers the
    rest.  The KKT conditions give lambda_1 = 60 + eps 100, the ramp multiplier
    mu = lambda_1 - 10 - eps 200 and lambda_0 = 10 + eps 100 - mu (negative: load in the
    first hour would buy ramp headroom); dc/deta_A = -0.2 mu through R = 0.2 eta_A."""
    net, eta = network(1, gens=[(0, 10.0, 500.0), (0, 60.0, 500.0)], ramp={0: 0.2})
    sol = dispatch.solve(net, scenario([[100.0, 300.0]], G=2), eta, opts())
    np.testing.assert_allclose(sol.p[0], [100.0, 200.0], atol=1e-6)
    np.testing.assert_allclose(sol.p[1], [0.0, 100.0], atol=1e-6)
    lam1 = 60.0 + EPS * 100.0
    mu = lam1 - 10.0 - EPS * 200.0
    np.testing.assert_allclose(sol.price[0], [10.0 + EPS * 100.0 - mu, lam1], atol=1e-6)
    for g in (grad.envelope_grad(sol), grad.adjoint_grad(sol)):
        assert abs(g[0] + 0.2 * mu) < 1e-6 * mu and abs(g[1]) < 1e-6


@pytest.mark.parametrize("kappa", [0.0, 50.0])
def test_ramp_limits_gradient_routes(kappa):
    """Three buses, six hours, two ramping generators whose limits bind on the load's
    rise and fall: the adjoint gradient equals the central finite difference."""
    net, eta = network(3, gens=[(0, 12.0, 300.0, 0.5), (1, 25.0, 250.0, 0.4), (2, 70.0, 400.0, 0.3)],
                       lines=[(0, 1, 800.0, 400.0), (1, 2, 600.0, 400.0), (0, 2, 500.0, 400.0)],
                       ramp={0: 0.25, 1: 0.3})
    load = np.array([[30, 60, 120, 150, 90, 40], [40, 70, 110, 160, 80, 50], [20, 50, 90, 120, 70, 30]], float)
    sc = scenario(load, G=3)
    o = opts(kappa=kappa)
    sol = dispatch.solve(net, sc, eta, o)
    dp = np.abs(np.diff(sol.p[:2], axis=1))
    assert np.any(np.isclose(dp[0], 0.25 * eta[0], atol=1e-6)) and np.any(np.isclose(dp[1], 0.3 * eta[1], atol=1e-6))
    g = grad.adjoint_grad(sol)
    gf, ok = grad.fd_grad(net, sc, eta, o)
    assert ok.all()
    np.testing.assert_allclose(g, gf, atol=1e-6 * np.max(np.abs(gf)))


# ---------------------------------------------------------------- batteries
@pytest.mark.parametrize("case", ["power", "spare", "energy"])
def test_battery_arbitrage(case):
    """Dynamics sign, efficiencies, injection dis - ch and the soc bound coefficient."""
    P, dur = {"power": (30.0, 4.0), "spare": (200.0, 4.0), "energy": (60.0, 0.5)}[case]
    eff = math.sqrt(0.9)
    net, eta = network(1, gens=[(0, 10.0, 200.0), (0, 50.0, 200.0)], bats=[(0, P, dur, eff)])
    cf = np.array([[1.0, 0.0], [1.0, 1.0]])
    sol = dispatch.solve(net, scenario([[100.0, 100.0]], cf=cf), eta, opts())
    ch0, dis1, soc0 = closed.battery_arbitrage(P, dur, eff, eff, spare_cheap=100.0)
    assert abs(sol.ch[0, 0] - ch0) < 1e-6
    assert abs(sol.dis[0, 1] - dis1) < 1e-6
    assert abs(sol.soc[0, 0] - soc0) < 1e-6
    assert abs(sol.soc[0, 1]) < 1e-6
    assert sol.ch[0, 1] < 1e-6 and sol.dis[0, 0] < 1e-6
    if case == "power":
        # cost(P) = 10(100+P) + e/2(100+P)^2 + 50(100-0.9P) + e/2(100-0.9P)^2 + e/2(P^2 + 0.81 P^2)
        dC = 10 + EPS * (100 + P) - 0.9 * 50 - 0.9 * EPS * (100 - 0.9 * P) + EPS * 1.81 * P
        g = grad.adjoint_grad(sol)
        assert abs(g[2] - dC) < 1e-6 * abs(dC)
        assert abs(grad.envelope_grad(sol)[2] - dC) < 1e-6 * abs(dC)


# ---------------------------------------------------------------- brute force LP
SMALL_LPS = {
    "2bus": (2, [(0, 12.0, 80.0), (1, 45.0, 150.0)], [(0, 1, 800.0, 60.0)], [], [[30.0], [90.0]]),
    "3bus": (3, [(0, 12.0, 120.0), (1, 30.0, 60.0), (2, 70.0, 100.0)],
             [(0, 1, 800.0, 50.0), (1, 2, 600.0, 200.0), (0, 2, 400.0, 70.0)], [], [[20.0], [40.0], [110.0]]),
    "bat": (1, [(0, 15.0, 120.0)], [], [(0, 40.0, 2.0)], [[60.0, 130.0]]),
}


@pytest.mark.parametrize("name", list(SMALL_LPS))
def test_vertex_enumeration(name):
    """eps = 0: IPM optimum equals the cheapest vertex; eps > 0 lies in the bracket."""
    nb, gens, lines, bats, load = SMALL_LPS[name]
    net, eta = network(nb, gens=gens, lines=lines, bats=bats)
    sc = scenario(load, G=len(gens))
    if name == "bat":
        sc["cf"] = np.array([[1.0, 0.4]])
    qp = DispatchQP(net, sc, eta, opts(eps=0.0))
    A = qp.A.toarray()
    G = qp.Gm.toarray()
    best, xbest = closed.lp_vertex_enumeration(qp.q, A, qp.b, G, qp.h)
    lp = dispatch.solve(net, sc, eta, opts(eps=0.0))
    assert abs(lp.cost - best) < 1e-7 * max(1.0, abs(best))
    reg = dispatch.solve(net, sc, eta, opts())
    qd = DispatchQP(net, sc, eta, opts()).Qd
    upper = best + 0.5 * float(np.sum(qd * xbest ** 2))
    assert best - 1e-7 <= reg.cost <= upper + 1e-7


def test_highs_bound_medium_slice():
    """Library LP (HiGHS) on a 100-bus slice: eps = 0 optimum and the eps > 0 bracket."""
    from scipy.optimize import linprog
    nets, scens = synth.medium()
    nets, sl = synth.slice_hours(nets, scens[:1], 10, 3)
    eta = nets[0]["eta_min"]
    qp = DispatchQP(nets[0], sl[0], eta, opts(eps=0.0))
    res = linprog(qp.q, A_ub=qp.Gm, b_ub=qp.h, A_eq=qp.A, b_eq=qp.b, bounds=(None, None), method="highs")
    assert res.status == 0
    lp = dispatch.solve(nets[0], sl[0], eta, opts(eps=0.0))
    assert abs(lp.cost - res.fun) < 1e-7 * abs(res.fun)
    reg = dispatch.solve(nets[0], sl[0], eta, opts())
    qd = DispatchQP(nets[0], sl[0], eta, opts()).Qd
    upper = res.fun + 0.5 * float(np.sum(qd * res.x ** 2))
    assert res.fun - 1e-6 <= reg.cost <= upper + 1e-6


# ---------------------------------------------------------------- gradients
@pytest.mark.parametrize("kappa", [0.0, 50.0])
def test_gradient_routes_tiny(kappa):
    """FD vs implicit-function adjoint (and the envelope theorem for h = c)."""
    nets, scens = synth.tiny()
    eta = nets[0]["eta_min"] * 1.1
    o = opts(kappa=kappa)
    sol = dispatch.solve(nets[0], scens[0], eta, o)
    g_adj = grad.adjoint_grad(sol)
    g_fd, _ = grad.fd_grad(nets[0], scens[0], eta, o)
    scale = np.max(np.abs(g_fd))
    assert np.max(np.abs(g_adj - g_fd)) < 1e-5 * scale
    if kappa == 0.0:
        g_env = grad.envelope_grad(sol)
        assert np.max(np.abs(g_env - g_fd)) < 1e-5 * scale
        assert np.all(g_adj <= 1e-6 * scale)  # more capacity never raises cost
    else:
        # with an emissions weight the gradient is not the cost envelope
        g_env = grad.envelope_grad(sol)
        assert np.max(np.abs(g_env - g_adj)) > 1e-3 * scale


def test_cost_scaling_invariant():
    """Scaling every cost (and eps) by a scales the prices by a and keeps the dispatch."""
    nets, scens = synth.tiny()
    eta = nets[0]["eta_min"]
    a = 3.0
    s1 = dispatch.solve(nets[0], scens[0], eta, opts())
    net2 = dict(nets[0]); net2["gen_cost"] = nets[0]["gen_cost"] * a
    s2 = dispatch.solve(net2, scens[0], eta, opts(eps=EPS * a, voll=VOLL * a))
    np.testing.assert_allclose(s2.p, s1.p, atol=1e-5)
    np.testing.assert_allclose(s2.price, a * s1.price, rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------- KKT checker
def test_kkt_checker_detects_planted_mistakes():
    nets, scens = synth.tiny()
    sol = dispatch.solve(nets[0], scens[0], nets[0]["eta_min"], opts())
    good = kkt.residuals(sol.qp, sol.x, sol.price)
    assert good["primal"] < 1e-9 and good["dual"] < 1e-4
    x = sol.x.copy()
    x[sol.qp.vid("p", 2, 5)] += 1.0  # one generator off by 1 MW
    assert kkt.residuals(sol.qp, x, sol.price)["primal"] > 1e-4
    bad_price = sol.price.copy(); bad_price[1, 3] += 5.0
    assert kkt.residuals(sol.qp, sol.x, bad_price)["dual"] > 1e-3
    assert kkt.residuals(sol.qp, sol.x, -sol.price)["dual"] > 1e-2


# ---------------------------------------------------------------- plan step
def test_plan_step_projection():
    eta = np.array([1.0, 5.0, 9.0])
    d = np.array([10.0, -10.0, 0.5])
    out = plan.plan_step(eta, d, np.array([0.0, 0.0, 0.0]), np.array([8.0, 6.0, 8.0]), 0.2)
    np.testing.assert_allclose(out, [0.0, 6.0, 8.0])
