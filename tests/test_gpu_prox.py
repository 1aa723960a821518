"""The device proxes of one message-passing iteration (Section 2.1, Eq. 2's devices) against
brute-force minimisation of their objectives.

A user start at prices lambda and angles theta sets the bus duals u = -lambda / rho, every
generator and load at its best response to lambda, the line angle differences to theta's and
the bus power average p_bar to the terminals' mean.  One iteration then moves each device to
the minimiser of its own objective plus rho/2 |x - (x0 - p_bar0 - u0)|^2 (and, for a line,
rho_theta/2 |theta_j - theta_n|^2 at each end) over its box.  The test rebuilds those targets
on the CPU from the same start and minimises each 1-D objective by golden-section search in
FP64, with no use of the closed forms.  Prices are kept at least 1 $/MWh from every
generator's cost at its bus and below the value of lost load, so the start's outputs sit
exactly on their bounds in FP32 on both sides."""
import numpy as np
import pytest
import torch

from paper_2410_13055_gb300 import gx, synth

RHO, RHO_TH_C = 0.3, 0.1


def golden_min(f, lo, hi, iters=200):
    """Elementwise minimisers of convex 1-D functions on [lo, hi] by golden-section search
    (f takes and returns arrays of the shape of lo and hi)."""
    g = (np.sqrt(5.0) - 1.0) / 2.0
    a, b = np.array(lo, dtype=np.float64), np.array(hi, dtype=np.float64)
    for _ in range(iters):
        c, d = b - g * (b - a), a + g * (b - a)
        left = f(c) <= f(d)
        b = np.where(left, d, b)
        a = np.where(left, a, c)
    return 0.5 * (a + b)


def start_prices(net, T, rng):
    N = int(net["n_bus"])
    lam = rng.uniform(10.0, 120.0, size=(N, T))
    cost = net["gen_cost"]
    for n in range(N):
        cs = cost[net["gen_bus"] == n]
        for t in range(T):
            while np.any(np.abs(lam[n, t] - cs) < 1.0):
                lam[n, t] += 2.0
    return lam.astype(np.float32)


def after_one_iteration(net_d, sc, lam, theta, eta, eps, voll):
    """Each device's output after one iteration from the user start (lam, theta), by
    brute-force minimisation of its prox objective: generator output, load shed, line flow."""
    T = sc["T"]
    N, G, L = int(net_d["n_bus"]), net_d["gen_bus"].size, net_d["line_from"].size
    # the start, as the user start defines it (FP32 where it decides a bound)
    gb, cost = net_d["gen_bus"], net_d["gen_cost"].astype(np.float32)
    cap = (sc["cf"].astype(np.float32) * eta[:G, None]).astype(np.float32)
    p0 = np.where(lam[gb] > cost[:, None], cap, np.float32(0.0)).astype(np.float64)
    load = sc["load"].astype(np.float32).astype(np.float64)
    assert np.all(lam < voll - 1.0)
    xl0 = -load  # no shed below the value of lost load
    lf, lt = net_d["line_from"], net_d["line_to"]
    beta = net_d["line_beta"].astype(np.float64)
    d0 = (theta[lf] - theta[lt]).astype(np.float64)
    inj = np.zeros((N, T))
    cnt = np.ones(N)
    np.add.at(inj, gb, p0)
    np.add.at(cnt, gb, 1)
    inj += xl0
    np.add.at(inj, lf, -beta[:, None] * d0)
    np.add.at(inj, lt, beta[:, None] * d0)
    np.add.at(cnt, lf, 1)
    np.add.at(cnt, lt, 1)
    np.add.at(cnt, net_d["bat_bus"], 1)  # batteries start at zero output
    pbar0 = inj / cnt[:, None]
    u0 = -lam.astype(np.float64) / RHO
    e, r = float(eps), RHO

    # generators: min c p + eps/2 p^2 + rho/2 (p - v)^2 on [0, cap]
    v = p0 - pbar0[gb] - u0[gb]
    c = cost.astype(np.float64)[:, None]
    p_ref = golden_min(lambda p: c * p + e / 2 * p * p + r / 2 * (p - v) ** 2, np.zeros((G, T)),
                       cap.astype(np.float64))

    # loads: min VOLL sh + eps/2 sh^2 + rho/2 (sh - L - v)^2 on [0, L]
    v = xl0 - pbar0 - u0
    sh_ref = golden_min(lambda s: float(voll) * s + e / 2 * s * s + r / 2 * (s - load - v) ** 2, np.zeros((N, T)), load)

    # lines: the end angles (theta_f, theta_t) minimise
    #   rho/2 [(p_f - a_f)^2 + (p_t - a_t)^2] + rho_th/2 [(theta_f - theta_n(f))^2 + (theta_t - theta_n(t))^2]
    # with p_f = -beta (theta_f - theta_t) = -p_t, under |beta delta| <= eta_l and |delta| <= dtheta_max,
    # rho_th = rho * rho_theta_c * mean(beta^2).  Brute force over (delta, sigma = theta_f + theta_t),
    # nested: sigma is unconstrained.
    rth = RHO * RHO_TH_C * np.mean(beta ** 2)
    eta_l = eta[G:G + L].astype(np.float64)
    lim = np.minimum(eta_l / beta, net_d["line_dtheta"])
    bl = beta[:, None]
    af = -bl * d0 - pbar0[lf] - u0[lf]
    at = bl * d0 - pbar0[lt] - u0[lt]
    zf, zt = theta[lf].astype(np.float64), theta[lt].astype(np.float64)

    def obj_sigma(s, d):
        thf, tht = (s + d) / 2, (s - d) / 2
        return rth / 2 * ((thf - zf) ** 2 + (tht - zt) ** 2)

    def obj_delta(d):
        s_best = golden_min(lambda s: obj_sigma(s, d), zf + zt - 1.0, zf + zt + 1.0, iters=80)
        return r / 2 * ((-bl * d - af) ** 2 + (bl * d - at) ** 2) + obj_sigma(s_best, d)

    lim2 = np.broadcast_to(lim[:, None], (L, T))
    flow_ref = bl * golden_min(obj_delta, -lim2, lim2, iters=120)
    return p_ref, sh_ref, flow_ref, dict(v_gen=p0 - pbar0[gb] - u0[gb], af=af, at=at, d0=d0, lim=lim, rth=rth)


def _case(case):
    nets, scens = synth.tiny() if case == "tiny" else synth.medium(S=1, T=24)
    net_d, sc = nets[0], scens[0]
    rng = np.random.default_rng(11)
    lam = start_prices(net_d, sc["T"], rng)
    theta = rng.uniform(-0.05, 0.05, size=(int(net_d["n_bus"]), sc["T"])).astype(np.float32)
    eta = net_d["eta_min"].astype(np.float32) * np.float32(1.1)
    return nets, scens, lam, theta, eta


@pytest.mark.parametrize("case", ["tiny", "medium24"])
def test_brute_force_prox_equals_closed_forms(case):
    """The brute-force minimisers above against the proxes' closed forms (Section 2.1's device
    models): generator clip((rho v - c) / (rho + eps), 0, cap); line delta =
    (rho beta (a_t - a_f) + rho_th/2 (w_f - w_t)) / (2 rho beta^2 + rho_th/2), clipped."""
    nets, scens, lam, theta, eta = _case(case)
    net_d, sc = nets[0], scens[0]
    o = gx.default_opts()
    p_ref, sh_ref, flow_ref, aux = after_one_iteration(net_d, sc, lam, theta, eta, np.float32(o.eps), np.float32(o.voll))
    e, r = float(np.float32(o.eps)), RHO
    G = net_d["gen_bus"].size
    cap = (sc["cf"].astype(np.float32) * eta[:G, None]).astype(np.float64)
    p_cf = np.clip((r * aux["v_gen"] - net_d["gen_cost"][:, None]) / (r + e), 0.0, cap)
    assert np.max(np.abs(p_cf - p_ref)) <= 1e-7 * max(np.max(np.abs(p_cf)), 1.0)
    beta = net_d["line_beta"][:, None]
    d = (r * beta * (aux["at"] - aux["af"]) + aux["rth"] / 2 * aux["d0"]) / (2 * r * beta ** 2 + aux["rth"] / 2)
    d = np.clip(d, -aux["lim"][:, None], aux["lim"][:, None])
    assert np.max(np.abs(beta * d - flow_ref)) <= 1e-6 * max(np.max(np.abs(flow_ref)), 1.0)
    assert np.all(sh_ref >= 0) and np.all(sh_ref <= sc["load"] + 1e-9)


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["tiny", "medium24"])
def test_one_iteration_matches_brute_force_prox(case):
    nets, scens, lam, theta, eta = _case(case)
    net_d, sc = nets[0], scens[0]
    T = sc["T"]
    N, G, L = int(net_d["n_bus"]), net_d["gen_bus"].size, net_d["line_from"].size
    net = gx.Network(nets, scens, kappa=0.0, rho=RHO, rho_theta_c=RHO_TH_C, tol=1e-12, max_iter=1, check_every=1)
    assert net.opts.theta_weight == 0  # phase weights: the mean beta^2 of the network
    assert net.info[0]["Tp"] == T  # prices and angles below are [N x T] rows without padding
    rc = net.solve(torch.tensor(eta, device="cuda"), warm="user", warm_prices=torch.tensor(lam.ravel()),
                   warm_angles=torch.tensor(theta.ravel()))
    assert rc in (0, 1)
    torch.cuda.synchronize()
    p_gpu = net.array("p", 0).cpu().numpy().astype(np.float64)
    shed_gpu = net.array("shed", 0).cpu().numpy().astype(np.float64)
    flow_gpu = net.array("flow", 0).cpu().numpy().astype(np.float64)
    p_ref, sh_ref, flow_ref, _ = after_one_iteration(net_d, sc, lam, theta, eta, np.float32(net.opts.eps),
                                                     np.float32(net.opts.voll))
    assert p_gpu.shape == (G, T) and shed_gpu.shape == (N, T) and flow_gpu.shape == (L, T)
    scale = max(np.max(np.abs(p_ref)), 1.0)
    assert np.max(np.abs(p_gpu - p_ref)) <= 1e-4 * scale, np.max(np.abs(p_gpu - p_ref))
    load = sc["load"]
    assert np.max(np.abs(shed_gpu - sh_ref)) <= 1e-4 * max(np.max(load), 1.0), np.max(np.abs(shed_gpu - sh_ref))
    fscale = max(np.max(np.abs(flow_ref)), 1.0)
    assert np.max(np.abs(flow_gpu - flow_ref)) <= 1e-4 * fscale, np.max(np.abs(flow_gpu - flow_ref))
