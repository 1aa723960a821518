"""Training data, training loop and evaluation of the learned warm start.

The network learns nodal prices and angles from plan-derived features; its training
data are dispatch solutions that the CUDA solver itself produces for perturbed plans
(a battery-cost sweep of the planner's gradient descent, Section 3.3, plus
log-normal perturbations of those plans).  Everything numeric runs in the CUDA kernels
of libgx.so; this module only sequences the calls.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import gx, synth


def gamma_for_battery_cost(net, cost_per_kwh, T):
    """The planner's investment-cost vector with battery capital cost `cost_per_kwh`."""
    g = np.array(net["gamma"], dtype=np.float64)
    G, L = net["gen_bus"].size, net["line_from"].size
    g[G + L:] = synth.battery_gamma_annual(cost_per_kwh) * T / 8760.0
    return g


def targets(net: gx.Network):
    """[prices | angles] of the last solve in the warm-start layout; angles relative to
    bus 0 of each scenario-hour (the solver's angles are defined up to that constant)."""
    # prices clipped to [0, 200] $/MWh: the rare value-of-lost-load hours would dominate
    # the squared error; a warm start needs the ordinary price level right
    price = net.array("price").clone().clamp_(0.0, 200.0)
    theta = net.array("theta").clone()
    for s, inf in enumerate(net.info):
        off = sum(i["N"] * i["Tp"] for i in net.info[:s])
        v = theta[off:off + inf["N"] * inf["Tp"]].view(inf["N"], inf["Tp"])
        v -= v[0:1, :].clone()
    return torch.cat([price, theta])


def plan_path(net, nets, eta0, gamma, eta_min, eta_max, alpha, steps):
    """Plans along `steps` implicit-gradient steps; returns the list of plans visited."""
    eta = eta0.clone()
    g = torch.zeros_like(eta)
    out = [eta.clone()]
    for k in range(steps):
        net.solve(eta, warm="cold" if k == 0 else "prev")
        net.grad(eta, out=g, warm="cold" if k == 0 else "prev")
        net.plan_step(eta, g, gamma, eta_min, eta_max, alpha)
        out.append(eta.clone())
    return out


def make_dataset(net, nets, costs, steps=8, keep_every=2, n_perturb=2, sigma=0.1, seed=100, alpha_frac=2e-2):
    """(plan, target) pairs: plans on gradient paths at each battery cost, plus log-normal
    perturbations of them, each solved by the CUDA solver (to 1e-3)."""
    rng = np.random.default_rng(seed)
    dev = net.device
    eta_min = torch.tensor(nets[0]["eta_min"], dtype=torch.float32, device=dev)
    eta_max = torch.tensor(nets[0]["eta_max"], dtype=torch.float32, device=dev)
    T = net.info[0]["T"]
    plans = []
    for c in costs:
        gamma = torch.tensor(gamma_for_battery_cost(nets[0], c, T), dtype=torch.float32, device=dev)
        g0 = torch.zeros_like(eta_min)
        net.solve(eta_min, warm="cold")
        net.grad(eta_min, out=g0)
        alpha = alpha_frac * float(eta_min.median()) / max(float((gamma + g0).abs().max()), 1e-30)
        path = plan_path(net, nets, eta_min, gamma, eta_min, eta_max, alpha, steps)
        plans += path[::keep_every]
    samples = []
    for p in plans:
        for k in range(n_perturb + 1):
            eta = p.clone()
            if k > 0:
                f = torch.tensor(rng.lognormal(0.0, sigma, size=eta.numel()), dtype=torch.float32, device=dev)
                eta = torch.minimum(torch.maximum(eta * f, eta_min), eta_max)
            net.solve(eta, warm="prev")
            samples.append((eta.clone(), targets(net)))
    return samples


def train(gnn: gx.WarmStartGNN, samples, epochs=30, lr=2e-3, w_theta=10.0, seed=0, log=None):
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        tot = 0.0
        lr_ep = lr * (0.5 * (1 + np.cos(np.pi * ep / max(epochs, 1))) * 0.9 + 0.1)
        for i in order:
            eta, tgt = samples[i]
            tot += gnn.train_step(eta, tgt, lr=float(lr_ep), w_theta=w_theta)
        hist.append(tot / len(samples))
        if log:
            log(f"epoch {ep} loss {hist[-1]:.4e}")
    return hist


def compare_starts(net, gnn, pairs):
    """For each (eta_a, eta_b): solve at eta_a, then at eta_b from a cold start, from
    eta_a's state (previous plan), from the learned start with its selection rule
    (GX_WARM_LEARNED: per scenario, the learned start or the previous plan's, whichever
    has the smaller residual at the first check) and from the network's prediction alone
    (a user start, no rule).  Forward and adjoint iterations, wall time (prediction
    included) and, for the rule, the share of scenarios that kept the learned start."""
    net.attach_gnn(gnn)
    rows = []
    for eta_a, eta_b in pairs:
        r = {}
        for mode in ("cold", "prev", "learned", "learned_only"):
            net.solve(eta_a, warm="cold")
            net.grad(eta_a)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "learned_only":
                w = gnn.predict(eta_b)
                M = w.numel() // 2
                net.solve(eta_b, warm="user", warm_prices=w[:M], warm_angles=w[M:])
            else:
                net.solve(eta_b, warm=mode)
            it_f = net.last_stats["iters_max"]
            # every start's adjoint begins at the negated forward duals (exact for the
            # h = c part; measured faster than the previous plan's adjoint state)
            net.grad(eta_b, warm="cold")
            torch.cuda.synchronize()
            r[mode] = dict(fwd=it_f, adj=net.last_grad_stats["iters_max"], ms=1e3 * (time.perf_counter() - t0))
            if mode == "learned":
                r[mode]["kept_learned"] = float(np.mean(net.array("warm").cpu().numpy() == 1))
        rows.append(r)
    return rows
