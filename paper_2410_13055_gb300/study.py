"""Planner-level studies on top of the hot path: stochastic implicit gradient descent
(Section 2.2) with a scenario sampler, the outer-loop warm-start study (Section 3.2) and
the battery-cost sweep (Section 3.3).

Every dispatch, adjoint and plan step runs in libgx.so; this module only samples
scenario batches, evaluates the planner objective and keeps the books.

    python -m paper_2410_13055_gb300.study warm --out warm.json
    python -m paper_2410_13055_gb300.study battery --out battery.json

Synthetic stand-in for the paper's 100-node, 16-day WECC cases: the 100-bus network of
``synth.medium`` with 16 scenarios of T = 24 hours.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import synth


def batches(S: int, B: int, seed: int):
    """Endless stream of scenario batches: B distinct scenarios drawn uniformly (Section
    2.2's stochastic estimate of the gradient)."""
    rng = np.random.default_rng(seed)
    while True:
        yield np.sort(rng.choice(S, size=min(B, S), replace=False)).astype(np.int32)


def within(history, target: float, rel: float = 0.02):
    """First iteration whose objective is within `rel` of `target` (Section 3.2's rule:
    converged once the loss is within 2 % of the best cold-start loss); None if never."""
    for it, J in history:
        if J <= target + rel * abs(target):
            return it
    return None


def within_gap(history, start: float, target: float, frac: float = 0.02):
    """First iteration whose objective has closed all but `frac` of the gap between a
    cold start's initial objective `start` and `target` (J - target <= frac (start -
    target)); None if never.  A stricter companion to the 2 % rule where the objective's
    fixed part dwarfs what the plan can change."""
    gap = start - target
    for it, J in history:
        if J - target <= frac * gap:
            return it
    return None


class Planner:
    """Implicit gradient descent on one bound network (``gx.Network``) of S scenarios."""

    def __init__(self, net, nets):
        import torch
        self.net = net
        dev = net.device
        cat = lambda k: torch.tensor(np.concatenate([n[k] for n in nets]), dtype=torch.float32, device=dev)
        self.eta_min, self.eta_max = cat("eta_min"), cat("eta_max")
        self.grad = torch.zeros_like(self.eta_min)

    def objective(self, eta, gamma):
        """gamma^T eta + sum_s w_s h_s(x*_s(eta)) over every scenario (Eq. 1)."""
        self.net.solve(eta, warm="prev")
        h = float((self.net.array("h").double().cpu().numpy() * self.net.weights).sum())
        return float((gamma.double() * eta.double()).sum()) + h

    def sgd(self, eta0, gamma, alpha, iters, batch, seed=0, eval_every=10, log=None):
        """`iters` projected steps eta <- clip(eta - alpha (gamma + g_B), eta_min, eta_max),
        g_B the gradient over a sampled batch (weights rescaled to the whole set).  Returns
        the final plan and the objective history [(iteration, J)]."""
        eta = eta0.clone()
        draw = batches(self.net.S, batch, seed)
        hist = [(0, self.objective(eta, gamma))]
        t0 = time.perf_counter()
        for it in range(1, iters + 1):
            idx = next(draw)
            self.net.solve(eta, batch=idx, warm="prev")
            self.net.grad(eta, out=self.grad, warm="prev")
            self.net.plan_step(eta, self.grad, gamma, self.eta_min, self.eta_max, alpha)
            if it % eval_every == 0 or it == iters:
                hist.append((it, self.objective(eta, gamma)))
                if log:
                    log(f"iter {it} J {hist[-1][1]:.6e} ({time.perf_counter() - t0:.1f} s)")
        return eta, hist


def _setup(kappa, seed=1, S=16, T=24):
    import torch
    from . import gx
    nets, scens = synth.medium(seed=seed, S=S, T=T)
    net = gx.Network(nets, scens, kappa=kappa, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    pl = Planner(net, nets)
    gamma = torch.tensor(nets[0]["gamma"], dtype=torch.float32, device=net.device)
    return nets, net, pl, gamma


def step_size(pl, gamma, frac):
    """alpha = frac * median(eta_min) / |gamma + g(eta_min)|_inf (a fixed step, set once)."""
    pl.net.solve(pl.eta_min, warm="cold")
    pl.net.grad(pl.eta_min, out=pl.grad)
    return frac * float(pl.eta_min.median()) / max(float((gamma + pl.grad).abs().max()), 1e-30)


def warm_start_study(kappas=(100.0, 150.0, 175.0, 225.0, 250.0, 300.0), ref_kappa=200.0, iters=300, batch=4,
                     alpha_frac=0.02, eval_every=5, seed=0, log=None):
    """Section 3.2 on the synthetic 100-bus, 16 x 24 h case: for each carbon weight, SGD
    from no expansion (eta_min) and from the solution at `ref_kappa`; iterations until
    the loss is within 2 % of the best cold-start loss, and their ratio."""
    nets, net, pl, gamma = _setup(ref_kappa)
    alpha = step_size(pl, gamma, alpha_frac)
    eta_ref, hist_ref = pl.sgd(pl.eta_min, gamma, alpha, iters, batch, seed=seed, eval_every=eval_every)
    rows = []
    for k in kappas:
        net.set_opts(kappa=k)
        _, hc = pl.sgd(pl.eta_min, gamma, alpha, iters, batch, seed=seed + 1, eval_every=eval_every)
        _, hw = pl.sgd(eta_ref, gamma, alpha, iters, batch, seed=seed + 1, eval_every=eval_every)
        best = min(J for _, J in hc)
        row = dict(kappa=k, best_cold=best, best_warm=min(J for _, J in hw), cold_history=hc, warm_history=hw)
        for tag, rel in (("", 0.02), ("_05", 0.005)):
            ic, iw = within(hc, best, rel), within(hw, best, rel)
            # 0 warm iterations: the warm plan already meets the threshold (speedup counted
            # against one iteration)
            row["cold_iters" + tag], row["warm_iters" + tag] = ic, iw
            row["speedup" + tag] = (ic / max(iw, 1)) if (ic is not None and iw is not None) else None
        # the same for 98 % of the improvement a cold run achieves over its start
        ic, iw = within_gap(hc, hc[0][1], best), within_gap(hw, hc[0][1], best)
        row["cold_iters_gap"], row["warm_iters_gap"] = ic, iw
        row["speedup_gap"] = (ic / max(iw, 1)) if (ic is not None and iw is not None) else None
        rows.append(row)
        if log:
            log(f"kappa {k}: to 2 %: cold {row['cold_iters']} warm {row['warm_iters']}; "
                f"to 0.5 %: cold {row['cold_iters_05']} warm {row['warm_iters_05']}; "
                f"to 98 % of the cold gain: cold {row['cold_iters_gap']} warm {row['warm_iters_gap']}")
    return dict(ref_kappa=ref_kappa, alpha=alpha, batch=batch, iters=iters, ref_history=hist_ref, rows=rows)


def asset_classes(net_desc):
    """Index groups of the plan vector: gas, solar, wind generators, lines, batteries."""
    G, L = net_desc["gen_bus"].size, net_desc["line_from"].size
    kind = np.asarray(net_desc.get("gen_kind", np.zeros(G, dtype=int)))
    out = {}
    for name, code in (("gas", 0), ("solar", 1), ("wind", 2)):
        out[name] = np.where(kind == code)[0]
    out["lines"] = G + np.arange(L)
    out["batteries"] = G + L + np.arange(net_desc["bat_bus"].size)
    return out


def battery_cost_sweep(costs=None, kappa=200.0, iters=150, batch=4, alpha_frac=0.02, eval_every=10, seed=0,
                       log=None, S=16, T=24):
    """Section 3.3: battery capital costs from low to high, each run warm-started from the
    previous cost's plan; expansion (MW above existing) per asset class at each cost."""
    import torch
    from .warmstart import gamma_for_battery_cost
    costs = list(costs) if costs is not None else list(np.linspace(40.0, 800.0, 20))
    nets, net, pl, _ = _setup(kappa, S=S, T=T)
    T = net.info[0]["T"]
    groups = asset_classes(nets[0])
    eta = pl.eta_min.clone()
    rows = []
    alpha = None
    for k, c in enumerate(costs):
        gamma = torch.tensor(gamma_for_battery_cost(nets[0], c, T), dtype=torch.float32, device=net.device)
        if alpha is None:
            alpha = step_size(pl, gamma, alpha_frac)
        eta, hist = pl.sgd(eta, gamma, alpha, iters if k == 0 else max(iters // 3, 10), batch, seed=seed + k,
                           eval_every=eval_every)
        e = eta.double().cpu().numpy()
        e0 = pl.eta_min.double().cpu().numpy()
        rows.append(dict(cost_per_kwh=float(c), objective=hist[-1][1],
                         expansion_mw={g: float((e[ix] - e0[ix]).sum()) for g, ix in groups.items()}))
        if log:
            log(f"battery ${c:.0f}/kWh: " + ", ".join(f"{g} {v:.0f}" for g, v in rows[-1]["expansion_mw"].items()))
    return dict(kappa=kappa, alpha=alpha, rows=rows)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["warm", "battery"])
    ap.add_argument("--out", default=None)
    ap.add_argument("--iters", type=int, default=None)
    ap.add_argument("--batch", type=int, default=4)
    args = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)
    t0 = time.time()
    if args.study == "warm":
        rep = warm_start_study(iters=args.iters or 300, batch=args.batch, log=log)
        for tag in ("", "_05", "_gap"):
            sp = [r["speedup" + tag] for r in rep["rows"] if r["speedup" + tag] is not None]
            rep["mean_speedup" + tag] = float(np.mean(sp)) if sp else None
    else:
        rep = battery_cost_sweep(iters=args.iters or 150, batch=args.batch, log=log)
    rep["wall_s"] = time.time() - t0
    summary = {k: v for k, v in rep.items() if k not in ("rows", "ref_history")}
    print(json.dumps(summary), flush=True)
    if args.out:
        json.dump(rep, open(args.out, "w"), indent=1, default=float)


if __name__ == "__main__":
    main()
