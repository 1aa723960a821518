"""Autotuner of the solver's launch and penalty parameters, cached per shape bucket.

For a bound network it times a short implicit-gradient sequence (a cold solve and
gradient, then `steps` previous-plan steps) for candidate settings, one parameter at a
time from the defaults (coordinate descent), and keeps the fastest setting whose
planner objective stays within `h_tol` of a tight reference solve at the same plan and
whose gradient there is no less accurate than the defaults' (within a factor `g_slack`)
against a tight reference gradient (equal residual tolerances do not give equal
accuracy across penalties; the adjoint penalty changes the gradient and not h).  Parameters:
the execution path (per-iteration kernels replayed as CUDA graphs, or one persistent
cluster-resident launch per loop for the scenarios that fit), the kernel schedule (how
the bus kernel brings its device rows in: per-thread loads, bulk copies into shared
memory, or per-thread asynchronous copies; one or two warps per battery), residual-check
chunk length (the CUDA-graph size), power penalty rho, phase penalty scale, adjoint
penalty, battery inner iterations.  Results are cached as JSON, keyed by (buses, hours,
scenarios) rounded to powers of two.

``tune_schedule`` is the quick form for the kernel schedule alone: schedules do not change
the iterates (the bus kernel variants are bitwise equal), so it times a fixed number of
iterations per candidate and keeps the fastest.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np
import torch

from typing import TYPE_CHECKING

if TYPE_CHECKING:  # the library is loaded by the functions that run it
    from . import gx

SCHEDULE = {"bus_staged": [0, 1, 2], "bat_warps": [2, 1]}

SPACE = {
    "persistent": [False, True],
    "bus_staged": SCHEDULE["bus_staged"],
    "bat_warps": SCHEDULE["bat_warps"],
    "check_every": [10, 20, 40],
    "rho": [0.1, 0.15, 0.2, 0.3, 0.5],
    "rho_theta_c": [0.03, 0.1],
    "adj_rho": [0.001, 0.002, 0.004],
    "inner_iters": [2, 3],
}


def bucket(net: gx.Network):
    p2 = lambda x: 1 << max(0, int(math.ceil(math.log2(max(x, 1)))))
    N = max(i["N"] for i in net.info)
    T = max(i["T"] for i in net.info)
    return f"N{p2(N)}_T{p2(T)}_S{p2(net.S)}"


def default_cache_path():
    return os.environ.get("GX_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gx", "autotune.json"))


def _run(net, eta0, gamma, eta_min, eta_max, steps, alpha):
    eta = eta0.clone()
    g = torch.zeros_like(eta)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps + 1):
        warm = "cold" if k == 0 else "prev"
        net.solve(eta, warm=warm)
        net.grad(eta, out=g, warm=warm)
        if k < steps:
            net.plan_step(eta, g, gamma, eta_min, eta_max, alpha)
    torch.cuda.synchronize()
    h = float((net.array("h").cpu().numpy() * net.weights).sum())
    return time.perf_counter() - t0, eta, h


def accept(h, h_ref, g_err, g_base, h_tol=2e-3, g_slack=1.25):
    """The accuracy guard: the candidate's planner objective within h_tol of the tight
    reference and its gradient error at most g_slack times the defaults'."""
    return abs(h - h_ref) <= h_tol * abs(h_ref) and g_err <= g_slack * g_base + 1e-6


def _grad_err(net, eta, g_ref):
    net.solve(eta, warm="cold")
    g = net.grad(eta, warm="cold")
    torch.cuda.synchronize()
    return float((g.double() - g_ref).norm() / max(float(g_ref.norm()), 1e-30))


def _apply(net, opts):
    """Options, execution path and kernel schedule of a setting."""
    net.set_opts(**{k: v for k, v in opts.items() if k not in ("persistent",) and k not in SCHEDULE})
    if "persistent" in opts:
        net.use_persistent(bool(opts["persistent"]))
    sched = {k: int(v) for k, v in opts.items() if k in SCHEDULE}
    if sched:
        net.set_schedule(**sched)


def tune_schedule(net: gx.Network, eta, iters=200, space=None, log=None):
    """Pick the fastest kernel schedule for `net` at plan `eta`: for each candidate, time
    `iters` forward and `iters` adjoint iterations with every scenario iterating (the
    tolerances are set out of reach for the timing, then restored).  The schedules
    compute the same iterates, so only time decides.  Leaves the state of the last
    timing run in the workspace (callers start their solves cold).  Returns
    dict(best=..., trials=[...])."""
    space = space or SCHEDULE
    keep = {k: getattr(net.opts, k) for k in ("tol", "adj_tol", "max_iter", "adj_max_iter")}
    net.solve(eta, warm="cold")
    net.grad(eta, warm="cold")
    every = net.opts.check_every
    n = max(every, iters // every * every)
    net.set_opts(tol=1e-30, adj_tol=1e-30, max_iter=n, adj_max_iter=n)
    cands = [dict(bus_staged=b, bat_warps=w) for b in space["bus_staged"] for w in space["bat_warps"]]
    trials = []
    for cand in cands:
        net.set_schedule(**cand)
        net.solve(eta, warm="prev")  # captures the loop graphs of this schedule, untimed
        net.grad(eta, warm="prev")
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        net.solve(eta, warm="prev")
        net.grad(eta, warm="prev")
        b.record()
        torch.cuda.synchronize()
        us = 1e3 * a.elapsed_time(b) / (2 * n)
        # the same run again with the kernels' timer stamps on: per-launch kernel times
        net.profile(True)
        net.solve(eta, warm="prev")  # (switching the stamps on re-captures the graphs)
        net.grad(eta, warm="prev")
        net.profile(True)  # reset the counters, keep the graphs
        net.solve(eta, warm="prev")
        net.grad(eta, warm="prev")
        prof = net.profile_read()
        net.profile(False)
        kern = {k + "_us": round(1e3 * v["ms"] / max(v["samples"], 1), 3) for k, v in prof.items() if k != "k_crs"}
        trials.append(dict(cand, us_per_iteration=round(us, 3), **kern))
        if log:
            log(trials[-1])
    best = min(trials, key=lambda t: t["us_per_iteration"])
    best = {k: best[k] for k in SCHEDULE}
    net.set_schedule(**best)
    net.set_opts(**keep)
    return dict(best=best, trials=trials, iterations=n)


def pick_schedule(trials, default, margin):
    """The schedule to keep from timed trials (dicts with the schedule's keys and
    `ms_per_step`): the fastest, if it beats the default schedule's time by more than
    `margin` (a fraction) or the default was not timed; else the default."""
    fastest = min(trials, key=lambda t: t["ms_per_step"])
    t_def = next((t["ms_per_step"] for t in trials if {k: t[k] for k in SCHEDULE} == default), None)
    pick = fastest if (t_def is None or fastest["ms_per_step"] < (1.0 - margin) * t_def) else dict(default)
    return {k: pick[k] for k in SCHEDULE}


def tune_schedule_step(net: gx.Network, eta, step=None, steps=2, reps=2, margin=0.02, space=None, log=None,
                       flush=None):
    """Pick the fastest kernel schedule on the workload's own steps.  From the current
    (previous plan's) forward and adjoint state and plan `eta`, each candidate runs `steps`
    consecutive previous-plan steps (`step(eta)`: solve, gradient and plan step in place;
    default: solve and gradient only, at a fixed plan), `reps` times from the same restored
    state and plan, keeping its best time; the first run of a candidate also captures its
    graphs.  The schedule in force when the tuner is called (bind's default) is kept unless
    a candidate is faster by more than `margin`: a single step's timing cannot tell apart
    schedules closer than that.  `flush()`, if given, runs before each step outside its
    timing (the caller's cache flush, so the steps are timed as the caller times them).
    State and plan are restored at the end.  Unlike
    `tune_schedule`, this times the steps' real mix of launches, including the ones where
    most scenarios have converged.  Returns dict(best=..., default=..., trials=[...])."""
    space = space or SCHEDULE
    if step is None:
        def step(e):
            net.solve(e, warm="prev")
            net.grad(e, warm="prev")
    default = net.schedule()
    sx, sa, se = net.state(False).clone(), net.state(True).clone(), eta.clone()

    def restore():
        net.state(False).copy_(sx)
        net.state(True).copy_(sa)
        eta.copy_(se)

    cands = [dict(bus_staged=b, bat_warps=w) for b in space["bus_staged"] for w in space["bat_warps"]]
    trials = []
    for cand in cands:
        net.set_schedule(**cand)
        best_ms = None
        for _ in range(reps):
            restore()
            torch.cuda.synchronize()
            evs = []
            for _ in range(steps):
                if flush is not None:
                    flush()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                step(eta)
                b.record()
                evs.append((a, b))
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs) / steps
            best_ms = ms if best_ms is None else min(best_ms, ms)
        trials.append(dict(cand, ms_per_step=round(best_ms, 4)))
        if log:
            log(trials[-1])
    best = pick_schedule(trials, default, margin)
    net.set_schedule(**best)
    # one more run captures the chosen schedule's graphs, so the caller's next step is not
    # charged for it; then state and plan go back to the previous plan's
    restore()
    step(eta)
    restore()
    torch.cuda.synchronize()
    return dict(best=best, default=default, trials=trials)


def tune(net: gx.Network, nets, steps=3, h_tol=2e-3, g_slack=1.25, cache=None, log=None, alpha_frac=1e-2):
    """Tune `net`'s options in place; returns the chosen option dict."""
    cache = cache or default_cache_path()
    key = bucket(net)
    dev = net.device
    eta_min = torch.tensor(np.concatenate([n["eta_min"] for n in nets]), dtype=torch.float32, device=dev)
    eta_max = torch.tensor(np.concatenate([n["eta_max"] for n in nets]), dtype=torch.float32, device=dev)
    gamma = torch.tensor(np.concatenate([n["gamma"] for n in nets]), dtype=torch.float32, device=dev)
    base = {k: getattr(net.opts, k) for k in SPACE if k != "persistent" and k not in SCHEDULE}
    base["persistent"] = False
    base.update(net.schedule())
    g0 = torch.zeros_like(eta_min)
    net.solve(eta_min, warm="cold")
    net.grad(eta_min, out=g0)
    alpha = alpha_frac * float(eta_min.median()) / max(float((gamma + g0).abs().max()), 1e-30)

    def apply(opts):
        _apply(net, opts)

    def measure(opts):
        apply(opts)
        return _run(net, eta_min, gamma, eta_min, eta_max, steps, alpha)

    t_best, eta_end, _ = measure(base)
    # tight reference objective at the plan the defaults reach
    from . import gx
    ref = gx.Network(nets, [dict(sc) for sc in net.scens_desc], opts=gx.default_opts(
        **{**{k: getattr(net.opts, k) for k, _ in gx.Opts._fields_}, "tol": 1e-5, "max_iter": 200000}))
    ref.set_opts(adj_tol=1e-5, adj_max_iter=200000)
    ref.solve(eta_end)
    g_ref = ref.grad(eta_end).double().clone()
    torch.cuda.synchronize()
    h_ref = float((ref.array("h").cpu().numpy() * ref.weights).sum())
    del ref
    g_base = _grad_err(net, eta_end, g_ref)
    best = dict(base)
    trials = [dict(base, time_s=t_best, g_rel=g_base)]
    for name, vals in SPACE.items():
        for v in vals:
            if v == best[name]:
                continue
            cand = dict(best, **{name: v})
            t, eta_c, _ = measure(cand)
            g_err = _grad_err(net, eta_end, g_ref)
            h = float((net.array("h").cpu().numpy() * net.weights).sum())
            ok = accept(h, h_ref, g_err, g_base, h_tol, g_slack)
            trials.append(dict(cand, time_s=t, h_rel=abs(h - h_ref) / abs(h_ref), g_rel=g_err, ok=ok))
            if log:
                log(trials[-1])
            if ok and t < t_best:
                best, t_best = cand, t
    apply(best)
    entry = dict(best=best, time_s=t_best, trials=trials)
    try:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        db = json.load(open(cache)) if os.path.exists(cache) else {}
        db[key] = entry
        json.dump(db, open(cache, "w"), indent=1)
    except OSError:
        pass
    return best


def load(net: gx.Network, cache=None):
    """Apply a cached setting for `net`'s shape bucket; returns it (or None)."""
    cache = cache or default_cache_path()
    if not os.path.exists(cache):
        return None
    db = json.load(open(cache))
    e = db.get(bucket(net))
    if e:
        _apply(net, dict(e["best"]))
        return e["best"]
    return None


def main(argv=None):
    """python -m paper_2410_13055_gb300.autotune schedule --config medium|scale|batching
    [--scenarios S] [--iters N]: every kernel schedule's time per iteration and per-launch
    kernel times (timer stamps) with every scenario iterating, as JSON."""
    import argparse
    from . import gx, synth
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["schedule"])
    ap.add_argument("--config", default="medium", choices=["medium", "scale", "batching"])
    ap.add_argument("--scenarios", type=int, default=None)
    ap.add_argument("--iters", type=int, default=200)
    args = ap.parse_args(argv)
    make = {"medium": synth.medium, "scale": synth.scale, "batching": synth.batching}[args.config]
    nets, scens = make(S=args.scenarios) if args.scenarios else make()
    net = gx.Network(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000, rho=0.2)
    eta = torch.tensor(np.concatenate([n["eta_min"] for n in nets]), dtype=torch.float32, device=net.device)
    rep = tune_schedule(net, eta, iters=args.iters)
    print(json.dumps(dict(config=args.config, scenarios=net.S, **rep)), flush=True)


if __name__ == "__main__":
    main()
