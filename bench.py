"""Throughput of the dispatch + implicit-gradient hot path on one GB300.

A step is one implicit-gradient iteration of the planner (Section 2.2): solve every
scenario's dispatch (Eq. 2) to a 1e-3 relative residual, solve the adjoint of the
active KKT system to 1e-3 for d h / d eta, and take the projected plan step.  The
metric is device-hours dispatched + differentiated per second:
    device-hours = sum_s (generators + lines + batteries + loads) * T_s   per step.

Default workload: the 100-bus network of 16 weekly scenarios (T = 168), emissions
weight kappa = 50 $/t (so h != c and the adjoint is required).  Starts: "prev"
(the previous plan's dispatch and adjoint state, the interactive warm start of
Section 2.2) is the headline; "cold" is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config medium|scale|batching|tiny]
                    [--impl gx|reference]

--impl reference times the FP64 oracle (interior point + KKT adjoint) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import resource
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2410_13055_gb300 import synth  # noqa: E402

KAPPA = 50.0
METRIC = "device-hours dispatched+differentiated/s at 1e-3 residual"
UNIT = "device-hours/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        # raw samples: GX_BENCH_CLOCKS_DIR if set, else the system temporary directory
        base = os.environ.get("GX_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(base, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def build_workload(config, rank=0, ws=1, scenarios=None):
    """The scenarios rank `rank` of `ws` solves (weak scaling: every rank gets the one-GPU
    workload's size).  Returns (nets, scens, shared): `shared` is True when the ranks plan
    one network together, so a plan step sums their partial gradients.

    medium     16 x ws scenarios of the 100-bus network, split by sharding.shard
    batching   64 x ws scenarios of their own networks, split by sharding.shard (no network
               spans two ranks: no collective)
    scale      52 weekly scenarios per rank, drawn from the rank's own seed on the common
               2000-bus network (the global set is too large to draw on every rank)
    tiny       the 5-bus case, one per rank
    """
    from paper_2410_13055_gb300 import sharding
    if config == "medium":
        S = scenarios or 16
        nets, scens = synth.medium(seed=1, S=S * ws)
        idx = sharding.shard(nets, scens, ws)[rank]
        nets, scens, _ = sharding.local_problem(nets, scens, idx)
        return nets, scens, ws > 1
    if config == "batching":
        nets, scens = synth.batching(seed=2, S=(scenarios or 64) * ws)
        idx = sharding.shard(nets, scens, ws)[rank]
        nets, scens, _ = sharding.local_problem(nets, scens, idx)
        return nets, scens, False
    if config == "scale":
        S = scenarios or 52
        nets, scens = synth.scale(seed=3, S=S, scen_seed=None if rank == 0 else 3000 + rank, weight=1.0 / (S * ws))
        return nets, scens, ws > 1
    if config == "tiny":
        nets, scens = synth.tiny(seed=0)
        for sc in scens:
            sc["weight"] = 1.0 / ws
        return nets, scens, ws > 1
    raise SystemExit(f"unknown config {config}")


def algorithmic_bytes(nets, scens):
    """Compulsory bytes of one k_bus / k_line / k_bat launch for each scenario: every array
    element the kernel must touch, read or written once (per hour of each row).

    k_bus   generators x r/w 8 + cf 4 (non-firm rows); load x r/w 8 + L 4;
            bus u, pbar, z r/w 24; line delta 4 + q at both ends 8; battery x 4
    k_line  line delta, sigma, q_f, q_t r/w 32; bus pbar, u, z read 12 per bus-hour
    k_bat   battery x, z(3), y(3) r/w 56 + pivots 4; bus pbar, u read 8
    """
    out = []
    for sc in scens:
        n = nets[sc["net"]]
        T = sc["T"]
        G, L, B, N = n["gen_bus"].size, n["line_from"].size, n["bat_bus"].size, n["n_bus"]
        nonfirm = int(np.sum(np.any(sc["cf"] != 1.0, axis=1)))
        bat_buses = np.unique(n["bat_bus"]).size
        out.append({"k_bus": T * (8 * G + 4 * nonfirm + 12 * N + 24 * N + 12 * L + 4 * B),
                    "k_line": T * (32 * L + 12 * N),
                    "k_bat": T * (60 * B + 8 * bat_buses)})
    return out


# DRAM bytes (read + write) per launch from one ncu capture of the solver kernels; valid only
# while gx_kernels.cu is the source that was profiled.
PROFILED = {
    "sha256_prefix": "8e66a2280c707af5",
    # forward launches, all scenarios iterating, cold cache (ncu flushes before each pass)
    "medium": {"scenarios": 16, "source": "profiles/launches_medium_bench.md (dram capture, same command)",
               "traffic": {"k_bus": 16.84e6, "k_line": 9.80e6, "k_bat": 5.33e6}},
    "scale": {"scenarios": 13, "source": "profiles/bus_kernel_staged_scale13.md",
              "traffic": {"k_bus": 387.8e6, "k_line": 209.0e6, "k_bat": 43.9e6}},
    "batching": {"scenarios": 64, "source": "profiles/solver_kernels_batching64.md",
                 "traffic": {"k_bus": 103.86e6, "k_line": 56.73e6, "k_bat": 19.05e6}},
}


def profiled_traffic(config, n_scen, kernel):
    """DRAM bytes per launch from the capture of this workload, scaled by scenarios (the Scale
    capture is of 13 of its 52 identical-size weeks, above L2, where traffic grows in
    proportion; the others are of the whole workload); None if the kernels changed since, or
    the workload has no capture."""
    import hashlib
    src = os.path.join(ROOT, "paper_2410_13055_gb300", "csrc", "gx_kernels.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    cap = PROFILED.get(config)
    if sha != PROFILED["sha256_prefix"] or cap is None or kernel not in cap["traffic"]:
        return None
    return cap["traffic"][kernel] * n_scen / cap["scenarios"]


def roofline(config, prof, active, per_scen, n_scen, iters_per_step, ms_per_step):
    """The dominant per-iteration kernel against the measured HBM copy rate.

    achieved = algorithmic bytes of a sampled launch / its CUDA-event time.  A converged
    scenario's blocks exit at once, so a sampled launch is credited with the bytes of the
    scenarios still iterating in it (gx_profile_active), not of the whole batch."""
    peak, peak_kind = _peaks()
    kinds = {k: v for k, v in prof.items() if k in ("k_bus", "k_line", "k_bat") and v["samples"] > 0}
    if not kinds:
        return None
    rec = {}
    for k, v in kinds.items():
        avg_ms = v["ms"] / v["samples"]
        nbytes = float(sum(int(active[s]) * per_scen[s][k] for s in range(n_scen))) / v["samples"]
        rec[k] = {"avg_launch_us": round(avg_ms * 1e3, 3), "bytes_per_launch": round(nbytes, 1),
                  "achieved_gbs": round(nbytes / (avg_ms / 1e3) / 1e9, 1), "launches": v["launches"],
                  "total_ms": round(avg_ms * v["launches"], 3)}
    dom = max(rec, key=lambda k: rec[k]["total_ms"])
    d = rec[dom]
    tr = profiled_traffic(config, n_scen, dom)
    if tr is not None:
        # the capture is of all-scenario launches: scale to the average sampled launch's share
        all_bytes = float(sum(per_scen[s][dom] for s in range(n_scen)))
        tr = round(tr * d["bytes_per_launch"] / max(all_bytes, 1.0), 1)
    it_us = rec.get("k_bus", {"avg_launch_us": 0.0})["avg_launch_us"] + max(
        rec.get("k_line", {"avg_launch_us": 0.0})["avg_launch_us"], rec.get("k_bat", {"avg_launch_us": 0.0})["avg_launch_us"])
    return {"bound": "hbm", "kernel": dom, "achieved": d["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": round(d["achieved_gbs"] / peak, 4), "traffic": tr,
            "traffic_note": (f"ncu dram read+write of an all-scenario launch (cold cache), scaled by scenarios and "
                             f"by the sampled launches' active share, from {PROFILED[config]['source']}"
                             if tr is not None else "kernel changed since the ncu capture, or no capture"),
            "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
            "bytes_per_launch": d["bytes_per_launch"], "avg_launch_us": d["avg_launch_us"],
            "bytes_counted": "scenarios still iterating in each sampled launch",
            "timing": ("device-timer stamps inside the kernels (earliest block start, latest block end) on the "
                       "last iteration of every residual-check chunk, same launch mode as the headline"),
            "kernels": rec,
            "check": {"sampled_iteration_us": round(it_us, 3), "iterations_per_step": iters_per_step,
                      "sampled_ms_per_step": round(it_us * iters_per_step / 1e3, 3),
                      "ms_per_step": round(ms_per_step, 3)}}


def measure(config, args, steps, warmup, dist=None, learned=False, cold=True, scenarios=None, accuracy=False):
    """Time `steps` previous-plan implicit-gradient steps of one workload (after `warmup`
    steps from a cold start), then a profiled pass of the same steps (kernel times and the
    roofline), an end-to-end pass through host buffers, and optionally cold and learned
    starts.  Returns the workload's record (times are the max over ranks)."""
    import torch
    from paper_2410_13055_gb300 import gx
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    nets, scens, shared = build_workload(config, rank, ws, scenarios)
    dh = synth.device_hours(nets, scens)
    net = gx.Network(nets, scens, kappa=KAPPA, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000,
                     check_every=args.check_every, rho=args.rho, inner_iters=args.inner_iters,
                     adj_inner_iters=args.adj_inner_iters)
    net.use_persistent(args.persistent)
    net.use_graphs(args.graphs != "eager", args.graphs == "loop")
    resident = sum(1 for c in net.persistent_info() if c > 0)
    eta_min = torch.tensor(np.concatenate([n["eta_min"] for n in nets]), dtype=torch.float32, device=dev)
    eta_max = torch.tensor(np.concatenate([n["eta_max"] for n in nets]), dtype=torch.float32, device=dev)
    gamma = torch.tensor(np.concatenate([n["gamma"] for n in nets]), dtype=torch.float32, device=dev)
    eta = eta_min.clone()
    grad = torch.zeros_like(eta)
    flush = torch.empty(int(256e6) // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    state = {"alpha": None, "launches": 0, "iters": [], "adj_iters": []}
    reduce_grad = dist is not None and shared

    def step(warm):
        rc = net.solve(eta, warm=warm)
        # previous-plan adjoint state for the small steps of a plan loop (measured faster
        # than the negated-forward-dual start there; the latter wins after large changes)
        net.grad(eta, out=grad, warm="cold" if warm == "cold" else "prev")
        if reduce_grad:
            # the one collective of a plan step: the ranks' partial gradients of one network
            from paper_2410_13055_gb300.sharding import allreduce_sum
            allreduce_sum(grad)
        if state["alpha"] is None:
            d = (gamma + grad).abs().max().item()
            state["alpha"] = 1e-2 * float(eta_min.median().item()) / max(d, 1e-30)
        net.plan_step(eta, grad, gamma, eta_min, eta_max, state["alpha"])
        state["launches"] += net.last_stats["launches"] + net.last_grad_stats["launches"] + 1
        state["iters"].append(net.last_stats["iters_max"])
        state["adj_iters"].append(net.last_grad_stats["iters_max"])
        return rc

    step("cold")  # warm-up (also settles the plan trajectory's step size)
    for _ in range(max(warmup - 1, 0)):
        step("prev")
    torch.cuda.synchronize()
    # kernel schedule picked by the autotuner on this workload's own next step (each
    # candidate from the same restored state; the bus-kernel variants take bitwise the
    # same iterates), untimed; the state is restored afterwards
    tuned = None
    if args.bus_staged is not None:
        net.set_schedule(bus_staged=args.bus_staged)
    elif not args.no_tune and not args.persistent:
        from paper_2410_13055_gb300 import autotune
        def plain_step(e):  # the timed step, without the bookkeeping
            net.solve(e, warm="prev")
            net.grad(e, out=grad, warm="prev")
            if reduce_grad:
                from paper_2410_13055_gb300.sharding import allreduce_sum
                allreduce_sum(grad)
            net.plan_step(e, grad, gamma, eta_min, eta_max, state["alpha"])

        tuned = autotune.tune_schedule_step(net, eta, step=plain_step, steps=args.tune_steps, reps=args.tune_reps,
                                            flush=lambda: flush.fill_(1.0))

    def timed(warm, K):
        state["launches"], state["iters"], state["adj_iters"] = 0, [], []
        evs = []
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push(f"timed_{warm}")  # lets a profiler pick the timed launches
        for _ in range(K):
            flush.fill_(1.0)  # L2 flush between steps, outside the per-step events
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            step(warm)
            b.record()
            evs.append((a, b))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = [a.elapsed_time(b) for a, b in evs]
        state["step_ms"] = ms
        return float(np.sum(ms)), list(state["iters"]), list(state["adj_iters"]), state["launches"]

    def rank_max(*vals):
        if dist is None:
            return list(vals)
        t = torch.tensor(list(vals), dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.tolist()

    clocks = Clocks(local)
    clocks.start()
    # plan and iteration state at the start of the headline steps, so that the e2e pass
    # replays exactly these steps (gx_network_state_range)
    snap = (eta.clone(), net.state(False).clone(), net.state(True).clone())
    ms_prev, it_prev, ait_prev, launches = timed("prev", steps)
    ms_median = float(np.median(state["step_ms"]))
    clk = clocks.stop()
    # kernel times from a second pass of the same steps in the same launch mode: the
    # kernels stamp their sampled launches with the device timer (gx_profile_enable), which
    # stays out of the headline timing
    eta.copy_(snap[0]); net.state(False).copy_(snap[1]); net.state(True).copy_(snap[2])
    net.profile(True)
    ms_prof, pit, pait, _ = timed("prev", steps)
    prof = net.profile_read()
    active = net.profile_active()
    net.profile(False)
    step("prev")  # re-captures the loop graphs (switching the timing drops them), untimed
    ms_step = ms_prev / steps

    # e2e: the same steps through the C ABI with host buffers (pinned): the plan comes from
    # host memory, the plan step runs on the device, and the updated plan, the gradient and
    # the scenario costs go back to host memory, all inside the timed region.  The
    # headline's plan and solver state are restored first, so the pass replays the
    # headline's steps (same iterations) and the difference is the host traffic.
    eta.copy_(snap[0]); net.state(False).copy_(snap[1]); net.state(True).copy_(snap[2])
    e2e_its = []
    eta_h = eta.cpu().pin_memory()
    grad_h = torch.empty_like(grad, device="cpu").pin_memory()
    cost_h = torch.empty(net.S, dtype=torch.float64).pin_memory()
    cost_dev = net.array("cost")
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        eta.copy_(eta_h, non_blocking=True)
        step("prev")
        e2e_its.append((net.last_stats["iters_max"], net.last_grad_stats["iters_max"]))
        eta_h.copy_(eta, non_blocking=True)
        grad_h.copy_(grad, non_blocking=True)
        cost_h.copy_(cost_dev, non_blocking=True)
    b.record()
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / steps

    acc = accuracy_check(net, eta, grad) if accuracy else None
    rec_learned = None
    if learned:
        rec_learned = measure_learned(net, eta, grad, gamma, eta_min, eta_max, state["alpha"], flush, dh, steps, dev)
    ms_cold = None
    it_cold, ait_cold = [], []
    if cold:
        kc = max(1, min(steps, 3))
        ms_cold, it_cold, ait_cold, _ = timed("cold", kc)
        ms_cold /= kc
    ms_step, e2e_ms, ms_median = rank_max(ms_step, e2e_ms, ms_median)
    if ms_cold is not None:
        ms_cold = rank_max(ms_cold)[0]
    value = ws * dh / (ms_step / 1e3)
    iters_step = float(np.mean(pit) + np.mean(pait))
    per_scen = algorithmic_bytes(nets, scens)
    roof = roofline(config, prof, active, per_scen, len(scens), iters_step, ms_step)
    resident_prof = prof.get("k_crs")
    if resident_prof and roof is not None:
        iters = float(sum(pit) + sum(pait))
        roof["resident"] = {"launches": resident_prof["launches"], "ms": round(resident_prof["ms"], 3),
                            "us_per_iteration": round(1e3 * resident_prof["ms"] / max(iters, 1.0), 3)}
    path = ((f"cluster-resident persistent launches for {resident} of {len(scens)} scenarios, "
             "per-iteration kernels (CUDA graphs) for the rest") if args.persistent
            else {"loop": "per-iteration kernels, the whole loop one CUDA graph (device-side convergence test)",
                  "chunk": "per-iteration kernels, one CUDA graph per residual-check chunk",
                  "eager": "per-iteration kernels launched one by one"}[args.graphs])
    return {
        "workload": config, "scenarios": len(scens), "device_hours_per_step": dh, "steps": steps,
        "value": round(value, 1), "ms_per_step": round(ms_step, 4), "ms_per_step_median": round(ms_median, 4),
        "path": path,
        "iterations": {"prev_fwd_median": float(np.median(it_prev)), "prev_adj_median": float(np.median(ait_prev)),
                       "cold_fwd_median": float(np.median(it_cold)) if it_cold else None,
                       "cold_adj_median": float(np.median(ait_cold)) if ait_cold else None},
        "cold": round(ws * dh / (ms_cold / 1e3), 1) if ms_cold else None,
        "learned": rec_learned,
        "roofline": roof,
        "e2e": {"value": round(ws * dh / (e2e_ms / 1e3), 1), "unit": UNIT, "h2d_bytes_per_step": int(eta.numel() * 4),
                "d2h_bytes_per_step": int(2 * eta.numel() * 4 + net.S * 8),
                "replays_headline_steps": [list(x) for x in e2e_its] == [[a, b] for a, b in zip(it_prev, ait_prev)],
                "note": "headline's plan and solver state restored first; no L2 flush between its steps"},
        "clocks": clk, "gpu_launches": int(launches), "alpha": state["alpha"], "accuracy": acc,
        "schedule": {"chosen": net.schedule(), "default": tuned["default"] if tuned else None,
                     "by": "autotune.tune_schedule_step" if tuned else ("--bus-staged" if args.bus_staged is not None
                                                                        else "bind default"),
                     "trials_ms_per_step": ({f"bus{t['bus_staged']}_bat{t['bat_warps']}": t["ms_per_step"]
                                             for t in tuned["trials"]} if tuned else None)},
    }


def tight_reference(net, eta, tight=1e-5, cap=40000, ref_rho=0.3):
    """Cold solve and gradient to `tight` at the library's default penalty (which converges
    further in FP32; the fixed point does not depend on the penalty), the network's options
    restored afterwards.  Returns (weighted objective, gradient, forward stats, adjoint stats);
    the iteration state is left at the reference's."""
    import torch
    from paper_2410_13055_gb300 import gx
    saved = gx.Opts.from_buffer_copy(net.opts)
    g_t = torch.empty(net.K, dtype=torch.float32, device=eta.device)
    net.set_opts(rho=ref_rho, tol=tight, adj_tol=tight, max_iter=cap, adj_max_iter=cap)
    try:
        net.solve(eta, warm="cold")
        fwd = dict(net.last_stats)
        obj_t = float(net.array("obj")[0])
        net.grad(eta, out=g_t, warm="cold")
        adj = dict(net.last_grad_stats)
    finally:
        net.set_opts(saved)
    return obj_t, g_t, fwd, adj


def accuracy_check(net, eta, grad, tight=1e-5, cap=40000, ref_rho=0.3):
    """How far the metric's 1e-3 stop is from a tight solve, at the plan the headline's e2e pass
    ends on (outside every timed region; the plan and iteration state are restored after).
    Metric side: previous-plan solves to 1e-3 at the bench's power penalty, as the next step
    would run them.  Reference: cold solves to `tight` at the library's default penalty, which
    converges further in FP32 (the fixed point does not depend on the penalty); the residuals
    it reached are reported with it."""
    import torch
    snap = (eta.clone(), net.state(False).clone(), net.state(True).clone())
    g_m = torch.empty_like(grad)
    net.solve(eta, warm="prev")
    obj_m = float(net.array("obj")[0])
    net.grad(eta, out=g_m, warm="prev")
    its_m = (net.last_stats["iters_max"], net.last_grad_stats["iters_max"])
    try:
        obj_t, g_t, fwd, adj = tight_reference(net, eta, tight, cap, ref_rho)
    finally:
        eta.copy_(snap[0]); net.state(False).copy_(snap[1]); net.state(True).copy_(snap[2])
    gm, gt = g_m.double(), g_t.double()
    return {"plan": "the plan the headline's e2e pass ends on",
            "grad_rel_err_l2": round(float((gm - gt).norm() / gt.norm().clamp_min(1e-30)), 6),
            "grad_rel_err_max_entry": round(float((gm - gt).abs().max() / gt.abs().max().clamp_min(1e-30)), 6),
            "obj_rel_err": float(abs(obj_m - obj_t) / max(abs(obj_t), 1e-30)),
            "iterations_at_1e-3": list(its_m),
            "reference": {"tol": tight, "rho": ref_rho, "start": "cold", "cap": cap,
                          "forward_converged": f"{fwd['n_converged']}/{fwd['n_scen']}",
                          "adjoint_converged": f"{adj['n_converged']}/{adj['n_scen']}",
                          "forward_residual_max": [fwd["max_primal"], fwd["max_dual"]],
                          "adjoint_residual_max": [adj["max_primal"], adj["max_dual"]],
                          "iterations": [fwd["iters_max"], adj["iters_max"]]}}


def measure_learned(net, eta, grad, gamma, eta_min, eta_max, alpha, flush, dh, steps, dev):
    """The learned start through the C ABI (GX_WARM_LEARNED): the graph network trained by
    paper_2410_13055_gb300.train_warmstart on this network (weights in
    paper_2410_13055_gb300/weights/), its prediction inside the solve, and the selection
    rule (per scenario, the learned start or the previous plan's state, whichever has the
    smaller residual at the first check), on the plan path continued from the headline's.
    Then the learned start alone (no previous solution: gx_network_forget) against a cold
    start on the same plans, both checked against one tight solve at the first of them."""
    import torch
    from paper_2410_13055_gb300 import gx
    wpath = os.path.join(ROOT, "paper_2410_13055_gb300", "weights", "warmstart_medium.npy")
    if not os.path.exists(wpath):
        return None
    gnn = gx.WarmStartGNN(net, seed=0)
    gnn.set_params(np.load(wpath))
    net.attach_gnn(gnn)
    eta_l = eta.clone()
    it_l, ms_l, kept = [], [], []
    torch.cuda.synchronize()
    for _ in range(max(1, min(steps, 5))):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        net.solve(eta_l, warm="learned")
        it_l.append(net.last_stats["iters_max"])
        net.grad(eta_l, out=grad, warm="prev")
        net.plan_step(eta_l, grad, gamma, eta_min, eta_max, alpha)
        b.record()
        torch.cuda.synchronize()
        ms_l.append(a.elapsed_time(b))
        kept.append(float(np.mean(net.array("warm").cpu().numpy() == 1)))
    # no previous solution (gx_network_forget): the learned start alone against a cold start,
    # paired on the same plans, both adjoints from the negated forward duals
    pair = {"cold": {"ms": [], "fwd": [], "adj": []}, "learned": {"ms": [], "fwd": [], "adj": []}}
    first = {}
    for i in range(max(1, min(steps, 3))):
        for mode in ("cold", "learned"):
            net.forget()
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            net.solve(eta_l, warm=mode)
            fwd = net.last_stats["iters_max"]
            net.grad(eta_l, out=grad, warm="cold")
            b.record()
            torch.cuda.synchronize()
            pair[mode]["ms"].append(a.elapsed_time(b))
            pair[mode]["fwd"].append(fwd)
            pair[mode]["adj"].append(net.last_grad_stats["iters_max"])
            if i == 0:
                first[mode] = (float(net.array("obj")[0]), grad.clone())
        if i == 0:
            # both stops against one tight solve at the first plan (untimed)
            obj_t, g_t, _, _ = tight_reference(net, eta_l)
            gt = g_t.double()
            for mode, (obj_m, g_m) in first.items():
                first[mode] = {"obj_rel_err": float(abs(obj_m - obj_t) / max(abs(obj_t), 1e-30)),
                               "grad_rel_err_l2": round(float((g_m.double() - gt).norm() / gt.norm().clamp_min(1e-30)), 6)}
        net.plan_step(eta_l, grad, gamma, eta_min, eta_max, alpha)
    net.attach_gnn(None)
    alone = {m: {"value": round(dh / (float(np.mean(v["ms"])) / 1e3), 1), "fwd_iters_median": float(np.median(v["fwd"])),
                 "adj_iters_median": float(np.median(v["adj"])), "accuracy_first_plan": first.get(m)}
             for m, v in pair.items()}
    alone["steps"] = len(pair["cold"]["ms"])
    alone["note"] = ("gx_network_forget before each solve; solve + gradient on the same plans, the plan stepped "
                     "with the learned run's gradient; no plan step inside the timing")
    return {"value": round(dh / (float(np.mean(ms_l)) / 1e3), 1), "fwd_iters_median": float(np.median(it_l)),
            "kept_learned_fraction": round(float(np.mean(kept)), 4),
            "rule": "GX_WARM_LEARNED: per scenario, learned start or previous plan's by the first check's residual",
            "no_previous_solution": alone,
            "weights": "paper_2410_13055_gb300/weights/warmstart_medium.npy"}


def run_gx(args):
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    head = measure(args.config, args, args.steps, args.warmup, dist,
                   learned=(args.config == "medium" and not args.quick and ws == 1), cold=not args.quick,
                   scenarios=args.scenarios, accuracy=(not args.quick and ws == 1))
    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "ms_per_step": head["ms_per_step"], "iterations": head["iterations"],
                              "roofline": head["roofline"], "launches": head["gpu_launches"]}), flush=True)
        return
    # the workloads where the HBM roofline is judged (medium is L2-resident): a few timed
    # steps each, in the same JSON line
    subs = {}
    if args.config == "medium" and not args.no_sub:
        for cfg, k in (("scale", 3), ("batching", 10)):
            r = measure(cfg, args, k, 3, dist, learned=False, cold=False)
            for key in ("clocks", "learned", "cold", "alpha", "accuracy"):
                r.pop(key, None)
            subs[cfg] = r
    per_scen = None
    if args.config == "batching" and args.per_scenario:
        per_scen = per_scenario_batching(args, head)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = cpu_baseline(args) if not args.no_cpu_baseline else None
    cpu_ref = cpu_reference() if (not args.no_cpu_baseline and args.config == "medium") else None
    out = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "ms_per_step_median": head["ms_per_step_median"],
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.config, "scenarios": head["scenarios"],
                   "device_hours_per_step": head["device_hours_per_step"],
                   "start": "prev (previous plan's dispatch and adjoint state)",
                   "kappa": KAPPA, "rho": args.rho, "inner_iters": args.inner_iters,
                   "adj_inner_iters": args.adj_inner_iters or args.inner_iters,
                   "tol": 1e-3, "l2": "256 MB buffer written between steps, outside the per-step events",
                   "parallelism": f"x{ws} ranks, scenarios sharded (sharding.shard), weak scaling",
                   "path": head["path"]},
        "iterations": head["iterations"],
        "schedule": head["schedule"],
        "modes": {"prev": head["value"], "cold": head["cold"],
                  "learned": head["learned"]["value"] if head["learned"] else None},
        "learned": head["learned"],
        "accuracy": head["accuracy"],
        "roofline": head["roofline"],
        "cpu_baseline": cpu,
        "cpu_reference": cpu_ref,
        "e2e": head["e2e"],
        "clocks": head["clocks"],
        "gpu_launches": head["gpu_launches"],
        "workloads": subs or None,
    }
    if per_scen is not None:
        out["per_scenario"] = per_scen
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def per_scenario_batching(args, head):
    """Batching: the same steps with one network (and launch sequence) per scenario."""
    import torch
    from paper_2410_13055_gb300 import gx
    ws, rank = _dist()
    nets, scens, _ = build_workload("batching", rank, ws)
    offs = np.cumsum([0] + [int(n["K"]) for n in nets])
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    singles = []
    for sc in scens:
        k = sc["net"]
        one = dict(sc, net=0, weight=1.0)
        nt = gx.Network([nets[k]], [one], kappa=KAPPA, tol=1e-3, adj_tol=1e-3, max_iter=50000,
                        adj_max_iter=50000, check_every=args.check_every, rho=args.rho, inner_iters=args.inner_iters,
                        adj_inner_iters=args.adj_inner_iters)
        nt.use_persistent(args.persistent)
        singles.append((nt, nets[k]))
    e_s = [torch.tensor(n["eta_min"], dtype=torch.float32, device=dev) for _, n in singles]
    g_s = [torch.zeros_like(e) for e in e_s]
    aux = [tuple(torch.tensor(n[key], dtype=torch.float32, device=dev) for key in ("gamma", "eta_min", "eta_max"))
           for _, n in singles]
    for (nt, _), e, g in zip(singles, e_s, g_s):  # warm-up: cold then previous-plan
        nt.solve(e, warm="cold"); nt.grad(e, out=g)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    alpha = head["alpha"]
    for _ in range(args.steps):
        for (nt, _), e, g, (gm, lo, hi) in zip(singles, e_s, g_s, aux):
            nt.solve(e, warm="prev")
            nt.grad(e, out=g, warm="prev")
            nt.plan_step(e, g, gm, lo, hi, alpha)
    b.record()
    torch.cuda.synchronize()
    ms_single = a.elapsed_time(b) / args.steps
    return {"batched_ms_per_step": head["ms_per_step"], "per_scenario_ms_per_step": round(ms_single, 3),
            "speedup": round(ms_single / head["ms_per_step"], 2), "scenarios_checked": int(offs.size - 1),
            "note": "same workload, one network and launch sequence per scenario, solved one after another"}


def _cores_used(cpu_s, wall_s):
    return max(1, int(round(cpu_s / max(wall_s, 1e-9))))


def oracle_step(nets, scens, hours):
    """FP64 oracle on the first scenario restricted to `hours` hours: solve + adjoint gradient."""
    from oracle import dispatch, grad as ograd
    n2, s2 = synth.slice_hours(nets, scens[:1], 0, hours)
    opts = synth.default_opts(kappa=KAPPA)
    sol = dispatch.solve(n2[0], s2[0], n2[0]["eta_min"], opts)
    ograd.adjoint_grad(sol)
    return synth.device_hours(n2, s2)


def cpu_baseline(args, hours=24):
    nets, scens, _ = build_workload(args.config)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    dh = oracle_step(nets, scens, hours)
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu_s = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return {"value": round(dh / wall, 2), "unit": UNIT, "cores": _cores_used(cpu_s, wall), "kind": "oracle",
            "sample": f"{args.config} network, scenario 0, hours 0-{hours - 1} ({dh} device-hours): "
                      f"FP64 interior-point dispatch + KKT adjoint gradient, {wall:.1f} s",
            "host_threads_available": os.cpu_count()}


def _timed(fn):
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    out = fn()
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu_s = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return out, wall, _cores_used(cpu_s, wall)


def cpu_probe(which):
    """One CPU timing of the reference points (run in a child process so its thread count can
    be fixed through the environment): the FP64 oracle on the 5-bus case, or on the medium
    network's scenario 0, hours 0-23."""
    if which == "tiny":
        nets, scens = synth.tiny()
        dh, wall, cores = _timed(lambda: oracle_step(nets, scens, 24))
    else:
        nets, scens, _ = build_workload("medium")
        dh, wall, cores = _timed(lambda: oracle_step(nets, scens, 24))
    print(json.dumps({"device_hours": dh, "wall_s": wall, "cores": cores}), flush=True)


def cpu_reference():
    """The CPU reference points of the measurement plan, on the host cores.

    * HiGHS (scipy's LP solver) on one full medium scenario (100 buses, 168 h) with eps = 0:
      the library LP at full size, where the interior-point oracle does not fit.  Dispatch
      only: an LP solver gives no implicit gradient.
    * The FP64 oracle (interior point + KKT adjoint gradient) on the 5-bus case (in full),
      with every host thread and with one, and on the medium slice with one thread (the
      all-thread slice is cpu_baseline)."""
    from scipy.optimize import linprog
    from oracle.qp import DispatchQP
    out = {}
    nets, scens, _ = build_workload("medium")
    qp = DispatchQP(nets[0], scens[0], nets[0]["eta_min"], synth.default_opts(eps=0.0))
    res, wall, cores = _timed(lambda: linprog(qp.q, A_ub=qp.Gm, b_ub=qp.h, A_eq=qp.A, b_eq=qp.b,
                                              bounds=(None, None), method="highs"))
    dh = synth.device_hours(nets, scens[:1])
    out["highs_lp_medium_scenario"] = {"value": round(dh / wall, 2), "unit": UNIT, "wall_s": round(wall, 2),
                                       "cores": cores, "status": int(res.status),
                                       "sample": "medium network, scenario 0, 168 h, eps = 0 LP (dispatch only)"}
    env1 = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for name, which, env in (("oracle_tiny", "tiny", None), ("oracle_tiny_1thread", "tiny", env1),
                             ("oracle_medium_slice_1thread", "slice", env1)):
        r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-probe", which],
                           capture_output=True, text=True, env=env or dict(os.environ), timeout=600)
        try:
            d = json.loads(r.stdout.strip().splitlines()[-1])
            out[name] = {"value": round(d["device_hours"] / d["wall_s"], 2), "unit": UNIT,
                         "wall_s": round(d["wall_s"], 2), "cores": d["cores"],
                         "sample": ("5-bus case, 24 h, in full" if which == "tiny" else
                                    "medium network, scenario 0, hours 0-23") +
                                   ": FP64 interior-point dispatch + KKT adjoint gradient"}
        except Exception:
            out[name] = {"error": (r.stderr or r.stdout)[-300:]}
    out["host_threads_available"] = os.cpu_count()
    return out


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    nets, scens, _ = build_workload(args.config)
    hours = 6
    for _ in range(args.warmup):
        oracle_step(nets, scens, hours)
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    dh = 0
    for _ in range(args.steps):
        dh += oracle_step(nets, scens, hours)
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu_s = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    v = dh / wall
    sample = (f"{args.config} network, scenario 0, hours 0-{hours - 1} per step: FP64 interior-point dispatch + "
              f"KKT adjoint gradient")
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * wall / args.steps, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.config, "kappa": KAPPA, "sample_hours": hours},
           "cpu_baseline": {"value": round(v, 2), "unit": UNIT, "cores": _cores_used(cpu_s, wall), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(v, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="medium")
    ap.add_argument("--impl", default="gx", choices=["gx", "reference"])
    ap.add_argument("--check-every", type=int, default=20)
    # Power penalty of the dispatch.  At the 1e-3 tolerance 0.2 beats the library default
    # 0.3 on every workload's previous-plan steps (medium +24 %, Scale +47 %) with a
    # slightly more accurate gradient (4.9 % vs 5.6 % mean error against tight solves on
    # five medium plans); the default 0.3 converges better to tight tolerances.
    ap.add_argument("--rho", type=float, default=0.2)
    ap.add_argument("--inner-iters", type=int, default=2, help="battery inner iterations per outer iteration")
    ap.add_argument("--adj-inner-iters", type=int, default=1,
                    help="battery inner iterations per adjoint iteration (0: --inner-iters); one is faster on "
                         "every workload here")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--scenarios", type=int, default=None,
                    help="scenario count of the medium (default 16) or scale (default 52) workload")
    ap.add_argument("--quick", action="store_true", help="timed previous-plan steps only (profiling runs)")
    ap.add_argument("--persistent", action="store_true",
                    help="cluster-resident persistent launches for the scenarios that fit shared memory")
    ap.add_argument("--graphs", default="loop", choices=["loop", "chunk", "eager"],
                    help="launch mode of the iteration kernels: the whole loop as one graph with a device-side "
                         "convergence test (default), one graph per residual-check chunk (ncu cannot profile the "
                         "kernel nodes of a graph with conditional nodes), or kernel by kernel")
    ap.add_argument("--per-scenario", action="store_true",
                    help="batching config: also time one network and launch sequence per scenario")
    ap.add_argument("--no-sub", action="store_true",
                    help="medium config: skip the scale and batching sub-records")
    ap.add_argument("--tune-steps", type=int, default=2, help="previous-plan steps per schedule trial")
    ap.add_argument("--tune-reps", type=int, default=2, help="repetitions of each schedule trial (best kept)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's default kernel schedule instead of autotuning it per workload")
    ap.add_argument("--bus-staged", type=int, default=None, choices=[0, 1, 2],
                    help="force the bus kernel variant (gx_network_set_schedule) instead of autotuning it")
    ap.add_argument("--cpu-probe", default=None, choices=["tiny", "slice"], help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_probe:
        cpu_probe(args.cpu_probe)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gx(args)


if __name__ == "__main__":
    main()
