"""Train the learned warm start on the 100-bus network and compare it with cold and
previous-plan starts.

    python -m paper_2410_13055_gb300.train_warmstart --out weights.npy --report report.json

Training data: plans along implicit-gradient paths for battery capital costs
$100-400/kWh in $25 steps (Section 3.3's sweep), plus log-normal(0, sigma)
perturbations of them, each solved by the CUDA solver.  Test pairs (seeded
separately): (plan at cost c, plan at cost c +- $25) and (consecutive plans on a
path); each start is timed to a 1e-3 residual for the dispatch and the adjoint.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import gx, synth
from .warmstart import compare_starts, gamma_for_battery_cost, make_dataset, plan_path, targets, train

KAPPA = 50.0


def build(seed=1, S=16):
    nets, scens = synth.medium(seed=seed, S=S)
    net = gx.Network(nets, scens, kappa=KAPPA, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    return nets, scens, net


def test_pairs(net, nets, n_pairs, seed=1000, steps=10, alpha_frac=4e-2):
    rng = np.random.default_rng(seed)
    dev = net.device
    eta_min = torch.tensor(nets[0]["eta_min"], dtype=torch.float32, device=dev)
    eta_max = torch.tensor(nets[0]["eta_max"], dtype=torch.float32, device=dev)
    T = net.info[0]["T"]
    pairs = []
    for k in range(n_pairs):
        c = float(rng.uniform(175.0, 325.0))
        ends = []
        for cc in (c, c + (75.0 if rng.random() < 0.5 else -75.0)):
            gamma = torch.tensor(gamma_for_battery_cost(nets[0], cc, T), dtype=torch.float32, device=dev)
            g0 = torch.zeros_like(eta_min)
            net.solve(eta_min, warm="cold")
            net.grad(eta_min, out=g0)
            alpha = alpha_frac * float(eta_min.median()) / max(float((gamma + g0).abs().max()), 1e-30)
            path = plan_path(net, nets, eta_min, gamma, eta_min, eta_max, alpha, steps)
            ends.append(path)
        if k % 2 == 0:
            pairs.append(("cost", ends[0][-1], ends[1][-1]))
        else:
            pairs.append(("step", ends[0][-2], ends[0][-1]))
    return pairs


def time_kernels(reps=20, S=16):
    """CUDA-event time of one prediction and one training step (with its loss read-back) of
    the warm-start network on the medium network (S x 168 h scenarios)."""
    nets, scens, net = build(S=S)
    gnn = gx.WarmStartGNN(net, seed=7)
    eta = torch.tensor(nets[0]["eta_min"], dtype=torch.float32, device="cuda")
    out = torch.empty(2 * gnn.M, dtype=torch.float32, device="cuda")
    tgt = torch.randn(2 * gnn.M, dtype=torch.float32, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"rows": gnn.M, "reps": reps}
    for name, fn in (("predict_us", lambda: gnn.predict(eta, out)),
                     ("train_step_us", lambda: gnn.train_step(eta, tgt, lr=1e-4))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        res[name] = round(1e3 * a.elapsed_time(b) / reps, 1)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--time-kernels", action="store_true",
                    help="only time one prediction and one training step on the medium network")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--out", default=None)
    ap.add_argument("--report", default=None)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--pairs", type=int, default=20)
    ap.add_argument("--costs", type=int, default=13)
    ap.add_argument("--w-theta", type=float, default=0.1)
    ap.add_argument("--weights", default=None, help="evaluate these parameters instead of training")
    args = ap.parse_args(argv)
    if args.time_kernels:
        print(json.dumps(time_kernels(args.reps)), flush=True)
        return
    t0 = time.time()
    nets, scens, net = build()
    gnn = gx.WarmStartGNN(net, seed=7)
    samples, hist, t_data, t_train = [], [float("nan")], 0.0, 0.0
    if args.weights:
        gnn.set_params(np.load(args.weights))
    else:
        costs = list(np.linspace(100.0, 400.0, args.costs))
        samples = make_dataset(net, nets, costs, steps=8, keep_every=2, n_perturb=2, sigma=0.1, seed=100)
        t_data = time.time() - t0
        t1 = time.time()
        hist = train(gnn, samples, epochs=args.epochs, lr=args.lr, w_theta=args.w_theta,
                     log=lambda m: print(m, flush=True))
        torch.cuda.synchronize()
        t_train = time.time() - t1
    if args.out:
        np.save(args.out, gnn.params())
    pairs = test_pairs(net, nets, args.pairs)
    rows = compare_starts(net, gnn, [(a, b) for _, a, b in pairs])
    summ = {}
    for mode in ("cold", "prev", "learned", "learned_only"):
        summ[mode] = {k: float(np.median([r[mode][k] for r in rows])) for k in ("fwd", "adj", "ms")}
    summ["learned"]["kept_learned"] = float(np.mean([r["learned"]["kept_learned"] for r in rows]))
    tot = lambda r, m: r[m]["fwd"] + r[m]["adj"]
    wins = sum(1 for r in rows if tot(r, "learned") < tot(r, "prev"))
    wins_only = sum(1 for r in rows if tot(r, "learned_only") < tot(r, "prev"))
    wins_cold = sum(1 for r in rows if tot(r, "learned_only") < tot(r, "cold"))
    # prediction error on held-out plans (the first scenario-hours of each test plan)
    errs = []
    for _, _, eta_b in pairs:
        net.solve(eta_b, warm="cold")
        tgt = targets(net)
        pred = gnn.predict(eta_b)
        M = tgt.numel() // 2
        errs.append(float(torch.sqrt(torch.mean((pred[:M].clamp(0, 200) - tgt[:M]) ** 2))))
    rep = dict(samples=len(samples), data_s=t_data, train_s=t_train, loss_first=hist[0], loss_last=hist[-1],
               price_rmse_test=float(np.median(errs)),
               pairs=len(rows), kinds=[k for k, _, _ in pairs], median=summ, learned_beats_prev=wins,
               learned_only_beats_prev=wins_only, learned_only_beats_cold=wins_cold,
               fallback_rate=1.0 - summ["learned"]["kept_learned"], rows=rows)
    print(json.dumps({k: v for k, v in rep.items() if k != "rows"}), flush=True)
    if args.report:
        json.dump(rep, open(args.report, "w"), indent=1)


if __name__ == "__main__":
    main()
