"""The learned warm start: trained on the GPU by the project's kernels on solutions the
solver produces; what it gains over a cold start on held-out plans; its selection rule
through the C ABI (GX_WARM_LEARNED); and the bound that keeps any price/angle predictor
from beating the previous plan's start on a plan step."""
import numpy as np
import pytest
import torch

from paper_2410_13055_gb300 import gx, synth
from paper_2410_13055_gb300.warmstart import compare_starts, make_dataset, targets, train

pytestmark = pytest.mark.gpu


def _rmse(gnn, net, eta):
    net.solve(eta, warm="cold")
    tgt = targets(net)
    M = tgt.numel() // 2
    pred = gnn.predict(eta)
    return float(torch.sqrt(torch.mean((pred[:M].clamp(0, 200) - tgt[:M]) ** 2)))


def test_trained_network_beats_untrained_and_cold_start():
    nets, scens = synth.medium(S=4)
    net = gx.Network(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    samples = make_dataset(net, nets, [150.0, 250.0, 350.0], steps=4, keep_every=2, n_perturb=1, seed=100)
    test = make_dataset(net, nets, [200.0, 300.0], steps=2, keep_every=2, n_perturb=1, seed=1000)
    gnn = gx.WarmStartGNN(net, seed=3)
    e_test = [e for e, _ in test]
    before = np.median([_rmse(gnn, net, e) for e in e_test])
    train(gnn, samples, epochs=25, lr=2e-3, w_theta=0.1)
    after = np.median([_rmse(gnn, net, e) for e in e_test])
    assert after < before / 3, (before, after)
    rows = compare_starts(net, gnn, [(e_test[i], e_test[i + 1]) for i in range(0, len(e_test) - 1, 2)])
    cold = np.median([r["cold"]["fwd"] for r in rows])
    learned = np.median([r["learned"]["fwd"] for r in rows])
    assert learned <= cold, (cold, learned, [r["prev"]["fwd"] for r in rows])


def _medium_net(S=4, T=48):
    nets, scens = synth.medium(S=S, T=T)
    net = gx.Network(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000, rho=0.2)
    return nets, net


def _next_plan(net, nets, eta, frac=1e-2):
    g = net.grad(eta, warm="prev")
    gamma = torch.tensor(nets[0]["gamma"], dtype=torch.float32, device="cuda")
    lo = torch.tensor(nets[0]["eta_min"], dtype=torch.float32, device="cuda")
    hi = torch.tensor(nets[0]["eta_max"], dtype=torch.float32, device="cuda")
    alpha = frac * float(lo.median()) / float((gamma + g).abs().max())
    e2 = eta.clone()
    net.plan_step(e2, g, gamma, lo, hi, alpha)
    return e2


def test_learned_mode_selection_rule_through_the_abi():
    import os
    nets, net = _medium_net()
    eta = torch.tensor(nets[0]["eta_min"] * 1.05, dtype=torch.float32, device="cuda")
    with pytest.raises(gx.GxError) as e:
        net.solve(eta, warm="learned")  # no network attached
    assert e.value.status == -6
    gnn = gx.WarmStartGNN(net, seed=0)
    w = os.path.join(os.path.dirname(gx.__file__), "weights", "warmstart_medium.npy")
    gnn.set_params(np.load(w))
    net.attach_gnn(gnn)
    # no previous solution: every scenario takes the learned start
    assert net.solve(eta, warm="learned") == 0
    torch.cuda.synchronize()
    assert np.all(net.array("warm").cpu().numpy() == 1)
    e2 = _next_plan(net, nets, eta)
    sx, sa = net.state(False).clone(), net.state(True).clone()
    assert net.solve(e2, warm="prev") == 0
    it_prev = net.array("iters").cpu().numpy().copy()
    cost_prev = net.array("cost").cpu().numpy().copy()
    net.state(False).copy_(sx)
    net.state(True).copy_(sa)
    assert net.solve(e2, warm="learned") == 0
    torch.cuda.synchronize()
    chosen = net.array("warm").cpu().numpy()
    it_l = net.array("iters").cpu().numpy()
    assert set(chosen.tolist()) <= {0, 1}
    # the rule costs at most one trial chunk over the start it keeps: where the previous
    # plan's start won, its iterations are those of the plain previous-plan solve
    every = net.opts.check_every
    assert np.all(it_l[chosen == 0] == it_prev[chosen == 0]), (chosen, it_l, it_prev)
    assert np.all(it_l <= np.maximum(it_prev, every) + 5000)
    assert np.allclose(net.array("cost").cpu().numpy(), cost_prev, rtol=2e-3)
    # with the previous solution dropped, every scenario takes the learned start again
    net.forget()
    with pytest.raises(gx.GxError) as e:
        net.grad(e2, warm="prev")
    assert e.value.status == -6
    assert net.solve(e2, warm="learned") == 0
    torch.cuda.synchronize()
    assert np.all(net.array("warm").cpu().numpy() == 1)
    assert np.all(net.array("status").cpu().numpy() == 0)


def test_exact_prices_do_not_beat_the_previous_plan_start():
    """The bound behind the learned start's result: even the exact prices and angles of the
    new plan's solution (what a perfect predictor would output), applied as a start, need
    more forward iterations than the previous plan's full state: the slow modes of the
    iteration are in the device-side state (battery schedules, line phase copies), not in
    the prices."""
    nets, net = _medium_net(S=4, T=168)
    eta = torch.tensor(nets[0]["eta_min"] * 1.05, dtype=torch.float32, device="cuda")
    net.solve(eta, warm="cold")
    e2 = _next_plan(net, nets, eta)
    sx = net.state(False).clone()
    net.solve(e2, warm="prev")
    it_prev = net.last_stats["iters_max"]
    price, theta = net.array("price").clone(), net.array("theta").clone()
    net.state(False).copy_(sx)
    net.solve(e2, warm="user", warm_prices=price, warm_angles=theta)
    it_exact = net.last_stats["iters_max"]
    assert it_exact > it_prev, (it_exact, it_prev)
