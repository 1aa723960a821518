"""Uneven batches, full-size workloads and edge cases on the GPU."""
import numpy as np
import pytest

from cases import network, scenario
from gpu_util import eta_tensor, gpu_net, pack_x, ref_groups, rel, solution
from oracle import dispatch, grad as ograd, kkt
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-6, max_iter=200000, adj_tol=1e-5, adj_max_iter=200000, check_every=50)


def _small_uneven():
    """Three networks of different sizes with ragged horizons (T = 5, 24, 13)."""
    nets, scens = [], []
    for k, (nb, nl, ng, nbt, T) in enumerate([(6, 8, 14, 2, 5), (9, 13, 20, 3, 24), (4, 5, 9, 1, 13)]):
        net, sc = synth.custom(nb, nl, ng, nbt, T, S=1, seed=40 + k, net_index=k)
        sc[0]["weight"] = 1.0 / 3
        nets.append(net)
        scens.append(sc[0])
    return nets, scens


def test_uneven_batch_matches_oracle_per_scenario():
    nets, scens = _small_uneven()
    eta = np.concatenate([n["eta_min"] for n in nets])
    net = gpu_net(nets, scens, kappa=50.0, **TIGHT)
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    g = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0
    refs = dispatch.solve_all(nets, scens, eta, synth.default_opts(kappa=50.0))
    off = 0
    for s, ref in enumerate(refs):
        sol = solution(net, s, ref_groups(ref.qp))
        assert abs(sol["cost"] - ref.cost) / ref.cost <= 1e-4, s
        assert rel(sol["price"], ref.price) <= 1e-3, s
        K = nets[s]["K"]
        gs = net.array("grad_s", s).cpu().numpy()
        assert rel(gs, ograd.adjoint_grad(ref)) <= 1e-3, s
        # the combined gradient of a network that only one scenario uses is w_s dh_s
        assert rel(g[off:off + K], scens[s]["weight"] * gs) <= 1e-5
        off += K


def test_batch_subset_leaves_other_scenarios_untouched():
    nets, scens = synth.tiny()
    s2 = [dict(scens[0]), dict(scens[0])]
    s2[1]["load"] = scens[0]["load"] * 0.9
    for s in s2:
        s["weight"] = 0.5
    net = gpu_net(nets, s2, **TIGHT)
    e = eta_tensor(nets[0]["eta_min"])
    assert net.solve(e, batch=[1]) == 0
    p0 = net.array("p", 0).cpu().numpy()
    assert np.all(p0 == 0.0)  # scenario 0 was never solved
    ref = dispatch.solve(nets[0], s2[1], nets[0]["eta_min"], synth.default_opts())
    assert abs(float(net.array("cost", 1).cpu()[0]) - ref.cost) / ref.cost <= 1e-4


def test_no_lines_no_batteries_single_hour():
    """Degenerate shapes: one bus, no lines, no batteries, T = 1."""
    net_d, eta = network(1, gens=[(0, 20.0, 100.0), (0, 40.0, 100.0)])
    sc = scenario([[150.0]], G=2)
    net = gpu_net([net_d], [sc], **TIGHT)
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    p = net.array("p", 0).cpu().numpy()
    ref = dispatch.solve(net_d, sc, eta, synth.default_opts())
    np.testing.assert_allclose(p, ref.p, atol=1e-2)
    g = net.grad(e).cpu().numpy()
    np.testing.assert_allclose(g, ograd.adjoint_grad(ref), rtol=1e-3, atol=1e-3)


@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_user_warm_start_from_oracle_prices_converges_fast(tol):
    """Starting from the oracle's prices and angles beats a cold start at the bench's
    tolerance and at 1e-5.  (Near the FP32 floor, 1e-6, the last decade's iteration count
    is dominated by rounding noise and either start can take longer.)"""
    import torch
    nets, scens = synth.tiny()
    eta = nets[0]["eta_min"]
    ref = dispatch.solve(nets[0], scens[0], eta, synth.default_opts())
    net = gpu_net(nets, scens, **{**TIGHT, "tol": tol})
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    cold_iters = net.last_stats["iters_max"]
    inf = net.info[0]
    pr = torch.zeros(inf["N"], inf["Tp"], device="cuda")
    th = torch.zeros_like(pr)
    pr[:, :inf["T"]] = torch.tensor(ref.price, dtype=torch.float32)
    th[:, :inf["T"]] = torch.tensor(ref.th, dtype=torch.float32)
    assert net.solve(e, warm="user", warm_prices=pr, warm_angles=th) == 0
    assert net.last_stats["iters_max"] < (0.5 if tol >= 1e-3 else 0.9) * cold_iters


def test_iteration_cap_reports_not_converged():
    nets, scens = synth.tiny()
    net = gpu_net(nets, scens, tol=1e-9, max_iter=40, check_every=20)
    rc = net.solve(eta_tensor(nets[0]["eta_min"]))
    assert rc == 1
    assert int(net.array("status", 0).cpu()[0]) == 1
    assert int(net.array("iters", 0).cpu()[0]) == 40


def test_medium_full_size_properties():
    """16 x 168 h at the bench's tolerance: every scenario converges; balance holds;
    bounds hold; the gradient agrees with a GPU central difference along a random
    direction (solves at 1e-6); sampled scenario cost within 1e-3 of the oracle on
    its first 24 hours is not comparable (coupled horizon), so the check uses the
    planner identity h = cost + kappa * emissions instead."""
    import torch
    nets, scens = synth.medium()
    eta = nets[0]["eta_min"] * 1.05
    kappa = 50.0
    net = gpu_net(nets, scens, kappa=kappa, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    assert net.last_stats["n_converged"] == 16
    for s in (0, 7, 15):
        p = net.array("p", s).cpu().numpy()
        cap = (eta[:300][:, None] * scens[s]["cf"]).astype(np.float32)
        assert np.all(p >= 0) and np.all(p <= cap * (1 + 1e-6) + 1e-4)
        sh = net.array("shed", s).cpu().numpy()
        assert np.all(sh >= -1e-4) and np.all(sh <= scens[s]["load"] + 1e-3)
    g = net.grad(e)
    assert net.last_grad_status == 0
    # directional derivative of sum_s w_s h_s, tight solves
    tight = gpu_net(nets, scens, kappa=kappa, tol=1e-6, max_iter=200000, check_every=100)
    rng = np.random.default_rng(0)
    d = rng.standard_normal(eta.size) * eta * 1e-3
    vals = []
    for sgn in (+1, -1):
        assert tight.solve(eta_tensor(eta + sgn * d)) in (0, 1)
        torch.cuda.synchronize()
        hs = tight.array("h").cpu().numpy()
        vals.append(float(np.sum(hs * np.array([sc["weight"] for sc in scens]))))
    fd = (vals[0] - vals[1]) / 2.0
    lin = float(np.dot(g.double().cpu().numpy(), d))
    assert abs(fd - lin) <= 2e-2 * abs(fd), (fd, lin)


@pytest.mark.parametrize("case", ["tiny", "medium4"])
def test_graph_modes_match_eager_launches_bitwise(case):
    """The device-side loop (one graph with a conditional WHILE node), one graph per chunk
    and kernel-by-kernel launches run the same kernels in the same order: identical
    iteration counts and bitwise-identical dispatch and gradient, forward and adjoint,
    over two plan steps (the second from the previous plan's state)."""
    nets, scens = synth.tiny() if case == "tiny" else synth.medium(S=4, T=48)
    e0 = eta_tensor(np.concatenate([n["eta_min"] for n in nets]))
    out = []
    for mode in ((True, True), (True, False), (False, True)):
        net = gpu_net(nets, scens, kappa=50.0, tol=1e-5, adj_tol=1e-4, max_iter=50000, adj_max_iter=50000)
        net.use_graphs(*mode)
        e = e0.clone()
        res = []
        for k in range(2):
            assert net.solve(e, warm="cold" if k == 0 else "prev") == 0
            f_it = net.last_stats["iters_max"]
            g = net.grad(e, warm="cold" if k == 0 else "prev").cpu().numpy().copy()
            res.append((net.array("p").cpu().numpy().copy(), g, f_it, net.last_grad_stats["iters_max"]))
            e = (e * 1.01).contiguous()
        out.append(res)
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert a[2] == b[2] and a[3] == b[3]
            assert np.array_equal(a[0], b[0])
            assert np.array_equal(a[1], b[1])


def test_device_loop_respects_the_iteration_cap():
    """With a cap below the iterations needed, the device-side loop stops at the cap and
    reports GX_NOT_CONVERGED, like the host-checked loop."""
    nets, scens = synth.tiny()
    e = eta_tensor(nets[0]["eta_min"])
    for mode in ((True, True), (True, False)):
        net = gpu_net(nets, scens, kappa=50.0, tol=1e-9, max_iter=60, check_every=20)
        net.use_graphs(*mode)
        assert net.solve(e) == 1
        assert net.last_stats["iters_max"] == 60 and net.last_stats["n_converged"] == 0


def test_scale_full_size_properties():
    """The full Scale workload (2000 buses, 52 x 168 h) at the bench's 1e-3 tolerance,
    checked through properties that hold at any size (the dense oracle cannot hold it):
    every scenario converges; on sampled scenarios bounds hold, every bus-hour's power
    balance computed from the reported injections, flows and battery powers is within
    the residual tolerance, flows respect their limits, and prices satisfy the generator
    optimality condition lambda = c + eps p at generators strictly inside their bounds;
    with kappa = 0 (h = cost) every capacity gradient entry is <= 0."""
    nets, scens = synth.scale()
    n = nets[0]
    G, L = n["gen_bus"].size, n["line_from"].size
    eta = n["eta_min"] * 1.05
    eps = synth.default_opts()["eps"]
    net = gpu_net(nets, scens, kappa=0.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    assert net.last_stats["n_converged"] == 52
    for s in (0, 25, 51):
        sc = scens[s]
        p = net.array("p", s).double().cpu().numpy()
        cap = eta[:G][:, None] * sc["cf"]
        assert np.all(p >= -1e-4) and np.all(p <= cap * (1 + 1e-5) + 1e-3)
        sh = net.array("shed", s).double().cpu().numpy()
        assert np.all(sh >= -1e-3) and np.all(sh <= sc["load"] + 1e-3)
        f = net.array("flow", s).double().cpu().numpy()
        assert np.all(np.abs(f) <= eta[G:G + L][:, None] * (1 + 1e-5) + 1e-3)
        ch = net.array("ch", s).double().cpu().numpy()
        dis = net.array("dis", s).double().cpu().numpy()
        inj = np.zeros_like(sc["load"])
        np.add.at(inj, n["gen_bus"], p)
        np.add.at(inj, n["bat_bus"], dis - ch)
        inj += sh - sc["load"]
        np.add.at(inj, n["line_from"], -f)
        np.add.at(inj, n["line_to"], f)
        # the primal residual bounds |imbalance| / |load| by the tolerance; the reported
        # battery powers are the inner box copies, within the inner residual of the x-step
        assert np.linalg.norm(inj) <= 5e-3 * np.linalg.norm(sc["load"]), np.linalg.norm(inj) / np.linalg.norm(sc["load"])
        lam = net.array("price", s).double().cpu().numpy()
        interior = (p > 1.0) & (p < cap - 1.0)
        lam_g = lam[n["gen_bus"]]
        stat = np.abs(lam_g - (n["gen_cost"][:, None] + eps * p))[interior]
        # a 1e-3 relative dual residual on prices of tens of $/MWh
        assert np.median(stat) <= 0.05 and np.quantile(stat, 0.99) <= 0.5, (np.median(stat), np.quantile(stat, 0.99))
    g = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0
    assert np.max(g) <= 1e-3 * np.max(np.abs(g)), np.max(g)


def test_set_opts_between_solve_and_grad():
    """Changing the adjoint penalty after a solve takes effect in the next gradient call
    (its battery pivots are refreshed there too): the gradient equals that of a network
    created with the new penalty, bit for bit."""
    import torch
    nets, scens = synth.medium(S=2, T=48)
    e = eta_tensor(nets[0]["eta_min"] * 1.05)
    kw = dict(kappa=50.0, tol=1e-4, adj_tol=1e-4, max_iter=50000, adj_max_iter=50000)
    a = gpu_net(nets, scens, adj_rho=0.002, **kw)
    assert a.solve(e) == 0
    a.grad(e)
    a.set_opts(adj_rho=0.004)
    g_a = a.grad(e, warm="cold").clone()
    it_a = a.last_grad_stats["iters_max"]
    b = gpu_net(nets, scens, adj_rho=0.004, **kw)
    assert b.solve(e) == 0
    g_b = b.grad(e, warm="cold").clone()
    assert a.last_grad_status == 0 and b.last_grad_status == 0
    assert it_a == b.last_grad_stats["iters_max"]
    assert torch.equal(g_a, g_b)
