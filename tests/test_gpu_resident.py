"""The cluster-resident persistent path (one launch per forward or adjoint loop, state
in thread-block-cluster shared memory) against the FP64 oracle and against the
per-iteration kernels on the same inputs."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net, pack_x, ref_groups, rel, solution
from oracle import dispatch, grad as ograd, kkt
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-6, max_iter=200000, adj_tol=1e-5, adj_max_iter=200000, check_every=50)
ACT_TOL = 1e-3


def _resident(nets, scens, **kw):
    net = gpu_net(nets, scens, **kw)
    net.use_persistent(True)
    return net


def _small_uneven():
    nets, scens = [], []
    for k, (nb, nl, ng, nbt, T) in enumerate([(6, 8, 14, 2, 5), (9, 13, 20, 3, 24), (4, 5, 9, 1, 13)]):
        net, sc = synth.custom(nb, nl, ng, nbt, T, S=1, seed=40 + k, net_index=k)
        sc[0]["weight"] = 1.0 / 3
        nets.append(net)
        scens.append(sc[0])
    return nets, scens


@pytest.mark.parametrize("kappa", [0.0, 50.0])
def test_resident_tiny_matches_oracle(kappa):
    nets, scens = synth.tiny()
    eta = nets[0]["eta_min"] * 1.1
    net = _resident(nets, scens, kappa=kappa, **TIGHT)
    assert net.persistent_info() == [1]
    e = eta_tensor(eta)
    assert net.solve(e) == 0, net.last_stats
    assert net.last_stats["launches"] < 40  # the loop is one launch, not one per iteration
    ref = dispatch.solve(nets[0], scens[0], eta, synth.default_opts(kappa=kappa))
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0, net.last_grad_stats
    assert rel(gg, ograd.adjoint_grad(ref)) <= 1e-3


def test_resident_uneven_batch_matches_oracle():
    """Three networks, ragged horizons (5, 24, 13 h): each scenario its own cluster."""
    nets, scens = _small_uneven()
    eta = np.concatenate([n["eta_min"] for n in nets])
    net = _resident(nets, scens, kappa=50.0, **TIGHT)
    assert all(c >= 1 for c in net.persistent_info())
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    net.grad(e)
    assert net.last_grad_status == 0
    refs = dispatch.solve_all(nets, scens, eta, synth.default_opts(kappa=50.0))
    for s, ref in enumerate(refs):
        sol = solution(net, s, ref_groups(ref.qp))
        assert abs(sol["cost"] - ref.cost) / ref.cost <= 1e-4, s
        assert rel(sol["price"], ref.price) <= 1e-3, s
        assert rel(net.array("grad_s", s).cpu().numpy(), ograd.adjoint_grad(ref)) <= 1e-3, s


def _run(nets, scens, persistent, steps=3, batch=None, **kw):
    import torch
    net = gpu_net(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000, **kw)
    net.use_persistent(persistent)
    dev = torch.device("cuda")
    cat = lambda k: torch.tensor(np.concatenate([n[k] for n in nets]), dtype=torch.float32, device=dev)
    emin, emax, gam = cat("eta_min"), cat("eta_max"), cat("gamma")
    eta = emin.clone()
    g = torch.zeros_like(eta)
    out = []
    for k in range(steps):
        w = "cold" if k == 0 else "prev"
        net.solve(eta, warm=w, batch=batch)
        f = net.last_stats["iters_max"]
        net.grad(eta, out=g, warm=w)
        h = net.array("h").double().cpu().numpy().copy()
        out.append((f, net.last_grad_stats["iters_max"], h, g.double().cpu().numpy().copy()))
        net.plan_step(eta, g, gam, emin, emax, 1e-3)
    return net, out


def test_resident_matches_iteration_kernels_on_medium():
    """Same iterates up to the summation order of the residual partials: equal iteration
    counts, objectives and gradients to FP32 rounding over three plan steps."""
    nets, scens = synth.medium(S=4)
    net1, a = _run(nets, scens, False)
    net2, b = _run(nets, scens, True)
    assert net1.persistent_info() == [0] * 4
    assert all(c > 0 for c in net2.persistent_info())
    for (f1, a1, h1, g1), (f2, a2, h2, g2) in zip(a, b):
        assert (f1, a1) == (f2, a2)
        assert np.max(np.abs(h1 - h2) / np.abs(h1)) <= 1e-5
        assert rel(g2, g1) <= 1e-4


def test_mixed_resident_and_streaming_batch():
    """A scenario too large for a cluster's shared memory runs on the per-iteration
    kernels in the same call as resident ones; results match the all-streaming run and
    a batch subset leaves the other scenarios untouched."""
    big, sb = synth.custom(700, 1050, 2100, 200, 168, S=1, seed=71, net_index=0)
    small, ss = synth.custom(12, 18, 36, 4, 24, S=2, seed=72, net_index=1)
    nets = [big, small]
    scens = [sb[0]] + ss
    for s in scens:
        s["weight"] = 1.0 / 3
    net1, a = _run(nets, scens, False, steps=2)
    net2, b = _run(nets, scens, True, steps=2)
    info = net2.persistent_info()
    assert info[0] == 0 and info[1] > 0 and info[2] > 0, info
    for (f1, a1, h1, g1), (f2, a2, h2, g2) in zip(a, b):
        assert (f1, a1) == (f2, a2)
        assert np.max(np.abs(h1 - h2) / np.abs(h1)) <= 1e-5
        assert rel(g2, g1) <= 1e-4
    # batch of the resident scenarios only: the large one keeps its previous state
    import torch
    p_big = net2.array("p", 0).clone()
    e = torch.tensor(np.concatenate([n["eta_min"] for n in nets]), dtype=torch.float32, device="cuda")
    assert net2.solve(e, warm="cold", batch=[1, 2]) == 0
    assert torch.equal(net2.array("p", 0), p_big)


def test_resident_groups_sharing_one_kernel():
    """Networks of one horizon class but different sizes: their clusters differ in size
    and shared-memory image yet share one kernel instantiation (launch groups of several
    sizes in one call); results match the per-iteration kernels."""
    nets, scens = [], []
    for k, nb in enumerate([8, 60, 140, 260]):
        n, sc = synth.custom(nb, int(1.5 * nb), 3 * nb, max(1, int(0.3 * nb)), 24, S=1, seed=90 + k, net_index=k)
        sc[0]["weight"] = 0.25
        nets.append(n)
        scens.append(sc[0])
    net1, a = _run(nets, scens, False, steps=2)
    net2, b = _run(nets, scens, True, steps=2)
    info = net2.persistent_info()
    assert len(set(info)) >= 2 and all(c > 0 for c in info), info
    for (f1, a1, h1, g1), (f2, a2, h2, g2) in zip(a, b):
        assert (f1, a1) == (f2, a2)
        assert np.max(np.abs(h1 - h2) / np.abs(h1)) <= 1e-5
        assert rel(g2, g1) <= 1e-4
