"""The autograd wrapper: backward equals the oracle's implicit gradient and a GPU
central difference of the forward."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net, rel
from oracle import dispatch, grad as ograd
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle_and_central_difference():
    import torch

    from paper_2410_13055_gb300.autograd import planner_objective
    nets, scens = synth.tiny()
    kappa = 50.0
    net = gpu_net(nets, scens, kappa=kappa, tol=1e-6, adj_tol=1e-5, max_iter=200000, adj_max_iter=200000,
                  check_every=50)
    eta0 = nets[0]["eta_min"] * 1.1
    eta = eta_tensor(eta0).requires_grad_(True)
    val = planner_objective(eta, net)
    val.backward()
    g = eta.grad.double().cpu().numpy()
    ref = dispatch.solve(nets[0], scens[0], eta0, synth.default_opts(kappa=kappa))
    assert abs(float(val.detach()) - ref.h) / abs(ref.h) <= 1e-4
    assert rel(g, ograd.adjoint_grad(ref)) <= 1e-3
    # central difference of the forward along a random direction
    rng = np.random.default_rng(3)
    d = rng.standard_normal(eta0.size) * eta0 * 1e-3
    with torch.no_grad():
        fp = float(planner_objective(eta_tensor(eta0 + d), net))
        fm = float(planner_objective(eta_tensor(eta0 - d), net))
    fd = (fp - fm) / 2.0
    assert abs(fd - float(g @ d)) <= 1e-2 * abs(fd)
