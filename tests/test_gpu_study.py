"""Stochastic implicit gradient descent on the GPU path (Section 2.2) and the warm-start
effect of Section 3.2 on a small case."""
import numpy as np
import pytest

from paper_2410_13055_gb300 import study, synth

pytestmark = pytest.mark.gpu


def test_sgd_descends_and_warm_start_converges_faster():
    import torch
    from paper_2410_13055_gb300 import gx
    nets, scens = synth.medium(S=4, T=24)
    net = gx.Network(nets, scens, kappa=200.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    pl = study.Planner(net, nets)
    gamma = torch.tensor(nets[0]["gamma"], dtype=torch.float32, device="cuda")
    alpha = study.step_size(pl, gamma, 0.02)
    eta1, h1 = pl.sgd(pl.eta_min, gamma, alpha, 40, batch=2, seed=0, eval_every=5)
    assert h1[-1][1] < h1[0][1]                       # the planner objective went down
    assert torch.all(eta1 >= pl.eta_min) and torch.all(eta1 <= pl.eta_max)
    # a nearby problem (carbon weight 200 -> 175): from the previous solution the loss
    # reaches 2 % of the cold run's best in fewer iterations than from no expansion
    net.set_opts(kappa=175.0)
    _, hc = pl.sgd(pl.eta_min, gamma, alpha, 40, batch=2, seed=1, eval_every=5)
    _, hw = pl.sgd(eta1, gamma, alpha, 40, batch=2, seed=1, eval_every=5)
    best = min(J for _, J in hc)
    ic, iw = study.within(hc, best), study.within(hw, best)
    assert iw is not None and ic is not None and iw < ic, (ic, iw)
