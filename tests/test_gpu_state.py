"""The iteration state exported by gx_network_state_range: saving it after a call and
writing it back restores that warm start exactly (same iterates, bit for bit)."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu


def test_state_checkpoint_restores_warm_start():
    import torch
    nets, scens = synth.medium(S=3, T=24)
    net = gpu_net(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=20000, adj_max_iter=20000)
    eta = nets[0]["eta_min"] * 1.1
    e = eta_tensor(eta)
    assert net.solve(e) == 0
    net.grad(e)
    fs, ad = net.state(False), net.state(True)
    assert fs.numel() > 0 and ad.numel() > 0
    assert fs.data_ptr() + fs.numel() * 4 <= ad.data_ptr()  # disjoint ranges, forward first
    f0, a0 = fs.clone(), ad.clone()
    e2 = eta_tensor(eta * 1.05)

    def run():
        assert net.solve(e2, warm="prev") == 0
        g = net.grad(e2, warm="prev").clone()
        return (net.array("p").clone(), net.array("price").clone(), g, net.last_stats["iters_max"],
                net.last_grad_stats["iters_max"])

    r1 = run()
    assert not torch.equal(fs, f0)  # the call moved the state
    fs.copy_(f0)
    ad.copy_(a0)
    r2 = run()
    for x, y in zip(r1[:3], r2[:3]):
        assert torch.equal(x, y)
    assert r1[3:] == r2[3:]
