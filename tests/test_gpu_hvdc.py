"""HVDC transport lines on the CUDA path against the FP64 oracle: dispatch, prices, the
capacity gradient of every asset (HVDC lines included), and the cluster-resident path."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net, pack_x, ref_groups, rel, solution
from oracle import dispatch, grad as ograd, kkt
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-6, max_iter=200000, adj_tol=1e-5, adj_max_iter=200000, check_every=50)
ACT_TOL = 1e-3


def _islands():
    """Two AC islands (buses 0-2 with cheap generation, 3-5 with expensive generation and
    most of the load) joined only by two HVDC links that bind in the peak hours."""
    import math
    from cases import network, scenario
    gens = [(0, 15.0, 400.0, 0.2), (1, 22.0, 300.0, 0.3), (2, 30.0, 300.0, 0.4),
            (3, 55.0, 400.0, 0.5), (4, 70.0, 300.0, 0.6), (5, 90.0, 300.0, 0.6)]
    lines = [(0, 1, 900.0, 500.0), (1, 2, 700.0, 500.0), (0, 2, 500.0, 500.0),
             (3, 4, 800.0, 500.0), (4, 5, 600.0, 500.0),
             (1, 3, 1.0, 120.0), (2, 5, 1.0, 90.0)]
    net, eta = network(6, gens=gens, lines=lines, bats=[(4, 60.0)], dc=(5, 6))
    t = np.arange(24)
    shape = 1.0 + 0.4 * np.sin(2 * math.pi * (t - 8) / 24)
    load = np.outer([40.0, 50.0, 30.0, 160.0, 140.0, 120.0], shape)
    return [net], [scenario(load, G=6)], eta


def _case(kind):
    if kind == "islands":
        nets, scens, _ = _islands()
        return nets, scens
    net, sc = synth.custom(24, 36, 72, 6, 24, S=1, seed=81)
    return [synth.add_hvdc(net, 3, seed=82, cap=(60.0, 150.0))], sc


@pytest.mark.parametrize("kind", ["islands", "custom24"])
@pytest.mark.parametrize("persistent", [False, True])
def test_hvdc_parity(kind, persistent):
    nets, scens = _case(kind)
    eta = nets[0]["eta_min"] * 1.05
    net = gpu_net(nets, scens, kappa=50.0, **TIGHT)
    net.use_persistent(persistent)
    e = eta_tensor(eta)
    assert net.solve(e) == 0, net.last_stats
    ref = dispatch.solve(nets[0], scens[0], eta, synth.default_opts(kappa=50.0))
    g = solution(net, 0, ref_groups(ref.qp))
    assert abs(g["cost"] - ref.cost) / ref.cost <= 1e-4
    res = kkt.residuals(ref.qp, pack_x(ref.qp, g), g["price"], act_tol=ACT_TOL)
    assert res["primal"] <= 1e-3 and res["dual"] <= 1e-3, res
    assert rel(g["price"], ref.price) <= 1e-3
    dc = np.where(nets[0]["line_dc"] == 1)[0]
    # A transport flow below its limit equals (lambda_to - lambda_from) / eps (its KKT
    # condition): 1000 MW per $/MWh of price gap, so its error is the price-gap error
    # amplified by 1/eps; at the limit both sit on the same bound.
    fr, to = nets[0]["line_from"][dc], nets[0]["line_to"][dc]
    gap_err = np.abs((g["price"][to] - g["price"][fr]) - (ref.price[to] - ref.price[fr]))
    eps = synth.default_opts()["eps"]
    tol = 1.05 * gap_err / eps + 1e-3 * np.max(np.abs(ref.flow[dc])) + 1e-6
    assert np.all(np.abs(g["flow"][dc] - ref.flow[dc]) <= tol)
    gg = net.grad(e).double().cpu().numpy()
    assert net.last_grad_status == 0, net.last_grad_stats
    g_ref = ograd.adjoint_grad(ref)
    assert rel(gg, g_ref) <= 2e-3, (rel(gg, g_ref), gg[nets[0]["gen_bus"].size + dc], g_ref[nets[0]["gen_bus"].size + dc])
