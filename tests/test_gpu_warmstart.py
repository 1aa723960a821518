"""The learned warm start: trained on the GPU by the project's kernels on solutions the
solver produces; what it gains over a cold start on held-out plans, next to the
previous-plan start (which it does not beat: see the design doc)."""
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
