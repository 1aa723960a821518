"""Pins of the FP64 warm-start network reference: backward = central differences."""
import numpy as np

from oracle import gnn
from paper_2410_13055_gb300 import synth


def test_gnn_backward_matches_central_differences():
    nets, scens = synth.tiny()
    n2, s2 = synth.slice_hours(nets, scens, 5, 3)
    X = gnn.features(n2[0], s2[0], n2[0]["eta_min"])
    A = gnn.agg_matrix(n2[0], 3)
    rng = np.random.default_rng(0)
    p = gnn.init_params(rng, H=8)
    target = rng.standard_normal((X.shape[0], 2))
    g = gnn.backward(p, X, A, target, w_theta=0.5)
    for name, W in p.items():
        flat = W.reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            h = 1e-6 * max(1.0, abs(old))
            flat[i] = old + h
            lp = gnn.loss(p, X, A, target, w_theta=0.5)
            flat[i] = old - h
            lm = gnn.loss(p, X, A, target, w_theta=0.5)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, an)


def test_gnn_features_and_aggregation():
    nets, scens = synth.tiny()
    X = gnn.features(nets[0], scens[0], nets[0]["eta_min"])
    assert X.shape == (5 * 24, gnn.F_IN)
    np.testing.assert_allclose(X[:, 0], scens[0]["load"].reshape(-1) / 100.0)
    np.testing.assert_allclose(X[:, 9], 1.0)
    A = gnn.agg_matrix(nets[0], 24)
    # rows are means: each row sums to 1 (every tiny bus has a line)
    np.testing.assert_allclose(A.sum(1), 1.0)


def test_sparse_aggregation_equals_dense_and_propagates_alike():
    """agg_matrix_sparse holds agg_matrix's entries (each row of a connected bus sums to 1),
    and forward/backward give the same results with either form."""
    nets, scens = synth.tiny()
    net = nets[0]
    A = gnn.agg_matrix(net, 24)
    As = gnn.agg_matrix_sparse(net, 24)
    assert np.array_equal(As.toarray(), A)
    rs = A.sum(axis=1)
    assert np.allclose(rs[rs > 0], 1.0)
    X = gnn.features(net, scens[0], net["eta_min"])
    rng = np.random.default_rng(3)
    p = gnn.init_params(rng, H=16)
    target = rng.standard_normal((X.shape[0], 2))
    yd, _ = gnn.forward(p, X, A)
    ys, _ = gnn.forward(p, X, As)
    assert np.allclose(yd, ys, rtol=1e-12, atol=1e-12)
    gd = gnn.backward(p, X, A, target)
    gs = gnn.backward(p, X, As, target)
    for k in gd:
        assert np.allclose(gd[k], gs[k], rtol=1e-12, atol=1e-12), k
