"""GPU warm-start network (BF16 tcgen05 tensor-core layers, FP32 accumulation) against the
FP64 CPU reference: activations within 2e-2 relative, gradients with cosine > 0.999.  Cases:
the 5-bus day (120 bus-hour rows: one partial 128-row tile) and a 20-bus, 72-hour network
(1,440 rows: eleven full tiles and a ragged one of 32 rows)."""
import numpy as np
import pytest

from gpu_util import eta_tensor, gpu_net
from oracle import gnn as ognn
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu

H, FIN = 64, 16


def pack(p):
    """CPU parameter dict -> the GPU's flat FP32 layout (input rows padded to 16)."""
    win = np.zeros((FIN, H)); win[:p["W_in"].shape[0]] = p["W_in"]
    parts = [win.ravel(), p["b_in"]]
    for k in range(3):
        parts += [p[f"W{k}"].ravel(), p[f"b{k}"]]
    parts += [p["W_out"].ravel(), p["b_out"]]
    return np.concatenate(parts).astype(np.float32)


def unpack_grads(v, p):
    out, o = {}, 0
    win = v[o:o + FIN * H].reshape(FIN, H); o += FIN * H
    out["W_in"] = win[:p["W_in"].shape[0]]
    out["b_in"] = v[o:o + H]; o += H
    for k in range(3):
        out[f"W{k}"] = v[o:o + 2 * H * H].reshape(2 * H, H); o += 2 * H * H
        out[f"b{k}"] = v[o:o + H]; o += H
    out["W_out"] = v[o:o + 2 * H].reshape(H, 2); o += 2 * H
    out["b_out"] = v[o:o + 2]
    return out


def _case(name):
    if name == "tiny":
        return synth.tiny()
    net, scens = synth.custom(20, 30, 60, 6, 72, S=1, seed=17, net_index=0)
    return [net], scens


CASES = ["tiny", "ragged"]


def _setup(case="tiny"):
    from paper_2410_13055_gb300 import gx
    nets, scens = _case(case)
    net = gpu_net(nets, scens)
    w = gx.WarmStartGNN(net, seed=1)
    rng = np.random.default_rng(4)
    p = ognn.init_params(rng, H=H)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    w.set_params(pack(p))
    eta = nets[0]["eta_min"] * 1.05
    X = ognn.features(nets[0], scens[0], eta)
    A = ognn.agg_matrix(nets[0], scens[0]["T"])
    return net, w, p, eta, X, A


@pytest.mark.parametrize("case", CASES)
def test_gnn_forward_matches_cpu_reference(case):
    net, w, p, eta, X, A = _setup(case)
    y_cpu, _ = ognn.forward(p, X, A)
    out = w.predict(eta_tensor(eta)).cpu().numpy()
    M = X.shape[0]
    y_gpu = np.stack([out[:M] / 100.0, out[M:]], axis=1)
    err = np.linalg.norm(y_gpu - y_cpu) / np.linalg.norm(y_cpu)
    assert err <= 2e-2, err


@pytest.mark.parametrize("case", CASES)
def test_gnn_gradients_match_cpu_reference(case):
    import torch
    net, w, p, eta, X, A = _setup(case)
    rng = np.random.default_rng(5)
    M = X.shape[0]
    target = rng.standard_normal((M, 2))
    g_cpu = ognn.backward(p, X, A, target, w_theta=0.5)
    tgt = torch.tensor(np.concatenate([100.0 * target[:, 0], target[:, 1]]), dtype=torch.float32, device="cuda")
    loss = w.train_step(eta_tensor(eta), tgt, lr=0.0, w_theta=0.5)
    assert abs(loss - ognn.loss(p, X, A, target, w_theta=0.5)) <= 2e-2 * abs(loss)
    g_gpu = unpack_grads(w.params(which=1), p)
    for k in g_cpu:
        a, b = g_gpu[k].ravel().astype(float), g_cpu[k].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        assert cos > 0.999, (k, cos)


def test_gnn_training_reduces_loss():
    import torch
    net, w, p, eta, X, A = _setup()
    M = X.shape[0]
    rng = np.random.default_rng(6)
    target = np.stack([np.sin(np.arange(M) / 7.0), 0.1 * np.cos(np.arange(M) / 5.0)], 1)
    tgt = torch.tensor(np.concatenate([100.0 * target[:, 0], target[:, 1]]), dtype=torch.float32, device="cuda")
    e = eta_tensor(eta)
    first = w.train_step(e, tgt, lr=1e-3)
    for _ in range(200):
        last = w.train_step(e, tgt, lr=1e-3)
    assert last < 0.5 * first, (first, last)


def test_gnn_predict_is_deterministic():
    """Each tile's MMAs run in a fixed order: two predictions are bitwise equal."""
    net, w, p, eta, X, A = _setup("ragged")
    e = eta_tensor(eta)
    a = w.predict(e).clone()
    b = w.predict(e).clone()
    import torch
    assert torch.equal(a, b)


def test_gnn_multi_tile_ring_matches_cpu_reference():
    """Two 168-hour scenarios of the 100-bus network: 33,600 rows, 263 tiles of 128 rows, so
    the persistent weight-gradient kernel (one CTA per SM) streams more than one tile through
    its ring in some CTAs, and the dense layers run 263 CTAs with a ragged last tile."""
    import scipy.sparse as sp
    import torch
    from paper_2410_13055_gb300 import gx
    nets, scens = synth.medium(S=2)
    net = gpu_net(nets, scens)
    w = gx.WarmStartGNN(net, seed=1)
    rng = np.random.default_rng(8)
    p = ognn.init_params(rng, H=H)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    w.set_params(pack(p))
    eta = nets[0]["eta_min"] * 1.05
    T = scens[0]["T"]
    X = np.concatenate([ognn.features(nets[0], sc, eta) for sc in scens])
    A1 = ognn.agg_matrix_sparse(nets[0], T)
    A = sp.block_diag([A1] * len(scens), format="csr")
    M = X.shape[0]
    assert M == w.M and M > 152 * 128, (M, w.M)
    y_cpu, _ = ognn.forward(p, X, A)
    out = w.predict(eta_tensor(eta)).cpu().numpy()
    y_gpu = np.stack([out[:M] / 100.0, out[M:]], axis=1)
    assert np.linalg.norm(y_gpu - y_cpu) / np.linalg.norm(y_cpu) <= 2e-2
    target = rng.standard_normal((M, 2))
    g_cpu = ognn.backward(p, X, A, target, w_theta=0.5)
    tgt = torch.tensor(np.concatenate([100.0 * target[:, 0], target[:, 1]]), dtype=torch.float32, device="cuda")
    loss = w.train_step(eta_tensor(eta), tgt, lr=0.0, w_theta=0.5)
    assert abs(loss - ognn.loss(p, X, A, target, w_theta=0.5)) <= 2e-2 * abs(loss)
    g_gpu = unpack_grads(w.params(which=1), p)
    for k in g_cpu:
        a, b = g_gpu[k].ravel().astype(float), g_cpu[k].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        assert cos > 0.999, (k, cos)
