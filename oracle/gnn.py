"""FP64 CPU reference of the warm-start graph network (forward, loss, backward).

Test infrastructure only (see the package docstring).

Nodes are bus-hours of one scenario; node (n, t) is connected to (m, t) when a line
joins buses n and m.  With features x (F per node), hidden width H and L layers:

    h_0 = relu(x W_in + b_in)
    h_k = h_{k-1} + relu([h_{k-1}, mean_{m in N(n)} h_{k-1,m}] W_k + b_k),  k = 1..L
    y   = h_L W_out + b_out                      (y[:, 0] ~ price / 100, y[:, 1] ~ angle)
    loss = mean_nodes((y_0 - lambda/100)^2 + w_theta (y_1 - theta)^2)

The mean over an empty neighbourhood is 0.  Backward is the chain rule written out;
the tests check it against central differences of `loss`.
"""
from __future__ import annotations

import numpy as np

F_IN = 10


def features(net, scen, eta):
    """Node features [N*T, F] of one scenario at plan eta (bus-major, hour-minor)."""
    N, T = int(net["n_bus"]), int(scen["T"])
    G, L = net["gen_bus"].size, net["line_from"].size
    eta = np.asarray(eta, float)
    eg, el, eb = eta[:G], eta[G:G + L], eta[G + L:]
    cap = np.asarray(scen["cf"], float) * eg[:, None]          # [G, T]
    cost = np.asarray(net["gen_cost"], float)
    avail = np.zeros((N, T)); costw = np.zeros((N, T)); free = np.zeros((N, T)); dear = np.zeros((N, T))
    np.add.at(avail, net["gen_bus"], cap)
    np.add.at(costw, net["gen_bus"], cap * cost[:, None])
    np.add.at(free, net["gen_bus"], cap * (cost[:, None] == 0))
    np.add.at(dear, net["gen_bus"], cap * (cost[:, None] > 0))
    bat = np.zeros(N); np.add.at(bat, net["bat_bus"], eb)
    lin = np.zeros(N); np.add.at(lin, net["line_from"], el); np.add.at(lin, net["line_to"], el)
    load = np.asarray(scen["load"], float)
    h = np.arange(T) % 24
    X = np.empty((N, T, F_IN))
    X[..., 0] = load / 100.0
    X[..., 1] = avail / 100.0
    X[..., 2] = np.where(dear > 0, costw / np.maximum(dear, 1e-9), 0.0) / 100.0
    X[..., 3] = free / 100.0
    X[..., 4] = bat[:, None] / 100.0
    X[..., 5] = lin[:, None] / 100.0
    X[..., 6] = np.sin(2 * np.pi * h / 24.0)[None, :]
    X[..., 7] = np.cos(2 * np.pi * h / 24.0)[None, :]
    X[..., 8] = (load - free) / 100.0
    X[..., 9] = 1.0
    return X.reshape(N * T, F_IN)


def neighbours(net):
    """Adjacency lists of the bus graph."""
    N = int(net["n_bus"])
    adj = [[] for _ in range(N)]
    for a, b in zip(net["line_from"].tolist(), net["line_to"].tolist()):
        adj[a].append(b)
        adj[b].append(a)
    return adj


def agg_matrix(net, T):
    """Sparse-free dense helper: A [N*T, N*T] with A[(n,t),(m,t)] = 1/deg(n) for m in N(n)."""
    N = int(net["n_bus"])
    adj = neighbours(net)
    A = np.zeros((N * T, N * T))
    for n in range(N):
        if not adj[n]:
            continue
        w = 1.0 / len(adj[n])
        for m in adj[n]:
            for t in range(T):
                A[n * T + t, m * T + t] += w
    return A


def agg_matrix_sparse(net, T):
    """The same matrix as agg_matrix in CSR form, for graphs too large to hold densely: entry
    ((n, t), (m, t)) = 1/deg(n) for every line joining n and m (parallel lines add up)."""
    import scipy.sparse as sp
    N = int(net["n_bus"])
    adj = neighbours(net)
    rows, cols, vals = [], [], []
    for n in range(N):
        if not adj[n]:
            continue
        w = 1.0 / len(adj[n])
        for m in adj[n]:
            for t in range(T):
                rows.append(n * T + t)
                cols.append(m * T + t)
                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N * T, N * T))  # duplicates are summed


def init_params(rng, H=64, L=3, F=F_IN):
    p = {"W_in": rng.standard_normal((F, H)) * np.sqrt(2.0 / F), "b_in": np.zeros(H)}
    for k in range(L):
        p[f"W{k}"] = rng.standard_normal((2 * H, H)) * np.sqrt(1.0 / (2 * H))
        p[f"b{k}"] = np.zeros(H)
    p["W_out"] = rng.standard_normal((H, 2)) * np.sqrt(1.0 / H)
    p["b_out"] = np.zeros(2)
    return p


def forward(p, X, A, L=3):
    cache = {}
    z0 = X @ p["W_in"] + p["b_in"]
    h = np.maximum(z0, 0.0)
    cache["z0"] = z0
    hs = [h]
    for k in range(L):
        a = A @ h
        cat = np.concatenate([h, a], axis=1)
        z = cat @ p[f"W{k}"] + p[f"b{k}"]
        cache[f"cat{k}"] = cat
        cache[f"z{k + 1}"] = z
        h = h + np.maximum(z, 0.0)
        hs.append(h)
    y = h @ p["W_out"] + p["b_out"]
    cache["hs"] = hs
    return y, cache


def loss(p, X, A, target, w_theta=1.0, L=3):
    y, _ = forward(p, X, A, L)
    d0 = y[:, 0] - target[:, 0]
    d1 = y[:, 1] - target[:, 1]
    return float(np.mean(d0 * d0 + w_theta * d1 * d1))


def backward(p, X, A, target, w_theta=1.0, L=3):
    y, cache = forward(p, X, A, L)
    M = X.shape[0]
    dy = np.empty_like(y)
    dy[:, 0] = 2.0 * (y[:, 0] - target[:, 0]) / M
    dy[:, 1] = 2.0 * w_theta * (y[:, 1] - target[:, 1]) / M
    g = {}
    hs = cache["hs"]
    g["W_out"] = hs[L].T @ dy
    g["b_out"] = dy.sum(0)
    dh = dy @ p["W_out"].T
    H = dh.shape[1]
    for k in reversed(range(L)):
        dz = dh * (cache[f"z{k + 1}"] > 0)
        g[f"W{k}"] = cache[f"cat{k}"].T @ dz
        g[f"b{k}"] = dz.sum(0)
        dcat = dz @ p[f"W{k}"].T
        dh = dh + dcat[:, :H] + A.T @ dcat[:, H:]
    dz0 = dh * (cache["z0"] > 0)
    g["W_in"] = X.T @ dz0
    g["b_in"] = dz0.sum(0)
    return g
