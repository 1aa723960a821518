"""Small hand-built networks used by the pin tests (inputs only, no method arithmetic)."""
import math

import numpy as np


def network(n_bus, gens=(), lines=(), bats=(), gamma=None, dc=(), ramp=None):
    """gens: (bus, cost, cap[, emis]); lines: (from, to, beta, cap[, dtheta]); bats: (bus, P[, dur, eff]);
    dc: indices of the lines that are HVDC transport links (their beta and dtheta are unused);
    ramp: {generator index: hourly ramp limit as a fraction of its capacity}."""
    gb = np.array([g[0] for g in gens], dtype=np.int64)
    gc = np.array([g[1] for g in gens], dtype=float)
    gcap = np.array([g[2] for g in gens], dtype=float)
    ge = np.array([g[3] if len(g) > 3 else 0.0 for g in gens], dtype=float)
    lf = np.array([l[0] for l in lines], dtype=np.int64)
    lt = np.array([l[1] for l in lines], dtype=np.int64)
    lb = np.array([l[2] for l in lines], dtype=float)
    lcap = np.array([l[3] for l in lines], dtype=float)
    ld = np.array([l[4] if len(l) > 4 else math.pi / 6 for l in lines], dtype=float)
    bb = np.array([b[0] for b in bats], dtype=np.int64)
    bP = np.array([b[1] for b in bats], dtype=float)
    bdur = np.array([b[2] if len(b) > 2 else 4.0 for b in bats], dtype=float)
    beff = np.array([b[3] if len(b) > 3 else math.sqrt(0.9) for b in bats], dtype=float)
    K = gb.size + lf.size + bb.size
    eta = np.concatenate([gcap, lcap, bP])
    net = dict(n_bus=int(n_bus), gen_bus=gb, gen_cost=gc, gen_emis=ge, gen_kind=np.zeros(gb.size, np.int64),
               line_from=lf, line_to=lt, line_beta=lb, line_dtheta=ld,
               bat_bus=bb, bat_dur=bdur, bat_eff_c=beff.copy(), bat_eff_d=beff.copy(),
               eta_min=0.5 * eta, eta_max=2.0 * eta + 1.0,
               gamma=np.zeros(K) if gamma is None else np.asarray(gamma, float), K=K)
    if len(dc):
        net["line_dc"] = np.isin(np.arange(lf.size), np.asarray(dc)).astype(np.uint8)
    if ramp:
        net["gen_ramp"] = np.zeros(gb.size)
        for g, r in ramp.items():
            net["gen_ramp"][g] = r
    return net, eta


def scenario(load, cf=None, G=0, weight=1.0):
    load = np.atleast_2d(np.asarray(load, float))
    T = load.shape[1]
    if cf is None:
        cf = np.ones((G, T))
    return dict(net=0, T=T, load=load, cf=np.atleast_2d(np.asarray(cf, float)).reshape(-1, T), weight=weight)
