"""The dispatch map x*_s(eta) of Eq. 2, solved in FP64 by the interior-point method.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .ipm import solve_qp
from .qp import DispatchQP


class Dispatch:
    """Solution of one scenario: primal arrays, nodal prices, multipliers, cost."""

    def __init__(self, qp: DispatchQP, res, kappa: float):
        self.qp = qp
        self.res = res
        self.x = res.x
        self.y = res.y
        self.z = res.z
        self.s = res.s
        v = qp.unpack(res.x)
        self.p, self.sh, self.th = v["p"], v["sh"], v["th"]
        self.ch, self.dis, self.soc = v["ch"], v["dis"], v["soc"]
        self.fdc = v["fdc"]
        self.flow = qp.flows(self.th, self.fdc)
        # nodal price lambda_nt = -y of the balance row
        self.price = -res.y[qp.row_bal:qp.row_bal + qp.N * qp.T].reshape(qp.N, qp.T)
        self.cost = qp.cost(res.x)
        self.kappa = float(kappa)
        self.h = qp.planner(res.x, kappa)
        self.emissions = float(qp.emis_vec @ res.x)
        self.converged = res.converged
        self.iters = res.iters


def solve(net, scen, eta, opts, tol=1e-11, max_iter=200) -> Dispatch:
    qp = DispatchQP(net, scen, eta, opts)
    res = solve_qp(qp.Q, qp.q, qp.A, qp.b, qp.Gm, qp.h, tol=tol, max_iter=max_iter)
    return Dispatch(qp, res, opts.get("kappa", 0.0))


def net_slices(nets):
    """Offsets of each network's block in the concatenated plan vector."""
    offs = [0]
    for n in nets:
        offs.append(offs[-1] + int(n["K"]))
    return offs


def solve_all(nets, scens, eta_full, opts, **kw):
    offs = net_slices(nets)
    out = []
    for sc in scens:
        k = sc["net"]
        out.append(solve(nets[k], sc, eta_full[offs[k]:offs[k + 1]], opts, **kw))
    return out
