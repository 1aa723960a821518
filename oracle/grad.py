"""Implicit gradient of the planner objective (Section 2.2), three independent routes.

Test infrastructure only (see the package docstring).

For one scenario, dh/deta = (d x*/d eta)^T grad h(x*).  Routes:

1. ``fd_grad``        central finite differences of h(x*(eta)) with fresh IPM solves;
2. ``envelope_grad``  h = c only: dc*/deta = -D^T z, z the inequality multipliers
                      (the derivative of the Lagrangian in eta at the optimum);
3. ``adjoint_grad``   the implicit function theorem on the KKT conditions restricted
                      to the active set A (Section 2.2 cites it for differentiating the
                      argmin):  solve
                          [Q  A^T  G_A^T] [w ]   [grad h]
                          [A   0    0   ] [zeta] = [  0   ]
                          [G_A 0    0   ] [xi]   [  0   ]
                      and return D_A^T xi.
The planner's full gradient is Delta = gamma + sum_s w_s dh_s/deta.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .dispatch import solve, net_slices


def envelope_grad(sol) -> np.ndarray:
    return -(sol.qp.D.T @ sol.z)


def active_set(sol, tol_mult=1e-6, tol_slack=1e-6):
    """Constraints at their bound with a multiplier clearly above zero.

    Both tests are relative: slack against the bound's magnitude, multiplier
    against the largest multiplier.  A weakly active constraint (at the bound
    with a vanishing multiplier) is treated as inactive, which gives the
    one-sided derivative in the direction that keeps it slack.
    """
    qp = sol.qp
    zscale = max(1.0, float(np.max(sol.z))) if sol.z.size else 1.0
    hscale = np.maximum(1.0, np.abs(qp.h))
    return np.where((sol.s < tol_slack * hscale) & (sol.z > tol_mult * zscale))[0]


def adjoint_grad(sol, kappa=None, act=None) -> np.ndarray:
    qp = sol.qp
    if kappa is None:
        kappa = sol.kappa
    if act is None:
        act = active_set(sol)
    g = qp.planner_grad(sol.x, kappa)
    GA = qp.Gm[act]
    n, me, ma = qp.n, qp.m_eq, act.size
    K = sp.bmat([[qp.Q, qp.A.T, GA.T], [qp.A, None, None], [GA, None, None]], format="csc")
    rhs = np.concatenate([g, np.zeros(me + ma)])
    try:
        sol_vec = spla.splu(K).solve(rhs)
        if not np.all(np.isfinite(sol_vec)):
            raise RuntimeError("non-finite")
    except Exception:
        sol_vec = spla.lsqr(K, rhs, atol=1e-14, btol=1e-14, iter_lim=100000)[0]
    xi = sol_vec[n + me:]
    return qp.D[act].T @ xi


def fd_grad(net, scen, eta, opts, idx=None, rel_step=1e-4, tol=1e-12):
    """Central differences of h(x*(eta)); returns (grad, same_active_flags)."""
    eta = np.asarray(eta, dtype=np.float64)
    K = eta.size
    idx = range(K) if idx is None else idx
    kappa = opts.get("kappa", 0.0)
    g = np.zeros(K)
    same = np.ones(K, bool)
    base = solve(net, scen, eta, opts, tol=tol)
    a0 = set(active_set(base).tolist())
    for k in idx:
        st = rel_step * max(abs(eta[k]), 1.0)
        ep = eta.copy(); ep[k] += st
        em = eta.copy(); em[k] -= st
        sp_ = solve(net, scen, ep, opts, tol=tol)
        sm_ = solve(net, scen, em, opts, tol=tol)
        g[k] = (sp_.qp.planner(sp_.x, kappa) - sm_.qp.planner(sm_.x, kappa)) / (2 * st)
        same[k] = (set(active_set(sp_).tolist()) == a0) and (set(active_set(sm_).tolist()) == a0)
    return g, same


def planner_gradient(nets, scens, sols, route="adjoint"):
    """Delta = gamma + sum_s w_s dh_s/deta over the concatenated plan vector."""
    offs = net_slices(nets)
    gam = np.concatenate([n["gamma"] for n in nets])
    delta = gam.copy()
    for sc, sol in zip(scens, sols):
        k = sc["net"]
        gs = adjoint_grad(sol) if route == "adjoint" else envelope_grad(sol)
        delta[offs[k]:offs[k + 1]] += sc["weight"] * gs
    return delta


def scenario_grads(nets, scens, sols):
    """Per-scenario dh_s/deta blocks (no gamma, no weights)."""
    return [adjoint_grad(sol) for sol in sols]
