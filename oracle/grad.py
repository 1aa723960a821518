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
    """-D^T z, plus y^T dA_k x + z^T dG_k x for plan entries that enter the constraint
    matrix (lines whose susceptance scales with capacity)."""
    qp = sol.qp
    g = -(qp.D.T @ sol.z)
    for k, dA in qp.dA.items():
        g[k] += float(sol.y @ (dA @ sol.x)) + float(sol.z @ (qp.dG[k] @ sol.x))
    return g


def active_set(sol, ratio=1.0):
    """Constraints identified as active at the interior-point solution.

    At an interior-point optimum an active constraint has slack s_i -> 0 with a
    positive multiplier z_i, an inactive one the reverse, so the indicator
    z_i / s_i separates them by many decades; a constraint counts as active when
    z_i > ratio * s_i.  Weakly active constraints (both tiny) fall on either side,
    which changes the derivative only by the (vanishing) multiplier involved.
    """
    return np.where(sol.z > ratio * sol.s)[0]


def independent_active(qp, act):
    """Drop the lower row of a box whose two bounds coincide and are both active.

    A generator with capacity factor 0 (or a battery of zero power) has
    0 <= x <= 0: both rows are tight and the constraint gradients are linearly
    dependent, so the active KKT matrix is singular.  One row fixes the variable;
    the upper one is kept because it is the row that depends on eta (its
    derivative cf * 1 is 0 there anyway).  Lines keep both their rows: their two
    limits never coincide (eta_l > 0, dtheta_max > 0).
    """
    kind = qp.kind
    ups = {}
    for i in act:
        tag = kind[i]
        if tag is not None and tag[0].endswith("_up"):
            ups[(tag[0][:-3], tag[1], tag[2])] = i
    keep = []
    for i in act:
        tag = kind[i]
        if tag is not None and tag[0].endswith("_lo") and tag[0][0] != "f" and tag[0][0] != "a":
            if (tag[0][:-3], tag[1], tag[2]) in ups:
                continue
        keep.append(i)
    return np.array(keep, dtype=np.int64)


def adjoint_grad(sol, kappa=None, act=None) -> np.ndarray:
    qp = sol.qp
    if kappa is None:
        kappa = sol.kappa
    if act is None:
        act = active_set(sol)
    act = independent_active(qp, act)
    g = qp.planner_grad(sol.x, kappa)
    GA = qp.Gm[act]
    n, me, ma = qp.n, qp.m_eq, act.size
    K = sp.bmat([[qp.Q, qp.A.T, GA.T], [qp.A, None, None], [GA, None, None]], format="csc")
    rhs = np.concatenate([g, np.zeros(me + ma)])
    # The active constraints can be linearly dependent (an idle battery held at full or
    # empty charge over consecutive hours: soc bounds + dynamics + ch, dis >= 0).  The
    # multipliers are then not unique, but the system is consistent and D_A^T xi is the
    # same for every solution (the dependent combinations have zero eta-derivative).
    # Solve it with a small regularisation of the multiplier block, then refine on the
    # exact system.
    nm = me + ma
    delta = 1e-9 * max(1.0, float(np.max(np.abs(qp.Qd))))
    Kreg = (K - sp.block_diag([sp.csc_matrix((n, n)), delta * sp.identity(nm)])).tocsc()
    lu = spla.splu(Kreg)
    sol_vec = lu.solve(rhs)
    for _ in range(20):
        r = rhs - K @ sol_vec
        if np.linalg.norm(r) <= 1e-12 * max(1.0, np.linalg.norm(rhs)):
            break
        sol_vec = sol_vec + lu.solve(r)
    if not np.all(np.isfinite(sol_vec)) or np.linalg.norm(K @ sol_vec - rhs) > 1e-8 * max(1.0, np.linalg.norm(rhs)):
        raise np.linalg.LinAlgError("active-set KKT system is inconsistent")
    xi = sol_vec[n + me:]
    out = qp.D[act].T @ xi
    # plan entries inside the constraint matrix: -[w^T (dA^T y + dG_A^T z_A) + zeta^T dA x
    # + xi^T dG_A x], from differentiating the KKT residual in eta
    if qp.dA:
        w, zeta = sol_vec[:n], sol_vec[n:n + me]
        zA = sol.z[act]
        for k, dA in qp.dA.items():
            dGA = qp.dG[k][act]
            out[k] -= float(w @ (dA.T @ sol.y + dGA.T @ zA)) + float(zeta @ (dA @ sol.x)) + float(xi @ (dGA @ sol.x))
    return out


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
