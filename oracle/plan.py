"""Projected gradient step on the plan (Section 2.2), FP64.

Test infrastructure only (see the package docstring).

eta^(i+1) = proj_[eta_min, eta_max](eta^(i) - alpha Delta^(i)).
"""
from __future__ import annotations

import numpy as np

from .dispatch import solve_all
from .grad import planner_gradient


def plan_step(eta, delta, eta_min, eta_max, alpha):
    return np.minimum(np.maximum(eta - alpha * delta, eta_min), eta_max)


def objective(nets, scens, eta, sols):
    """gamma^T eta + sum_s w_s h_s  (Eq. 1 with weights w_s, 1/S by default)."""
    gam = np.concatenate([n["gamma"] for n in nets])
    return float(gam @ eta + sum(sc["weight"] * s.h for sc, s in zip(scens, sols)))


def run(nets, scens, eta0, opts, alpha, steps):
    """`steps` projected gradient steps; returns the trajectory of plans and objectives."""
    eta_min = np.concatenate([n["eta_min"] for n in nets])
    eta_max = np.concatenate([n["eta_max"] for n in nets])
    eta = np.array(eta0, dtype=np.float64)
    traj, objs, deltas = [eta.copy()], [], []
    for _ in range(steps):
        sols = solve_all(nets, scens, eta, opts)
        objs.append(objective(nets, scens, eta, sols))
        d = planner_gradient(nets, scens, sols)
        deltas.append(d)
        eta = plan_step(eta, d, eta_min, eta_max, alpha)
        traj.append(eta.copy())
    return traj, objs, deltas
