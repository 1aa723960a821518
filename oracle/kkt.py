"""FP64 KKT residuals of any candidate dispatch (x, nodal prices).

Test infrastructure only (see the package docstring).

Given primal arrays and prices lambda (balance multipliers y = -lambda), the
remaining multipliers (battery dynamics, angle reference, and z >= 0 on the
constraints that the candidate holds at their bound) are chosen to minimise the
stationarity residual, so the result measures how far (x, lambda) is from
satisfying the KKT conditions of the QP in ``qp``:

    primal   = max(|A x - b|_inf, |max(G x - h, 0)|_inf) / (1 + |(b, h)|_inf)
    dual     = |Q x + q + A^T y + G^T z|_inf / (1 + |q|_inf)
    comp     = max_i z_i |h_i - G_i x| / (1 + |q|_inf)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import lsq_linear


def residuals(qp, x, price, act_tol=1e-5):
    x = np.asarray(x, float)
    rp_eq = qp.A @ x - qp.b
    rg = qp.Gm @ x - qp.h
    scale_bh = 1.0 + max(np.max(np.abs(qp.b)), np.max(np.abs(qp.h)))
    primal = max(np.max(np.abs(rp_eq)), np.max(np.maximum(rg, 0.0))) / scale_bh

    nb = qp.N * qp.T
    y_bal = -np.asarray(price, float).ravel()
    grad = qp.Qd * x + qp.q + qp.A[:nb].T @ y_bal
    near = np.where(-rg <= act_tol * np.maximum(1.0, np.abs(qp.h)))[0]
    Afree = qp.A[nb:].T  # dynamics + reference rows: free multipliers
    Gn = qp.Gm[near].T
    M = sp.hstack([Afree, Gn]).tocsr()
    nf = Afree.shape[1]
    lb = np.concatenate([np.full(nf, -np.inf), np.zeros(near.size)])
    ub = np.full(nf + near.size, np.inf)
    if M.shape[1]:
        sol = lsq_linear(M.toarray() if M.shape[0] * M.shape[1] < 4e7 else M, -grad, bounds=(lb, ub),
                         lsmr_tol="auto", tol=1e-13, max_iter=5000)
        mult = sol.x
        r = grad + M @ mult
        zn = mult[nf:]
    else:
        r = grad
        zn = np.zeros(0)
    scale_q = 1.0 + np.max(np.abs(qp.q))
    dual = np.max(np.abs(r)) / scale_q
    comp = float(np.max(zn * np.abs(rg[near]))) / scale_q if zn.size else 0.0
    return dict(primal=float(primal), dual=float(dual), comp=comp)
