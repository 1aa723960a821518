"""FP64 KKT residuals of any candidate dispatch (x, nodal prices).

Test infrastructure only (see the package docstring).

Given primal arrays and prices lambda (balance multipliers y = -lambda), the
remaining multipliers (battery dynamics, angle reference, and z >= 0 on the
constraints that the candidate holds at their bound) are chosen to minimise the
stationarity residual, so the result measures how far (x, lambda) is from
satisfying the KKT conditions of the QP in ``qp``:

    primal   = max(|A x - b|_inf, |max(G x - h, 0)|_inf) / (1 + |(b, h)|_inf)
    dual     = |(Q x + q + A^T y + G^T z) / colmax(A)|_inf / (1 + |q|_inf)
               (colmax: each variable's largest equality coefficient, >= 1)
    comp     = max_i z_i |h_i - G_i x| / (1 + |q|_inf)
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.optimize import lsq_linear
from scipy.sparse.csgraph import connected_components


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
    Afree = qp.A[nb:].T  # dynamics, reference and fixed-variable rows: free multipliers
    Gn = qp.Gm[near].T
    M = sp.hstack([Afree, Gn]).tocsc()
    nf = Afree.shape[1]
    lb_all = np.concatenate([np.full(nf, -np.inf), np.zeros(near.size)])
    r = grad.copy()
    zn = np.zeros(near.size)
    if M.shape[1]:
        # The multipliers only couple variables that share a row: solve the bounded
        # least-squares problem separately on each connected block (one generator-hour,
        # one battery's horizon, one hour of angles, ...).
        n, m = M.shape
        B = sp.bmat([[None, M], [M.T, None]]).tocsr()
        B.data[:] = 1.0
        ncomp, lab = connected_components(B, directed=False)
        vlab, clab = lab[:n], lab[n:]
        corder = np.argsort(clab, kind="stable")
        cstart = np.searchsorted(clab[corder], np.arange(ncomp + 1))
        vorder = np.argsort(vlab, kind="stable")
        vstart = np.searchsorted(vlab[vorder], np.arange(ncomp + 1))
        for k in range(ncomp):
            cols = corder[cstart[k]:cstart[k + 1]]
            if cols.size == 0:
                continue
            rows = vorder[vstart[k]:vstart[k + 1]]
            Mk = M[rows][:, cols].toarray()
            sol = lsq_linear(Mk, -grad[rows], bounds=(lb_all[cols], np.full(cols.size, np.inf)),
                             method="bvls", tol=1e-13, max_iter=2000)
            r[rows] = grad[rows] + Mk @ sol.x
            zc = cols >= nf
            zn[cols[zc] - nf] = sol.x[zc]
    scale_q = 1.0 + np.max(np.abs(qp.q))
    # Each variable's stationarity residual in its own units: divided by its column's
    # largest coefficient in the equality rows (beta for an angle, whose balance terms
    # are beta * price differences; 1 for powers), then relative to the cost scale.
    colmax = np.maximum(1.0, abs(qp.A).max(axis=0).toarray().ravel())
    dual = np.max(np.abs(r) / colmax) / scale_q
    comp = float(np.max(zn * np.abs(rg[near]))) / scale_q if zn.size else 0.0
    return dict(primal=float(primal), dual=float(dual), comp=comp)
