"""Mehrotra predictor-corrector interior-point method for a convex QP, FP64.

Test infrastructure only (see the package docstring).

Solves   min 1/2 x^T Q x + q^T x   s.t.  A x = b,  G x + s = h,  s >= 0
with multipliers y (equalities) and z >= 0 (inequalities).  The KKT conditions

    Q x + q + A^T y + G^T z = 0,   A x = b,   G x + s = h,   s o z = 0,  s, z >= 0

are followed by Newton steps on the perturbed complementarity s o z = sigma mu e
(the textbook primal-dual method; Mehrotra's choice of sigma and his
second-order correction).  Each Newton system is reduced to

    [ Q + G^T W G   A^T ] [dx]   [r1]
    [ A             -dI ] [dy] = [r2],     W = diag(z / s),

and solved with a sparse LU factorisation (a library primitive), reused for the
predictor and the corrector, with two steps of iterative refinement.  The best
iterate (smallest of the relative residuals and gap) is returned; it counts as
converged at 1e-8 when the end game stalls before `tol`.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class IPMResult:
    def __init__(self, x, y, z, s, iters, converged, info):
        self.x, self.y, self.z, self.s = x, y, z, s
        self.iters, self.converged, self.info = iters, converged, info


def _max_step(v, dv):
    neg = dv < 0
    if not np.any(neg):
        return 1.0
    return float(min(1.0, np.min(-v[neg] / dv[neg])))


def solve_qp(Q, q, A, b, G, h, tol=1e-11, max_iter=200, reg=1e-13, verbose=False):
    n = q.size
    me = b.size
    mi = h.size
    Q = sp.csc_matrix(Q)
    A = sp.csr_matrix(A)
    G = sp.csr_matrix(G)
    At = A.T.tocsr()
    Gt = G.T.tocsr()

    x = np.zeros(n)
    y = np.zeros(me)
    s = np.maximum(h - G @ x, 1.0)
    z = np.ones(mi)
    scale_q = 1.0 + np.max(np.abs(q)) if n else 1.0
    scale_b = 1.0 + (np.max(np.abs(b)) if me else 0.0)
    scale_h = 1.0 + (np.max(np.abs(h)) if mi else 0.0)

    converged = False
    it = 0
    info = {}
    best = (np.inf, None)
    stall = 0
    for it in range(1, max_iter + 1):
        rd = Q @ x + q + At @ y + Gt @ z
        rp = A @ x - b
        rg = G @ x + s - h
        mu = float(s @ z) / max(mi, 1)
        obj = 0.5 * x @ (Q @ x) + q @ x
        e_d = np.max(np.abs(rd)) / scale_q if n else 0.0
        e_p = np.max(np.abs(rp)) / scale_b if me else 0.0
        e_g = np.max(np.abs(rg)) / scale_h if mi else 0.0
        gap = float(s @ z) / (1.0 + abs(obj))
        info = dict(e_d=e_d, e_p=e_p, e_g=e_g, gap=gap, obj=obj)
        if verbose:
            print(it, info)
        merit = max(e_d, e_p, e_g, gap)
        if merit < best[0]:
            best = (merit, (x.copy(), y.copy(), z.copy(), s.copy(), dict(info)))
            stall = 0
        else:
            stall += 1
        if merit < tol:
            converged = True
            break
        # End game: once the iterate is accurate, W = z/s spans many decades and the
        # Newton systems lose accuracy; stop when the merit no longer improves and
        # return the best iterate.
        if stall >= 5 and best[0] < 1e-7:
            break

        w = z / s
        H = (Q + Gt @ sp.diags(w) @ G + reg * sp.identity(n)).tocsc()
        K = sp.bmat([[H, At], [A, -reg * sp.identity(me)]], format="csc")
        lu = spla.splu(K)

        K0 = sp.bmat([[H, At], [A, None]], format="csr")

        def direction(r_sz):
            # ds = -(r_sz + s dz)/z ;  dz = W (G dx + rg) - r_sz / s
            r1 = -rd - Gt @ (w * rg) + Gt @ (r_sz / s)
            rhs = np.concatenate([r1, -rp])
            sol = lu.solve(rhs)
            for _ in range(2):  # iterative refinement against the unregularised system
                sol = sol + lu.solve(rhs - K0 @ sol)
            dx, dy = sol[:n], sol[n:]
            dz = w * (G @ dx + rg) - r_sz / s
            ds = -(r_sz + s * dz) / z
            return dx, dy, dz, ds

        # predictor (affine scaling)
        dx, dy, dz, ds = direction(s * z)
        a_aff = min(_max_step(s, ds), _max_step(z, dz))
        mu_aff = float((s + a_aff * ds) @ (z + a_aff * dz)) / max(mi, 1)
        sigma = (mu_aff / mu) ** 3 if mu > 0 else 0.0
        # corrector
        dx, dy, dz, ds = direction(s * z + ds * dz - sigma * mu)
        alpha = 0.99 * min(_max_step(s, ds), _max_step(z, dz))
        alpha = min(alpha, 1.0)
        x = x + alpha * dx
        y = y + alpha * dy
        z = z + alpha * dz
        s = s + alpha * ds
        s = np.maximum(s, 1e-300)
        z = np.maximum(z, 1e-300)
    if not converged and best[1] is not None:
        x, y, z, s, info = best[1]
        converged = best[0] < 1e-8
    return IPMResult(x, y, z, s, it, converged, info)
