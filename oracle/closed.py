"""Independent closed forms and brute force that pin the oracle.

Test infrastructure only (see the package docstring).  None of these calls the
interior-point method; they are what its results are checked against.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def waterfill(costs, caps, load, eps, voll, iters=200):
    """Single bus, one hour: generators (cost c_g, cap u_g) plus load shedding.

    With the eps/2 p^2 regularisation each generator's output at price lam is
    clip((lam - c_g)/eps, 0, u_g) (its marginal cost c_g + eps p meets lam), and
    the shed variable is a generator of cost VOLL and capacity L.  The price
    solves sum(output) = L; the sum is continuous and nondecreasing in lam, so
    bisection finds it.  Returns (p[G], shed, lam).
    """
    costs = np.asarray(costs, float)
    caps = np.asarray(caps, float)

    def supply(lam):
        p = np.clip((lam - costs) / eps, 0.0, caps)
        s = min(max((lam - voll) / eps, 0.0), load)
        return p, s

    lo = min(costs.min() if costs.size else voll, voll) - 1.0
    hi = voll + eps * load + 1.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        p, s = supply(mid)
        if p.sum() + s < load:
            lo = mid
        else:
            hi = mid
    lam = 0.5 * (lo + hi)
    p, s = supply(lam)
    return p, s, lam


def merit_order(costs, caps, load):
    """eps -> 0 limit: fill cheapest first; the price is the marginal unit's cost."""
    order = np.argsort(costs, kind="stable")
    p = np.zeros(len(costs))
    rem = load
    lam = None
    for g in order:
        take = min(caps[g], rem)
        p[g] = take
        rem -= take
        if rem <= 1e-12:
            lam = costs[g]
            break
    return p, lam


def two_bus_congested(c0, c1, L0, L1, eta_l, eps):
    """Cheap generator at bus 0, dear one at bus 1, one line 0->1 at its limit.

    Flow f = eta_l, p0 = L0 + f, p1 = L1 - f; prices lam_n = c_n + eps p_n; the
    derivative of the hourly cost in eta_l is -(lam1 - lam0).
    """
    p0 = L0 + eta_l
    p1 = L1 - eta_l
    lam0 = c0 + eps * p0
    lam1 = c1 + eps * p1
    return p0, p1, lam0, lam1, -(lam1 - lam0)


def battery_arbitrage(P, dur, eff_c, eff_d, spare_cheap):
    """Two hours on one bus: cheap energy in hour 0, dear energy in hour 1.

    The battery charges as much as it can in hour 0 (bounded by its power P,
    its energy dur*P / eff_c and the cheap generator's spare capacity), then
    empties in hour 1 (soc_1 = 0): dis_1 = eff_c * eff_d * ch_0.  Valid when the
    round trip is profitable and the discharge stays below P and the hour-1 load.
    """
    ch0 = min(P, dur * P / eff_c, spare_cheap)
    soc0 = eff_c * ch0
    dis1 = eff_d * soc0
    return ch0, dis1, soc0


def lp_vertex_enumeration(c, A, b, G, h, tol=1e-9, chunk=20000):
    """Brute force: minimise c^T x over the vertices of {A x = b, G x <= h}.

    Every vertex is the solution of A x = b together with n - rank(A) inequality
    rows held tight.  All such square systems are solved, infeasible points are
    dropped, and the cheapest remaining vertex is returned (bounded LPs only).
    """
    A = np.atleast_2d(np.asarray(A, float))
    G = np.atleast_2d(np.asarray(G, float))
    n = c.size
    me = A.shape[0]
    k = n - me
    best, best_x = math.inf, None
    combos = itertools.combinations(range(G.shape[0]), k)
    while True:
        block = list(itertools.islice(combos, chunk))
        if not block:
            break
        idx = np.array(block, dtype=np.int64)
        M = np.empty((len(block), n, n))
        M[:, :me, :] = A[None]
        M[:, me:, :] = G[idx]
        rhs = np.empty((len(block), n))
        rhs[:, :me] = b[None]
        rhs[:, me:] = h[idx]
        # |det M| against Hadamard's bound (product of row norms): near zero = singular
        det = np.abs(np.linalg.det(M))
        hb = np.prod(np.linalg.norm(M, axis=2), axis=1)
        ok = det > 1e-10 * hb
        if not np.any(ok):
            continue
        X = np.linalg.solve(M[ok], rhs[ok][..., None])[..., 0]
        feas = np.all(X @ G.T <= h[None] + tol * (1 + np.abs(h[None])), axis=1)
        if not np.any(feas):
            continue
        X = X[feas]
        vals = X @ c
        j = int(np.argmin(vals))
        if vals[j] < best:
            best, best_x = float(vals[j]), X[j]
    return best, best_x
