"""Dense/sparse assembly of one scenario's dispatch QP (Eq. 2), FP64.

Test infrastructure only (see the package docstring).

Variables, each a row of T hours, stacked in this order::

    p    [G, T]   generator output, MW
    sh   [N, T]   load shed at each bus, MW (served load is L - sh)
    th   [N, T]   bus voltage angle, rad
    ch   [B, T]   battery charging power, MW
    dis  [B, T]   battery discharging power, MW
    soc  [B, T]   battery state of charge at the end of hour t, MWh
    fdc  [Ld, T]  flow on each HVDC (transport) line, MW, from -> to

Objective c(x) = 1/2 x^T Q x + q^T x with
    sum_gt (c_g p + eps/2 p^2) + sum_nt (VOLL sh + eps/2 sh^2) + sum_bt eps/2 (ch^2 + dis^2)
    + sum_dc,t eps/2 fdc^2.

Capacity-dependent susceptance (``net["line_beta_ref"]`` > 0 for an AC line): the line's
susceptance scales with its planned capacity, beta_l(eta) = line_beta_l eta_l / ref_l, as when
capacity is added by parallel circuits.  The constraint matrix then depends on eta (the A(eta)
of Eq. 2); ``dA[k]`` and ``dG[k]`` hold its derivatives for such a line's plan entry k.

HVDC lines (``net["line_dc"]`` = 1) are transport links (Sections 2.1 and 3 name HVDC
among the planned assets): their flow is a free variable limited by eta_l, with no
angle coupling and no angle-difference limit, regularised like the other free
injections so the dispatch stays unique.

Equalities A x = b:
    balance (n,t): sum_{g at n} p + sum_{b at n} (dis - ch) + sh
                   - sum_{l from n} f_l + sum_{l to n} f_l = L_nt,
                   f_l = beta_l (th_f - th_t) for AC lines, fdc_l for HVDC lines
    dynamics (b,t): soc_t - soc_{t-1} - eff_c ch_t + dis_t / eff_d = 0,  soc_{-1} = 0
    reference (component, t): th_ref = 0   (angles are fixed up to a constant per island of
                              the AC lines)
    pinned: p_gt = 0 where cf_gt eta_g = 0, sh_nt = 0 where L_nt = 0 (coinciding bounds)

Inequalities G x <= h(eta) = h0 + D eta  (the capacity dependence b(eta) of Eq. 2):
    p <= cf eta_g,  -p <= 0,  sh <= L,  -sh <= 0,
    +-beta (th_f - th_t) <= eta_l,  +-(th_f - th_t) <= dtheta_max   (AC lines),
    +-fdc <= eta_l   (HVDC lines),
    +-(p_t - p_{t-1}) <= r_g eta_g, t >= 1   (ramping generators: 0 < r_g < 1, the hourly
                                             ramp limit as a fraction of capacity),
    ch <= eta_b, -ch <= 0, dis <= eta_b, -dis <= 0, soc <= dur eta_b, -soc <= 0.

The nodal price is lambda_nt = -y_nt, y the multiplier of the balance row in
the Lagrangian c(x) + y^T (A x - b) + z^T (G x - h).

The planner objective of Eq. 1 for this scenario is
    h(x) = c(x) + kappa * sum_gt e_g p_gt      (emissions-aware planning, Section 2.1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def components(n_bus, lf, lt):
    """Connected components of the bus graph (union-find); returns a label per bus."""
    parent = list(range(n_bus))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in zip(lf.tolist(), lt.tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(i) for i in range(n_bus)])
    _, lab = np.unique(roots, return_inverse=True)
    return lab


class DispatchQP:
    """One scenario's QP with index maps back to the device arrays."""

    def __init__(self, net, scen, eta, opts):
        N = int(net["n_bus"])
        T = int(scen["T"])
        G = net["gen_bus"].size
        L = net["line_from"].size
        B = net["bat_bus"].size
        eps = float(opts["eps"])
        voll = float(opts["voll"])
        self.N, self.T, self.G, self.L, self.B = N, T, G, L, B
        self.K = G + L + B
        dc = np.asarray(net.get("line_dc", np.zeros(L)), dtype=bool)
        self.dc_lines = np.where(dc)[0]
        self.ac_lines = np.where(~dc)[0]
        Ld = self.dc_lines.size
        self.Ld = Ld
        dc_row = {int(l): j for j, l in enumerate(self.dc_lines)}
        # effective susceptances: fixed, or scaling with the line's capacity
        bref = np.asarray(net.get("line_beta_ref", np.zeros(L)), dtype=np.float64)
        beta0 = np.asarray(net["line_beta"], dtype=np.float64)
        self.scaling = np.where((bref > 0) & ~dc)[0]
        self.beta = beta0.copy()
        self.beta[self.scaling] = beta0[self.scaling] * eta[G + self.scaling] / bref[self.scaling]
        dA_entries = {int(G + l): ([], [], []) for l in self.scaling}  # rows, cols, vals of dA / deta_k
        dG_entries = {int(G + l): ([], [], []) for l in self.scaling}
        eta = np.asarray(eta, dtype=np.float64)
        assert eta.shape == (self.K,)
        self.eta = eta.copy()
        eg, el, eb = eta[:G], eta[G:G + L], eta[G + L:]

        # --- variable offsets
        off = {}
        o = 0
        for name, rows in (("p", G), ("sh", N), ("th", N), ("ch", B), ("dis", B), ("soc", B), ("fdc", Ld)):
            off[name] = o
            o += rows * T
        self.n = o
        self.off = off

        def vid(name, row, t):
            return off[name] + row * T + t

        self.vid = vid
        tt = np.arange(T)

        # --- objective
        Qd = np.zeros(self.n)
        q = np.zeros(self.n)
        for name, rows in (("p", G), ("sh", N), ("ch", B), ("dis", B), ("fdc", Ld)):
            Qd[off[name]:off[name] + rows * T] = eps
        q[off["p"]:off["p"] + G * T] = np.repeat(net["gen_cost"], T)
        q[off["sh"]:off["sh"] + N * T] = voll
        self.Qd = Qd
        self.Q = sp.diags(Qd).tocsc()
        self.q = q
        self.emis_vec = np.zeros(self.n)
        self.emis_vec[off["p"]:off["p"] + G * T] = np.repeat(net["gen_emis"], T)

        # --- equalities
        rows, cols, vals = [], [], []
        b = []
        r = 0
        self.row_bal = r
        load = np.asarray(scen["load"], dtype=np.float64)
        for n in range(N):
            for t in range(T):
                b.append(load[n, t])
        for g in range(G):
            n = int(net["gen_bus"][g])
            rows += list(r + n * T + tt)
            cols += [vid("p", g, t) for t in range(T)]
            vals += [1.0] * T
        for n in range(N):
            rows += list(r + n * T + tt)
            cols += [vid("sh", n, t) for t in range(T)]
            vals += [1.0] * T
        for bb in range(B):
            n = int(net["bat_bus"][bb])
            rows += list(r + n * T + tt)
            cols += [vid("dis", bb, t) for t in range(T)]
            vals += [1.0] * T
            rows += list(r + n * T + tt)
            cols += [vid("ch", bb, t) for t in range(T)]
            vals += [-1.0] * T
        for l in range(L):
            f, to, beta = int(net["line_from"][l]), int(net["line_to"][l]), float(self.beta[l])
            if l in dc_row:
                # HVDC: the flow variable leaves bus f and enters bus to
                for t in range(T):
                    rows += [r + f * T + t, r + to * T + t]
                    cols += [vid("fdc", dc_row[l], t), vid("fdc", dc_row[l], t)]
                    vals += [-1.0, 1.0]
                continue
            # flow f_lt = beta (th_f - th_t) leaves bus f and enters bus to
            for t in range(T):
                rows += [r + f * T + t, r + f * T + t, r + to * T + t, r + to * T + t]
                cols += [vid("th", f, t), vid("th", to, t), vid("th", f, t), vid("th", to, t)]
                vals += [-beta, beta, beta, -beta]
                if G + l in dA_entries:  # d beta / d eta_l = beta / eta_l
                    db = beta / float(eta[G + l])
                    e = dA_entries[G + l]
                    e[0].extend([r + f * T + t, r + f * T + t, r + to * T + t, r + to * T + t])
                    e[1].extend([vid("th", f, t), vid("th", to, t), vid("th", f, t), vid("th", to, t)])
                    e[2].extend([-db, db, db, -db])
        r += N * T
        self.row_dyn = r
        for bb in range(B):
            ec, ed = float(net["bat_eff_c"][bb]), float(net["bat_eff_d"][bb])
            for t in range(T):
                rows.append(r + bb * T + t); cols.append(vid("soc", bb, t)); vals.append(1.0)
                if t > 0:
                    rows.append(r + bb * T + t); cols.append(vid("soc", bb, t - 1)); vals.append(-1.0)
                rows.append(r + bb * T + t); cols.append(vid("ch", bb, t)); vals.append(-ec)
                rows.append(r + bb * T + t); cols.append(vid("dis", bb, t)); vals.append(1.0 / ed)
                b.append(0.0)
        r += B * T
        self.row_ref = r
        lab = components(N, np.asarray(net["line_from"])[self.ac_lines], np.asarray(net["line_to"])[self.ac_lines])
        self.comp = lab
        self.ref_bus = np.array([int(np.where(lab == c)[0][0]) for c in range(lab.max() + 1)])
        for rb in self.ref_bus:
            for t in range(T):
                rows.append(r); cols.append(vid("th", int(rb), t)); vals.append(1.0)
                b.append(0.0)
                r += 1
        # A box whose bounds coincide (zero capacity factor, zero load) fixes its
        # variable: written as an equality so the interior-point method never has
        # to squeeze two slacks to zero.  Both bounds have zero eta-derivative there
        # (cf = 0; the load does not depend on eta).
        cf_in = np.asarray(scen["cf"], dtype=np.float64)
        self.pinned = set()
        for g in range(G):
            for t in range(T):
                if cf_in[g, t] * eg[g] == 0.0:
                    rows.append(r); cols.append(vid("p", g, t)); vals.append(1.0); b.append(0.0); r += 1
                    self.pinned.add(("p", g, t))
        for n in range(N):
            for t in range(T):
                if load[n, t] == 0.0:
                    rows.append(r); cols.append(vid("sh", n, t)); vals.append(1.0); b.append(0.0); r += 1
                    self.pinned.add(("sh", n, t))
        self.m_eq = r
        self.A = sp.csr_matrix((vals, (rows, cols)), shape=(r, self.n))
        self.b = np.array(b)

        # --- inequalities G x <= h0 + D eta
        grows, gcols, gvals = [], [], []
        h0 = []
        drows, dcols, dvals = [], [], []
        kind = []  # (tag, device, t) per row, for reading multipliers back
        m = 0

        def add_row(entries, rhs0, dk=None, dv=0.0, tag=None):
            nonlocal m
            for c, v in entries:
                grows.append(m); gcols.append(c); gvals.append(v)
            h0.append(rhs0)
            if dk is not None:
                drows.append(m); dcols.append(dk); dvals.append(dv)
            kind.append(tag)
            m += 1

        cf = np.asarray(scen["cf"], dtype=np.float64)
        for g in range(G):
            for t in range(T):
                if ("p", g, t) in self.pinned:
                    continue
                add_row([(vid("p", g, t), 1.0)], 0.0, g, cf[g, t], ("p_up", g, t))
                add_row([(vid("p", g, t), -1.0)], 0.0, tag=("p_lo", g, t))
        ramp = np.asarray(net.get("gen_ramp", np.zeros(G)), dtype=np.float64)
        self.ramp_gens = np.where((ramp > 0.0) & (ramp < 1.0))[0]
        for g in self.ramp_gens:
            r = float(ramp[g])
            for t in range(1, T):
                a, b0 = vid("p", g, t), vid("p", g, t - 1)
                add_row([(a, 1.0), (b0, -1.0)], 0.0, int(g), r, ("r_up", int(g), t))
                add_row([(a, -1.0), (b0, 1.0)], 0.0, int(g), r, ("r_lo", int(g), t))
        for n in range(N):
            for t in range(T):
                if ("sh", n, t) in self.pinned:
                    continue
                add_row([(vid("sh", n, t), 1.0)], load[n, t], tag=("sh_up", n, t))
                add_row([(vid("sh", n, t), -1.0)], 0.0, tag=("sh_lo", n, t))
        for l in range(L):
            f, to = int(net["line_from"][l]), int(net["line_to"][l])
            if l in dc_row:
                for t in range(T):
                    v = vid("fdc", dc_row[l], t)
                    add_row([(v, 1.0)], 0.0, G + l, 1.0, ("f_up", l, t))
                    add_row([(v, -1.0)], 0.0, G + l, 1.0, ("f_lo", l, t))
                continue
            beta = float(self.beta[l])
            dth = float(net["line_dtheta"][l])
            for t in range(T):
                a, c = vid("th", f, t), vid("th", to, t)
                if G + l in dG_entries:
                    db = beta / float(eta[G + l])
                    e = dG_entries[G + l]
                    e[0].extend([m, m, m + 1, m + 1])
                    e[1].extend([a, c, a, c])
                    e[2].extend([db, -db, -db, db])
                add_row([(a, beta), (c, -beta)], 0.0, G + l, 1.0, ("f_up", l, t))
                add_row([(a, -beta), (c, beta)], 0.0, G + l, 1.0, ("f_lo", l, t))
                add_row([(a, 1.0), (c, -1.0)], dth, tag=("a_up", l, t))
                add_row([(a, -1.0), (c, 1.0)], dth, tag=("a_lo", l, t))
        for bb in range(B):
            dur = float(net["bat_dur"][bb])
            for t in range(T):
                add_row([(vid("ch", bb, t), 1.0)], 0.0, G + L + bb, 1.0, ("ch_up", bb, t))
                add_row([(vid("ch", bb, t), -1.0)], 0.0, tag=("ch_lo", bb, t))
                add_row([(vid("dis", bb, t), 1.0)], 0.0, G + L + bb, 1.0, ("dis_up", bb, t))
                add_row([(vid("dis", bb, t), -1.0)], 0.0, tag=("dis_lo", bb, t))
                add_row([(vid("soc", bb, t), 1.0)], 0.0, G + L + bb, dur, ("soc_up", bb, t))
                add_row([(vid("soc", bb, t), -1.0)], 0.0, tag=("soc_lo", bb, t))
        self.m_in = m
        self.Gm = sp.csr_matrix((gvals, (grows, gcols)), shape=(m, self.n))
        self.dA = {k: sp.csr_matrix((v, (r_, c_)), shape=(self.m_eq, self.n)) for k, (r_, c_, v) in dA_entries.items()}
        self.dG = {k: sp.csr_matrix((v, (r_, c_)), shape=(m, self.n)) for k, (r_, c_, v) in dG_entries.items()}
        self.h0 = np.array(h0)
        self.D = sp.csr_matrix((dvals, (drows, dcols)), shape=(m, self.K))
        self.h = self.h0 + self.D @ eta
        self.kind = kind
        self.eps, self.voll = eps, voll
        self.net, self.scen = net, scen

    # ---- helpers --------------------------------------------------------------
    def unpack(self, x):
        T = self.T
        o = self.off
        return dict(
            p=x[o["p"]:o["p"] + self.G * T].reshape(self.G, T),
            sh=x[o["sh"]:o["sh"] + self.N * T].reshape(self.N, T),
            th=x[o["th"]:o["th"] + self.N * T].reshape(self.N, T),
            ch=x[o["ch"]:o["ch"] + self.B * T].reshape(self.B, T),
            dis=x[o["dis"]:o["dis"] + self.B * T].reshape(self.B, T),
            soc=x[o["soc"]:o["soc"] + self.B * T].reshape(self.B, T),
            fdc=x[o["fdc"]:o["fdc"] + self.Ld * T].reshape(self.Ld, T),
        )

    def pack(self, p, sh, th, ch, dis, soc, fdc=None):
        """x from device arrays; `fdc` may be the flows of all L lines (the HVDC rows are taken)."""
        if fdc is None:
            fdc = np.zeros((self.Ld, self.T))
        fdc = np.asarray(fdc, dtype=np.float64)
        if fdc.shape[0] == self.L and self.L != self.Ld:
            fdc = fdc[self.dc_lines]
        return np.concatenate([np.ravel(p), np.ravel(sh), np.ravel(th), np.ravel(ch), np.ravel(dis), np.ravel(soc),
                               np.ravel(fdc)])

    def cost(self, x):
        """Operating cost c(x) of Eq. 2 (with the eps regularisation), FP64."""
        return float(0.5 * x @ (self.Qd * x) + self.q @ x)

    def planner(self, x, kappa):
        """Planner objective h(x) = c(x) + kappa * emissions (Section 2.1)."""
        return self.cost(x) + float(kappa) * float(self.emis_vec @ x)

    def planner_grad(self, x, kappa):
        return self.Qd * x + self.q + float(kappa) * self.emis_vec

    def flows(self, th, fdc=None):
        """Flow of every line, from -> to: beta (th_f - th_t) on AC lines, the flow
        variable on HVDC lines."""
        lf, lt = self.net["line_from"], self.net["line_to"]
        f = self.beta[:, None] * (th[lf] - th[lt])
        if self.Ld:
            f[self.dc_lines] = fdc if fdc is not None else 0.0
        return f
