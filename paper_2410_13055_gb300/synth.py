"""Seeded synthetic networks and scenarios shaped like the paper's Western-US cases.

This module only draws inputs. It holds none of the dispatch arithmetic, so the
FP64 oracle and the CUDA path can both be fed from it without sharing any of
the method's code.

The paper plans generation, storage and transmission capacity on PyPSA-USA
Western Interconnect cases of 100 to 500 nodes with 24-hour scenarios
(Section 3, "Results"; Section 3.1 gives the 500-node mix: 1799 generators,
1191 AC lines, 576 batteries).  That data is not available here, so these
generators stand in for it with the same kinds of devices and per-bus ratios:

* tiny      5-bus ring + 2 chords, 6 generators, 2 batteries, T=24, 1 scenario
* medium    100-bus random geometric graph, 150 lines, 300 generators
            (gas / solar / wind thirds), 50 batteries, T=168, 16 scenarios
* batching  64 scenarios, each with its own network of 50..500 buses
            (1.5 lines, 3 generators, 0.3 batteries per bus) and T in {24,72,168}
* scale     2000 buses, 3000 lines, 8000 generators, 500 batteries, 52 weekly
            scenarios of T=168

Data format (plain dicts of numpy arrays; FP64, indices int64):

network
    n_bus                 number of buses N
    gen_bus, gen_cost     [G] bus index, marginal cost $/MWh
    gen_emis, gen_kind    [G] emission rate t/MWh, 0 = gas, 1 = solar, 2 = wind
    line_from, line_to    [L] bus indices
    line_beta             [L] MW per rad (100 MVA base x susceptance in p.u.)
    line_dtheta           [L] angle-difference limit, rad
    bat_bus               [Bt]
    bat_dur               [Bt] hours of energy at full power
    bat_eff_c, bat_eff_d  [Bt] charge / discharge efficiency
    eta_min, eta_max      [K] plan bounds, K = G + L + Bt, layout [gen | line | battery]
    gamma                 [K] investment cost per MW for one scenario period
scenario
    net                   index into the list of networks
    T                     hours
    load                  [N, T] MW
    cf                    [G, T] capacity factor in [0, 1]
    weight                scenario weight w_s (1/S by default)
"""
from __future__ import annotations

import math

import numpy as np

GAS, SOLAR, WIND = 0, 1, 2

# Annualised investment costs, $/MW-yr (a synthetic stand-in for ATB figures).
GAMMA_ANNUAL = {GAS: 60e3, SOLAR: 70e3, WIND: 110e3}
GAMMA_LINE_ANNUAL = 30e3
BATTERY_COST_PER_KWH = 250.0
CAPITAL_RECOVERY = 0.1


def battery_gamma_annual(cost_per_kwh: float, duration_h: float = 4.0) -> float:
    """$/MW-yr for a battery of the given duration at a capital cost in $/kWh."""
    return cost_per_kwh * duration_h * 1000.0 * CAPITAL_RECOVERY


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _solar_cf(rng, n, T):
    h = np.arange(T) % 24
    shape = np.maximum(0.0, np.sin(np.pi * (h - 6) / 12.0))
    days = (T + 23) // 24
    amp = rng.beta(5.0, 2.0, size=(n, days))
    amp_t = np.repeat(amp, 24, axis=1)[:, :T]
    return shape[None, :] * amp_t


def _wind_cf(rng, n, T, mu=0.35, rho=0.9, sigma=0.25):
    x = np.empty((n, T))
    x[:, 0] = mu + sigma * rng.standard_normal(n)
    innov = sigma * math.sqrt(1.0 - rho * rho)
    for t in range(1, T):
        x[:, t] = mu + rho * (x[:, t - 1] - mu) + innov * rng.standard_normal(n)
    return np.clip(x, 0.0, 1.0)


def _daily_load(rng, base, T, amp_frac, phase_h, noise=0.05):
    t = np.arange(T)[None, :]
    shape = 1.0 + amp_frac * np.sin(2 * np.pi * (t - 8.0 - phase_h[:, None]) / 24.0)
    L = base[:, None] * shape * (1.0 + noise * rng.standard_normal((base.size, T)))
    return np.maximum(L, 0.0)


def _geometric_graph(rng, n, n_lines):
    """Random geometric graph: minimum spanning tree plus the shortest extra edges."""
    pts = rng.random((n, 2))
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    # Prim's MST on the complete graph.
    in_tree = np.zeros(n, bool)
    best = np.full(n, np.inf)
    parent = np.full(n, -1)
    best[0] = 0.0
    edges = []
    for _ in range(n):
        cand = np.where(in_tree, np.inf, best)
        v = int(np.argmin(cand))
        in_tree[v] = True
        if parent[v] >= 0:
            edges.append((int(parent[v]), v))
        upd = (~in_tree) & (d[v] < best)
        best[upd] = d[v][upd]
        parent[upd] = v
    have = {(min(a, b), max(a, b)) for a, b in edges}
    extra = n_lines - len(edges)
    if extra > 0:
        iu, ju = np.triu_indices(n, 1)
        order = np.argsort(d[iu, ju], kind="stable")
        for k in order:
            e = (int(iu[k]), int(ju[k]))
            if e in have:
                continue
            have.add(e)
            edges.append(e)
            if len(edges) == n_lines:
                break
    e = np.array(edges, dtype=np.int64)
    return e[:, 0], e[:, 1]


def _finish_network(net, gen_kind, gen_cap, line_cap, bat_cap, bat_cost_kwh, T_period):
    G, L, B = gen_kind.size, line_cap.size, bat_cap.size
    eta_min = np.concatenate([gen_cap, line_cap, bat_cap]).astype(np.float64)
    gmax = np.where(gen_kind == GAS, 2.0, 3.0) * gen_cap
    lmax = 2.0 * line_cap
    bmax = 3.0 * np.maximum(bat_cap, 50.0)
    eta_max = np.concatenate([gmax, lmax, bmax])
    scale = T_period / 8760.0
    g_gam = np.array([GAMMA_ANNUAL[int(k)] for k in gen_kind]) * scale
    l_gam = np.full(L, GAMMA_LINE_ANNUAL * scale)
    b_gam = np.full(B, battery_gamma_annual(bat_cost_kwh) * scale)
    net["eta_min"] = eta_min
    net["eta_max"] = eta_max
    net["gamma"] = np.concatenate([g_gam, l_gam, b_gam])
    net["K"] = G + L + B
    return net


def _bus_network(rng, n_bus, n_lines, n_gen, n_bat, T_period, bat_cost_kwh=BATTERY_COST_PER_KWH,
                 gen_scale=1.0):
    lf, lt = _geometric_graph(rng, n_bus, n_lines)
    L = lf.size
    beta = 100.0 * rng.lognormal(math.log(10.0), 0.5, size=L)
    line_cap = rng.uniform(100.0, 400.0, size=L)
    kinds = np.array([GAS, SOLAR, WIND])[np.arange(n_gen) % 3]
    rng.shuffle(kinds)
    gen_bus = rng.integers(0, n_bus, size=n_gen)
    cost = np.where(kinds == GAS, rng.uniform(20.0, 80.0, size=n_gen), 0.0)
    emis = np.where(kinds == GAS, rng.uniform(0.35, 0.6, size=n_gen), 0.0)
    gen_cap = gen_scale * rng.uniform(50.0, 300.0, size=n_gen)
    bat_bus = rng.integers(0, n_bus, size=n_bat)
    bat_cap = rng.uniform(0.0, 200.0, size=n_bat)
    net = dict(
        n_bus=int(n_bus),
        gen_bus=gen_bus.astype(np.int64), gen_cost=cost, gen_emis=emis, gen_kind=kinds.astype(np.int64),
        line_from=lf, line_to=lt, line_beta=beta, line_dtheta=np.full(L, math.pi / 6),
        bat_bus=bat_bus.astype(np.int64), bat_dur=np.full(n_bat, 4.0),
        bat_eff_c=np.full(n_bat, math.sqrt(0.9)), bat_eff_d=np.full(n_bat, math.sqrt(0.9)),
    )
    return _finish_network(net, kinds, gen_cap, line_cap, bat_cap, bat_cost_kwh, T_period)


def _bus_scenario(rng, net, net_idx, T, weight, load_base):
    N = net["n_bus"]
    kinds = net["gen_kind"]
    G = kinds.size
    cf = np.ones((G, T))
    sol = np.where(kinds == SOLAR)[0]
    win = np.where(kinds == WIND)[0]
    if sol.size:
        cf[sol] = _solar_cf(rng, sol.size, T)
    if win.size:
        cf[win] = _wind_cf(rng, win.size, T)
    phase = rng.uniform(-2.0, 2.0, size=N)
    load = _daily_load(rng, load_base, T, 0.4, phase)
    return dict(net=net_idx, T=int(T), load=load, cf=cf, weight=float(weight))


def tiny(seed: int = 0):
    """5-bus ring with 2 chords (7 lines), 6 generators, 2 batteries, 5 loads, T=24, S=1."""
    rng = _rng(seed)
    T = 24
    lf = np.array([0, 1, 2, 3, 4, 0, 1], dtype=np.int64)
    lt = np.array([1, 2, 3, 4, 0, 2, 3], dtype=np.int64)
    beta = 100.0 * rng.uniform(5.0, 20.0, size=7)
    line_cap = rng.uniform(100.0, 400.0, size=7)
    gen_bus = np.array([0, 0, 1, 2, 3, 4], dtype=np.int64)
    cost = rng.uniform(10.0, 100.0, size=6)
    gen_cap = rng.uniform(50.0, 300.0, size=6)
    emis = rng.uniform(0.3, 0.9, size=6)
    bat_bus = np.array([1, 3], dtype=np.int64)
    bat_cap = rng.uniform(0.0, 200.0, size=2)
    kinds = np.zeros(6, dtype=np.int64)
    net = dict(
        n_bus=5, gen_bus=gen_bus, gen_cost=cost, gen_emis=emis, gen_kind=kinds,
        line_from=lf, line_to=lt, line_beta=beta, line_dtheta=np.full(7, math.pi / 6),
        bat_bus=bat_bus, bat_dur=np.full(2, 4.0),
        bat_eff_c=np.full(2, math.sqrt(0.9)), bat_eff_d=np.full(2, math.sqrt(0.9)),
    )
    net = _finish_network(net, kinds, gen_cap, line_cap, bat_cap, BATTERY_COST_PER_KWH, T)
    t = np.arange(T)
    shape = 150.0 + 100.0 * np.sin(2 * np.pi * (t - 8) / 24.0)
    load = shape[None, :] * (1.0 + 0.05 * rng.standard_normal((5, T)))
    scen = dict(net=0, T=T, load=np.maximum(load, 0.0), cf=np.ones((6, T)), weight=1.0)
    return [net], [scen]


def medium(seed: int = 1, S: int = 16, T: int = 168, bat_cost_kwh: float = BATTERY_COST_PER_KWH,
           scen_seed: int | None = None):
    """100-bus geometric graph, 150 lines, 300 generators, 50 batteries, 100 loads, T=168, S=16.

    With `scen_seed`, the scenarios (weather and load draws) come from their own seed
    while the network stays that of `seed` (independent scenario shards of one network)."""
    rng = _rng(seed)
    net = _bus_network(rng, 100, 150, 300, 50, T, bat_cost_kwh=bat_cost_kwh)
    base = rng.uniform(50.0, 150.0, size=100)
    srng = rng if scen_seed is None else _rng(scen_seed)
    scens = [_bus_scenario(srng, net, 0, T, 1.0 / S, base) for _ in range(S)]
    return [net], scens


def batching(seed: int = 2, S: int = 64):
    """S scenarios, each on its own network of 50..500 buses, horizon drawn from {24, 72, 168}."""
    rng = _rng(seed)
    nets, scens = [], []
    for s in range(S):
        N = int(rng.integers(50, 501))
        T = int(rng.choice([24, 72, 168]))
        net = _bus_network(rng, N, int(round(1.5 * N)), 3 * N, max(1, int(round(0.3 * N))), T)
        base = rng.uniform(50.0, 150.0, size=N)
        nets.append(net)
        scens.append(_bus_scenario(rng, net, s, T, 1.0 / S, base))
    return nets, scens


def scale(seed: int = 3, S: int = 52, T: int = 168, scen_seed: int | None = None, weight: float | None = None):
    """2000 buses, 3000 lines, 8000 generators, 500 batteries, 2000 loads, 52 weeks of T=168.

    With `scen_seed`, the scenarios come from their own seed on the network of `seed`;
    `weight` overrides the scenario weight 1/S (one shard of a larger set)."""
    rng = _rng(seed)
    net = _bus_network(rng, 2000, 3000, 8000, 500, T, gen_scale=0.75)
    base = rng.uniform(50.0, 150.0, size=2000)
    srng = rng if scen_seed is None else _rng(scen_seed)
    w = 1.0 / S if weight is None else weight
    scens = [_bus_scenario(srng, net, 0, T, w, base) for _ in range(S)]
    return [net], scens


def custom(n_bus, n_lines, n_gen, n_bat, T, S=1, seed=0, net_index=0):
    """A network of the given size with the medium case's distributions and S scenarios."""
    rng = _rng(seed)
    net = _bus_network(rng, n_bus, n_lines, n_gen, n_bat, T)
    base = rng.uniform(50.0, 150.0, size=n_bus)
    scens = [_bus_scenario(rng, net, net_index, T, 1.0 / S, base) for _ in range(S)]
    return net, scens


def add_hvdc(net, n_dc, seed=0, cap=(200.0, 600.0)):
    """Append `n_dc` HVDC transport lines between random bus pairs not already joined
    (the paper's WECC case plans 3 HVDC lines next to 1191 AC lines).  Their plan entries
    go at the end of the line block: eta_min = U[cap], eta_max = 2 eta_min, gamma = the
    line rate.  Returns a new network dict (inputs only)."""
    rng = _rng(seed)
    N = int(net["n_bus"])
    G, L = net["gen_bus"].size, net["line_from"].size
    have = set(zip(net["line_from"].tolist(), net["line_to"].tolist()))
    pairs = []
    while len(pairs) < n_dc:
        a, b = (int(x) for x in rng.choice(N, size=2, replace=False))
        if (a, b) not in have and (b, a) not in have:
            have.add((a, b))
            pairs.append((a, b))
    out = dict(net)
    fa = np.array([p[0] for p in pairs], dtype=np.int64)
    ta = np.array([p[1] for p in pairs], dtype=np.int64)
    c = rng.uniform(cap[0], cap[1], size=n_dc)
    out["line_from"] = np.concatenate([net["line_from"], fa])
    out["line_to"] = np.concatenate([net["line_to"], ta])
    out["line_beta"] = np.concatenate([net["line_beta"], np.ones(n_dc)])
    out["line_dtheta"] = np.concatenate([net["line_dtheta"], np.full(n_dc, math.pi / 6)])
    out["line_dc"] = np.concatenate([np.asarray(net.get("line_dc", np.zeros(L)), np.uint8), np.ones(n_dc, np.uint8)])
    rate = net["gamma"][G] if L else GAMMA_LINE_ANNUAL / 8760.0
    ins = lambda v, new: np.concatenate([v[:G + L], new, v[G + L:]])
    out["eta_min"] = ins(net["eta_min"], c)
    out["eta_max"] = ins(net["eta_max"], 2.0 * c)
    out["gamma"] = ins(net["gamma"], np.full(n_dc, rate))
    out["K"] = int(net["K"]) + n_dc
    return out


def add_ramps(net, rate=(0.1, 0.3), share=1.0, seed=0):
    """Give a share of the gas generators an hourly ramp limit drawn from U[rate] as a
    fraction of their capacity (``gen_ramp``; renewables stay unlimited).  Returns a new
    network dict (inputs only)."""
    rng = _rng(seed)
    G = net["gen_bus"].size
    out = dict(net)
    ramp = np.zeros(G)
    gas = np.where(np.asarray(net.get("gen_kind", np.zeros(G))) == GAS)[0]
    pick = gas[rng.random(gas.size) < share]
    ramp[pick] = rng.uniform(rate[0], rate[1], size=pick.size)
    out["gen_ramp"] = ramp
    return out


def add_scaling(net, share=0.3, seed=0):
    """Let a share of the AC lines gain susceptance with capacity (``line_beta_ref`` = their
    existing capacity eta_min, so beta is the given one at eta_min and grows in proportion
    as circuits are added).  Returns a new network dict (inputs only)."""
    rng = _rng(seed)
    G, L = net["gen_bus"].size, net["line_from"].size
    out = dict(net)
    dc = np.asarray(net.get("line_dc", np.zeros(L)), bool)
    pick = (rng.random(L) < share) & ~dc
    out["line_beta_ref"] = np.where(pick, np.asarray(net["eta_min"][G:G + L], float), 0.0)
    return out


CONFIGS = {"tiny": tiny, "medium": medium, "batching": batching, "scale": scale}


def make(name: str, **kw):
    return CONFIGS[name](**kw)


def device_hours(nets, scens) -> int:
    """sum_s (generators + lines + batteries + loads) * T_s."""
    tot = 0
    for sc in scens:
        n = nets[sc["net"]]
        devs = n["gen_bus"].size + n["line_from"].size + n["bat_bus"].size + n["n_bus"]
        tot += devs * sc["T"]
    return int(tot)


def slice_hours(nets, scens, t0: int, T: int):
    """Scenarios restricted to hours [t0, t0+T) (a bounded sample of a workload)."""
    out = []
    for sc in scens:
        out.append(dict(net=sc["net"], T=int(T), load=sc["load"][:, t0:t0 + T].copy(),
                        cf=sc["cf"][:, t0:t0 + T].copy(), weight=sc["weight"]))
    return nets, out


def default_opts(**kw):
    """Model constants shared by both sides as *inputs* (not method arithmetic)."""
    o = dict(eps=1e-3, voll=1000.0, kappa=0.0)
    o.update(kw)
    return o
