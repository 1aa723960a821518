"""Input generators: seeded, shaped like the documented workloads, and the device-model
extension helpers leave the base network's arrays untouched (inputs only, no method
arithmetic)."""
import numpy as np

from paper_2410_13055_gb300 import synth


def test_generators_are_seeded():
    a, sa = synth.medium(S=2, T=24)
    b, sb = synth.medium(S=2, T=24)
    for k in ("gen_cost", "line_beta", "eta_min", "gamma"):
        assert np.array_equal(a[0][k], b[0][k])
    assert np.array_equal(sa[1]["load"], sb[1]["load"]) and np.array_equal(sa[1]["cf"], sb[1]["cf"])
    c, _ = synth.medium(seed=2, S=2, T=24)
    assert not np.array_equal(a[0]["gen_cost"], c[0]["gen_cost"])


def test_medium_shapes():
    nets, scens = synth.medium(S=3, T=48)
    n = nets[0]
    assert int(n["n_bus"]) == 100 and n["line_from"].size == 150
    assert n["gen_bus"].size == 300 and n["bat_bus"].size == 50
    assert n["K"] == 500 and n["eta_min"].size == 500
    assert all(s["load"].shape == (100, 48) and s["cf"].shape == (300, 48) for s in scens)
    assert np.all((scens[0]["cf"] >= 0) & (scens[0]["cf"] <= 1))
    assert np.all(n["eta_max"] >= n["eta_min"])


def test_add_scaling_marks_a_share_of_ac_lines():
    nets, _ = synth.medium(S=1, T=24)
    base = nets[0]
    G, L = base["gen_bus"].size, base["line_from"].size
    out = synth.add_scaling(base, share=0.3, seed=5)
    ref = out["line_beta_ref"]
    picked = ref > 0
    assert 0.15 < picked.mean() < 0.45
    assert np.allclose(ref[picked], base["eta_min"][G:G + L][picked])
    assert "line_beta_ref" not in base and np.array_equal(out["line_beta"], base["line_beta"])
    # HVDC links never scale
    dc = synth.add_hvdc(base, 3, seed=1, cap=(60.0, 150.0))
    ref_dc = synth.add_scaling(dc, share=1.0, seed=2)["line_beta_ref"]
    assert np.all(ref_dc[dc["line_dc"] == 1] == 0) and np.all(ref_dc[dc["line_dc"] == 0] > 0)


def test_add_ramps_limits_gas_units_only():
    nets, _ = synth.medium(S=1, T=24)
    base = nets[0]
    out = synth.add_ramps(base, rate=(0.1, 0.3), share=1.0, seed=7)
    r = out["gen_ramp"]
    gas = np.asarray(base["gen_kind"]) == synth.GAS
    assert np.all((r[gas] >= 0.1) & (r[gas] <= 0.3)) and np.all(r[~gas] == 0)
    assert "gen_ramp" not in base


def test_add_hvdc_appends_transport_lines():
    nets, _ = synth.medium(S=1, T=24)
    base = nets[0]
    G, L = base["gen_bus"].size, base["line_from"].size
    out = synth.add_hvdc(base, 3, seed=1, cap=(60.0, 150.0))
    assert out["line_from"].size == L + 3 and out["K"] == base["K"] + 3
    assert np.all(out["line_dc"][:L] == 0) and np.all(out["line_dc"][L:] == 1)
    assert np.all(out["line_from"][L:] != out["line_to"][L:])
    cap = out["eta_min"][G + L:G + L + 3]
    assert np.all((cap >= 60.0) & (cap <= 150.0))
    # the plan vector keeps generators first and batteries last
    assert np.array_equal(out["eta_min"][:G + L], base["eta_min"][:G + L])
    assert np.array_equal(out["eta_min"][G + L + 3:], base["eta_min"][G + L:])


def _connected(n_bus, lf, lt):
    adj = [[] for _ in range(n_bus)]
    for a, b in zip(lf.tolist(), lt.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    seen, stack = {0}, [0]
    while stack:
        for w in adj[stack.pop()]:
            if w not in seen:
                seen.add(w)
                stack.append(w)
    return len(seen) == n_bus


def _simple_graph(lf, lt):
    pairs = {(min(a, b), max(a, b)) for a, b in zip(lf.tolist(), lt.tolist())}
    return len(pairs) == lf.size and np.all(lf != lt)


def test_tiny_recipe():
    nets, scens = synth.tiny()
    n, sc = nets[0], scens[0]
    assert int(n["n_bus"]) == 5 and n["line_from"].size == 7 and n["gen_bus"].size == 6 and n["bat_bus"].size == 2
    # a ring over the five buses plus two chords
    ring = {(min(a, (a + 1) % 5), max(a, (a + 1) % 5)) for a in range(5)}
    pairs = {(min(a, b), max(a, b)) for a, b in zip(n["line_from"].tolist(), n["line_to"].tolist())}
    assert ring <= pairs and len(pairs - ring) == 2 and _simple_graph(n["line_from"], n["line_to"])
    assert np.all((n["line_beta"] >= 500) & (n["line_beta"] <= 2000))
    G, L = 6, 7
    assert np.all((n["eta_min"][G:G + L] >= 100) & (n["eta_min"][G:G + L] <= 400))
    assert np.all((n["gen_cost"] >= 10) & (n["gen_cost"] <= 100))
    assert np.all((n["eta_min"][:G] >= 50) & (n["eta_min"][:G] <= 300))
    assert np.all((n["eta_min"][G + L:] >= 0) & (n["eta_min"][G + L:] <= 200))
    assert sc["T"] == 24 and np.all(sc["cf"] == 1.0) and n["K"] == 15
    # 150 + 100 sin(...) with 5 % noise: between 50 and 250 MW up to the noise
    assert np.all(sc["load"] >= 0.75 * 50) and np.all(sc["load"] <= 1.25 * 250)
    assert synth.device_hours(nets, scens) == 20 * 24


def test_medium_recipe():
    nets, scens = synth.medium(S=2, T=168)
    n = nets[0]
    assert _connected(100, n["line_from"], n["line_to"]) and _simple_graph(n["line_from"], n["line_to"])
    kinds = np.asarray(n["gen_kind"])
    assert [int(np.sum(kinds == k)) for k in (synth.GAS, synth.SOLAR, synth.WIND)] == [100, 100, 100]
    gas = kinds == synth.GAS
    assert np.all((n["gen_cost"][gas] >= 20) & (n["gen_cost"][gas] <= 80)) and np.all(n["gen_cost"][~gas] == 0)
    assert np.all(n["gen_emis"][~gas] == 0) and np.all(n["gen_emis"][gas] > 0)
    # susceptance: 100 x LogNormal(ln 10, 0.5) p.u., median near 1000 MW/rad
    assert 700 < np.median(n["line_beta"]) < 1400
    cf = scens[0]["cf"]
    hour = np.arange(168) % 24
    solar = kinds == synth.SOLAR
    night = (hour <= 6) | (hour >= 18)
    # sin(pi (h - 6) / 12) is zero at 6 h and 18 h up to rounding, negative at night
    assert np.all(cf[np.ix_(solar, night)] <= 1e-12) and np.all(cf[np.ix_(solar, ~night)] > 0)
    wind = cf[kinds == synth.WIND]
    assert np.all((wind >= 0) & (wind <= 1))
    # AR(1) with rho = 0.9 (clipping to [0, 1] lowers the sample value a little)
    a, b = wind[:, :-1].ravel(), wind[:, 1:].ravel()
    assert np.corrcoef(a, b)[0, 1] > 0.75
    assert abs(np.mean(wind) - 0.35) < 0.05
    # a daily load cycle: a day apart the loads agree far better than half a day apart
    load = scens[0]["load"]
    d24 = np.mean(np.abs(load[:, 24:] - load[:, :-24]))
    d12 = np.mean(np.abs(load[:, 12:] - load[:, :-12]))
    assert d24 < 0.5 * d12
    # plan bounds and period investment costs
    G, L = 300, 150
    assert np.allclose(n["eta_max"][:G][gas], 2 * n["eta_min"][:G][gas])
    assert np.allclose(n["eta_max"][:G][~gas], 3 * n["eta_min"][:G][~gas])
    assert np.allclose(n["eta_max"][G:G + L], 2 * n["eta_min"][G:G + L])
    assert np.allclose(n["gamma"][:G][gas], 60e3 * 168 / 8760)
    assert synth.device_hours(nets, scens) == 600 * 168 * 2
    assert abs(sum(s["weight"] for s in scens) - 1.0) < 1e-12


def test_batching_recipe():
    nets, scens = synth.batching()
    assert len(nets) == len(scens) == 64
    Ts = set()
    for s, (n, sc) in enumerate(zip(nets, scens)):
        N = int(n["n_bus"])
        assert 50 <= N <= 500 and sc["net"] == s
        assert n["line_from"].size == int(round(1.5 * N)) and n["gen_bus"].size == 3 * N
        assert n["bat_bus"].size == max(1, int(round(0.3 * N)))
        assert sc["T"] in (24, 72, 168) and sc["load"].shape == (N, sc["T"])
        assert _connected(N, n["line_from"], n["line_to"])
        Ts.add(sc["T"])
    assert Ts == {24, 72, 168}
    assert abs(sum(sc["weight"] for sc in scens) - 1.0) < 1e-12


def test_scale_recipe():
    nets, scens = synth.scale(S=1)
    n = nets[0]
    assert int(n["n_bus"]) == 2000 and n["line_from"].size == 3000
    assert n["gen_bus"].size == 8000 and n["bat_bus"].size == 500 and n["K"] == 11500
    assert _connected(2000, n["line_from"], n["line_to"])
    # 52 weekly scenarios of this network: 117.9M device-hours per step
    assert 52 * synth.device_hours(nets, scens) == 117_936_000
