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
