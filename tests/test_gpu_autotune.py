"""The autotuner picks a setting that meets the accuracy guard and caches it."""
import json

import pytest

from gpu_util import gpu_net
from paper_2410_13055_gb300 import autotune, synth

pytestmark = pytest.mark.gpu


def test_autotune_tiny_caches_a_valid_setting(tmp_path):
    nets, scens = synth.tiny()
    net = gpu_net(nets, scens, kappa=50.0, tol=1e-3, adj_tol=1e-3, max_iter=50000, adj_max_iter=50000)
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(net, nets, steps=2, cache=cache)
    assert set(best) == set(autotune.SPACE)
    db = json.load(open(cache))
    key = autotune.bucket(net)
    assert db[key]["best"] == best
    trials = db[key]["trials"]
    g_base = trials[0]["g_rel"]
    # every rejected candidate failed the objective or the gradient guard
    assert all(t.get("ok", True) or t["h_rel"] > 2e-3 or t["g_rel"] > 1.25 * g_base for t in trials)
    assert all(t["g_rel"] <= 1.25 * g_base + 1e-6 for t in trials if t.get("ok"))
    net2 = gpu_net(nets, scens)
    assert autotune.load(net2, cache) == best
    assert abs(net2.opts.rho - best["rho"]) < 1e-12
