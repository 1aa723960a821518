"""gx_network_create's host-side validation, one corrupted field at a time (no GPU: create
does no device work).  Every corruption of a valid descriptor returns GX_ERR_INVALID_ARG with
a message, and nothing crosses the ABI but the status."""
import copy
import os

import numpy as np
import pytest

from test_abi import gx_create

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gx():
    from paper_2410_13055_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2410_13055_gb300 import gx as mod
    return mod


def _tiny():
    from paper_2410_13055_gb300 import synth
    nets, scens = synth.tiny()
    return copy.deepcopy(nets), copy.deepcopy(scens)


def _set(arr_key, idx, value):
    def f(nets, scens):
        a = np.array(nets[0][arr_key], dtype=np.asarray(nets[0][arr_key]).dtype)
        a[idx] = value
        nets[0][arr_key] = a
    return f


NET_CASES = {
    "gen_bus above range": (_set("gen_bus", 2, 5), "gen_bus out of range"),
    "gen_bus negative": (_set("gen_bus", 0, -1), "gen_bus out of range"),
    "gen_cost NaN": (_set("gen_cost", 1, np.nan), "non-finite generator data"),
    "gen_emis inf": (_set("gen_emis", 3, np.inf), "non-finite generator data"),
    "line on one bus": (_set("line_to", 0, 0), "both ends"),
    "line end above range": (_set("line_to", 4, 7), None),
    "line end negative": (_set("line_from", 2, -2), None),
    "line_beta zero": (_set("line_beta", 1, 0.0), "line_beta must be > 0"),
    "line_beta negative": (_set("line_beta", 6, -10.0), "line_beta must be > 0"),
    "line_dtheta zero": (_set("line_dtheta", 3, 0.0), "line_dtheta must be > 0"),
    "bat_bus above range": (_set("bat_bus", 1, 9), "bat_bus out of range"),
    "bat_dur zero": (_set("bat_dur", 0, 0.0), "bat_dur must be > 0"),
    "bat_eff_c above 1": (_set("bat_eff_c", 0, 1.2), None),
    "bat_eff_d zero": (_set("bat_eff_d", 1, 0.0), None),
}


def _scen(key, value):
    def f(nets, scens):
        scens[0][key] = value
    return f


def _scen_arr(key, idx, value):
    def f(nets, scens):
        a = np.array(scens[0][key], dtype=np.float64)
        a[idx] = value
        scens[0][key] = a
    return f


def _horizon(T):
    def f(nets, scens):
        # arrays of the claimed length, so only the horizon itself is wrong
        scens[0]["T"] = T
        scens[0]["load"] = np.full((5, max(T, 1)), 100.0)
        scens[0]["cf"] = np.ones((6, max(T, 1)))
    return f


SCEN_CASES = {
    "net index out of range": (_scen("net", 1), "net index out of range"),
    "zero horizon": (_horizon(0), "T must be in"),
    "horizon above the maximum": (_horizon(300), "T must be in"),
    "zero weight": (_scen("weight", 0.0), "weight must be > 0"),
    "NaN weight": (_scen("weight", float("nan")), "weight must be > 0"),
    "negative load": (_scen_arr("load", (2, 5), -1.0), None),
    "NaN load": (_scen_arr("load", (0, 0), np.nan), None),
    "cf above 1": (_scen_arr("cf", (1, 3), 1.5), None),
    "cf negative": (_scen_arr("cf", (4, 7), -0.1), None),
}

OPT_CASES = {
    "eps": 0.0, "voll": -1.0, "kappa": -1.0, "rho": 0.0, "adj_rho": float("nan"), "rho_theta_c": 0.0,
    "inner_iters": 0, "adj_inner_iters": 1001, "tol": 0.0, "max_iter": 0, "check_every": 0,
    "theta_weight": 2, "adj_rho_theta_c": -0.1,
}


def _expect_invalid(gx, nets, scens, text, opts=None):
    with pytest.raises(gx.GxError) as e:
        gx_create(gx, nets, scens, opts)
    assert e.value.status == -1
    msg = str(e.value)
    assert msg and (text is None or text in msg), msg


def test_untouched_tiny_creates(gx):
    nets, scens = _tiny()
    h, K, nbytes = gx_create(gx, nets, scens)
    assert K == 15 and nbytes > 0
    gx._lib.gx_network_destroy(h)


@pytest.mark.parametrize("case", sorted(NET_CASES))
def test_network_corruption_rejected(gx, case):
    nets, scens = _tiny()
    corrupt, text = NET_CASES[case]
    corrupt(nets, scens)
    _expect_invalid(gx, nets, scens, text)


@pytest.mark.parametrize("case", sorted(SCEN_CASES))
def test_scenario_corruption_rejected(gx, case):
    nets, scens = _tiny()
    corrupt, text = SCEN_CASES[case]
    corrupt(nets, scens)
    _expect_invalid(gx, nets, scens, text)


@pytest.mark.parametrize("field", sorted(OPT_CASES))
def test_option_corruption_rejected(gx, field):
    nets, scens = _tiny()
    o = gx.default_opts()
    setattr(o, field, OPT_CASES[field])
    _expect_invalid(gx, nets, scens, None, o)
