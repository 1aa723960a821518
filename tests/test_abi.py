"""The C-ABI library loads, exports every entry point declared in include/gx.h, and
validates descriptors on the host (no GPU needed: create does no device work)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gx():
    from paper_2410_13055_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2410_13055_gb300 import gx as mod
    return mod


def declared_symbols():
    with open(os.path.join(ROOT, "include", "gx.h")) as f:
        txt = f.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gx_[a-z_0-9]+)\s*\(", txt)))


def test_header_symbols_exported(gx):
    lib = ctypes.CDLL(gx.lib_path())
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(gx.exported_symbols())


def test_create_validates_on_host(gx):
    from paper_2410_13055_gb300 import synth
    nets, scens = synth.tiny()
    # a line with both ends on one bus is rejected
    bad = dict(nets[0]); bad["line_to"] = bad["line_from"].copy()
    with pytest.raises(gx.GxError) as e:
        gx_create(gx, [bad], scens)
    assert e.value.status == -1 and "both ends" in str(e.value)
    bad = dict(nets[0]); bad["gen_bus"] = nets[0]["gen_bus"] + 10
    with pytest.raises(gx.GxError):
        gx_create(gx, [bad], scens)
    sc = dict(scens[0]); sc["load"] = -scens[0]["load"]
    with pytest.raises(gx.GxError):
        gx_create(gx, nets, [sc])
    sc = dict(scens[0]); sc["cf"] = scens[0]["cf"] * 2
    with pytest.raises(gx.GxError):
        gx_create(gx, nets, [sc])
    h, K, nbytes = gx_create(gx, nets, scens)
    assert K == nets[0]["K"] and nbytes > 0
    off, cnt = ctypes.c_size_t(), ctypes.c_size_t()
    assert gx._lib.gx_network_array(h, gx.ARR["p"], 0, ctypes.byref(off), ctypes.byref(cnt)) == 0
    assert cnt.value == 6 * 24 and off.value % 4 == 0
    assert gx._lib.gx_network_array(h, 99, 0, ctypes.byref(off), ctypes.byref(cnt)) == -1
    # solve before bind is an ordering error, not a crash
    st = gx.Stats()
    assert gx._lib.gx_dispatch_solve_batch(h, ctypes.c_void_p(16), None, 0, 0, None, ctypes.byref(st), None) == -6
    assert gx._lib.gx_network_forget(h) == -6
    assert gx._lib.gx_network_forget(None) == -6
    gx._lib.gx_network_destroy(h)


def test_scaling_susceptance_validated_on_host(gx):
    """line_beta_ref must be finite and >= 0; a valid one adds the per-call tables of the
    scaling lines to the workspace."""
    from paper_2410_13055_gb300 import synth
    nets, scens = synth.tiny()
    L = nets[0]["line_from"].size
    bad = dict(nets[0]); bad["line_beta_ref"] = np.full(L, -1.0)
    with pytest.raises(gx.GxError) as e:
        gx_create(gx, [bad], scens)
    assert "line_beta_ref" in str(e.value)
    bad["line_beta_ref"] = np.full(L, np.nan)
    with pytest.raises(gx.GxError):
        gx_create(gx, [bad], scens)
    h0, _, b0 = gx_create(gx, nets, scens)
    ok = dict(nets[0]); ok["line_beta_ref"] = np.where(np.arange(L) % 2 == 0, 100.0, 0.0)
    h1, K, b1 = gx_create(gx, [ok], scens)
    assert K == nets[0]["K"] and b1 >= b0
    gx._lib.gx_network_destroy(h0)
    gx._lib.gx_network_destroy(h1)


def test_opts_validation(gx):
    o = gx.default_opts()
    assert o.eps > 0 and o.rho > 0 and o.inner_iters >= 1
    assert o.adj_rho_theta_c == 0 and o.adj_rho_inner_c == 0  # 0: the forward's scales
    from paper_2410_13055_gb300 import synth
    nets, scens = synth.tiny()
    o.rho = -1.0
    with pytest.raises(gx.GxError):
        gx_create(gx, nets, scens, o)
    o = gx.default_opts()
    o.adj_rho_theta_c = -0.1
    with pytest.raises(gx.GxError):
        gx_create(gx, nets, scens, o)


def test_state_ranges_on_host(gx):
    """The forward and adjoint iteration states are two disjoint ranges of the workspace,
    forward first, each holding at least the 16 state arrays' rows."""
    from paper_2410_13055_gb300 import synth
    nets, scens = synth.tiny()
    h, K, nbytes = gx_create(gx, nets, scens)
    off, nb = ctypes.c_size_t(), ctypes.c_size_t()
    ranges = []
    for which in (0, 1):
        assert gx._lib.gx_network_state_range(h, which, ctypes.byref(off), ctypes.byref(nb)) == 0
        ranges.append((off.value, nb.value))
    (f0, fb), (a0, ab) = ranges
    assert fb == ab and fb > 0 and f0 % 256 == 0 and a0 % 256 == 0
    assert f0 + fb <= a0 and a0 + ab <= nbytes
    n = nets[0]
    N, L, G, B = int(n["n_bus"]), n["line_from"].size, n["gen_bus"].size, n["bat_bus"].size
    Tp = (scens[0]["T"] + 3) // 4 * 4
    rows = G + 4 * N + 4 * L + 7 * B  # generators; load, u, pbar, theta; line delta, sigma, q_f, q_t; battery
    assert fb >= 4 * rows * Tp
    assert gx._lib.gx_network_state_range(h, 2, ctypes.byref(off), ctypes.byref(nb)) == -1
    gx._lib.gx_network_destroy(h)


def gx_create(gx, nets, scens, opts=None):
    """Create only (no bind), through the same descriptor marshalling as gx.Network."""
    N = gx.Network.__new__(gx.Network)
    # reuse the constructor's marshalling up to create by calling it with a fake device
    keep = []
    nd = (gx.NetworkDesc * len(nets))()
    for k, n in enumerate(nets):
        arrs = dict(gen_bus=np.ascontiguousarray(n["gen_bus"], np.int32),
                    gen_cost=np.ascontiguousarray(n["gen_cost"], np.float64),
                    gen_emis=np.ascontiguousarray(n["gen_emis"], np.float64),
                    line_from=np.ascontiguousarray(n["line_from"], np.int32),
                    line_to=np.ascontiguousarray(n["line_to"], np.int32),
                    line_beta=np.ascontiguousarray(n["line_beta"], np.float64),
                    line_dtheta=np.ascontiguousarray(n["line_dtheta"], np.float64),
                    bat_bus=np.ascontiguousarray(n["bat_bus"], np.int32),
                    bat_dur=np.ascontiguousarray(n["bat_dur"], np.float64),
                    bat_eff_c=np.ascontiguousarray(n["bat_eff_c"], np.float64),
                    bat_eff_d=np.ascontiguousarray(n["bat_eff_d"], np.float64))
        keep.append(arrs)
        d = nd[k]
        d.n_bus, d.n_gen, d.n_line, d.n_bat = int(n["n_bus"]), arrs["gen_bus"].size, arrs["line_from"].size, \
            arrs["bat_bus"].size
        for name, a in arrs.items():
            setattr(d, name, a.ctypes.data_as(gx._i32p if a.dtype == np.int32 else gx._f64p))
        if "line_beta_ref" in n:
            br = np.ascontiguousarray(n["line_beta_ref"], np.float64)
            keep.append(br)
            d.line_beta_ref = br.ctypes.data_as(gx._f64p)
    sd = (gx.ScenarioDesc * len(scens))()
    for s, sc in enumerate(scens):
        load = np.ascontiguousarray(sc["load"], np.float64)
        cf = np.ascontiguousarray(sc["cf"], np.float64)
        keep.append((load, cf))
        sd[s].net, sd[s].T, sd[s].weight = sc["net"], sc["T"], sc["weight"]
        sd[s].load = load.ctypes.data_as(gx._f64p)
        sd[s].cf = cf.ctypes.data_as(gx._f64p)
    o = opts if opts is not None else gx.default_opts()
    h = ctypes.c_void_p()
    rc = gx._lib.gx_network_create(nd, len(nets), sd, len(scens), ctypes.byref(o), ctypes.byref(h))
    if rc != 0:
        raise gx.GxError(rc, "create")
    return h, gx._lib.gx_network_K(h), gx._lib.gx_network_device_bytes(h)


def test_host_switches_validate_their_arguments(gx):
    """Launch-mode switches and option changes on a created (unbound) network: valid
    values are accepted, invalid ones return GX_ERR_INVALID_ARG, and the weighting of
    the phase penalties is fixed at create."""
    from paper_2410_13055_gb300 import synth
    nets, scens = synth.tiny()
    h, _, _ = gx_create(gx, nets, scens)
    lib = gx._lib
    for m in (0, 1, 2):
        assert lib.gx_network_use_graphs(h, m) == 0
    assert lib.gx_network_use_graphs(h, 3) == -1
    assert lib.gx_network_use_persistent(h, 1) == 0 and lib.gx_network_use_persistent(h, 0) == 0
    o = gx.default_opts()
    o.adj_rho = 0.004
    o.adj_rho_theta_c = 0.05
    assert lib.gx_network_set_opts(h, ctypes.byref(o)) == 0
    o.theta_weight = 1
    assert lib.gx_network_set_opts(h, ctypes.byref(o)) == -1
    o = gx.default_opts()
    o.check_every = 0
    assert lib.gx_network_set_opts(h, ctypes.byref(o)) == -1
    lib.gx_network_destroy(h)
