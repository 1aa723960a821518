"""Thin ctypes binding of the C ABI in include/gx.h (argument marshalling only).

Every step of the dispatch solve, the adjoint gradient and the plan step runs in the
CUDA kernels of ``libgx.so``; this module only converts numpy / torch arguments into
pointers and sizes.  PyTorch provides the device memory (one uint8 workspace tensor
per network) and the CUDA stream.  Importing this module raises if the library has
not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgx.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2410_13055_gb300.build` "
                      "(the CUDA library is the only implementation; there is no fallback)")
_lib = C.CDLL(LIB_PATH)

# ---------------------------------------------------------------------------- C types
GX_OK, GX_NOT_CONVERGED = 0, 1
GX_WARM = {"cold": 0, "prev": 1, "user": 2, "learned": 3}
ARR = dict(p=0, shed=1, flow=2, theta=3, ch=4, dis=5, soc=6, price=7, cost=8, h=9, iters=10, resid=11,
           status=12, grad_s=13, adj_iters=14, obj=15, warm=16)
_ARR_DTYPE = dict(cost="float64", h="float64", resid="float64", grad_s="float64", obj="float64", iters="int32",
                  status="int32", adj_iters="int32", warm="int32")

_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)


class NetworkDesc(C.Structure):
    _fields_ = [("n_bus", C.c_int), ("n_gen", C.c_int), ("n_line", C.c_int), ("n_bat", C.c_int),
                ("gen_bus", _i32p), ("gen_cost", _f64p), ("gen_emis", _f64p),
                ("line_from", _i32p), ("line_to", _i32p), ("line_beta", _f64p), ("line_dtheta", _f64p),
                ("bat_bus", _i32p), ("bat_dur", _f64p), ("bat_eff_c", _f64p), ("bat_eff_d", _f64p),
                ("line_dc", C.POINTER(C.c_uint8)), ("gen_ramp", _f64p),
                ("line_beta_ref", _f64p)]


class ScenarioDesc(C.Structure):
    _fields_ = [("net", C.c_int), ("T", C.c_int), ("load", _f64p), ("cf", _f64p), ("weight", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("eps", C.c_double), ("voll", C.c_double), ("kappa", C.c_double),
                ("rho", C.c_double), ("rho_theta_c", C.c_double), ("theta_weight", C.c_int),
                ("rho_inner_c", C.c_double), ("inner_iters", C.c_int),
                ("tol", C.c_double), ("max_iter", C.c_int), ("check_every", C.c_int),
                ("tol_active", C.c_double), ("adj_tol", C.c_double), ("adj_max_iter", C.c_int),
                ("grad_envelope", C.c_int), ("adj_rho", C.c_double),
                ("adj_rho_theta_c", C.c_double), ("adj_rho_inner_c", C.c_double), ("adj_inner_iters", C.c_int)]


class Schedule(C.Structure):
    _fields_ = [("bus_staged", C.c_int), ("bat_warps", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters_max", C.c_int), ("n_converged", C.c_int), ("n_scen", C.c_int), ("launches", C.c_int),
                ("max_primal", C.c_double), ("max_dual", C.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = C.c_void_p
_sz = C.c_size_t
_SIGS = {
    "gx_opts_default": (C.c_int, [C.POINTER(Opts)]),
    "gx_status_string": (C.c_char_p, [C.c_int]),
    "gx_last_error_message": (C.c_char_p, []),
    "gx_network_create": (C.c_int, [C.POINTER(NetworkDesc), C.c_int, C.POINTER(ScenarioDesc), C.c_int,
                                    C.POINTER(Opts), C.POINTER(_vp)]),
    "gx_network_destroy": (C.c_int, [_vp]),
    "gx_network_device_bytes": (_sz, [_vp]),
    "gx_network_K": (C.c_int, [_vp]),
    "gx_network_S": (C.c_int, [_vp]),
    "gx_network_bind": (C.c_int, [_vp, _vp, _sz, _vp]),
    "gx_network_set_opts": (C.c_int, [_vp, C.POINTER(Opts)]),
    "gx_network_forget": (C.c_int, [_vp]),
    "gx_network_array": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(_sz), C.POINTER(_sz)]),
    "gx_network_state_range": (C.c_int, [_vp, C.c_int, C.POINTER(_sz), C.POINTER(_sz)]),
    "gx_network_scenario_info": (C.c_int, [_vp, C.c_int] + [C.POINTER(C.c_int)] * 7),
    "gx_dispatch_solve_batch": (C.c_int, [_vp, _vp, C.POINTER(C.c_int), C.c_int, C.c_int, _vp,
                                          C.POINTER(Stats), _vp]),
    "gx_dispatch_grad_batch": (C.c_int, [_vp, _vp, C.c_int, _vp, C.POINTER(Stats), _vp]),
    "gx_plan_step": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_float, _vp]),
    "gx_profile_enable": (C.c_int, [_vp, C.c_int]),
    "gx_network_use_graphs": (C.c_int, [_vp, C.c_int]),
    "gx_network_use_persistent": (C.c_int, [_vp, C.c_int]),
    "gx_network_set_schedule": (C.c_int, [_vp, C.POINTER(Schedule)]),
    "gx_network_get_schedule": (C.c_int, [_vp, C.POINTER(Schedule)]),
    "gx_network_persistent_info": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "gx_profile_read": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "gx_profile_active": (C.c_int, [_vp, C.POINTER(C.c_longlong)]),
    "gx_dispatch_cost_noalloc": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "gx_gnn_num_params": (_sz, []),
    "gx_gnn_create": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(_vp)]),
    "gx_gnn_device_bytes": (_sz, [_vp]),
    "gx_gnn_bind": (C.c_int, [_vp, _vp, _sz, C.c_uint64, _vp]),
    "gx_gnn_set_params": (C.c_int, [_vp, _vp, _sz, _vp]),
    "gx_gnn_get_params": (C.c_int, [_vp, _vp, _sz, C.c_int, _vp]),
    "gx_gnn_predict": (C.c_int, [_vp, _vp, _vp, _vp]),
    "gx_gnn_train_step": (C.c_int, [_vp, _vp, _vp, C.c_float, C.c_float, C.POINTER(C.c_double), _vp]),
    "gx_gnn_destroy": (C.c_int, [_vp]),
    "gx_network_attach_gnn": (C.c_int, [_vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


class GxError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.gx_last_error_message().decode()
        super().__init__(f"{where}: {_lib.gx_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _check(status, where, allow_not_converged=True):
    if status < 0 or (status > 0 and not allow_not_converged):
        raise GxError(status, where)
    return status


def default_opts(**kw) -> Opts:
    o = Opts()
    _check(_lib.gx_opts_default(C.byref(o)), "gx_opts_default")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class Network:
    """A batch of dispatch scenarios bound to a torch-allocated device workspace.

    nets / scens are the plain dicts of ``paper_2410_13055_gb300.synth``.  Model
    constants (eps, voll, kappa) and solver options go in ``opts``.
    """

    def __init__(self, nets, scens, opts: Opts | None = None, device="cuda", **opt_kw):
        import torch
        self._keep = []
        nd = (NetworkDesc * len(nets))()
        for k, n in enumerate(nets):
            arrs = dict(
                gen_bus=np.ascontiguousarray(n["gen_bus"], np.int32),
                gen_cost=np.ascontiguousarray(n["gen_cost"], np.float64),
                gen_emis=np.ascontiguousarray(n["gen_emis"], np.float64),
                line_from=np.ascontiguousarray(n["line_from"], np.int32),
                line_to=np.ascontiguousarray(n["line_to"], np.int32),
                line_beta=np.ascontiguousarray(n["line_beta"], np.float64),
                line_dtheta=np.ascontiguousarray(n["line_dtheta"], np.float64),
                bat_bus=np.ascontiguousarray(n["bat_bus"], np.int32),
                bat_dur=np.ascontiguousarray(n["bat_dur"], np.float64),
                bat_eff_c=np.ascontiguousarray(n["bat_eff_c"], np.float64),
                bat_eff_d=np.ascontiguousarray(n["bat_eff_d"], np.float64),
            )
            self._keep.append(arrs)
            d = nd[k]
            d.n_bus, d.n_gen = int(n["n_bus"]), arrs["gen_bus"].size
            d.n_line, d.n_bat = arrs["line_from"].size, arrs["bat_bus"].size
            for name, a in arrs.items():
                ct = _i32p if a.dtype == np.int32 else _f64p
                setattr(d, name, a.ctypes.data_as(ct))
            if "line_dc" in n and np.any(n["line_dc"]):
                dc = np.ascontiguousarray(n["line_dc"], np.uint8)
                arrs["line_dc"] = dc
                d.line_dc = dc.ctypes.data_as(C.POINTER(C.c_uint8))
            if "gen_ramp" in n and np.any(np.asarray(n["gen_ramp"]) > 0):
                rp = np.ascontiguousarray(n["gen_ramp"], np.float64)
                arrs["gen_ramp"] = rp
                d.gen_ramp = rp.ctypes.data_as(_f64p)
            if "line_beta_ref" in n and np.any(np.asarray(n["line_beta_ref"]) > 0):
                br = np.ascontiguousarray(n["line_beta_ref"], np.float64)
                arrs["line_beta_ref"] = br
                d.line_beta_ref = br.ctypes.data_as(_f64p)
        sd = (ScenarioDesc * len(scens))()
        for s, sc in enumerate(scens):
            load = np.ascontiguousarray(sc["load"], np.float64)
            cf = np.ascontiguousarray(sc["cf"], np.float64)
            self._keep.append((load, cf))
            d = sd[s]
            d.net, d.T, d.weight = int(sc["net"]), int(sc["T"]), float(sc["weight"])
            d.load = load.ctypes.data_as(_f64p)
            d.cf = cf.ctypes.data_as(_f64p)
        self.opts = opts if opts is not None else default_opts(**opt_kw)
        h = C.c_void_p()
        _check(_lib.gx_network_create(nd, len(nets), sd, len(scens), C.byref(self.opts), C.byref(h)),
               "gx_network_create", False)
        self._h = h
        self._keep = None  # the library copied the descriptors
        self.K = _lib.gx_network_K(h)
        self.S = _lib.gx_network_S(h)
        self.nbytes = _lib.gx_network_device_bytes(h)
        self.device = torch.device(device)
        self.ws = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._off0 = (-base) % 256
        _check(_lib.gx_network_bind(h, C.c_void_p(base + self._off0), C.c_size_t(self.nbytes),
                                    _stream_handle(None)), "gx_network_bind", False)
        self.info = [self.scenario_info(s) for s in range(self.S)]
        self.weights = np.array([float(sc["weight"]) for sc in scens])
        self.nets_desc, self.scens_desc = nets, scens
        self.eta_offsets = []
        off = 0
        for n in nets:
            self.eta_offsets.append(off)
            off += int(n["gen_bus"].size + n["line_from"].size + n["bat_bus"].size)
        self.last_stats = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.gx_network_destroy(h)
            self._h = None

    # ------------------------------------------------------------------ metadata
    def scenario_info(self, s):
        vals = [C.c_int() for _ in range(7)]
        _check(_lib.gx_network_scenario_info(self._h, s, *[C.byref(v) for v in vals]), "scenario_info", False)
        return dict(zip(["T", "Tp", "N", "G", "L", "B", "eta_offset"], [v.value for v in vals]))

    def set_opts(self, opts: Opts | None = None, **kw):
        if opts is None:
            opts = Opts.from_buffer_copy(self.opts)
            for k, v in kw.items():
                setattr(opts, k, v)
        _check(_lib.gx_network_set_opts(self._h, C.byref(opts)), "gx_network_set_opts", False)
        self.opts = opts

    def forget(self):
        """Drop the previous solution: the next warm="prev" solve starts cold, and warm="learned"
        takes the learned start for every scenario."""
        _check(_lib.gx_network_forget(self._h), "gx_network_forget", False)

    def state(self, adjoint=False):
        """A float32 torch view (no copy) of the forward or adjoint iteration state; clone it
        to checkpoint a warm start, copy it back before a warm="prev" call to restore it."""
        import torch
        off, nb = C.c_size_t(), C.c_size_t()
        _check(_lib.gx_network_state_range(self._h, 1 if adjoint else 0, C.byref(off), C.byref(nb)),
               "gx_network_state_range", False)
        start = self._off0 + off.value
        return self.ws[start:start + nb.value].view(torch.float32)

    def array(self, which, scen=-1):
        """A torch view (no copy) of an output array inside the workspace."""
        import torch
        off, cnt = C.c_size_t(), C.c_size_t()
        _check(_lib.gx_network_array(self._h, ARR[which], scen, C.byref(off), C.byref(cnt)), "gx_network_array",
               False)
        dt = getattr(torch, _ARR_DTYPE.get(which, "float32"))
        esz = torch.tensor([], dtype=dt).element_size()
        start = self._off0 + off.value
        v = self.ws[start:start + cnt.value * esz].view(dt)
        if scen >= 0 and which in ("p", "shed", "flow", "theta", "ch", "dis", "soc", "price"):
            inf = self.info[scen]
            rows = {"p": "G", "shed": "N", "flow": "L", "theta": "N", "ch": "B", "dis": "B", "soc": "B",
                    "price": "N"}[which]
            v = v.view(inf[rows], inf["Tp"])[:, :inf["T"]]
        return v

    # ------------------------------------------------------------------ compute
    def solve(self, eta, batch=None, warm="cold", warm_prices=None, warm_angles=None, stream=None):
        """Eq. 2 for every scenario of the batch at plan eta (FP32 CUDA tensor [K])."""
        import torch
        assert eta.is_cuda and eta.dtype == torch.float32 and eta.numel() == self.K and eta.is_contiguous()
        wd = None
        if warm == "user":
            wd = torch.cat([warm_prices.reshape(-1), warm_angles.reshape(-1)]).to(self.device, torch.float32)
        idx, nb = None, 0
        if batch is not None:
            arr = (C.c_int * len(batch))(*[int(b) for b in batch])
            idx, nb = arr, len(batch)
        st = Stats()
        rc = _lib.gx_dispatch_solve_batch(self._h, _ptr(eta), idx, nb, GX_WARM[warm], _ptr(wd), C.byref(st),
                                          _stream_handle(stream))
        _check(rc, "gx_dispatch_solve_batch")
        self.last_stats = st.asdict()
        self.last_status = rc
        return rc

    def grad(self, eta, out=None, warm="cold", stream=None):
        """sum_s w_s dh_s/deta at the last solve (FP32 [K])."""
        import torch
        if out is None:
            out = torch.zeros(self.K, dtype=torch.float32, device=self.device)
        st = Stats()
        rc = _lib.gx_dispatch_grad_batch(self._h, _ptr(eta), GX_WARM[warm], _ptr(out), C.byref(st),
                                         _stream_handle(stream))
        _check(rc, "gx_dispatch_grad_batch")
        self.last_grad_stats = st.asdict()
        self.last_grad_status = rc
        return out

    def attach_gnn(self, gnn):
        """The learned start of warm="learned" (gx_network_attach_gnn); None detaches."""
        _check(_lib.gx_network_attach_gnn(self._h, gnn._h if gnn is not None else None), "gx_network_attach_gnn",
               False)
        self._gnn = gnn  # keeps it alive while attached

    def use_graphs(self, on=True, device_loop=True):
        """Launch mode of the per-iteration kernels (gx_network_use_graphs): the whole loop
        as one graph with a device-side convergence test (default), one graph per
        residual-check chunk (device_loop=False), or kernel by kernel (on=False)."""
        mode = 0 if not on else (2 if device_loop else 1)
        _check(_lib.gx_network_use_graphs(self._h, mode), "gx_network_use_graphs", False)

    def set_schedule(self, bus_staged=None, bat_warps=None):
        """Kernel schedule (gx_network_set_schedule); None keeps a field as it is."""
        sc = Schedule()
        _check(_lib.gx_network_get_schedule(self._h, C.byref(sc)), "gx_network_get_schedule", False)
        if bus_staged is not None:
            sc.bus_staged = int(bus_staged)
        if bat_warps is not None:
            sc.bat_warps = int(bat_warps)
        _check(_lib.gx_network_set_schedule(self._h, C.byref(sc)), "gx_network_set_schedule", False)

    def schedule(self):
        sc = Schedule()
        _check(_lib.gx_network_get_schedule(self._h, C.byref(sc)), "gx_network_get_schedule", False)
        return {"bus_staged": sc.bus_staged, "bat_warps": sc.bat_warps}

    def use_persistent(self, on=True):
        """Cluster-resident persistent launches for the scenarios that fit (default) or the
        per-iteration kernels for every scenario."""
        _check(_lib.gx_network_use_persistent(self._h, int(bool(on))), "gx_network_use_persistent", False)

    def persistent_info(self):
        """Per scenario: CTAs of its resident cluster, 0 if it runs on the per-iteration kernels."""
        out = []
        for s in range(self.S):
            v = C.c_int(0)
            _check(_lib.gx_network_persistent_info(self._h, s, C.byref(v)), "gx_network_persistent_info", False)
            out.append(v.value)
        return out

    def profile(self, on=True):
        """Sampled CUDA-event timing of the bus / line / battery kernels and of the
        cluster-resident launches (see gx_profile_enable)."""
        _check(_lib.gx_profile_enable(self._h, int(bool(on))), "gx_profile_enable", False)

    def profile_read(self):
        ms = (C.c_double * 4)()
        sm = (C.c_longlong * 4)()
        ln = (C.c_longlong * 4)()
        _check(_lib.gx_profile_read(self._h, ms, sm, ln), "gx_profile_read", False)
        names = ["k_bus", "k_line", "k_bat", "k_crs"]
        return {names[k]: {"ms": ms[k], "samples": sm[k], "launches": ln[k]} for k in range(4) if sm[k] > 0}

    def profile_active(self):
        """Per scenario: sampled iterations it was still iterating in (gx_profile_active)."""
        out = (C.c_longlong * self.S)()
        _check(_lib.gx_profile_active(self._h, out), "gx_profile_active", False)
        return np.array(out[:], dtype=np.int64)

    def plan_step(self, eta, grad, gamma, eta_min, eta_max, alpha, stream=None):
        rc = _lib.gx_plan_step(self._h, _ptr(eta), _ptr(grad), _ptr(gamma), _ptr(eta_min), _ptr(eta_max),
                               C.c_float(alpha), _stream_handle(stream))
        _check(rc, "gx_plan_step", False)
        return eta


class WarmStartGNN:
    """The learned warm start of a bound ``Network`` (kernels in csrc/gx_gnn.cu)."""

    def __init__(self, net: Network, seed=0):
        import torch
        h = C.c_void_p()
        _check(_lib.gx_gnn_create(net._h, 64, 3, C.byref(h)), "gx_gnn_create", False)
        self._h = h
        self.net = net  # keeps the network alive
        self.nparam = int(_lib.gx_gnn_num_params())
        nb = _lib.gx_gnn_device_bytes(h)
        self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=net.device)
        base = self.ws.data_ptr()
        off = (-base) % 256
        _check(_lib.gx_gnn_bind(h, C.c_void_p(base + off), C.c_size_t(nb), C.c_uint64(seed), _stream_handle(None)),
               "gx_gnn_bind", False)
        self.M = int(sum(inf["N"] * inf["Tp"] for inf in net.info))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.gx_gnn_destroy(h)
            self._h = None

    def params(self, which=0):
        out = np.empty(self.nparam, np.float32)
        _check(_lib.gx_gnn_get_params(self._h, out.ctypes.data_as(C.c_void_p), out.size, which,
                                      _stream_handle(None)), "gx_gnn_get_params", False)
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(_lib.gx_gnn_set_params(self._h, p.ctypes.data_as(C.c_void_p), p.size, _stream_handle(None)),
               "gx_gnn_set_params", False)

    def predict(self, eta, out=None):
        """[2 * bus rows]: prices ($/MWh) then angles, the user warm-start layout."""
        import torch
        if out is None:
            out = torch.empty(2 * self.M, dtype=torch.float32, device=self.net.device)
        _check(_lib.gx_gnn_predict(self._h, _ptr(eta), _ptr(out), _stream_handle(None)), "gx_gnn_predict", False)
        return out

    def train_step(self, eta, target, lr, w_theta=1.0):
        loss = C.c_double()
        _check(_lib.gx_gnn_train_step(self._h, _ptr(eta), _ptr(target), C.c_float(lr), C.c_float(w_theta),
                                      C.byref(loss), _stream_handle(None)), "gx_gnn_train_step", False)
        return loss.value


def lib_path():
    return LIB_PATH


def exported_symbols():
    """Names the binding resolves in libgx.so (every entry point of include/gx.h)."""
    return EXPORTED
