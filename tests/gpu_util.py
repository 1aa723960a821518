"""Helpers for the GPU parity tests: run the CUDA path, read its outputs back in the
oracle's array format (FP64 numpy), and compare."""
import numpy as np


def gpu_net(nets, scens, **opt_kw):
    from paper_2410_13055_gb300 import gx
    return gx.Network(nets, scens, **opt_kw)


def eta_tensor(eta):
    import torch
    return torch.tensor(np.asarray(eta, np.float32), device="cuda")


def solution(net, s, ref_bus=None):
    """Scenario s of the last solve as float64 numpy arrays (oracle layout)."""
    import torch
    torch.cuda.synchronize()
    g = {k: net.array(k, s).double().cpu().numpy() for k in ("p", "shed", "theta", "ch", "dis", "soc", "price", "flow")}
    if ref_bus is not None:
        th = g["theta"].copy()
        # angles are defined up to a constant per island: subtract the reference bus's angle
        for comp_ref, members in ref_bus:
            th[members] -= th[comp_ref]
        g["theta"] = th
    g["cost"] = float(net.array("cost", s).cpu().numpy()[0])
    g["h"] = float(net.array("h", s).cpu().numpy()[0])
    g["iters"] = int(net.array("iters", s).cpu().numpy()[0])
    g["resid"] = net.array("resid", s).cpu().numpy().copy()
    return g


def ref_groups(qp):
    """(reference bus, member buses) for each island of the oracle's QP."""
    out = []
    for c, rb in enumerate(qp.ref_bus):
        out.append((int(rb), np.where(qp.comp == c)[0]))
    return out


def pack_x(qp, g):
    return qp.pack(g["p"], g["shed"], g["theta"], g["ch"], g["dis"], g["soc"], fdc=g["flow"])


def rel(a, b):
    a = np.asarray(a, float); b = np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))

