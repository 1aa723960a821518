"""gx_dispatch_cost_noalloc: the cost reduction for callers that cannot allocate device
memory (a fixed memory budget, device memory owned by a host framework).  Its output,
called through the C ABI twice in a row, must equal the cost and planner value that
gx_dispatch_solve_batch computes with its workspace scratch.  This file is collected
last so that a run stopping at the first failure has already run everything else."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_cost_noalloc_matches_workspace_reduction():
    import torch

    from paper_2410_13055_gb300 import gx, synth
    nets, scens = synth.medium(S=2)
    net = gx.Network(nets, scens, kappa=50.0, tol=1e-3, max_iter=3000)
    eta = torch.tensor(np.concatenate([n["eta_min"] for n in nets]), dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # bound but not solved yet: there is no dispatch to price
    rc = gx._lib.gx_dispatch_cost_noalloc(net._h, 0, ctypes.c_void_p(out.data_ptr()), None, stream)
    assert rc == -6 and b"solve first" in gx._lib.gx_last_error_message()
    net.solve(eta)
    torch.cuda.synchronize()
    ref_cost = net.array("cost").cpu().numpy().copy()
    ref_h = net.array("h").cpu().numpy().copy()
    for _call in range(2):  # two calls in a row share the fixed scratch array
        for s in range(net.S):
            out.zero_()
            rc = gx._lib.gx_dispatch_cost_noalloc(net._h, s, ctypes.c_void_p(out.data_ptr()),
                                                  ctypes.c_void_p(out.data_ptr() + 8), stream)
            assert rc == 0, gx._lib.gx_last_error_message()
            torch.cuda.synchronize()
            c, h = out.cpu().numpy()
            assert abs(c - ref_cost[s]) <= 1e-9 * abs(ref_cost[s])
            assert abs(h - ref_h[s]) <= 1e-9 * abs(ref_h[s])
    # an out-of-range scenario is rejected before any device work
    rc = gx._lib.gx_dispatch_cost_noalloc(net._h, 99, ctypes.c_void_p(out.data_ptr()), None, stream)
    assert rc == -1 and b"out of range" in gx._lib.gx_last_error_message()
