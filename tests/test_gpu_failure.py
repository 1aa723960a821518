"""Failure paths driven by inputs only (no device fault): a load that passes validation
(finite, >= 0) but overflows FP32 in the message passing (3e38 MW; its square is inf)
ends the solve with GX_ERR_NONFINITE at the first residual check, on both execution
paths; the per-scenario status says so, and the CUDA context stays usable."""
import pytest

from gpu_util import eta_tensor, gpu_net
from paper_2410_13055_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("persistent", [False, True])
def test_overflowing_input_returns_nonfinite_and_context_survives(persistent):
    import torch

    from paper_2410_13055_gb300 import gx
    nets, scens = synth.tiny()
    scens[0]["load"] = scens[0]["load"].copy()
    scens[0]["load"][0, 3] = 3e38
    net = gpu_net(nets, scens, tol=1e-6, max_iter=2000, check_every=20)
    net.use_persistent(persistent)
    if persistent:
        assert net.persistent_info()[0] > 0  # the 5-bus case runs on the resident path
    eta = eta_tensor(nets[0]["eta_min"])
    with pytest.raises(gx.GxError) as e:
        net.solve(eta)
    assert e.value.status == -2, e.value
    torch.cuda.synchronize()
    assert int(net.array("status").cpu()[0]) == -2
    assert int(net.array("iters").cpu()[0]) == 20  # stopped at the first check, not at the cap
    # the context is intact: the unmodified case solves on the same device
    n2, s2 = synth.tiny()
    ok = gpu_net(n2, s2, tol=1e-6, max_iter=200000, check_every=50)
    ok.use_persistent(persistent)
    assert ok.solve(eta_tensor(n2[0]["eta_min"])) == 0
