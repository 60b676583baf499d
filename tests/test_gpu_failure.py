"""Failure detection on the GPU without a fault: the kernels' bounded wait is
made to run out on a barrier that nothing completes; the kernel records the
time-out in the device status word and exits; the host reads the status and
the context keeps working."""
import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_and_context_survives():
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    assert sc5.device_status() == 0
    sc5.selftest_wait_timeout(2000)  # 2 ms
    torch.cuda.synchronize()
    assert sc5.device_status() == 1  # SC5_EDEVICE with the time-out code
    assert sc5.device_status() == 0  # read-and-clear
    with pytest.raises(sc5.Sepconv5Error):
        sc5.selftest_wait_timeout(0)
    # the context is intact: a normal run still matches the oracle
    P, H, W = 3, 67, 132
    A = synth.image(4, H, W)
    k = synth.kernel_normalised(4)
    out = torch.empty((P, H - 4, W - 4), dtype=torch.float32, device="cuda")
    plan = sc5.Plan(P, H, W, W, W - 4)
    plan.run(U.to_dev(A), out, k)
    torch.cuda.synchronize()
    plan.close()
    ref = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    assert U.max_abs(out.cpu().numpy(), ref) <= U.FP32_TOL
    assert sc5.device_status() == 0
