"""The offload call (sepconv5_run_host): host buffers in and out, band-pipelined
copies overlapping the kernels; the result equals the device-resident run bit
for bit (fused), and the whole-image path (two-pass, KEEP) matches too."""
import numpy as np
import pytest

from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W,algo,border,pad", [(67, 260, "fused", "valid", 0), (1030, 1000, "fused", "valid", 0),
                                                 (300, 516, "two_pass", "valid", 0), (131, 132, "fused", "keep", 0),
                                                 (1030, 1000, "fused", "valid", 4), (300, 516, "two_pass", "valid", 8)])
def test_run_host_matches_device_run(H, W, algo, border, pad):
    """pad > 0: output rows with padding, which the call must leave as it was."""
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    A = synth.image(H + W, H, W)
    k = synth.kernel_normalised(H)
    hout, wout = (H, W) if border == "keep" else (H - 4, W - 4)
    plan = sc5.Plan(3, H, W, W, wout + pad, border=border, algo=algo)
    src = torch.from_numpy(A).pin_memory()
    dst = torch.full((3, hout, wout + pad), float("nan")).pin_memory()
    plan.run_host(src, dst, k)
    plan.run_host(src, dst, k)  # second call reuses the plan's staging buffers
    dev_out = torch.full((3, hout, wout + pad), float("nan"), device="cuda")
    plan.run(U.to_dev(A), dev_out, k)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    plan.close()
    got = dst.numpy()
    assert np.array_equal(got[:, :, :wout], dev_out.cpu().numpy()[:, :, :wout])
    assert U.is_finite_all(got[:, :, :wout])
    assert np.all(np.isnan(got[:, :, wout:])), "row padding written"
