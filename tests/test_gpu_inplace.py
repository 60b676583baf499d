"""In-place convolution (sepconv5_run_inplace): the image Listing 1 leaves in
A -- interior replaced by the result, 2-pixel frame unchanged -- computed by
Listing 1's two-pass structure and by the single pass with copy-back."""
import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("H,W", [(5, 8), (67, 132), (300, 520)])
def test_inplace_all_algorithms(H, W):
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    A = synth.image(H + W, H, W)
    k = synth.kernel_normalised(H + W)
    ref = oracle.keep_frame(A.astype(np.float64), oracle.direct(A.astype(np.float64), k.astype(np.float64)))
    frame = np.ones((H, W), bool)
    frame[2:-2, 2:-2] = False
    res = {}
    for algo in ("two_pass", "fused", "direct"):
        img = U.to_dev(A)
        plan = sc5.Plan(3, H, W, W, W, border="keep", algo=algo)
        plan.run_inplace(img, k)
        torch.cuda.synchronize()
        plan.close()
        assert sc5.device_status() == 0
        got = img.cpu().numpy()
        assert np.array_equal(got[:, frame], A[:, frame]), algo
        assert U.max_abs(got, ref) <= U.FP32_TOL, algo
        res[algo] = got
    assert np.array_equal(res["two_pass"], res["fused"])  # same FP32 evaluation order


def test_inplace_bf16_and_refusals():
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    H, W = 64, 136
    x = synth.image(12, H, W)
    codes = synth.to_storage(x, "bf16")
    k = synth.kernel_normalised(12)
    vals = U.decode(codes, "bf16")
    ref = oracle.direct(vals, k.astype(np.float64))
    img = U.to_dev(codes)
    plan = sc5.Plan(3, H, W, W, W, "bf16", "bf16", "keep", "fused")
    plan.run_inplace(img, k)
    torch.cuda.synchronize()
    got = U.from_dev(img, "bf16")
    assert np.array_equal(got[:, :2], codes[:, :2]) and np.array_equal(got[:, :, -2:], codes[:, :, -2:])
    inner = U.decode(got[:, 2:-2, 2:-2], "bf16")
    assert np.all(np.abs(inner - ref) <= U.stored_tolerance(ref, "bf16", 1.0, U.FP32_TOL))
    plan.close()
    valid = sc5.Plan(3, H, W, W, W - 4, "bf16", "bf16", "valid", "fused")
    with pytest.raises(sc5.Sepconv5Error):
        valid.run_inplace(img, k)
    valid.close()
