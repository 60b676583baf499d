"""Pixel-interleaved (HWC) 3-plane images through the fused kernel: the
result, de-interleaved, equals bit for bit the planar fused result of the
same image and lies within the bound of the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


def to_hwc(A, pitch):
    P, H, W = A.shape
    X = np.zeros((H, pitch), A.dtype)
    X[:, :3 * W] = np.transpose(A, (1, 2, 0)).reshape(H, 3 * W)
    return X


def from_hwc(X, W):
    H = X.shape[0]
    return np.ascontiguousarray(np.transpose(X[:, :3 * W].reshape(H, W, 3), (2, 0, 1)))


@pytest.mark.parametrize("H,W", [(5, 5), (9, 70), (67, 259), (130, 133), (300, 517)])
def test_hwc_f32(H, W):
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    A = synth.image(H * 31 + W, H, W)
    k = synth.kernel_normalised(H + 2 * W)
    ref = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    pitch = U.round_up(3 * W, 4) + 4
    X = to_hwc(A, pitch)
    X[:, 3 * W:] = np.nan  # padding must never be read
    opitch = U.round_up(3 * (W - 4), 4)
    Y = torch.full((H - 4, opitch), float("nan"), device="cuda")
    plan = sc5.Plan(3, H, W, pitch, opitch, layout="hwc")
    plan.run(U.to_dev(X), Y, k)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    plan.close()
    y = Y.cpu().numpy()
    assert U.sentinel_intact(y[:, 3 * (W - 4):], "f32")
    got = from_hwc(y, W - 4)
    assert U.max_abs(got, ref) <= U.FP32_TOL
    out = torch.empty((3, H - 4, W - 4), device="cuda")
    pp = U.pitch_for(W, "f32")
    Ap = np.zeros((3, H, pp), np.float32)
    Ap[:, :, :W] = A
    planar = sc5.Plan(3, H, W, pp, W - 4)
    planar.run(U.to_dev(Ap), out, k)
    torch.cuda.synchronize()
    planar.close()
    assert np.array_equal(got, out.cpu().numpy())


@pytest.mark.parametrize("dtype,out_dtype", [("bf16", "bf16"), ("bf16", "f32"), ("f16", "f16"),
                                             ("fp8e4m3", "fp8e4m3"), ("fp8e4m3", "f32")])
def test_hwc_narrow_formats(dtype, out_dtype):
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    H, W = 70, 300
    x = synth.image(71, H, W)
    scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
    codes = synth.to_storage(x, dtype, scale)
    es = {"bf16": 2, "f16": 2, "fp8e4m3": 1}[dtype]
    pitch = U.round_up(3 * W * es, 16) // es
    X = to_hwc(codes, pitch)
    oscale = scale if out_dtype != "f32" else 1.0
    opitch = U.round_up(3 * (W - 4), 4)
    Y = U.empty_dev((H - 4, opitch), out_dtype)
    plan = sc5.Plan(3, H, W, pitch, opitch, dtype, out_dtype, layout="hwc")
    plan.run(U.to_dev(X), Y, synth.kernel_normalised(71), scale, oscale)
    torch.cuda.synchronize()
    plan.close()
    got = U.decode(from_hwc(U.from_dev(Y, out_dtype), W - 4), out_dtype, oscale)
    ref = oracle.direct(U.decode(codes, dtype, scale), synth.kernel_normalised(71).astype(np.float64))
    if out_dtype == "f32":
        assert U.max_abs(got, ref) <= U.FP32_TOL
    else:
        assert np.all(np.abs(got - ref) <= U.stored_tolerance(ref, out_dtype, oscale, U.FP32_TOL))


def test_hwc_refusals():
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(2, 64, 64, 192, 180, layout="hwc")  # 3 planes only
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, 190, 180, layout="hwc")  # pitch below 3W
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, 192, 180, algo="two_pass", layout="hwc")
