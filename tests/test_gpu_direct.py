"""The direct single-pass kernel (25 products per output; Eq. 1 with a
general 5x5 matrix K, summed in the row-major order of Eq. 3) against the
FP64 oracle's direct_K.  Bound: max-abs 2e-4 for inputs in [0,255] and
sum|K| = 1; impulses, deltas and integer data are exact."""
import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc5():
    import torch  # noqa: F401
    from paper_1711_09791_gb300 import sepconv5
    sepconv5.load()
    return sepconv5


def _general_K(seed):
    K = synth.rng(seed).uniform(-1, 1, size=(5, 5))
    K /= np.abs(K).sum()
    return K.astype(np.float32)


def _run(sc5, A_dev, P, H, W, pitch, K=None, k=None, dtype="f32", out_dtype=None, border="valid", **kw):
    import torch
    out_dtype = dtype if out_dtype is None else out_dtype
    hout, wout = (H, W) if border == "keep" else (H - 4, W - 4)
    op = U.pitch_for(wout, out_dtype)
    out = U.empty_dev((P, hout, op), out_dtype)
    plan = sc5.Plan(P, H, W, pitch, op, dtype, out_dtype, border, "direct", **kw)
    if K is not None:
        plan.run_K(A_dev, out, K)
    else:
        plan.run(A_dev, out, k)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    plan.close()
    return U.from_dev(out, out_dtype)[:, :, :wout]


@pytest.mark.parametrize("H,W", [(5, 5), (9, 13), (67, 259), (130, 133), (300, 517)])
def test_general_K_against_oracle(sc5, H, W):
    pitch = U.pitch_for(W, "f32", extra=4)
    A = synth.image(H * 7 + W, H, W, pitch=pitch)
    K = _general_K(H + W)
    ref = oracle.direct_K(A[:, :, :W].astype(np.float64), K.astype(np.float64))
    A_dev = U.to_dev(A)
    for (th, tw, st) in [(0, 0, 0), (64, 128, 3), (32, 128, 4)]:
        got = _run(sc5, A_dev, 3, H, W, pitch, K=K, tile_h=th, tile_w=tw, stages=st)
        assert U.max_abs(got, ref) <= U.FP32_TOL, (th, tw, st)


def test_impulse_and_deltas_exact(sc5):
    K = (np.arange(25, dtype=np.float32).reshape(5, 5) - 12.0) / 16.0  # exact in FP32, not symmetric
    A = np.zeros((3, 9, 12), np.float32)
    A[:, 4, 4] = 1.0
    got = _run(sc5, U.to_dev(A), 3, 9, 12, 12, K=K)
    assert np.array_equal(got[:, :, :5], np.broadcast_to(K[::-1, ::-1], (3, 5, 5)))
    img = synth.image(3, 40, 68)
    for (i, j) in [(0, 0), (0, 4), (2, 2), (3, 1), (4, 4)]:
        D = np.zeros((5, 5), np.float32)
        D[i, j] = 1.0
        got = _run(sc5, U.to_dev(img), 3, 40, 68, 68, K=D)
        assert np.array_equal(got, img[:, i:i + 36, j:j + 64]), (i, j)


def test_integer_data_exact(sc5):
    A = synth.integer_image(8, 70, 132)
    K = synth.rng(8).integers(-3, 4, size=(5, 5)).astype(np.float32)
    ref = oracle.direct_K(A.astype(np.float64), K.astype(np.float64))
    got = _run(sc5, U.to_dev(A), 3, 70, 132, 132, K=K)
    assert np.array_equal(got.astype(np.float64), ref)


def test_separable_through_direct_form(sc5):
    """algo 'direct' with the taps k uses K = k k^T: the paper's single-pass
    algorithm on the separable kernel, against the oracle and the fused form."""
    import torch
    H, W = 131, 260
    A = synth.image(9, H, W)
    k = synth.kernel_normalised(9)
    ref = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    got = _run(sc5, U.to_dev(A), 3, H, W, W, k=k)
    assert U.max_abs(got, ref) <= U.FP32_TOL
    out = torch.empty((3, H - 4, W - 4), dtype=torch.float32, device="cuda")
    plan = sc5.Plan(3, H, W, W, W - 4)
    plan.run(U.to_dev(A), out, k)
    torch.cuda.synchronize()
    plan.close()
    assert U.max_abs(out.cpu().numpy(), got) <= U.FP32_TOL


@pytest.mark.parametrize("dtype", ["bf16", "fp8e4m3"])
def test_general_K_narrow_formats(sc5, dtype):
    H, W = 100, 300
    x = synth.image(10, H, W)
    scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
    codes = synth.to_storage(x, dtype, scale)
    pitch = U.pitch_for(W, dtype)
    padded = np.zeros((3, H, pitch), codes.dtype)
    padded[:, :, :W] = codes
    K = _general_K(10)
    ref = oracle.direct_K(U.decode(padded, dtype, scale)[:, :, :W], K.astype(np.float64))
    import torch
    out = torch.empty((3, H - 4, U.pitch_for(W - 4, "f32")), dtype=torch.float32, device="cuda")
    plan = sc5.Plan(3, H, W, pitch, out.shape[2], dtype, "f32", "valid", "direct")
    plan.run_K(U.to_dev(padded), out, K, in_scale=scale, out_scale=1.0)
    torch.cuda.synchronize()
    plan.close()
    assert U.max_abs(out.cpu().numpy()[:, :, :W - 4], ref) <= U.FP32_TOL


def test_keep_border_and_refusals(sc5):
    H, W = 50, 72
    A = synth.image(11, H, W)
    K = _general_K(11)
    got = _run(sc5, U.to_dev(A), 3, H, W, W, K=K, border="keep")
    frame = np.ones((H, W), bool)
    frame[2:-2, 2:-2] = False
    assert np.array_equal(got[:, frame], A[:, frame])
    ref = oracle.direct_K(A.astype(np.float64), K.astype(np.float64))
    assert U.max_abs(got[:, 2:-2, 2:-2], ref) <= U.FP32_TOL
    import torch
    plan = sc5.Plan(3, H, W, W, W - 4)  # not a direct plan
    out = torch.empty((3, H - 4, W - 4), dtype=torch.float32, device="cuda")
    with pytest.raises(sc5.Sepconv5Error):
        plan.run_K(U.to_dev(A), out, K)
    plan.close()


def test_direct_8192_every_pixel(sc5):
    """The direct single pass (25 products per output) on the 3 x 8192 x 8192
    FP32 image in the launch configuration the benchmark times (the
    planner's default direct plan): every output pixel against the FP64
    oracle in bands of 512 output rows."""
    import torch
    P, H, W = 3, 8192, 8192
    A = synth.image(2, H, W)
    k = synth.kernel_normalised(2)
    out = torch.empty((P, H - 4, W - 4), dtype=torch.float32, device="cuda")
    plan = sc5.Plan(P, H, W, W, W - 4, algo="direct")
    plan.run(U.to_dev(A), out, k)
    torch.cuda.synchronize()
    plan.close()
    assert sc5.device_status() == 0
    got = out.cpu().numpy()
    del out
    k64 = k.astype(np.float64)
    for r0 in range(0, H - 4, 512):
        r1 = min(H - 4, r0 + 512)
        ref = oracle.direct(A[:, r0:r1 + 4, :].astype(np.float64), k64)
        assert U.max_abs(got[:, r0:r1, :], ref) <= U.FP32_TOL, r0
