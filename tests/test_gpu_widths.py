"""Separable kernels of other odd widths (3, 7, 9) through the fused kernel,
against the FP64 oracle's direct_n (Eq. 1 with K = k k^T of width n)."""
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


def _k(n, seed):
    u = synth.rng(seed).uniform(0, 1, n)
    return (u / u.sum()).astype(np.float32)


def _run(sc5, A_dev, P, H, W, pitch, k, n, dtype="f32", out_dtype=None, border="valid", in_scale=1.0, out_scale=1.0):
    import torch
    out_dtype = dtype if out_dtype is None else out_dtype
    hout, wout = (H, W) if border == "keep" else (H - n + 1, W - n + 1)
    op = U.pitch_for(wout, out_dtype)
    out = U.empty_dev((P, hout, op), out_dtype)
    plan = sc5.Plan(P, H, W, pitch, op, dtype, out_dtype, border, "fused", taps=n)
    plan.run(A_dev, out, k, in_scale, out_scale)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    plan.close()
    return U.from_dev(out, out_dtype)[:, :, :wout]


@pytest.mark.parametrize("n", [3, 7, 9])
def test_widths_against_oracle(sc5, n):
    for (H, W) in [(n, n), (n + 3, 70), (67, 259), (300, 517)]:
        pitch = U.pitch_for(W, "f32", extra=4)
        A = synth.image(n * 1000 + H + W, H, W, pitch=pitch)
        k = _k(n, H * W + n)
        ref = oracle.direct_n(A[:, :, :W].astype(np.float64), k.astype(np.float64))
        got = _run(sc5, U.to_dev(A), 3, H, W, pitch, k, n)
        assert got.shape == ref.shape
        assert U.max_abs(got, ref) <= U.FP32_TOL, (n, H, W)


def test_width9_compiled_shapes_agree(sc5):
    """Width 9 has two compiled shapes (2 and 3 stages): same bits, within the bound."""
    import torch
    H, W, n = 300, 517, 9
    pitch = U.pitch_for(W, "f32")
    A = synth.image(99, H, W, pitch=pitch)
    k = _k(n, 99)
    ref = oracle.direct_n(A[:, :, :W].astype(np.float64), k.astype(np.float64))
    A_dev = U.to_dev(A)
    op = U.pitch_for(W - n + 1, "f32")
    res = []
    for st in (3, 2):
        out = U.empty_dev((3, H - n + 1, op), "f32")
        plan = sc5.Plan(3, H, W, pitch, op, "f32", "f32", "valid", "fused", 128, 128, st, taps=n)
        plan.run(A_dev, out, k)
        torch.cuda.synchronize()
        assert sc5.device_status() == 0
        plan.close()
        res.append(U.from_dev(out, "f32")[:, :, :W - n + 1])
    assert np.array_equal(res[0], res[1])
    assert U.max_abs(res[0], ref) <= U.FP32_TOL


@pytest.mark.parametrize("n", [3, 7, 9])
def test_width_deltas_exact_and_keep_frame(sc5, n):
    H, W = 40, 136
    A = synth.image(n, H, W)
    r = (n - 1) // 2
    for t in (0, r, n - 1):
        k = np.zeros(n, np.float32)
        k[t] = 1.0
        got = _run(sc5, U.to_dev(A), 3, H, W, W, k, n)
        assert np.array_equal(got, A[:, t:t + H - n + 1, t:t + W - n + 1]), (n, t)
    k = _k(n, 5)
    got = _run(sc5, U.to_dev(A), 3, H, W, W, k, n, border="keep")
    frame = np.ones((H, W), bool)
    frame[r:H - r, r:W - r] = False
    assert np.array_equal(got[:, frame], A[:, frame])
    ref = oracle.direct_n(A.astype(np.float64), k.astype(np.float64))
    assert U.max_abs(got[:, r:H - r, r:W - r], ref) <= U.FP32_TOL


@pytest.mark.parametrize("dtype,out_dtype", [("bf16", "f32"), ("bf16", "bf16"), ("fp8e4m3", "fp8e4m3")])
def test_widths_narrow_formats(sc5, dtype, out_dtype):
    for n in (3, 9):
        H, W = 70, 300
        x = synth.image(n + 77, H, W)
        scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
        codes = synth.to_storage(x, dtype, scale)
        pitch = U.pitch_for(W, dtype)
        padded = np.zeros((3, H, pitch), codes.dtype)
        padded[:, :, :W] = codes
        k = _k(n, n + 77)
        ref = oracle.direct_n(U.decode(padded, dtype, scale)[:, :, :W], k.astype(np.float64))
        oscale = scale if out_dtype != "f32" else 1.0
        got = _run(sc5, U.to_dev(padded), 3, H, W, pitch, k, n, dtype, out_dtype, in_scale=scale, out_scale=oscale)
        val = U.decode(got, out_dtype, oscale)
        if out_dtype == "f32":
            assert U.max_abs(val, ref) <= U.FP32_TOL
        else:
            assert np.all(np.abs(val - ref) <= U.stored_tolerance(ref, out_dtype, oscale, U.FP32_TOL))


def test_width_refusals(sc5):
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, taps=4)
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, algo="two_pass", taps=7)
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 8, 64, taps=9)  # H < taps
