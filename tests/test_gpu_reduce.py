"""GPU parity of the pyramid REDUCE step (SC5_ALGO_REDUCE) through the C ABI.

* Every storage pair on ragged sizes: bitwise equal to the fused result at
  every second row and column, and within the format's bound of the FP64
  oracle's REDUCE step on the decoded inputs.
* A five-level FP32 pyramid: level L of the GPU chain against L oracle steps
  applied to the original image (the oracle never sees a GPU result), within
  L times the FP32 bound.
* 3 x 8192 x 8192 FP32: every output against the oracle's REDUCE step.
* Plans and calls the step does not support are refused.
"""
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


PAIRS = [("f32", "f32"), ("bf16", "bf16"), ("bf16", "f32"), ("f16", "f16"), ("f16", "f32"),
         ("fp8e4m3", "fp8e4m3"), ("fp8e4m3", "f32")]
SIZES = [(5, 5), (6, 7), (37, 131), (130, 261), (300, 517)]


def _stored(x, dtype):
    scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
    codes = synth.to_storage(x, dtype, scale)
    P, H, W = codes.shape
    pitch = U.pitch_for(W, dtype)
    padded = np.zeros((P, H, pitch), codes.dtype)
    padded[:, :, :W] = codes
    return padded, scale


def _reduce(sc5, A_dev, H, W, pitch, k, in_dtype, out_dtype, in_scale, out_scale, P=3):
    import torch
    Ho, Wo = sc5.reduce_dims(H, W)
    op = U.pitch_for(Wo, out_dtype)
    out = U.empty_dev((P, Ho, op), out_dtype)
    plan = sc5.Plan(P, H, W, pitch, op, in_dtype, out_dtype, algo="reduce")
    plan.run(A_dev, out, k, in_scale, out_scale)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    plan.close()
    res = U.from_dev(out, out_dtype)
    assert U.sentinel_intact(res[:, :, Wo:], out_dtype), "wrote past Wo"
    return res[:, :, :Wo], out


def _fused(sc5, A_dev, H, W, pitch, k, in_dtype, out_dtype, in_scale, out_scale, P=3):
    import torch
    op = U.pitch_for(W - 4, out_dtype)
    out = U.empty_dev((P, H - 4, op), out_dtype)
    plan = sc5.Plan(P, H, W, pitch, op, in_dtype, out_dtype)
    plan.run(A_dev, out, k, in_scale, out_scale)
    torch.cuda.synchronize()
    plan.close()
    return U.from_dev(out, out_dtype)[:, :, :W - 4]


@pytest.mark.parametrize("in_dtype,out_dtype", PAIRS)
@pytest.mark.parametrize("H,W", SIZES)
def test_reduce_equals_fused_at_even_positions_and_oracle(sc5, in_dtype, out_dtype, H, W):
    x = synth.image(H * 31 + W, H, W)
    padded, scale = _stored(x, in_dtype)
    pitch = padded.shape[2]
    k = synth.kernel_normalised(H + W)
    out_scale = 1.0 if out_dtype == "f32" else scale
    A_dev = U.to_dev(padded)
    got, _ = _reduce(sc5, A_dev, H, W, pitch, k, in_dtype, out_dtype, scale, out_scale)
    full = _fused(sc5, A_dev, H, W, pitch, k, in_dtype, out_dtype, scale, out_scale)
    assert np.array_equal(got, full[:, ::2, ::2])
    ref = oracle.reduce2(U.decode(padded[:, :, :W], in_dtype, scale), k)
    dec = U.decode(got, out_dtype, out_scale)
    assert dec.shape == ref.shape
    if out_dtype == "f32":
        assert U.max_abs(dec, ref) <= U.FP32_TOL
    else:
        assert np.all(np.abs(dec - ref) <= U.stored_tolerance(ref, out_dtype, out_scale, U.FP32_TOL))


@pytest.mark.parametrize("in_dtype,out_dtype", PAIRS)
def test_every_compiled_reduce_shape(sc5, in_dtype, out_dtype):
    """Each (input rows per tile, stages) a plan accepts runs the same
    arithmetic: bitwise the fused result at even rows and columns."""
    import torch
    H, W = 300, 517
    padded, scale = _stored(synth.image(5, H, W), in_dtype)
    pitch = padded.shape[2]
    k = synth.kernel_normalised(5)
    out_scale = 1.0 if out_dtype == "f32" else scale
    A_dev = U.to_dev(padded)
    full = _fused(sc5, A_dev, H, W, pitch, k, in_dtype, out_dtype, scale, out_scale)[:, ::2, ::2]
    Ho, Wo = sc5.reduce_dims(H, W)
    op = U.pitch_for(Wo, out_dtype)
    seen = set()
    for th in (32, 64, 96, 128, 256):
        for st in range(1, 9):
            try:
                plan = sc5.Plan(3, H, W, pitch, op, in_dtype, out_dtype, algo="reduce", tile_h=th, stages=st)
            except sc5.Sepconv5Error as e:
                assert e.status == sc5.EINVAL
                continue
            info = plan.info()
            assert (info["tile_h"], info["stages"]) == (th, st)
            out = U.empty_dev((3, Ho, op), out_dtype)
            plan.run(A_dev, out, k, scale, out_scale)
            torch.cuda.synchronize()
            assert sc5.device_status() == 0
            plan.close()
            assert np.array_equal(U.from_dev(out, out_dtype)[:, :, :Wo], full), (th, st)
            seen.add((th, st))
    assert len(seen) == 4, seen


def test_five_level_pyramid(sc5):
    import torch
    H = W = 1030
    pitch = U.pitch_for(W, "f32")
    x = synth.image(17, H, W, pitch=pitch)  # NaN in the padding columns
    k = synth.kernel_binomial()
    cur = U.to_dev(x)
    h, w = H, W
    ref = x[:, :, :W].astype(np.float64)
    for level in range(1, 6):
        got, out = _reduce(sc5, cur, h, w, pitch, k, "f32", "f32", 1.0, 1.0)
        ref = oracle.reduce2(ref, k)
        assert got.shape == ref.shape
        assert U.max_abs(got, ref) <= level * U.FP32_TOL, level
        cur, pitch = out, out.shape[2]
        h, w = got.shape[1], got.shape[2]
    assert (h, w) == (29, 29)
    torch.cuda.synchronize()


def test_full_size_every_output(sc5):
    """3 x 8192 x 8192 FP32: every REDUCE output against the oracle's REDUCE
    step, in bands of 512 output rows (output row y is centred on input row
    2y + 2, so a band of rows [r0, r1) reads input rows [2 r0, 2 r1 + 3))."""
    import torch
    P, H, W = 3, 8192, 8192
    A = synth.image(2, H, W)
    k = synth.kernel_normalised(2)
    k64 = k.astype(np.float64)
    got, _ = _reduce(sc5, U.to_dev(A), H, W, W, k, "f32", "f32", 1.0, 1.0)
    Ho, Wo = sc5.reduce_dims(H, W)
    assert got.shape == (P, Ho, Wo)
    for r0 in range(0, Ho, 512):
        r1 = min(Ho, r0 + 512)
        ref = oracle.reduce2(A[:, 2 * r0:2 * r1 + 3, :].astype(np.float64), k64)
        assert ref.shape == (P, r1 - r0, Wo)
        err = U.max_abs(got[:, r0:r1, :], ref)
        assert err <= U.FP32_TOL, (r0, err)
    torch.cuda.synchronize()


def test_unsupported_reduce_plans_and_calls_refused(sc5):
    import torch
    with pytest.raises(sc5.Sepconv5Error) as e:
        sc5.Plan(3, 64, 64, 64, 30, algo="reduce", border="keep")
    assert e.value.status == sc5.EINVAL
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, 64, 29, algo="reduce")  # out_pitch < Wo = 30
    plan = sc5.Plan(3, 64, 68, 68, 32, algo="reduce")
    A = torch.zeros((3, 64, 68), dtype=torch.float32).pin_memory()
    out = torch.zeros((3, 30, 32), dtype=torch.float32).pin_memory()
    with pytest.raises(sc5.Sepconv5Error):
        plan.run_host(A, out, [0, 0, 1, 0, 0])
    assert plan.info()["tile_w"] == 128
    plan.close()


@pytest.mark.parametrize("in_dtype,out_dtype", [("f32", "f32"), ("bf16", "f32"), ("bf16", "bf16")])
def test_pyramid_api_matches_chained_plans(sc5, in_dtype, out_dtype):
    """sepconv5_pyramid_*: level sizes and pitches, and every level bitwise the
    result of chaining REDUCE plans by hand; FP32 levels also against the
    oracle's steps on the original image."""
    import torch
    H = W = 530
    x = synth.image(23, H, W)
    padded, scale = _stored(x, in_dtype)
    pitch = padded.shape[2]
    k = synth.kernel_normalised(23)
    out_scale = 1.0 if out_dtype == "f32" else scale
    A_dev = U.to_dev(padded)
    pyr = sc5.Pyramid(3, H, W, pitch, in_dtype, out_dtype, levels=4)
    assert pyr.level(0) == (H, W, pitch)
    bufs = []
    for lv in range(1, 5):
        h, w, p = pyr.level(lv)
        assert (h, w) == sc5.reduce_dims(*pyr.level(lv - 1)[:2])
        assert (p * sc5.DTYPE_BYTES[out_dtype]) % 16 == 0 and p >= w
        bufs.append(U.empty_dev((3, h, p), out_dtype))
    pyr.run(A_dev, bufs, k, scale, out_scale)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    pyr.close()
    cur, h, w, p, dt, s_in = A_dev, H, W, pitch, in_dtype, scale
    ref = U.decode(padded[:, :, :W], in_dtype, scale)
    for lv, buf in enumerate(bufs, start=1):
        want, out = _reduce(sc5, cur, h, w, p, k, dt, out_dtype, s_in, out_scale)
        got = U.from_dev(buf, out_dtype)[:, :, :want.shape[2]]
        assert np.array_equal(got, want), lv
        ref = oracle.reduce2(ref, k)
        if out_dtype == "f32":
            assert U.max_abs(got, ref) <= lv * U.FP32_TOL, lv
        cur, p, dt, s_in = out, out.shape[2], out_dtype, out_scale
        h, w = want.shape[1], want.shape[2]


def test_pyramid_graph_replay_matches_run(sc5):
    import torch
    H = W = 700
    A = U.to_dev(synth.image(31, H, W, pitch=U.pitch_for(W, "f32")))
    k = synth.kernel_normalised(31)
    pyr = sc5.Pyramid(3, H, W, U.pitch_for(W, "f32"), "f32", levels=3)
    shapes = [pyr.level(lv) for lv in range(1, 4)]
    run_bufs = [U.empty_dev((3, h, p), "f32") for h, w, p in shapes]
    graph_bufs = [U.empty_dev((3, h, p), "f32") for h, w, p in shapes]
    with pytest.raises(sc5.Sepconv5Error):
        pyr.replay()  # nothing captured yet
    pyr.run(A, run_bufs, k)
    pyr.capture(A, graph_bufs, k)
    torch.cuda.synchronize()
    for b in graph_bufs:  # capturing ran nothing
        assert U.sentinel_intact(U.from_dev(b, "f32"), "f32")
    pyr.replay()
    pyr.replay()
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    for (h, w, p), a, b in zip(shapes, run_bufs, graph_bufs):
        assert np.array_equal(U.from_dev(a, "f32")[:, :, :w], U.from_dev(b, "f32")[:, :, :w])
    pyr.close()


def test_pyramid_refusals(sc5):
    with pytest.raises(sc5.Sepconv5Error) as e:
        sc5.Pyramid(3, 40, 40, 40, "f32", levels=4)  # 40 -> 18 -> 7 -> 2: level 3 is too small to reduce
    assert e.value.status == sc5.EINVAL
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Pyramid(3, 64, 64, 64, "f32", "bf16", levels=1)  # levels in the input's format or FP32
    pyr = sc5.Pyramid(3, 40, 40, 40, "f32", levels=3)
    assert pyr.level(3) == (2, 2, 4)
    with pytest.raises(sc5.Sepconv5Error):
        pyr.level(4)
    pyr.close()
