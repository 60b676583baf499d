"""GPU parity at the edges of what a plan accepts, and for every compiled
shape of the 8/16-bit formats.

* The tallest image a plan takes (H = 524,280 rows) and an image of over four
  million columns, fused and two-pass, against the FP64 oracle on every
  output; sizes one past each limit are refused.
* Every compiled (tile, stages) shape of every 8/16-bit format pair on a
  ragged image that spans several tiles, so that interior strips (the
  kernels' guard-free path) and edge strips both occur: bitwise equal to the
  two-pass pair, and within the format's bound of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu

H_MAX = 65535 * 8  # rows a plan accepts


@pytest.fixture(scope="module")
def sc5():
    import torch  # noqa: F401
    from paper_1711_09791_gb300 import sepconv5
    sepconv5.load()
    return sepconv5


def _run(sc5, A_dev, H, W, in_pitch, k, algo="fused", in_dtype="f32", out_dtype=None, in_scale=1.0,
         out_scale=1.0, **shape):
    import torch
    out_dtype = in_dtype if out_dtype is None else out_dtype
    out_pitch = U.pitch_for(W - 4, out_dtype)
    out = U.empty_dev((3, H - 4, out_pitch), out_dtype)
    plan = sc5.Plan(3, H, W, in_pitch, out_pitch, in_dtype, out_dtype, "valid", algo, **shape)
    plan.run(A_dev, out, k, in_scale, out_scale)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    plan.close()
    res = U.from_dev(out, out_dtype)
    assert U.sentinel_intact(res[:, :, W - 4:], out_dtype), "wrote past the VALID width"
    return res[:, :, :W - 4]


@pytest.mark.parametrize("H,W", [(H_MAX, 8), (6, (1 << 22) + 5)])
def test_largest_extents_against_oracle(sc5, H, W):
    """The most rows a plan accepts, and over 4M columns with a ragged tail:
    every output of both forms against the oracle; the forms agree bitwise."""
    pitch = U.pitch_for(W, "f32")
    A = synth.image(H % 1000 + W % 1000, H, W, pitch=pitch)
    k = synth.kernel_normalised(7)
    ref = oracle.direct(A[:, :, :W].astype(np.float64), k.astype(np.float64))
    A_dev = U.to_dev(A)
    fused = _run(sc5, A_dev, H, W, pitch, k)
    two = _run(sc5, A_dev, H, W, pitch, k, algo="two_pass")
    assert U.max_abs(fused, ref) <= U.FP32_TOL
    assert np.array_equal(fused, two)


def test_sizes_past_the_limits_are_refused(sc5):
    with pytest.raises(sc5.Sepconv5Error) as e:
        sc5.Plan(3, H_MAX + 1, 8, 8, 4)
    assert e.value.status == sc5.EINVAL
    W = (1 << 30) + 4
    with pytest.raises(sc5.Sepconv5Error) as e:
        sc5.Plan(3, 5, W, W, W - 4)
    assert e.value.status == sc5.EINVAL


NARROW_PAIRS = [("bf16", "bf16"), ("bf16", "f32"), ("f16", "f16"), ("f16", "f32"),
                ("fp8e4m3", "fp8e4m3"), ("fp8e4m3", "f32")]


@pytest.mark.parametrize("in_dtype,out_dtype", NARROW_PAIRS)
def test_every_narrow_shape(sc5, in_dtype, out_dtype):
    H, W = 300, 517
    x = synth.image(41, H, W)
    scale = synth.fp8_scale(x) if in_dtype == "fp8e4m3" else 1.0
    codes = synth.to_storage(x, in_dtype, scale)
    pitch = U.pitch_for(W, in_dtype)
    padded = np.zeros((3, H, pitch), codes.dtype)
    padded[:, :, :W] = codes
    k = synth.kernel_normalised(41)
    ref = U.oracle_valid(padded, in_dtype, k, scale, W=W)
    out_scale = 1.0 if out_dtype == "f32" else scale
    A_dev = U.to_dev(padded)
    two = _run(sc5, A_dev, H, W, pitch, k, "two_pass", in_dtype, out_dtype, scale, out_scale)
    configs = sc5.fused_configs(in_dtype, out_dtype)
    assert len(configs) >= 2
    for (th, tw, st) in configs:
        got = _run(sc5, A_dev, H, W, pitch, k, "fused", in_dtype, out_dtype, scale, out_scale,
                   tile_h=th, tile_w=tw, stages=st)
        assert np.array_equal(got, two), (th, tw, st)
    dec = U.decode(two, out_dtype, out_scale)
    if out_dtype == "f32":
        assert U.max_abs(dec, ref) <= U.FP32_TOL
    else:
        assert np.all(np.abs(dec - ref) <= U.stored_tolerance(ref, out_dtype, out_scale, U.FP32_TOL))


BATCH_SHAPES = [(300, 517), (67, 259), (130, 133), (5, 5), (64, 1030), (261, 77)]


@pytest.mark.parametrize("in_dtype,out_dtype", NARROW_PAIRS)
def test_every_narrow_shape_in_a_batch(sc5, in_dtype, out_dtype):
    """The work-list kernel with every compiled shape of a pair (the tuner may
    pick any of them for a batch or a merged serving launch), on ragged
    images of several tile rows and columns, each image bitwise equal to its
    two-pass result (checked against the oracle above)."""
    import torch
    imgs, twos = [], []
    for i, (H, W) in enumerate(BATCH_SHAPES):
        x = synth.image(60 + i, H, W)
        scale = synth.fp8_scale(x) if in_dtype == "fp8e4m3" else 1.0
        codes = synth.to_storage(x, in_dtype, scale)
        pitch = U.pitch_for(W, in_dtype)
        padded = np.zeros((3, H, pitch), codes.dtype)
        padded[:, :, :W] = codes
        k = synth.kernel_normalised(60 + i)
        out_scale = 1.0 if out_dtype == "f32" else scale
        A_dev = U.to_dev(padded)
        twos.append(_run(sc5, A_dev, H, W, pitch, k, "two_pass", in_dtype, out_dtype, scale, out_scale))
        op = U.pitch_for(W - 4, out_dtype)
        imgs.append({"in": A_dev, "out": U.empty_dev((3, H - 4, op), out_dtype), "H": H, "W": W, "in_pitch": pitch,
                     "out_pitch": op, "k": k, "in_scale": scale, "out_scale": out_scale})
    for (th, tw, st) in sc5.fused_configs(in_dtype, out_dtype):
        for im in imgs:
            im["out"].copy_(U.empty_dev(tuple(im["out"].shape), out_dtype))
        plan = sc5.Plan(3, 64, 64, in_dtype=in_dtype, out_dtype=out_dtype, tile_h=th, tile_w=tw, stages=st)
        plan.run_batch(imgs)
        torch.cuda.synchronize()
        assert sc5.device_status() == 0
        plan.close()
        for im, two in zip(imgs, twos):
            res = U.from_dev(im["out"], out_dtype)
            assert U.sentinel_intact(res[:, :, im["W"] - 4:], out_dtype), (th, tw, st)
            assert np.array_equal(res[:, :, :im["W"] - 4], two), (th, tw, st, im["H"], im["W"])
