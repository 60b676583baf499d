"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every input comes from the seeded generators; every expected value from the
oracle.  FP32 bound: max-abs 2e-4 for inputs in [0, 255] and sum(k) = 1.
Integer-valued cases and delta kernels are exact in FP32, so there the bound
is bitwise equality.  The fused and two-pass forms use the same FP32
evaluation order, so they must agree bit for bit.
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


def _run(sc5, A_dev, P, H, W, in_pitch, k, algo="fused", in_dtype="f32", out_dtype=None, border="valid",
         out_pitch=None, in_scale=1.0, out_scale=1.0, **shape):
    import torch
    out_dtype = in_dtype if out_dtype is None else out_dtype
    Hout = H if border == "keep" else H - 4
    wout = W if border == "keep" else W - 4
    out_pitch = U.pitch_for(wout, out_dtype) if out_pitch is None else out_pitch
    out = U.empty_dev((P, Hout, out_pitch), out_dtype)
    plan = sc5.Plan(P, H, W, in_pitch, out_pitch, in_dtype, out_dtype, border, algo, **shape)
    plan.run(A_dev, out, k, in_scale, out_scale)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    plan.close()
    return U.from_dev(out, out_dtype), out_pitch


# ------------------------------------------------------------------ FP32


def test_c1_512_binomial_fused_and_two_pass(sc5):
    """3 x 512 x 512 FP32, k = [1,4,6,4,1]/16, both forms against the oracle."""
    P, H, W = 3, 512, 512
    A = synth.image(1, H, W)
    k = synth.kernel_binomial()
    ref = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    A_dev = U.to_dev(A)
    outs = {}
    for algo in ("fused", "two_pass"):
        out, op = _run(sc5, A_dev, P, H, W, W, k, algo=algo, out_pitch=512)
        assert U.sentinel_intact(out[:, :, W - 4:], "f32"), "wrote past the VALID width"
        outs[algo] = out[:, :, :W - 4]
        assert U.max_abs(outs[algo], ref) <= U.FP32_TOL
    assert np.array_equal(outs["fused"], outs["two_pass"])


SHAPES = [(5, 5), (6, 7), (9, 13), (37, 131), (67, 259), (130, 133), (300, 517)]


@pytest.mark.parametrize("H,W", SHAPES)
def test_ragged_shapes_every_fused_shape(sc5, H, W):
    P = 3
    pitch = U.pitch_for(W, "f32", extra=4)
    A = synth.image(H * 1000 + W, H, W, pitch=pitch)  # NaN in the padding columns
    k = synth.kernel_normalised(H + W)
    ref = oracle.direct(A[:, :, :W].astype(np.float64), k.astype(np.float64))
    A_dev = U.to_dev(A)
    two, _ = _run(sc5, A_dev, P, H, W, pitch, k, algo="two_pass")
    two = two[:, :, :W - 4]
    assert U.max_abs(two, ref) <= U.FP32_TOL
    for (th, tw, st) in sc5.fused_configs("f32"):
        out, _ = _run(sc5, A_dev, P, H, W, pitch, k, tile_h=th, tile_w=tw, stages=st)
        assert U.is_finite_all(out[:, :, :W - 4])
        assert U.max_abs(out[:, :, :W - 4], ref) <= U.FP32_TOL, (th, tw, st)
        assert np.array_equal(out[:, :, :W - 4], two), (th, tw, st)


@pytest.mark.parametrize("algo", ["fused", "two_pass"])
def test_shifted_delta_kernels_exact(sc5, algo):
    """k = e_t moves the image by t-2 on both axes, exactly (pins orientation)."""
    P, H, W = 3, 70, 133
    pitch = U.pitch_for(W, "f32")
    A = synth.image(5, H, W, pitch=pitch)
    A_dev = U.to_dev(A)
    for t in range(5):
        k = np.zeros(5, np.float32)
        k[t] = 1.0
        out, _ = _run(sc5, A_dev, P, H, W, pitch, k, algo=algo, out_pitch=W - 4)
        assert np.array_equal(out, A[:, t:t + H - 4, t:t + W - 4]), t


@pytest.mark.parametrize("algo", ["fused", "two_pass"])
def test_exact_integers_bitwise(sc5, algo):
    """Integer pixels and k = [1,4,6,4,1]: every partial sum is an integer
    below 2^24, so FP32 is exact and must equal the oracle bit for bit."""
    P, H, W = 3, 133, 301
    A = synth.integer_image(9, H, W)
    k = np.array([1, 4, 6, 4, 1], np.float32)
    ref = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    pitch = U.pitch_for(W, "f32")
    Ap = np.zeros((P, H, pitch), np.float32)
    Ap[:, :, :W] = A
    out, _ = _run(sc5, U.to_dev(Ap), P, H, W, pitch, k, algo=algo, out_pitch=W - 4)
    assert np.array_equal(out.astype(np.float64), ref)


def test_hpass_and_vpass_separately(sc5):
    """Each pass of the two-pass form against its own oracle pass."""
    import torch
    P, H, W = 3, 41, 203
    A = synth.image(12, H, W, pitch=U.pitch_for(W, "f32"))
    pitch = A.shape[2]
    k = synth.kernel_normalised(12)
    k64 = k.astype(np.float64)
    plan = sc5.Plan(P, H, W, pitch, U.pitch_for(W - 4, "f32"), algo="two_pass")
    t_pitch = U.round_up(W - 4, 4) + 4
    T = torch.full((P, H, t_pitch), float("nan"), dtype=torch.float32, device="cuda")
    plan.hpass(U.to_dev(A), T, t_pitch, k)
    torch.cuda.synchronize()
    Th = T.cpu().numpy()
    assert U.sentinel_intact(Th[:, :, W - 4:], "f32")
    T_ref = oracle.hpass(A[:, :, :W].astype(np.float64), k64)
    assert U.max_abs(Th[:, :, :W - 4], T_ref) <= 1e-4  # 5 FP32 terms of size <= 255
    out = U.empty_dev((P, H - 4, plan.desc.out_pitch), "f32")
    plan.vpass(T, t_pitch, out, k)
    torch.cuda.synchronize()
    B = out.cpu().numpy()[:, :, :W - 4]
    B_ref = oracle.vpass(Th[:, :, :W - 4].astype(np.float64), k64)
    assert U.max_abs(B, B_ref) <= 1e-4
    assert U.max_abs(B, oracle.direct(A[:, :, :W].astype(np.float64), k64)) <= U.FP32_TOL
    plan.close()


@pytest.mark.parametrize("algo", ["fused", "two_pass"])
def test_keep_border(sc5, algo):
    """KEEP: the 2-pixel frame is the input, the interior the VALID result."""
    P, H, W = 3, 77, 150
    pitch = U.pitch_for(W, "f32")
    Ap = synth.image(21, H, W, pitch=pitch)
    A = np.ascontiguousarray(Ap[:, :, :W])
    k = synth.kernel_normalised(21)
    ref = oracle.keep_frame(A.astype(np.float64), oracle.direct(A.astype(np.float64), k.astype(np.float64)))
    out, _ = _run(sc5, U.to_dev(Ap), P, H, W, pitch, k, algo=algo, border="keep", out_pitch=W)
    frame = np.ones((H, W), bool)
    frame[2:-2, 2:-2] = False
    assert np.array_equal(out[:, frame], A[:, frame])
    assert U.max_abs(out[:, 2:-2, 2:-2], ref[:, 2:-2, 2:-2]) <= U.FP32_TOL


def test_c2_8192_every_pixel(sc5):
    """3 x 8192 x 8192 FP32 in the launch configuration the benchmark times
    (the planner's default plan): every output pixel against the FP64 oracle,
    in bands of 512 output rows (each oracle band reads its 4 halo rows from
    the image), and fused == two-pass bit for bit."""
    import torch
    P, H, W = 3, 8192, 8192
    A = synth.image(2, H, W)
    k = synth.kernel_normalised(2)
    k64 = k.astype(np.float64)
    A_dev = U.to_dev(A)
    outs = {}
    for algo in ("fused", "two_pass"):
        out = torch.empty((P, H - 4, W - 4), dtype=torch.float32, device="cuda")
        plan = sc5.Plan(P, H, W, W, W - 4, algo=algo)
        plan.run(A_dev, out, k)
        torch.cuda.synchronize()
        plan.close()
        outs[algo] = out
    assert sc5.device_status() == 0
    assert torch.equal(outs["fused"], outs["two_pass"])
    fused = outs["fused"].cpu().numpy()
    del outs, A_dev
    worst = 0.0
    for r0 in range(0, H - 4, 512):
        r1 = min(H - 4, r0 + 512)
        ref = oracle.direct(A[:, r0:r1 + 4, :].astype(np.float64), k64)
        err = U.max_abs(fused[:, r0:r1, :], ref)
        assert err <= U.FP32_TOL, (r0, err)
        worst = max(worst, err)
    assert np.isfinite(worst)


# ------------------------------------------------------------------ reduced precision


@pytest.mark.parametrize("dtype", ["bf16", "f16", "fp8e4m3"])
@pytest.mark.parametrize("out_f32", [False, True])
def test_reduced_precision_storage(sc5, dtype, out_f32):
    """Stored inputs are decoded exactly; the FP32 result is compared with the
    oracle on the decoded inputs (the kernel error), within half an ulp of the
    output format plus the FP32 bound."""
    P, H, W = 3, 131, 301
    x = synth.image(31, H, W)
    scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
    codes = synth.to_storage(x, dtype, scale)
    pitch = U.pitch_for(W, dtype)
    padded = np.zeros((P, H, pitch), codes.dtype)
    padded[:, :, :W] = codes
    k = synth.kernel_normalised(31)
    ref = U.oracle_valid(padded, dtype, k, scale, W=W)
    out_dtype = "f32" if out_f32 else dtype
    out_scale = 1.0 if out_f32 else scale
    A_dev = U.to_dev(padded)
    res = {}
    for algo in ("fused", "two_pass"):
        out, _ = _run(sc5, A_dev, P, H, W, pitch, k, algo=algo, in_dtype=dtype, out_dtype=out_dtype,
                      in_scale=scale, out_scale=out_scale)
        res[algo] = out[:, :, :W - 4]
    assert np.array_equal(res["fused"], res["two_pass"])
    got = U.decode(res["fused"], out_dtype, out_scale)
    # The FP32 evaluation runs on the codes (up to 448 for fp8, i.e. max|x| * scale),
    # so its error in real units is the FP32 bound for values up to 255.
    if out_f32:
        assert U.max_abs(got, ref) <= U.FP32_TOL
    else:
        tol = U.stored_tolerance(ref, out_dtype, out_scale, U.FP32_TOL)
        assert np.all(np.abs(got - ref) <= tol)


# ------------------------------------------------------------------ batches


def _batch_images(sc5, shapes, seed, dtype="f32", out_dtype=None):
    out_dtype = dtype if out_dtype is None else out_dtype
    imgs, host, keep = [], [], []
    for i, (H, W) in enumerate(shapes):
        x = synth.image(seed * 1000 + i, H, W)
        scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
        codes = synth.to_storage(x, dtype, scale)
        pitch = U.pitch_for(W, dtype)
        padded = np.zeros((3, H, pitch), codes.dtype)
        padded[:, :, :W] = codes
        A = U.to_dev(padded)
        op = U.pitch_for(W - 4, out_dtype)
        out = U.empty_dev((3, H - 4, op), out_dtype)
        k = synth.kernel_normalised(seed * 1000 + i)
        imgs.append({"in": A, "out": out, "H": H, "W": W, "in_pitch": pitch, "out_pitch": op, "k": k,
                     "in_scale": scale, "out_scale": 1.0 if out_dtype == "f32" else scale})
        host.append(padded)
        keep.extend([A, out])
    return imgs, host, keep


BATCH_SHAPES = [(5, 5), (64, 64), (100, 3000), (517, 300), (131, 129), (1030, 70), (6, 400), (260, 260),
                (64, 4096), (2000, 64), (77, 77), (9, 13)]


BATCH_PAIRS = [("f32", "f32"), ("bf16", "bf16"), ("bf16", "f32"), ("f16", "f16"), ("f16", "f32"),
               ("fp8e4m3", "fp8e4m3"), ("fp8e4m3", "f32")]


@pytest.mark.parametrize("dtype,out_dtype", BATCH_PAIRS)
def test_batch_matches_single_runs_and_oracle(sc5, dtype, out_dtype):
    """Every storage pair the batch kernel is built for (the stored-format
    batches the benchmark times included): one-shot and graph-replayed batches
    agree bit for bit with each other and with single-image runs, and with the
    FP64 oracle on the decoded inputs within the FP32 bound plus half an ulp of
    the output format."""
    import torch
    imgs, host, _keep = _batch_images(sc5, BATCH_SHAPES, 3, dtype, out_dtype)
    plan = sc5.Plan(3, 64, 64, in_dtype=dtype, out_dtype=out_dtype)
    plan.run_batch(imgs)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    batch_out = [U.from_dev(im["out"], out_dtype)[:, :, :im["W"] - 4].copy() for im in imgs]
    for i, im in enumerate(imgs):
        assert U.sentinel_intact(U.from_dev(im["out"], out_dtype)[:, :, im["W"] - 4:], out_dtype), i
    # the same images through the graph-captured batch
    for im in imgs:
        im["out"].fill_(float("nan") if out_dtype == "f32" else (-1 if out_dtype != "fp8e4m3" else 0xFF))
    b = sc5.Batch(plan, imgs)
    b.launch()
    b.launch()  # replay twice: same result
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    info = b.info()
    assert info["tiles"] > 0 and info["ctas"] > 0
    for i, im in enumerate(imgs):
        H, W = im["H"], im["W"]
        g = U.from_dev(im["out"], out_dtype)[:, :, :W - 4]
        assert np.array_equal(g, batch_out[i])
        single, _ = _run(sc5, im["in"], 3, H, W, im["in_pitch"], im["k"], in_dtype=dtype, out_dtype=out_dtype,
                         in_scale=im["in_scale"], out_scale=im["out_scale"], tile_h=info["tile_h"],
                         tile_w=info["tile_w"])
        assert np.array_equal(single[:, :, :W - 4], batch_out[i]), i
        ref = U.oracle_valid(host[i], dtype, im["k"], im["in_scale"], W=W)
        got = U.decode(batch_out[i], out_dtype, im["out_scale"])
        if out_dtype == "f32":
            assert U.max_abs(got, ref) <= U.FP32_TOL, i
        else:
            assert np.all(np.abs(got - ref) <= U.stored_tolerance(ref, out_dtype, im["out_scale"], U.FP32_TOL)), i
    b.close()
    plan.close()


# ------------------------------------------------------------------ errors and probes


def test_invalid_arguments(sc5):
    import torch
    A = torch.zeros((3, 64, 68), dtype=torch.float32, device="cuda")
    out = torch.zeros((3, 60, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(sc5.Sepconv5Error) as e:
        sc5.Plan(3, 4, 64)
    assert e.value.status == sc5.EINVAL
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, in_pitch=66)  # 264 bytes: not a multiple of 16
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, in_dtype="bf16", out_dtype="f16")  # pair not built
    plan = sc5.Plan(3, 64, 64, 68, 64)
    with pytest.raises(sc5.Sepconv5Error):
        plan.run(A.data_ptr() + 4, out, [0, 0, 1, 0, 0])  # misaligned input
    with pytest.raises(sc5.Sepconv5Error):
        plan.run(A, A, [0, 0, 1, 0, 0])  # overlap
    with pytest.raises(sc5.Sepconv5Error):
        plan.run(A, out, [0, 0, float("nan"), 0, 0])
    with pytest.raises(sc5.Sepconv5Error):
        plan.run(A, out, [0, 0, 1, 0, 0], in_scale=0.0)
    plan.close()


def test_empty_probe_and_launch_counter(sc5):
    import torch
    n0 = sc5.launch_count()
    sc5.empty_launches(10)
    torch.cuda.synchronize()
    assert sc5.launch_count() - n0 == 10
