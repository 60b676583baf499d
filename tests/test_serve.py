"""Serving runtime (serve_create / serve_submit / serve_poll / serve_destroy).

The requests are host images of several sizes, each with its own taps.  The
checks: every result equals, bit for bit, the same image convolved alone
through sepconv5_run (the fused arithmetic of a tile does not depend on what
else shares its launch), and lies within the stored-format bound of the FP64
oracle; requests that arrive while others run are merged into shared
launches; the HBM budget bounds what is resident; unknown tickets, bad
shapes and oversized requests are refused.
"""
import json
import os
import threading

import numpy as np
import pytest

from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu

SIZES = [(5, 5), (64, 64), (131, 301), (480, 640), (1080, 1920), (67, 1030)]
# fill of the output rows' padding, which the server must leave as it was
PAD_FILL = {"f32": float("nan"), "bf16": -1, "f16": -1, "fp8e4m3": 0xFF}


@pytest.fixture(scope="module")
def sc5():
    import torch  # noqa: F401
    from paper_1711_09791_gb300 import sepconv5
    sepconv5.load()
    return sepconv5


def _request(i, H, W, dtype):
    import torch
    x = synth.image(5000 + i, H, W)
    scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
    codes = synth.to_storage(x, dtype, scale)
    pitch = U.pitch_for(W, dtype)
    padded = np.zeros((3, H, pitch), codes.dtype)
    padded[:, :, :W] = codes
    tdt = {"bf16": torch.int16, "f16": torch.int16, "fp8e4m3": torch.uint8, "f32": torch.float32}[dtype]
    src = torch.from_numpy(padded.view(np.int16) if padded.dtype == np.uint16 else padded).pin_memory()
    op = U.pitch_for(W - 4, dtype)
    dst = torch.full((3, H - 4, op), PAD_FILL[dtype], dtype=tdt).pin_memory()
    k = synth.kernel_normalised(5000 + i)
    return {"in": src, "out": dst, "H": H, "W": W, "in_pitch": pitch, "out_pitch": op, "k": k,
            "in_scale": scale, "out_scale": scale}, padded


def _solo(sc5, req, dtype):
    import torch
    A = req["in"].cuda()
    out = req["out"].clone().cuda()  # same padding contents as the served buffer
    plan = sc5.Plan(3, req["H"], req["W"], req["in_pitch"], req["out_pitch"], in_dtype=dtype)
    plan.run(A, out, req["k"], req["in_scale"], req["out_scale"])
    torch.cuda.synchronize()
    plan.close()
    return out.cpu()


@pytest.mark.parametrize("dtype", ["bf16", "f32", "f16", "fp8e4m3"])
def test_same_alone_and_in_the_mix(sc5, dtype):
    import torch
    reqs = [_request(i, H, W, dtype) for i, (H, W) in enumerate(SIZES * 4)]
    # a 5 ms batching window: requests submitted close together share launches
    srv = sc5.Server(hbm_budget_bytes=1 << 30, dtype=dtype, max_inflight=64, n_streams=2, batch_window_us=5000)
    # submit from two client threads at once so requests arrive while others run
    tickets = [None] * len(reqs)

    def client(idx):
        for i in idx:
            t = None
            while t is None:
                t = srv.submit(reqs[i][0])
            tickets[i] = t

    ths = [threading.Thread(target=client, args=(list(range(j, len(reqs), 2)),)) for j in range(2)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    lats = [srv.poll(t, -1) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(lat is not None and lat > 0 for lat in lats)
    assert stats["completed"] == len(reqs) and stats["submitted"] == len(reqs)
    assert stats["merged_max"] > 1, "no two requests ever shared a launch"
    assert stats["launches"] < len(reqs)
    for (req, padded) in reqs:
        solo = _solo(sc5, req, dtype)
        W = req["W"]
        assert torch.equal(solo[:, :, :W - 4], req["out"][:, :, :W - 4]), (req["H"], W)
        pad = req["out"][:, :, W - 4:]
        assert (torch.isnan(pad).all() if dtype == "f32" else (pad == PAD_FILL[dtype]).all()), "row padding written"
        # real units: codes divided by the per-image scale (1 except for fp8)
        got = U.decode(U.from_dev(req["out"], dtype)[:, :, :W - 4], dtype, req["out_scale"])
        ref = U.oracle_valid(padded, dtype, req["k"], req["in_scale"], W=W)
        if dtype == "f32":
            assert U.max_abs(got, ref) <= U.FP32_TOL
        else:
            assert np.all(np.abs(got - ref) <= U.stored_tolerance(ref, dtype, req["out_scale"], U.FP32_TOL))


# The request sizes of the serving stream (640x480, 1920x1080, 4096x4096), two
# of the largest among them: the heaviest merged launch the server makes.
C5_MIX = [(4096, 4096), (480, 640), (1080, 1920), (480, 640), (4096, 4096), (1080, 1920), (480, 640),
          (1080, 1920)]


def test_c5_mix_with_4096_requests(sc5):
    """BF16 requests of the serving stream's three sizes, two of them
    4096 x 4096 (100.7 MB in and out each), submitted together under a 16 GB
    budget with merged launches of up to 8 requests: every result equals its
    solo sepconv5_run bit for bit and lies within the stored-format bound of
    the FP64 oracle on its decoded input.  One 4096^2 image is also served as
    FP32; with SC5_REPORT_DIR set, the measured errors of the BF16 and FP32
    results against the oracle on the FP32 image are written to
    error_serve.json."""
    import torch
    reqs = [_request(100 + i, H, W, "bf16") for i, (H, W) in enumerate(C5_MIX)]
    srv = sc5.Server(hbm_budget_bytes=16 << 30, dtype="bf16", max_inflight=64, n_streams=2, max_merge=8,
                     batch_window_us=20000)
    tickets = [srv.submit(r) for r, _ in reqs]
    assert all(t is not None for t in tickets)
    lats = [srv.poll(t, -1) for t in tickets]
    stats = srv.stats()
    srv.close()
    assert all(lat is not None and lat > 0 for lat in lats)
    assert stats["completed"] == len(reqs) and stats["merged_max"] > 1 and stats["launches"] < len(reqs)
    assert stats["resident_peak_bytes"] <= 16 << 30
    report = {}
    for i, (req, padded) in enumerate(reqs):
        H, W = req["H"], req["W"]
        solo = _solo(sc5, req, "bf16")
        assert torch.equal(solo[:, :, :W - 4], req["out"][:, :, :W - 4]), (H, W)
        assert (req["out"][:, :, W - 4:] == -1).all(), "row padding written"
        got = U.decode(U.from_dev(req["out"], "bf16")[:, :, :W - 4], "bf16")
        ref = U.oracle_valid(padded, "bf16", req["k"], W=W)
        assert np.all(np.abs(got - ref) <= U.stored_tolerance(ref, "bf16", 1.0, U.FP32_TOL)), (H, W)
        if H == 4096 and not report:
            x = synth.image(5000 + 100 + i, H, W)
            ref_x = oracle_direct(x, req["k"])
            report["bf16_served"] = _errors(got, ref_x, ref)
            # the same image and taps served as FP32, one launch per request
            f32_req, f32_padded = _request(100 + i, H, W, "f32")
            srv32 = sc5.Server(hbm_budget_bytes=16 << 30, dtype="f32", merge=False)
            t = srv32.submit(f32_req)
            assert srv32.poll(t, -1) is not None
            srv32.close()
            got32 = U.from_dev(f32_req["out"], "f32")[:, :, :W - 4].astype(np.float64)
            assert U.max_abs(got32, ref_x) <= U.FP32_TOL
            report["f32_served"] = _errors(got32, ref_x, ref_x)
    d = os.environ.get("SC5_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "error_serve.json"), "w") as f:
            json.dump({"request": "3 x 4096 x 4096, pixels uniform [0,255), normalised k, served through "
                                  "serve_submit / serve_poll", **report}, f, indent=1)


def oracle_direct(x, k):
    import oracle
    return oracle.direct(x.astype(np.float64), np.asarray(k, np.float64))


def _errors(got, ref_fp32_input, ref_stored_input):
    def stats(ref):
        d = np.abs(got - ref)
        big = np.abs(ref) > 1.0
        return {"max_abs": float(d.max()), "max_abs_over_255": float(d.max()) / 255.0,
                "max_rel_where_abs_ref_gt_1": float((d[big] / np.abs(ref[big])).max())}
    return {"vs_oracle_on_fp32_input": stats(ref_fp32_input), "vs_oracle_on_stored_input": stats(ref_stored_input)}


def test_one_launch_per_request_mode(sc5):
    reqs = [_request(i, H, W, "bf16") for i, (H, W) in enumerate(SIZES)]
    srv = sc5.Server(hbm_budget_bytes=1 << 30, dtype="bf16", merge=False)
    tickets = [srv.submit(r) for r, _ in reqs]
    assert all(srv.poll(t, -1) is not None for t in tickets)
    stats = srv.stats()
    srv.close()
    assert stats["merged_max"] == 1 and stats["launches"] == len(reqs)


def test_budget_bounds_resident_bytes(sc5):
    """A budget of about two requests: everything still completes, in waves,
    and the resident high-water mark never exceeds the budget."""
    reqs = [_request(i, 1080, 1920, "bf16") for i in range(8)]
    per = 3 * 1080 * reqs[0][0]["in_pitch"] * 2 + 3 * 1076 * reqs[0][0]["out_pitch"] * 2
    budget = int(2.2 * per)
    srv = sc5.Server(hbm_budget_bytes=budget, dtype="bf16")
    tickets = [srv.submit(r) for r, _ in reqs]
    assert all(t is not None for t in tickets)
    assert all(srv.poll(t, -1) is not None for t in tickets)
    stats = srv.stats()
    srv.close()
    assert stats["resident_peak_bytes"] <= budget
    assert stats["completed"] == 8
    # phase times: ordered percentiles, and the requests beyond the budget waited
    # in the queue for at least part of an earlier request's run
    for ph in ("queue", "stage", "run"):
        assert 0 <= stats[f"{ph}_us_p50"] <= stats[f"{ph}_us_p99"]
    assert stats["run_us_p50"] > 0
    assert stats["queue_us_p99"] >= 0.5 * stats["run_us_p50"], stats


def test_refusals(sc5):
    srv = sc5.Server(hbm_budget_bytes=1 << 24, dtype="bf16")
    big, _ = _request(0, 1080, 1920, "bf16")  # ~25 MB > 16 MiB budget
    with pytest.raises(sc5.Sepconv5Error) as e:
        srv.submit(big)
    assert e.value.status == sc5.EINVAL
    bad, _ = _request(1, 64, 64, "bf16")
    bad["in_pitch"] = 66  # 132 bytes: not a multiple of 16
    with pytest.raises(sc5.Sepconv5Error):
        srv.submit(bad)
    for key, value in (("k", [0.2, float("nan"), 0.2, 0.2, 0.2]), ("in_scale", float("inf")), ("out_scale", 0.0)):
        r, _ = _request(2, 64, 64, "bf16")
        r[key] = value
        with pytest.raises(sc5.Sepconv5Error) as e:
            srv.submit(r)
        assert e.value.status == sc5.EINVAL, key
    # pageable host buffers are refused: their copies would block the scheduler
    r, _ = _request(3, 64, 64, "bf16")
    for key in ("in", "out"):
        q = dict(r)
        q[key] = r[key].clone()  # a plain (pageable) CPU tensor
        assert not q[key].is_pinned()
        with pytest.raises(sc5.Sepconv5Error) as e:
            srv.submit(q)
        assert e.value.status == sc5.EINVAL and "page-locked" in str(e.value), key
    with pytest.raises(sc5.Sepconv5Error) as e:
        srv.poll(123456, 0)
    assert e.value.status == sc5.ENOTFOUND
    srv.close()
