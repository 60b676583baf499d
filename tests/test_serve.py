"""Serving runtime (serve_create / serve_submit / serve_poll / serve_destroy).

The requests are host images of several sizes, each with its own taps.  The
checks: every result equals, bit for bit, the same image convolved alone
through sepconv5_run (the fused arithmetic of a tile does not depend on what
else shares its launch), and lies within the stored-format bound of the FP64
oracle; requests that arrive while others run are merged into shared
launches; the HBM budget bounds what is resident; unknown tickets, bad
shapes and oversized requests are refused.
"""
import threading

import numpy as np
import pytest

from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu

SIZES = [(5, 5), (64, 64), (131, 301), (480, 640), (1080, 1920), (67, 1030)]


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
    dst = torch.full((3, H - 4, op), -1 if dtype != "f32" else float("nan"), dtype=tdt).pin_memory()
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


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
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
        assert (torch.isnan(pad).all() if dtype == "f32" else (pad == -1).all()), "row padding written"
        got = U.decode(U.from_dev(req["out"], dtype)[:, :, :W - 4], dtype)
        ref = U.oracle_valid(padded, dtype, req["k"], W=W)
        if dtype == "f32":
            assert U.max_abs(got, ref) <= U.FP32_TOL
        else:
            assert np.all(np.abs(got - ref) <= U.stored_tolerance(ref, dtype, 1.0, U.FP32_TOL))


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
    with pytest.raises(sc5.Sepconv5Error) as e:
        srv.poll(123456, 0)
    assert e.value.status == sc5.ENOTFOUND
    srv.close()
