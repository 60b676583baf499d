"""Degenerate inputs through the C ABI: empty batches are refused, a server that
never receives a request starts and stops cleanly, all-zero taps give exact
zeros, and the smallest image gives its single output in every form."""
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


def test_empty_batch_refused(sc5):
    plan = sc5.Plan(3, 64, 64)
    with pytest.raises(sc5.Sepconv5Error) as e:
        plan.run_batch([])
    assert e.value.status == sc5.EINVAL
    with pytest.raises(sc5.Sepconv5Error) as e:
        sc5.Batch(plan, [])
    assert e.value.status == sc5.EINVAL
    plan.close()


def test_idle_server(sc5):
    srv = sc5.Server(hbm_budget_bytes=1 << 24, dtype="bf16")
    st = srv.stats()
    srv.close()
    assert st["submitted"] == st["completed"] == st["launches"] == 0
    assert st["run_us_p99"] == 0 and st["queue_us_p50"] == 0


@pytest.mark.parametrize("algo", ["fused", "two_pass", "direct"])
def test_zero_taps_give_exact_zeros(sc5, algo):
    import torch
    H, W = 70, 131
    pitch = U.pitch_for(W, "f32")
    A = U.to_dev(synth.image(3, H, W, pitch=pitch, pad_value=0.0))
    op = U.pitch_for(W - 4, "f32")
    out = U.empty_dev((3, H - 4, op), "f32")
    plan = sc5.Plan(3, H, W, pitch, op, algo=algo)
    plan.run(A, out, [0.0] * 5)
    torch.cuda.synchronize()
    plan.close()
    got = U.from_dev(out, "f32")
    assert np.all(got[:, :, :W - 4] == 0.0) and not np.any(np.signbit(got[:, :, :W - 4]))


def test_smallest_image_every_form(sc5):
    """A 5 x 5 image has one VALID output per plane: Eq. 1 at its centre."""
    import torch
    A = synth.image(9, 5, 5, pitch=8)
    k = synth.kernel_normalised(9)
    ref = oracle.direct(A[:, :, :5].astype(np.float64), k)[:, 0, 0]
    A_dev = U.to_dev(A)
    for algo in ("fused", "two_pass", "direct", "reduce"):
        out = U.empty_dev((3, 1, 4), "f32")
        plan = sc5.Plan(3, 5, 5, 8, 4, algo=algo)
        plan.run(A_dev, out, k)
        torch.cuda.synchronize()
        plan.close()
        got = U.from_dev(out, "f32")
        assert np.max(np.abs(got[:, 0, 0] - ref)) <= U.FP32_TOL, algo
        assert U.sentinel_intact(got[:, :, 1:], "f32"), algo
    assert sc5.device_status() == 0
