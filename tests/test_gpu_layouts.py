"""Plane layouts: the 3R x C agglomeration of Sec. 6 (each row holds the rows
of all 3 planes side by side: pitch 3W, plane stride W) and mixed layouts
give, bit for bit, the stacked-plane results, which match the oracle."""
import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


def to_3rxc(A):
    P, H, W = A.shape
    return np.ascontiguousarray(np.transpose(A, (1, 0, 2)).reshape(H, P * W))


def from_3rxc(X, P):
    H, PW = X.shape
    return np.ascontiguousarray(np.transpose(X.reshape(H, P, PW // P), (1, 0, 2)))


@pytest.mark.parametrize("algo", ["fused", "two_pass", "direct"])
@pytest.mark.parametrize("border", ["valid", "keep"])
def test_3rxc_equals_stacked(algo, border):
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    P, H, W = 3, 101, 260
    A = synth.image(44, H, W)
    k = synth.kernel_normalised(44)
    wout, hout = (W, H) if border == "keep" else (W - 4, H - 4)
    # stacked reference run
    ref_out = torch.full((P, hout, wout), float("nan"), device="cuda")
    plan = sc5.Plan(P, H, W, W, wout, border=border, algo=algo)
    plan.run(U.to_dev(A), ref_out, k)
    # the same image row-interleaved, output row-interleaved too
    X = U.to_dev(to_3rxc(A))
    Y = torch.full((hout, P * wout), float("nan"), device="cuda")
    plan2 = sc5.Plan(P, H, W, P * W, P * wout, border=border, algo=algo, in_plane_stride=W, out_plane_stride=wout)
    plan2.run(X, Y, k)
    # row-interleaved input, stacked output
    Z = torch.full((P, hout, wout), float("nan"), device="cuda")
    plan3 = sc5.Plan(P, H, W, P * W, wout, border=border, algo=algo, in_plane_stride=W)
    plan3.run(X, Z, k)
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    ref = ref_out.cpu().numpy()
    assert np.array_equal(from_3rxc(Y.cpu().numpy(), P), ref)
    assert np.array_equal(Z.cpu().numpy(), ref)
    want = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    got = ref[:, 2:-2, 2:-2] if border == "keep" else ref
    assert U.max_abs(got, want) <= U.FP32_TOL
    for p_ in (plan, plan2, plan3):
        p_.close()


def test_overlapping_plane_strides_refused():
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, 64, 60, in_plane_stride=32)  # planes overlap within rows
    with pytest.raises(sc5.Sepconv5Error):
        sc5.Plan(3, 64, 64, 128, 60, in_plane_stride=66)  # 264 bytes: not a multiple of 16
