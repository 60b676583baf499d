"""The 256-image batch at full size (H and W log-uniform in [64, 4096],
about 241 Mpix x 3 planes), in the launch configuration the benchmark times:
autotuned shape, one persistent launch replayed from a CUDA graph.  Sampled
pixels of every image are checked against the FP64 oracle one by one (a 5x5
window per pixel), in FP32 and in every stored format (fp8 with its per-image
scale 448/max)."""
import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16", "fp8e4m3"])
def test_full_batch_sampled(dtype):
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    shapes = synth.batch_shapes(3, 256)
    sc5.autotune(1, [(dtype, dtype)])
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16,
           "fp8e4m3": torch.float8_e4m3fn}[dtype]
    es = sc5.DTYPE_BYTES[dtype]
    imgs = []
    for i, (h, w) in enumerate(shapes):
        x = torch.from_numpy(synth.image(3000 + i, h, w)).cuda()
        s = 448.0 / float(x.abs().max()) if dtype == "fp8e4m3" else 1.0
        pitch = -(-w * es // 16) * 16 // es
        A = torch.zeros((3, h, pitch), dtype=tdt, device="cuda")
        A[:, :, :w] = (x * s).to(tdt)
        op = -(-(w - 4) // 4) * 4
        out = torch.zeros((3, h - 4, op), dtype=tdt, device="cuda")
        imgs.append({"in": A, "out": out, "H": h, "W": w, "in_pitch": pitch, "out_pitch": op,
                     "k": synth.kernel_normalised(3000 + i), "in_scale": s, "out_scale": s})
    plan = sc5.Plan(3, 64, 64, in_dtype=dtype)
    b = sc5.Batch(plan, imgs)
    b.launch()
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    g = synth.rng(17)
    idx = torch.arange(5, device="cuda")
    for im in imgs:
        h, w, m = im["H"], im["W"], 64
        p, y, x = (torch.from_numpy(g.integers(0, n, m)).cuda() for n in (3, h - 4, w - 4))
        # always include the four corners of plane 0
        p[:4] = 0
        y[:4] = torch.tensor([0, 0, h - 5, h - 5], device="cuda")
        x[:4] = torch.tensor([0, w - 5, 0, w - 5], device="cuda")
        s = im["in_scale"]
        win = im["in"].float()[p[:, None, None], (y[:, None] + idx)[:, :, None], (x[:, None] + idx)[:, None, :]] / s
        ref = oracle.direct(win.double().cpu().numpy(), np.asarray(im["k"], np.float64))[:, 0, 0]
        got = (im["out"][p, y, x].float() / s).double().cpu().numpy()
        if dtype == "f32":
            assert U.max_abs(got, ref) <= U.FP32_TOL
        else:
            assert np.all(np.abs(got - ref) <= U.stored_tolerance(ref, dtype, s, U.FP32_TOL))
        assert not torch.isnan(im["out"][:, :, :w - 4].float()).any()
    b.close()
    plan.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_batch_ctas_timed_on_create(dtype):
    """ctas_per_sm = -1: the batch times every feasible CTA count on itself at
    creation; the outputs do not depend on the count (bitwise equal to an
    explicit one CTA per SM) and the grid is a whole number of CTAs per SM."""
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    shapes = synth.batch_shapes(5, 40)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[dtype]
    es = sc5.DTYPE_BYTES[dtype]
    runs = []
    for ctas in (1, -1):
        imgs = []
        for i, (h, w) in enumerate(shapes):
            x = torch.from_numpy(synth.image(5000 + i, h, w)).cuda()
            pitch = -(-w * es // 16) * 16 // es
            A = torch.zeros((3, h, pitch), dtype=tdt, device="cuda")
            A[:, :, :w] = x.to(tdt)
            op = -(-(w - 4) // 4) * 4
            imgs.append({"in": A, "out": torch.zeros((3, h - 4, op), dtype=tdt, device="cuda"), "H": h, "W": w,
                         "in_pitch": pitch, "out_pitch": op, "k": synth.kernel_normalised(5000 + i)})
        plan = sc5.Plan(3, 64, 64, in_dtype=dtype, ctas_per_sm=ctas)
        b = sc5.Batch(plan, imgs)
        b.launch()
        torch.cuda.synchronize()
        assert sc5.device_status() == 0
        info = b.info()
        n_sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert info["ctas"] % n_sms == 0 or info["ctas"] == info["tiles"]
        runs.append([im["out"].clone() for im in imgs])
        b.close()
        plan.close()
    for a, c in zip(*runs):
        assert torch.equal(a, c)
