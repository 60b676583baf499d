"""The allocation-free two-pass entry point (sepconv5_two_pass_noalloc).

It serves callers that may not allocate device memory (a framework's caching
allocator owns the GPU memory, a latency-bound loop cannot absorb the
synchronisation of cudaFree, or a host application forbids allocation calls):
its FP32 intermediate sits in a fixed 16 MiB array inside the library instead
of a plan's workspace.  This test calls it through the C ABI several times in a row,
largest image first, on different images, kernels and storage formats, and
checks each output against the regular two-pass plan (sepconv5_plan +
sepconv5_run): the kernels are the same, so the bits match, which is within
the FP32 bound the other tests use (max-abs 2e-4).
It also checks that a repeated call leaves the device's free memory
unchanged and that an image too large for the array is refused.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1711_09791_gb300 import synth
from tests import _util as U

pytestmark = pytest.mark.gpu

MAX_T_FLOATS = 4194304  # SC5_NOALLOC_MAX_T_FLOATS in include/sepconv5.h


@pytest.fixture(scope="module")
def lib():
    from paper_1711_09791_gb300 import sepconv5
    L = sepconv5.load()
    f = L.sepconv5_two_pass_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                  ctypes.POINTER(ctypes.c_float), ctypes.c_float, ctypes.c_float, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return L


DT = {"f32": 0, "bf16": 1, "f16": 2, "fp8e4m3": 3}


def _noalloc(lib, A, out, P, H, W, in_pitch, out_pitch, k, stream, in_dtype="f32", out_dtype="f32",
             in_scale=1.0, out_scale=1.0):
    taps = (ctypes.c_float * 5)(*[float(v) for v in k])
    return lib.sepconv5_two_pass_noalloc(A.data_ptr(), out.data_ptr(), P, H, W, in_pitch, out_pitch, DT[in_dtype],
                                         DT[out_dtype], taps, in_scale, out_scale, stream)


# Calls in a row, largest first: a later, smaller call with another row pitch
# and other taps reads back only what it wrote itself, so stale values the
# earlier calls left in the shared array must not reach its output.
CASES = [(302, 1152, 1152, "f32", "f32"), (301, 211, 517, "f32", "f32"), (303, 640, 480, "bf16", "bf16"),
         (304, 333, 777, "fp8e4m3", "f32")]


def test_noalloc_matches_two_pass_plan_on_calls_in_a_row(lib):
    import torch
    from paper_1711_09791_gb300 import sepconv5

    stream = torch.cuda.current_stream().cuda_stream
    for seed, H, W, dt, odt in CASES:
        P = 3
        assert P * H * U.round_up(W - 4, 4) <= MAX_T_FLOATS
        in_pitch = U.pitch_for(W, dt)
        out_pitch = U.pitch_for(W - 4, odt)
        x = synth.image(seed, H, W)
        s = synth.fp8_scale(x) if dt == "fp8e4m3" else 1.0
        codes = synth.to_storage(x, dt, s)
        padded = np.zeros((P, H, in_pitch), codes.dtype)
        padded[:, :, :W] = codes
        A = U.to_dev(padded)
        k = synth.kernel_normalised(seed)
        os_ = s if odt == "fp8e4m3" else 1.0
        want = U.empty_dev((P, H - 4, out_pitch), odt)
        plan = sepconv5.Plan(P, H, W, in_pitch, out_pitch, dt, odt, algo="two_pass")
        plan.run(A, want, k, s, os_, stream=stream)
        plan.close()
        got = U.empty_dev((P, H - 4, out_pitch), odt)
        st = _noalloc(lib, A, got, P, H, W, in_pitch, out_pitch, k, stream, dt, odt, s, os_)
        assert st == 0, lib.sepconv5_last_error().decode()
        torch.cuda.synchronize()
        w = U.from_dev(want, odt)
        g = U.from_dev(got, odt)
        assert np.array_equal(g[:, :, :W - 4], w[:, :, :W - 4]), (H, W, dt, odt)
        assert U.sentinel_intact(g[:, :, W - 4:], odt)
        # and within the bound of the other tests against the regular plan's values
        gv, wv = U.decode(g[:, :, :W - 4], odt, os_), U.decode(w[:, :, :W - 4], odt, os_)
        assert U.is_finite_all(gv)
        assert U.max_abs(gv, wv) <= U.FP32_TOL


def test_noalloc_repeated_call_allocates_nothing(lib):
    import torch

    stream = torch.cuda.current_stream().cuda_stream
    P, H, W = 3, 300, 400
    A = U.to_dev(synth.image(7, H, W))
    out = U.empty_dev((P, H - 4, W - 4), "f32")
    k = synth.kernel_binomial()
    assert _noalloc(lib, A, out, P, H, W, W, W - 4, k, stream) == 0  # first call: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(lib, A, out, P, H, W, W, W - 4, k, stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_images_beyond_the_limit(lib):
    import torch

    P, H, W = 3, 1200, 1200  # 3 * 1200 * 1196 floats > the 16 MiB array
    A = torch.zeros((P, H, W), dtype=torch.float32, device="cuda")
    out = torch.zeros((P, H - 4, W - 4), dtype=torch.float32, device="cuda")
    st = _noalloc(lib, A, out, P, H, W, W, W - 4, [0, 0, 1, 0, 0], None)
    assert st == 1  # SC5_EINVAL
    assert b"too large" in lib.sepconv5_last_error()
