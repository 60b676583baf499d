"""The timed CPU baseline of the benchmark (cpu_baseline/: FP32 two-pass with
OpenMP, Listing 1's loop structure with the horizontal pass over all rows)
against the FP64 oracle: within the FP32 bound on ragged shapes, and exactly
equal on integer images with the binomial kernel (every sum is exact in FP32)."""
import numpy as np
import pytest

import cpu_baseline
import oracle
from paper_1711_09791_gb300 import synth

FP32_TOL = 2e-4


@pytest.mark.parametrize("H,W", [(5, 5), (6, 7), (37, 131), (130, 133), (300, 517)])
def test_two_pass_within_fp32_bound(H, W):
    A = synth.image(H * 7 + W, H, W)
    k = synth.kernel_normalised(H + W)
    got = cpu_baseline.two_pass(A, k)
    ref = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    assert got.shape == ref.shape and np.max(np.abs(got - ref)) <= FP32_TOL


def test_two_pass_exact_on_integers():
    A = synth.integer_image(9, 61, 97)
    k = synth.kernel_binomial()
    got = cpu_baseline.two_pass(A, k)
    ref = oracle.direct(A.astype(np.float64), k.astype(np.float64))
    assert np.array_equal(got.astype(np.float64), ref)


def test_threads_and_model():
    assert cpu_baseline.threads() >= 1 and cpu_baseline.cpu_model()
