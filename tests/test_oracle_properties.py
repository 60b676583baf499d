"""Randomised pins of the FP64 oracle (hypothesis): over random shapes,
values and taps (not normalised, not symmetric, negative allowed) each oracle
routine matches an independent library computation of its definition --
scipy's 2-D correlation in 'valid' mode for Eq. 1 with any odd width and any
K, the same kept at every second row and column for the REDUCE step, numpy's
1-D correlation for each pass -- and the FP32 point evaluator matches the
full evaluation at random pixels.  Complements the fixed-case pins in
test_oracle_pins.py."""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

SETTINGS = settings(max_examples=40, deadline=None, derandomize=True)


@st.composite
def image_and_taps(draw, n_choices=(5,), min_extra=0):
    n = draw(st.sampled_from(n_choices))
    P = draw(st.integers(1, 3))
    H = draw(st.integers(n + min_extra, n + 19))
    W = draw(st.integers(n + min_extra, n + 19))
    seed = draw(st.integers(0, 2**31 - 1))
    g = np.random.default_rng(seed)
    A = g.uniform(-300.0, 300.0, (P, H, W))
    k = g.uniform(-3.0, 3.0, n)
    K = g.uniform(-3.0, 3.0, (n, n))
    return A, k, K


def _tol(A, K):
    # every term is bounded by max|A| * max|K|; n*n terms summed in FP64
    return 1e-13 * np.abs(A).max() * np.abs(K).sum() + 1e-300


@SETTINGS
@given(image_and_taps())
def test_direct_is_scipy_valid_correlation(case):
    from scipy.signal import correlate2d
    A, k, _ = case
    K = np.outer(k, k)
    B = oracle.direct(A, k)
    ref = np.stack([correlate2d(A[p], K, mode="valid") for p in range(A.shape[0])])
    assert B.shape == ref.shape
    assert np.max(np.abs(B - ref)) <= _tol(A, K)


@SETTINGS
@given(image_and_taps(n_choices=(3, 5, 7, 9)))
def test_direct_Kn_any_matrix_is_scipy_valid_correlation(case):
    from scipy.signal import correlate2d
    A, _, K = case
    B = oracle.direct_Kn(A, K)
    ref = np.stack([correlate2d(A[p], K, mode="valid") for p in range(A.shape[0])])
    assert B.shape == ref.shape
    assert np.max(np.abs(B - ref)) <= _tol(A, K)


@SETTINGS
@given(image_and_taps())
def test_general_K_of_rank_one_is_the_separable_form(case):
    A, k, _ = case
    B1 = oracle.direct(A, k)
    B2 = oracle.direct_K(A, np.outer(k, k))
    B3 = oracle.vpass(oracle.hpass(A, k), k)
    tol = _tol(A, np.outer(k, k))
    assert np.max(np.abs(B1 - B2)) <= tol
    assert np.max(np.abs(B1 - B3)) <= tol


@SETTINGS
@given(image_and_taps())
def test_passes_are_numpy_1d_correlations(case):
    A, k, _ = case
    T = oracle.hpass(A, k)
    P, H, W = A.shape
    ref_T = np.array([[np.correlate(A[p, y], k, mode="valid") for y in range(H)] for p in range(P)])
    assert np.max(np.abs(T - ref_T)) <= 1e-13 * np.abs(A).max() * np.abs(k).sum()
    B = oracle.vpass(T, k)
    ref_B = np.array([np.stack([np.correlate(T[p, :, x], k, mode="valid") for x in range(W - 4)], axis=1)
                      for p in range(P)])
    assert np.max(np.abs(B - ref_B)) <= 1e-13 * np.abs(T).max() * np.abs(k).sum()


@SETTINGS
@given(image_and_taps())
def test_reduce_is_the_valid_correlation_at_even_positions(case):
    from scipy.signal import correlate2d
    A, k, _ = case
    K = np.outer(k, k)
    R = oracle.reduce2(A, k)
    full = np.stack([correlate2d(A[p], K, mode="valid") for p in range(A.shape[0])])
    ref = full[:, ::2, ::2]
    assert R.shape == ref.shape == (A.shape[0], -(-(A.shape[1] - 4) // 2), -(-(A.shape[2] - 4) // 2))
    assert np.max(np.abs(R - ref)) <= _tol(A, K)


@SETTINGS
@given(image_and_taps(), st.integers(0, 2**31 - 1))
def test_points_match_the_full_evaluation(case, seed):
    A, k, _ = case
    A32 = np.ascontiguousarray(A.astype(np.float32))
    k32 = k.astype(np.float32)
    full = oracle.direct(A32.astype(np.float64), k32.astype(np.float64))
    g = np.random.default_rng(seed)
    P, Hv, Wv = full.shape
    pts = np.stack([g.integers(0, P, 16), g.integers(0, Hv, 16), g.integers(0, Wv, 16)], axis=1)
    got = oracle.points_f32(A32, k32, pts)
    want = full[pts[:, 0], pts[:, 1], pts[:, 2]]
    assert np.max(np.abs(got - want)) <= _tol(A32.astype(np.float64), np.outer(k32, k32))
