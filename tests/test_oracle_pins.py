"""Pins for the FP64 oracle: checks against facts fixed by the paper and by the
mathematics, never against a retyped copy of the oracle's own loops.

What each pin fixes:

* library routine   -- Eq. 1 on the VALID region is exactly scipy's 2-D
                       correlation in 'valid' mode; each 1-D pass is numpy's
                       1-D correlation in 'valid' mode along its axis.
* shifted deltas    -- k = e_t moves the image by t-2 along the pass axis:
                       orientation of k (Eq. 2; Listing 1 puts k[0] on j-2).
* impulse response  -- correlating a unit impulse returns K rotated by 180
                       degrees: orientation of a general K (first index = rows).
* golden table      -- the binomial [1,4,6,4,1] impulse response (hand table).
* constant image    -- a kernel summing to 1 preserves a constant.
* ramp / cosine     -- closed forms that depend on the sign and order of the
                       taps for a non-symmetric k.
* linearity         -- linear in A, quadratic in k.
* exact integers    -- Python integer brute force on small images.
* transpose         -- K = k k^T is symmetric, so conv(A^T) = conv(A)^T.
* separability      -- Eq. 1 with K = k k^T equals the horizontal pass
                       followed by the vertical pass (Sec. 1, Sec. 5.1).
* decoders          -- every bf16 / fp16 / fp8-e4m3 code against torch's and
                       numpy's own conversions, plus spot values of the formats.
* REDUCE step       -- scipy's 2-D correlation kept at even rows and columns;
                       the centre-tap delta picks A[2y+2][2x+2]; a ramp maps to
                       the ramp at the even centres; output sizes for odd and
                       even H-4, W-4.

A last test plants plausible mistakes in copies of the C source and checks
that at least one pin fails for each.
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SHAPES = [(5, 5), (6, 7), (8, 8), (9, 13), (17, 33)]


def _rand_image(seed, H, W, P=3):
    return synth.image(seed, H, W, planes=P).astype(np.float64)


def _nonsym_k(seed=11):
    k = synth.kernel_normalised(seed).astype(np.float64)
    assert not np.allclose(k, k[::-1])
    return k


# ---------------------------------------------------------------- the pins
def pin_scipy_correlate2d():
    from scipy.signal import correlate2d
    g = synth.rng(5)
    for (H, W) in SHAPES:
        A = _rand_image(H * 100 + W, H, W, P=2)
        K = g.uniform(-1, 1, size=(5, 5))
        B = oracle.direct_K(A, K)
        for p in range(2):
            ref = correlate2d(A[p], K, mode="valid")
            assert B[p].shape == ref.shape
            assert np.max(np.abs(B[p] - ref)) <= 1e-12 * 255 * 25


def pin_numpy_correlate_1d():
    k = _nonsym_k()
    for (H, W) in SHAPES:
        A = _rand_image(H + 7 * W, H, W, P=2)
        T = oracle.hpass(A, k)
        for p in range(2):
            for y in range(H):
                ref = np.correlate(A[p, y], k, mode="valid")
                assert np.max(np.abs(T[p, y] - ref)) <= 1e-12 * 255
        B = oracle.vpass(T, k)
        for p in range(2):
            for x in range(W - 4):
                ref = np.correlate(T[p, :, x], k, mode="valid")
                assert np.max(np.abs(B[p, :, x] - ref)) <= 1e-12 * 255


def pin_shifted_deltas():
    A = _rand_image(3, 9, 13)
    for t in range(5):
        e = np.zeros(5)
        e[t] = 1.0
        B = oracle.direct(A, e)
        # output (y, x) is centred on input (y+2, x+2); tap t sits at offset t-2
        assert np.array_equal(B, A[:, t:t + 5, t:t + 9])
        T = oracle.hpass(A, e)
        assert np.array_equal(T, A[:, :, t:t + 9])
        V = oracle.vpass(A, e)
        assert np.array_equal(V, A[:, t:t + 5, :])


def pin_impulse_response_general_K():
    K = np.arange(25, dtype=np.float64).reshape(5, 5) + 1.0  # not symmetric
    A = np.zeros((1, 9, 9))
    A[0, 4, 4] = 1.0
    B = oracle.direct_K(A, K)[0]
    assert np.array_equal(B, K[::-1, ::-1])
    # off-centre impulse: only the outputs whose window covers it are non-zero
    A = np.zeros((1, 7, 11))
    A[0, 1, 6] = 1.0
    B = oracle.direct_K(A, K)[0]
    for y in range(3):
        for x in range(7):
            i, j = 1 - y, 6 - x
            want = K[i, j] if (0 <= i < 5 and 0 <= j < 5) else 0.0
            assert B[y, x] == want


def pin_golden_binomial_table():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "binomial5x5_impulse.txt"))
            if ln.strip() and not ln.startswith("#")]
    table = np.array(rows, dtype=np.float64)
    A = np.zeros((3, 9, 9))
    A[:, 4, 4] = 1.0
    B = oracle.direct(A, [1, 4, 6, 4, 1])
    for p in range(3):
        assert np.array_equal(B[p], table)
    assert np.array_equal(oracle.outer([1, 4, 6, 4, 1]), table)
    assert table.sum() == 256


def pin_constant_image():
    k = _nonsym_k(21)
    for c in (0.0, 1.0, 127.5, 254.75):
        A = np.full((3, 8, 12), c)
        B = oracle.direct(A, k)
        s = float(np.sum(k)) ** 2  # k sums to 1 only up to rounding
        assert np.max(np.abs(B - c * s)) <= 8 * np.finfo(float).eps * max(c, 1.0)
        V = oracle.vpass(oracle.hpass(A, k), k)
        assert np.max(np.abs(V - c * s)) <= 8 * np.finfo(float).eps * max(c, 1.0)


def pin_ramp_closed_form():
    # A = a*y + b*x + c (input coordinates).  With sum(k) = S and first moment
    # mu = sum_t (t-2) k[t], the VALID output centred on input (yc, xc) is
    # S^2 c + a S (S yc + mu) + b S (S xc + mu).
    k = _nonsym_k(31)
    S = float(k.sum())
    mu = float(sum((t - 2) * k[t] for t in range(5)))
    a, b, c = 1.75, -0.5, 3.0
    H, W = 10, 14
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    A = (a * yy + b * xx + c)[None]
    B = oracle.direct(A, k)[0]
    yv, xv = np.meshgrid(np.arange(H - 4) + 2, np.arange(W - 4) + 2, indexing="ij")
    want = S * S * c + a * S * (S * yv + mu) + b * S * (S * xv + mu)
    assert np.max(np.abs(B - want)) <= 1e-12 * 64


def pin_cosine_closed_form():
    # A[y][x] = cos(w x + phi) is an eigenfunction of the row correlation:
    # sum_t k[t] cos(w (x+t) + phi) = Re(H e^{i(w(x+2)+phi)}), H = sum_t k[t] e^{i w (t-2)};
    # the column pass then multiplies by sum(k).
    k = _nonsym_k(41)
    w, phi = 0.7, 0.3
    H, W = 7, 29
    x = np.arange(W)
    A = np.broadcast_to(np.cos(w * x + phi), (H, W))[None].copy()
    B = oracle.direct(A, k)[0]
    Hw = sum(k[t] * np.exp(1j * w * (t - 2)) for t in range(5))
    xv = np.arange(W - 4) + 2
    want = float(k.sum()) * np.real(Hw * np.exp(1j * (w * xv + phi)))
    assert np.max(np.abs(B - want[None, :])) <= 1e-13 * 8


def pin_linearity():
    k = _nonsym_k(51)
    A1, A2 = _rand_image(1, 11, 9), _rand_image(2, 11, 9)
    al, be = 0.37, -1.9
    lhs = oracle.direct(al * A1 + be * A2, k)
    rhs = al * oracle.direct(A1, k) + be * oracle.direct(A2, k)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * 255 * 4
    lam = 2.5
    assert np.max(np.abs(oracle.direct(A1, lam * k) - lam * lam * oracle.direct(A1, k))) <= 1e-11 * 255


def pin_exact_integer_brute_force():
    kint = [1, 4, 6, 4, 1]
    kint2 = [3, -1, 0, 7, 2]
    for (H, W) in [(5, 5), (6, 7), (9, 13)]:
        A = synth.integer_image(H * W, H, W, planes=2)
        for kv in (kint, kint2):
            B = oracle.direct(A.astype(np.float64), kv)
            Ai = A.astype(np.int64).tolist()
            for p in range(2):
                for y in range(H - 4):
                    for x in range(W - 4):
                        s = 0
                        for i in range(5):
                            for j in range(5):
                                s += int(Ai[p][y + i][x + j]) * kv[i] * kv[j]
                        assert B[p, y, x] == float(s)


def pin_transpose_equivariance():
    k = _nonsym_k(61)
    A = _rand_image(7, 9, 14)
    B = oracle.direct(A, k)
    Bt = oracle.direct(np.ascontiguousarray(np.transpose(A, (0, 2, 1))), k)
    assert np.max(np.abs(Bt - np.transpose(B, (0, 2, 1)))) <= 1e-12 * 255


def pin_separable_equals_direct():
    k = _nonsym_k(71)
    for (H, W) in SHAPES:
        A = _rand_image(H * 3 + W, H, W)
        d = oracle.direct(A, k)
        two = oracle.vpass(oracle.hpass(A, k), k)
        assert np.max(np.abs(d - two)) <= 1e-12 * 255
        assert np.max(np.abs(oracle.direct_K(A, oracle.outer(k)) - d)) == 0.0


def pin_points_f32():
    k = synth.kernel_normalised(81)
    A = synth.image(8, 12, 37, pitch=44)  # NaN in the 7 padding columns
    full = oracle.direct(A[:, :, :37].astype(np.float64), k.astype(np.float64))
    pts = [(p, y, x) for p in range(3) for y in range(8) for x in range(33)]
    got = oracle.points_f32((A, 37), k, pts)
    want = np.array([full[p, y, x] for (p, y, x) in pts])
    assert np.max(np.abs(got - want)) <= 1e-12 * 255


def pin_decoders():
    import torch
    codes16 = np.arange(65536, dtype=np.uint16)
    bf = oracle.decode(codes16, "bf16")
    ref_bf = torch.from_numpy(codes16.view(np.int16).copy()).view(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(bf), np.isnan(ref_bf))
    assert np.array_equal(bf[~np.isnan(bf)], ref_bf[~np.isnan(ref_bf)])
    hf = oracle.decode(codes16, "f16")
    ref_hf = codes16.view(np.float16).astype(np.float64)
    assert np.array_equal(np.isnan(hf), np.isnan(ref_hf))
    assert np.array_equal(hf[~np.isnan(hf)], ref_hf[~np.isnan(ref_hf)])
    codes8 = np.arange(256, dtype=np.uint8)
    e4 = oracle.decode(codes8, "fp8e4m3")
    ref_e4 = torch.from_numpy(codes8.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(e4), np.isnan(ref_e4))
    assert np.array_equal(e4[~np.isnan(e4)], ref_e4[~np.isnan(ref_e4)])
    # spot values of the E4M3 layout: 448 largest finite, 2^-9 smallest subnormal,
    # 2^-6 smallest normal, S.1111.111 NaN, 1.0 = 0.0111.000
    assert e4[0x7E] == 448.0 and e4[0x01] == 2.0 ** -9 and e4[0x08] == 2.0 ** -6
    assert math.isnan(e4[0x7F]) and math.isnan(e4[0xFF]) and e4[0x38] == 1.0
    assert e4[0xFE] == -448.0
    # the per-image scale divides
    assert oracle.decode(np.array([0x7E], np.uint8), "fp8e4m3", scale=448.0 / 255.0)[0] == pytest.approx(255.0, rel=1e-15)


def pin_keep_frame():
    A = _rand_image(9, 8, 10)
    B = oracle.direct(A, synth.kernel_binomial())
    F = oracle.keep_frame(A, B)
    assert F.shape == A.shape
    assert np.array_equal(F[:, :2], A[:, :2]) and np.array_equal(F[:, -2:], A[:, -2:])
    assert np.array_equal(F[:, :, :2], A[:, :, :2]) and np.array_equal(F[:, :, -2:], A[:, :, -2:])
    assert np.array_equal(F[:, 2:-2, 2:-2], B)


WIDTHS = [1, 3, 7, 9]


def pin_width_n_scipy_correlate2d():
    from scipy.signal import correlate2d
    g = synth.rng(91)
    for n in WIDTHS:
        for (H, W) in [(n, n), (n + 3, n + 8), (20, 31)]:
            A = _rand_image(H * 13 + W + n, H, W, P=2)
            K = g.uniform(-1, 1, size=(n, n))
            B = oracle.direct_Kn(A, K)
            for p in range(2):
                ref = correlate2d(A[p], K, mode="valid")
                assert B[p].shape == ref.shape
                assert np.max(np.abs(B[p] - ref)) <= 1e-12 * 255 * n * n


def pin_width_n_deltas_and_impulse():
    for n in WIDTHS:
        r = (n - 1) // 2
        A = _rand_image(n, n + 6, n + 9)
        for (i, j) in [(0, 0), (0, n - 1), (r, r), (n - 1, 0)]:
            D = np.zeros((n, n))
            D[i, j] = 1.0
            assert np.array_equal(oracle.direct_Kn(A, D), A[:, i:i + 7, j:j + 10])
        K = np.arange(n * n, dtype=np.float64).reshape(n, n) + 1.0
        imp = np.zeros((1, 2 * n - 1, 2 * n - 1))
        imp[0, n - 1, n - 1] = 1.0
        assert np.array_equal(oracle.direct_Kn(imp, K)[0], K[::-1, ::-1])


def pin_width_n_constant_and_integers():
    for n in WIDTHS:
        k = synth.rng(n).uniform(0, 1, n)
        k /= k.sum()
        c = 97.25
        B = oracle.direct_n(np.full((1, n + 4, n + 5), c), k)
        assert np.max(np.abs(B - c * k.sum() ** 2)) <= 16 * np.finfo(float).eps * c
        A = synth.integer_image(n * 5, n + 3, n + 4, planes=1)
        kint = list(range(1, n + 1))
        B = oracle.direct_n(A.astype(np.float64), kint)
        Ai = A.astype(np.int64).tolist()
        for y in range(4):
            for x in range(5):
                s = sum(Ai[0][y + i][x + j] * kint[i] * kint[j] for i in range(n) for j in range(n))
                assert B[0, y, x] == float(s)


def pin_width_5_agrees_with_direct():
    A = _rand_image(55, 12, 17)
    k = _nonsym_k(55)
    assert np.max(np.abs(oracle.direct_n(A, k) - oracle.direct(A, k))) <= 1e-12 * 255


def pin_reduce_scipy_subsampled():
    from scipy.signal import correlate2d
    for (H, W) in [(5, 5), (6, 7), (9, 13), (18, 21), (17, 32)]:
        A = _rand_image(H * 7 + W, H, W, P=2)
        k = _nonsym_k(H + W)
        B = oracle.reduce2(A, k)
        for p in range(2):
            ref = correlate2d(A[p], np.outer(k, k), mode="valid")[::2, ::2]
            assert B[p].shape == ref.shape
            assert np.max(np.abs(B[p] - ref)) <= 1e-12 * 255


def pin_reduce_delta_and_ramp():
    A = _rand_image(77, 15, 20)
    e2 = [0.0, 0.0, 1.0, 0.0, 0.0]
    assert np.array_equal(oracle.reduce2(A, e2), A[:, 2:13:2, 2:18:2][:, :6, :8])
    H, W = 16, 23
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    R = (0.75 * y - 1.25 * x + 3.0)[None]
    k = np.array([1, 4, 6, 4, 1], np.float64) / 16
    B = oracle.reduce2(R, k)
    yo, xo = np.mgrid[0:B.shape[1], 0:B.shape[2]].astype(np.float64)
    assert np.max(np.abs(B[0] - (0.75 * (2 * yo + 2) - 1.25 * (2 * xo + 2) + 3.0))) <= 1e-12 * 64


def pin_reduce_sizes():
    for (H, W, Ho, Wo) in [(5, 5, 1, 1), (6, 6, 1, 1), (7, 8, 2, 2), (8, 9, 2, 3), (100, 101, 48, 49)]:
        assert oracle.reduce2(np.zeros((1, H, W)), [0, 0, 1, 0, 0]).shape == (1, Ho, Wo)


PINS = [v for n, v in sorted(globals().items()) if n.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def test_bad_sizes_rejected():
    with pytest.raises(ValueError):
        oracle.direct(np.zeros((1, 4, 9)), [0, 0, 1, 0, 0])
    with pytest.raises(ValueError):
        oracle.direct(np.zeros((1, 9, 4)), [0, 0, 1, 0, 0])
    with pytest.raises(ValueError):
        oracle.points_f32(np.zeros((1, 9, 9), np.float32), [0, 0, 1, 0, 0], [(0, 5, 0)])


# ---------------------------------------------------------------- mutants
MUTANTS = {
    "dropped kernel column": ("for (int j = 0; j < SC5O_TAPS; ++j)\n                        s += Ap[(y + i)",
                              "for (int j = 0; j < SC5O_TAPS - 1; ++j)\n                        s += Ap[(y + i)"),
    "reduce: dropped kernel column": ("for (int j = 0; j < SC5O_TAPS; ++j)\n                        s += Ap[(2 * y",
                                      "for (int j = 0; j < SC5O_TAPS - 1; ++j)\n                        s += Ap[(2 * y"),
    "transposed image operand": ("Ap[(y + i) * W + (x + j)] * K[i * SC5O_TAPS + j]",
                                 "Ap[(y + j) * W + (x + i)] * K[i * SC5O_TAPS + j]"),
    "width-n transposed image operand": ("Ap[(y + i) * W + (x + j)] * K[i * n + j]",
                                         "Ap[(y + j) * W + (x + i)] * K[i * n + j]"),
    "transposed K": ("* K[i * SC5O_TAPS + j];\n                Bp[y * Wv", "* K[j * SC5O_TAPS + i];\n                Bp[y * Wv"),
    "flipped horizontal taps": ("W + x + t] * k[t]", "W + x + t] * k[4 - t]"),
    "flipped vertical taps": ("T[(p * H + y + t) * Wt + x] * k[t]", "T[(p * H + y + 4 - t) * Wt + x] * k[t]"),
    "outer product index": ("K[i * SC5O_TAPS + j] = k[i] * k[j]", "K[i * SC5O_TAPS + j] = k[i] * k[4 - j]"),
    "sign error": ("s += Ap[(y + i) * W + (x + j)] * K[i * SC5O_TAPS + j]",
                   "s -= Ap[(y + i) * W + (x + j)] * K[i * SC5O_TAPS + j]"),
    "width-n sign error": ("s += Ap[(y + i) * W + (x + j)] * K[i * n + j]",
                           "s -= Ap[(y + i) * W + (x + j)] * K[i * n + j]"),
    "points row offset": ("(p * H + y + i) * pitch + x + j]", "(p * H + y + i) * pitch + x + i]"),
    "e4m3 bias": ("ldexp(1.0 + (double)m / 8.0, e - 7)", "ldexp(1.0 + (double)m / 8.0, e - 8)"),
    "e4m3 subnormal": ("ldexp((double)m, -9)", "ldexp((double)m, -10)"),
    "f16 bias": ("ldexp(1.0 + (double)m / 1024.0, e - 15)", "ldexp(1.0 + (double)m / 1024.0, e - 14)"),
    "scale multiplies": ("out[i] = v / scale;", "out[i] = v * scale;"),
    "width-n transposed K": ("* K[i * n + j];", "* K[j * n + i];"),
    "width-n dropped row": ("for (int64_t i = 0; i < n; ++i)\n                    for (int64_t j = 0; j < n; ++j)",
                            "for (int64_t i = 1; i < n; ++i)\n                    for (int64_t j = 0; j < n; ++j)"),
    "width-n VALID size": ("const int64_t Hv = H - n + 1, Wv = W - n + 1;", "const int64_t Hv = H - n + 1, Wv = W - n;"),
    "reduce: no column stride": ("Ap[(2 * y + i) * W + (2 * x + j)]", "Ap[(2 * y + i) * W + (x + j)]"),
    "reduce: odd phase": ("Ap[(2 * y + i) * W + (2 * x + j)]", "Ap[(2 * y + 1 + i) * W + (2 * x + j)]"),
    "reduce: output height rounded down": ("const int64_t Ho = (H - 4 + 1) / 2,", "const int64_t Ho = (H - 4) / 2,"),
}


@pytest.fixture(scope="module")
def mutant_dir():
    d = tempfile.mkdtemp(prefix="sc5o_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, mutant_dir, monkeypatch):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name!r} not unique"
    path_c = os.path.join(mutant_dir, name.replace(" ", "_") + ".c")
    path_so = path_c[:-2] + ".so"
    open(path_c, "w").write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-o", path_so, path_c, "-lm"])
    monkeypatch.setattr(oracle, "_lib", oracle._bind(path_so))
    failed = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"no pin catches the planted mistake {name!r}"
