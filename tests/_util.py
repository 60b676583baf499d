"""Helpers shared by the tests: device buffers from numpy arrays, decoding of
stored outputs (through the oracle's pinned decoders), and the error bounds.

Tolerances (written out in the tests that use them):
  * FP32 output, inputs in [0, 255], sum(k) = 1: max-abs 2e-4 against the FP64
    oracle (about 13 ulp of FP32 at 255; the separable FP32 evaluation rounds
    10 products and 8 sums, a few ulp).
  * stored outputs (bf16 / f16 / fp8e4m3): half an ulp of the stored format at
    the result (rounding to nearest), plus the FP32 part above scaled to the
    stored code's units.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

FP32_TOL = 2e-4


def torch_mod():
    import torch
    return torch


def to_dev(a: np.ndarray):
    torch = torch_mod()
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint16:
        t = torch.from_numpy(a.view(np.int16).copy())
    elif a.dtype == np.uint8:
        t = torch.from_numpy(a.copy())
    else:
        t = torch.from_numpy(a.copy())
    return t.cuda()


def from_dev(t, dtype: str) -> np.ndarray:
    a = t.cpu().numpy()
    if dtype in ("bf16", "f16"):
        return a.view(np.uint16)
    if dtype == "fp8e4m3":
        return a.view(np.uint8)
    return a


def empty_dev(shape, dtype: str, fill="sentinel"):
    """Device buffer pre-filled with a sentinel (NaN, or the code 0xFF.. of
    the format) so that unwritten and overwritten pixels can be told apart."""
    torch = torch_mod()
    if dtype == "f32":
        return torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    if dtype in ("bf16", "f16"):
        return torch.full(shape, -1, dtype=torch.int16, device="cuda")  # 0xFFFF: a NaN in both
    if dtype == "fp8e4m3":
        return torch.full(shape, 0xFF, dtype=torch.uint8, device="cuda")  # E4M3 NaN
    raise ValueError(dtype)


def sentinel_intact(a: np.ndarray, dtype: str) -> bool:
    if dtype == "f32":
        return bool(np.all(np.isnan(a)))
    if dtype in ("bf16", "f16"):
        return bool(np.all(a == 0xFFFF))
    return bool(np.all(a == 0xFF))


def decode(codes: np.ndarray, dtype: str, scale: float = 1.0) -> np.ndarray:
    return oracle.decode(codes, dtype, scale)


def ulp(dtype: str, x: np.ndarray) -> np.ndarray:
    """Spacing of the stored format at |x| (normal range; subnormal floor)."""
    mant = {"bf16": 7, "f16": 10, "fp8e4m3": 3, "f32": 23}[dtype]
    emin = {"bf16": -126, "f16": -14, "fp8e4m3": -6, "f32": -126}[dtype]
    ax = np.maximum(np.abs(x), np.finfo(np.float64).tiny)
    e = np.maximum(np.floor(np.log2(ax)), emin)
    return np.exp2(e - mant)


def stored_tolerance(ref: np.ndarray, dtype: str, out_scale: float, fp32_tol: float) -> np.ndarray:
    """Bound on |decoded output - ref| (real units) when the FP32 result is
    rounded to `dtype` after multiplying by out_scale: half an ulp at the
    (slightly enlarged) code, plus the FP32 evaluation error."""
    code = np.abs(ref) * out_scale + fp32_tol * out_scale
    return (0.5 * ulp(dtype, code) + fp32_tol * out_scale) / out_scale * (1 + 1e-6)


def oracle_valid(A_codes: np.ndarray, dtype: str, k, in_scale: float = 1.0, W: int | None = None) -> np.ndarray:
    """FP64 oracle result (VALID) on the decoded stored input [P][H][pitch]."""
    vals = decode(A_codes, dtype, in_scale)
    if W is not None:
        vals = vals[:, :, :W]
    return oracle.direct(vals, np.asarray(k, np.float64))


def max_abs(a, b) -> float:
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return float(np.max(d)) if d.size else 0.0


def round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


def pitch_for(W: int, dtype: str, extra: int = 0) -> int:
    es = {"f32": 4, "bf16": 2, "f16": 2, "fp8e4m3": 1}[dtype]
    return round_up(W * es, 16) // es + extra


def is_finite_all(a: np.ndarray) -> bool:
    return bool(np.all(np.isfinite(a)))


def nan_count(a) -> int:
    return int(np.count_nonzero(np.isnan(a)))


def almost_power_of_two(x: float) -> bool:
    return abs(math.log2(x) - round(math.log2(x))) < 1e-12
