"""Seeded synthetic inputs for the separable width-5 convolution.

This module is shared by the oracle side and the CUDA side of the tests and by
the benchmark.  It draws images, kernel vectors, batch shapes and request
streams from fixed seeds, and converts FP32 images into the stored formats
(bfloat16, binary16, FP8 E4M3 with a per-image scale).  It contains none of
the convolution's arithmetic.

The paper's own test images (square 1152^2 .. 8748^2, 3 colour planes, Sec. 4)
are not available; uniform pixel values in [0, 255) stand in for them.  The
kernel is a width-5 vector (Sec. 1): either the binomial [1,4,6,4,1]/16 (a
Gaussian approximation) or five uniform(0,1) draws normalised to sum 1.
"""
from __future__ import annotations

import math

import numpy as np

PLANES = 3
E4M3_MAX = 448.0


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def image(seed: int, H: int, W: int, planes: int = PLANES, pitch: int | None = None,
          lo: float = 0.0, hi: float = 255.0, pad_value: float = float("nan")) -> np.ndarray:
    """Planar FP32 image [planes][H][pitch], values uniform in [lo, hi).

    Columns W..pitch-1 are padding filled with ``pad_value`` (NaN by default,
    so that a kernel reading past the logical width poisons its result)."""
    pitch = W if pitch is None else int(pitch)
    if pitch < W:
        raise ValueError("pitch < W")
    vals = rng(seed).uniform(lo, hi, size=(planes, H, W)).astype(np.float32)
    if pitch == W:
        return vals
    out = np.full((planes, H, pitch), pad_value, np.float32)
    out[:, :, :W] = vals
    return out


def integer_image(seed: int, H: int, W: int, planes: int = PLANES, hi: int = 256) -> np.ndarray:
    """Planar FP32 image of integers uniform in [0, hi)."""
    return rng(seed).integers(0, hi, size=(planes, H, W)).astype(np.float32)


def kernel_binomial() -> np.ndarray:
    """k = [1, 4, 6, 4, 1] / 16 (exact in FP32)."""
    return (np.array([1, 4, 6, 4, 1], np.float64) / 16.0).astype(np.float32)


def kernel_normalised(seed: int) -> np.ndarray:
    """Five uniform(0,1) draws divided by their sum, rounded to FP32."""
    u = rng(seed).uniform(0.0, 1.0, size=5)
    return (u / u.sum()).astype(np.float32)


def batch_shapes(seed: int, n: int = 256, lo: int = 64, hi: int = 4096) -> list[tuple[int, int]]:
    """n (H, W) pairs, each side drawn independently log-uniform in [lo, hi]."""
    g = rng(seed)
    out = []
    for _ in range(n):
        H = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        W = int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))
        out.append((max(lo, min(hi, H)), max(lo, min(hi, W))))
    return out


def fp8_scale(x: np.ndarray) -> float:
    """Per-image scale s = 448 / max|x| so that x * s fills the E4M3 range."""
    m = float(np.max(np.abs(x)))
    return E4M3_MAX / m if m > 0 else 1.0


def to_storage(x: np.ndarray, dtype: str, scale: float = 1.0) -> np.ndarray:
    """Round an FP32 array to a stored format (round to nearest even).

    Returns float32 for "f32", uint16 codes for "bf16" and "f16", uint8 codes
    for "fp8e4m3" (the code stores x * scale, saturated at +-448)."""
    import torch  # CPU conversions only

    x = np.ascontiguousarray(x, dtype=np.float32)
    if dtype == "f32":
        return x.copy()
    if dtype == "bf16":
        t = torch.from_numpy(x).to(torch.bfloat16)
        return t.view(torch.int16).numpy().view(np.uint16).copy()
    if dtype == "f16":
        return x.astype(np.float16).view(np.uint16).copy()
    if dtype == "fp8e4m3":
        y = np.clip(x.astype(np.float64) * scale, -E4M3_MAX, E4M3_MAX).astype(np.float32)
        t = torch.from_numpy(y).to(torch.float8_e4m3fn)
        return t.view(torch.uint8).numpy().copy()
    raise ValueError(f"unknown dtype {dtype!r}")


ELEM_BYTES = {"f32": 4, "bf16": 2, "f16": 2, "fp8e4m3": 1}

SERVE_SIZES = [(480, 640), (1080, 1920), (4096, 4096)]  # (H, W)


def serve_stream(seed: int, n: int, rate_per_s: float) -> list[tuple[float, int, int]]:
    """Poisson arrival stream: n tuples (arrival time in s, size class, k seed)."""
    g = rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += g.exponential(1.0 / rate_per_s)
        out.append((t, int(g.integers(0, len(SERVE_SIZES))), int(seed) * 1_000_003 + i))
    return out
