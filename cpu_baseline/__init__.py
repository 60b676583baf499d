"""Timed CPU baseline of the benchmark: the paper's two-pass form in FP32 with
OpenMP over every host core (``sc5_cpu_twopass.c``; loop structure of
Listing 1, Sec. 5.1, with the horizontal pass over all rows).

Benchmark infrastructure only: it shares no code with the CUDA library or
with the FP64 oracle.  The C source is compiled here with gcc
(``-O3 -fopenmp``, portable flags: the same source builds on x86-64 and
AArch64 hosts) into ``cpu_baseline/_build``.
"""
from __future__ import annotations

import ctypes
import os
import statistics
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc5_cpu_twopass.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsc5cpu.so")
FLAGS = ["-O3", "-fopenmp", "-std=c11", "-fPIC", "-shared"]

_lib = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *FLAGS, "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I = ctypes.c_void_p, ctypes.c_int64
        lib.sc5cpu_two_pass.argtypes = [P, I, I, I, P, P, P]
        lib.sc5cpu_two_pass.restype = ctypes.c_int
        lib.sc5cpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the OpenMP loops run on (OMP_NUM_THREADS, else every core)."""
    return int(_load().sc5cpu_threads())


def two_pass(A: np.ndarray, k, T: np.ndarray | None = None, B: np.ndarray | None = None) -> np.ndarray:
    """VALID result [P][H-4][W-4] (FP32) of a C-contiguous FP32 [P][H][W] image."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    P, H, W = A.shape
    k = np.ascontiguousarray(k, dtype=np.float32).reshape(5)
    T = np.empty((H, W - 4), np.float32) if T is None else T
    B = np.empty((P, H - 4, W - 4), np.float32) if B is None else B
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    if _load().sc5cpu_two_pass(ptr(A), P, H, W, ptr(k), ptr(T), ptr(B)) != 0:
        raise ValueError("two_pass: image smaller than 5 x 5")
    return B


def time_two_pass(A: np.ndarray, k, reps: int = 5) -> float:
    """Median wall time (s) of `reps` calls after one warm-up call."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    P, H, W = A.shape
    T = np.empty((H, W - 4), np.float32)
    B = np.empty((P, H - 4, W - 4), np.float32)
    two_pass(A, k, T, B)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        two_pass(A, k, T, B)
        times.append(time.perf_counter() - t0)
    return statistics.median(times)


def cpu_model() -> str:
    """The host CPU's model name (lscpu), or the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return os.uname().machine
