"""FP64 CPU oracle for the separable width-5 convolution (arXiv 1711.09791).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
timed CPU baseline of ``bench.py`` are the only users.  The product library
never imports, links or runs anything here, and nothing here imports the
product package.

The arithmetic lives in ``sepconv5_oracle.c`` (plain C, IEEE double); this
module compiles it with gcc into ``oracle/_build`` and marshals numpy arrays
to it.  Each wrapper names the passage of the paper it follows:

* :func:`direct`        -- Eq. 1 with K = k k^T (Sec. 1), single-pass form
* :func:`direct_K`      -- Eq. 1 with a general 5x5 K (Sec. 5.1, the
                           "general algorithm" with four nested loops)
* :func:`direct_Kn`     -- Eq. 1 with a general n x n K, any odd width n
* :func:`direct_n`      -- Eq. 1 with K = k k^T for a width-n vector k
* :func:`hpass`         -- the horizontal 1D pass (Sec. 5.1, Listing 1)
* :func:`vpass`         -- the vertical 1D pass (Sec. 5.1, Listing 1)
* :func:`points_f32`    -- Eq. 1 at chosen output pixels of an FP32 image
* :func:`decode`        -- exact decoding of bf16 / fp16 / fp8-e4m3 codes
* :func:`keep_frame`    -- the "copy the 2-pixel frame" output (Listing 1's
                           in-place result, whose frame keeps the input)
* :func:`reduce2`       -- one pyramid REDUCE step: Eq. 1 (K = k k^T) kept at
                           every second row and column (the "scaling" of the
                           stereo pipeline, Sec. 1, which the paper does not
                           define: this is the reading taken)

Output convention (the VALID region, Sec. 5: convolution starts at pixel
(2,2) and the edges are ignored): plane p of the result is (H-4) x (W-4) and
output (y, x) is centred on input (y+2, x+2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sepconv5_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsc5oracle.so")

DTYPE_CODES = {"f32": 0, "bf16": 1, "f16": 2, "fp8e4m3": 3}

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags: the same source gives the
    same doubles on x86-64 and AArch64; FMA contraction is switched off)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-fno-fast-math",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    """Open a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int64
    lib.sc5o_direct_K.argtypes = [P, I, I, I, P, P]
    lib.sc5o_direct.argtypes = [P, I, I, I, P, P]
    lib.sc5o_hpass.argtypes = [P, I, I, I, P, P]
    lib.sc5o_vpass.argtypes = [P, I, I, I, P, P]
    lib.sc5o_points_f32.argtypes = [P, I, I, I, I, P, P, I, P]
    lib.sc5o_decode.argtypes = [ctypes.c_int, P, I, ctypes.c_double, P]
    lib.sc5o_outer.argtypes = [P, P]
    lib.sc5o_direct_Kn.argtypes = [P, I, I, I, I, P, P]
    lib.sc5o_direct_Kn.restype = ctypes.c_int
    lib.sc5o_reduce.argtypes = [P, I, I, I, P, P]
    lib.sc5o_reduce.restype = ctypes.c_int
    for f in ("sc5o_direct_K", "sc5o_direct", "sc5o_hpass", "sc5o_vpass",
              "sc5o_points_f32", "sc5o_decode"):
        getattr(lib, f).restype = ctypes.c_int
    lib.sc5o_outer.restype = None
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as3(A) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim == 2:
        A = A[None]
    if A.ndim != 3:
        raise ValueError("image must be [H][W] or [P][H][W]")
    return A


def _k5(k) -> np.ndarray:
    k = np.ascontiguousarray(k, dtype=np.float64).reshape(-1)
    if k.size != 5:
        raise ValueError("k must have 5 taps")
    return k


def outer(k) -> np.ndarray:
    """K[i][j] = k[i] k[j] (Sec. 1)."""
    k = _k5(k)
    K = np.empty((5, 5), np.float64)
    _load().sc5o_outer(_ptr(k), _ptr(K))
    return K


def direct_K(A, K) -> np.ndarray:
    """Eq. 1 with a general 5x5 K; VALID output [P][H-4][W-4] in FP64."""
    A = _as3(A)
    K = np.ascontiguousarray(K, dtype=np.float64).reshape(5, 5)
    P, H, W = A.shape
    B = np.empty((P, H - 4, W - 4), np.float64)
    if _load().sc5o_direct_K(_ptr(A), P, H, W, _ptr(K), _ptr(B)) != 0:
        raise ValueError("direct_K: image smaller than 5x5")
    return B


def direct(A, k) -> np.ndarray:
    """Eq. 1 with K = k k^T (single-pass form); VALID output in FP64."""
    A = _as3(A)
    k = _k5(k)
    P, H, W = A.shape
    B = np.empty((P, H - 4, W - 4), np.float64)
    if _load().sc5o_direct(_ptr(A), P, H, W, _ptr(k), _ptr(B)) != 0:
        raise ValueError("direct: image smaller than 5x5")
    return B


def direct_Kn(A, K) -> np.ndarray:
    """Eq. 1 with a general n x n K (n odd); VALID output [P][H-n+1][W-n+1]."""
    A = _as3(A)
    K = np.ascontiguousarray(K, dtype=np.float64)
    n = K.shape[0]
    if K.shape != (n, n) or n % 2 == 0:
        raise ValueError("K must be square with odd width")
    P, H, W = A.shape
    if H < n or W < n:
        raise ValueError("direct_Kn: image smaller than the kernel")
    B = np.empty((P, H - n + 1, W - n + 1), np.float64)
    if _load().sc5o_direct_Kn(_ptr(A), P, H, W, n, _ptr(K), _ptr(B)) != 0:
        raise ValueError("direct_Kn: bad sizes")
    return B


def direct_n(A, k) -> np.ndarray:
    """Eq. 1 with K[i][j] = k[i] k[j] for a vector k of odd length n."""
    k = np.ascontiguousarray(k, dtype=np.float64).reshape(-1)
    return direct_Kn(A, np.outer(k, k))


def reduce2(A, k) -> np.ndarray:
    """One REDUCE step: [P][ceil((H-4)/2)][ceil((W-4)/2)] in FP64, output (y, x)
    centred on input (2y+2, 2x+2)."""
    A = _as3(A)
    k = _k5(k)
    P, H, W = A.shape
    B = np.empty((P, (H - 3) // 2, (W - 3) // 2), np.float64)
    if _load().sc5o_reduce(_ptr(A), P, H, W, _ptr(k), _ptr(B)) != 0:
        raise ValueError("reduce2: image smaller than 5x5")
    return B


def hpass(A, k) -> np.ndarray:
    """Horizontal pass over all rows: T [P][H][W-4] in FP64."""
    A = _as3(A)
    k = _k5(k)
    P, H, W = A.shape
    T = np.empty((P, H, W - 4), np.float64)
    if _load().sc5o_hpass(_ptr(A), P, H, W, _ptr(k), _ptr(T)) != 0:
        raise ValueError("hpass: W < 5")
    return T


def vpass(T, k) -> np.ndarray:
    """Vertical pass: B [P][H-4][Wt] in FP64."""
    T = _as3(T)
    k = _k5(k)
    P, H, Wt = T.shape
    B = np.empty((P, H - 4, Wt), np.float64)
    if _load().sc5o_vpass(_ptr(T), P, H, Wt, _ptr(k), _ptr(B)) != 0:
        raise ValueError("vpass: H < 5")
    return B


def points_f32(A, k, pts) -> np.ndarray:
    """Eq. 1 (K = k k^T) at VALID output pixels pts[:, (p, y, x)] of an FP32
    image A [P][H][pitch] whose logical width is W = A.shape[2] unless given
    as a (A, W) tuple."""
    W = None
    if isinstance(A, tuple):
        A, W = A
    if A.dtype != np.float32 or A.ndim != 3 or not A.flags.c_contiguous:
        raise ValueError("points_f32 wants a C-contiguous float32 [P][H][pitch] array")
    P, H, pitch = A.shape
    W = pitch if W is None else int(W)
    k = _k5(k)
    pts = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    out = np.empty(len(pts), np.float64)
    if _load().sc5o_points_f32(_ptr(A), P, H, W, pitch, _ptr(k), _ptr(pts),
                               len(pts), _ptr(out)) != 0:
        raise ValueError("points_f32: bad sizes or point outside the VALID region")
    return out


def decode(codes: np.ndarray, dtype: str, scale: float = 1.0) -> np.ndarray:
    """Exact value of stored codes (uint16 for bf16/f16, uint8 for fp8e4m3,
    float32 for f32), divided by the per-image scale."""
    code = DTYPE_CODES[dtype]
    want = {0: np.float32, 1: np.uint16, 2: np.uint16, 3: np.uint8}[code]
    c = np.ascontiguousarray(codes)
    if c.dtype != want:
        c = c.view(want) if c.dtype.itemsize == np.dtype(want).itemsize else None
        if c is None:
            raise ValueError(f"decode({dtype}) wants {np.dtype(want).name} codes")
    c = np.ascontiguousarray(c)
    out = np.empty(c.shape, np.float64)
    if _load().sc5o_decode(code, _ptr(c), c.size, float(scale), _ptr(out)) != 0:
        raise ValueError("decode: bad dtype or scale")
    return out


def keep_frame(A, B_valid) -> np.ndarray:
    """Full-size result whose 2-pixel frame is the input and whose interior is
    the VALID result -- the image Listing 1 leaves in A (its loops write only
    rows and columns 2..n-3)."""
    A = _as3(A)
    out = A.copy()
    out[:, 2:-2, 2:-2] = B_valid
    return out
