"""ctypes binding of libsepconv5 (C ABI in ``include/sepconv5.h``).

Argument marshalling only: every step of the convolution runs in the CUDA
library.  Device buffers may be given as integers (addresses) or as objects
with a ``data_ptr()`` method (e.g. torch tensors); streams as integers or
objects with a ``cuda_stream`` attribute.  If the library has not been built
this module raises on load -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, byref, c_char_p, c_double, c_float, c_int32, c_int64, c_size_t, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsepconv5.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sepconv5.h")

OK, EINVAL, ENOMEM, ECUDA, EAGAIN, ETIMEDOUT, ENOTFOUND, EDEVICE = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EAGAIN", "ETIMEDOUT", "ENOTFOUND", "EDEVICE"]
DTYPES = {"f32": 0, "bf16": 1, "f16": 2, "fp8e4m3": 3}
DTYPE_BYTES = {"f32": 4, "bf16": 2, "f16": 2, "fp8e4m3": 1}
BORDERS = {"valid": 0, "keep": 1}
LAYOUTS = {"planar": 0, "hwc": 1}
ALGOS = {"fused": 0, "two_pass": 1, "direct": 2, "reduce": 3}


class Sepconv5Error(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{func}: {name}: {message}")


class PlanDesc(ctypes.Structure):
    _fields_ = [("planes", c_int32), ("H", c_int32), ("W", c_int32),
                ("in_pitch", c_int64), ("out_pitch", c_int64),
                ("in_dtype", c_int32), ("out_dtype", c_int32), ("border", c_int32), ("algo", c_int32),
                ("tile_h", c_int32), ("tile_w", c_int32), ("stages", c_int32), ("ctas_per_sm", c_int32),
                ("in_plane_stride", c_int64), ("out_plane_stride", c_int64), ("taps", c_int32),
                ("layout", c_int32)]


class Image(ctypes.Structure):
    _fields_ = [("in_", c_void_p), ("out", c_void_p), ("H", c_int32), ("W", c_int32),
                ("in_pitch", c_int64), ("out_pitch", c_int64), ("k", c_float * 5),
                ("in_scale", c_float), ("out_scale", c_float)]


class PyramidDesc(ctypes.Structure):
    _fields_ = [("planes", c_int32), ("H", c_int32), ("W", c_int32), ("in_pitch", c_int64),
                ("in_dtype", c_int32), ("out_dtype", c_int32), ("levels", c_int32)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_size_t), ("max_inflight", c_int32), ("dtype", c_int32),
                ("planes", c_int32), ("n_streams", c_int32), ("max_merge", c_int32), ("merge", c_int32),
                ("batch_window_us", c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", c_uint64), ("completed", c_uint64), ("launches", c_uint64),
                ("rejected", c_uint64), ("merged_max", c_uint64), ("resident_peak_bytes", c_size_t),
                ("queue_us_p50", c_double), ("queue_us_p99", c_double), ("stage_us_p50", c_double),
                ("stage_us_p99", c_double), ("run_us_p50", c_double), ("run_us_p99", c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Open the library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsepconv5.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    V, P = c_void_p, c_void_p
    sigs = {
        "sepconv5_plan": [POINTER(PlanDesc), POINTER(V)],
        "sepconv5_plan_destroy": [V],
        "sepconv5_plan_info": [V, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)],
        "sepconv5_run": [V, V, V, POINTER(c_float), c_float, c_float, V],
        "sepconv5_run_host": [V, V, V, POINTER(c_float), c_float, c_float, V],
        "sepconv5_run_K": [V, V, V, POINTER(c_float), c_float, c_float, V],
        "sepconv5_run_inplace": [V, V, POINTER(c_float), c_float, V],
        "sepconv5_hpass": [V, V, V, c_int64, POINTER(c_float), V],
        "sepconv5_vpass": [V, V, c_int64, V, POINTER(c_float), c_float, c_float, V],
        "sepconv5_two_pass_noalloc": [V, V, c_int32, c_int32, c_int32, c_int64, c_int64, c_int32, c_int32,
                                      POINTER(c_float), c_float, c_float, V],
        "sepconv5_device_status": [V, POINTER(c_int32)],
        "sepconv5_run_batch": [V, c_int32, POINTER(Image), V],
        "sepconv5_batch_create": [V, c_int32, POINTER(Image), POINTER(V)],
        "sepconv5_batch_launch": [V, V],
        "sepconv5_batch_info": [V, POINTER(c_int64), POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)],
        "sepconv5_batch_destroy": [V],
        "sepconv5_fused_configs": [c_int32, c_int32, POINTER(c_int32), c_int32, POINTER(c_int32)],
        "sepconv5_autotune": [c_int32, POINTER(c_int32), c_int32, c_char_p],
        "sepconv5_tune_load": [c_char_p],
        "sepconv5_tune_lookup": [c_int32, c_int32, c_int32, c_int32, POINTER(c_int32), POINTER(c_int32),
                                 POINTER(c_int32), POINTER(c_int32)],
        "sepconv5_tune_lookup_batch": [c_int32, c_int32, c_int32, c_int32, POINTER(c_int32), POINTER(c_int32),
                                 POINTER(c_int32), POINTER(c_int32)],
        "sepconv5_pyramid_create": [POINTER(PyramidDesc), POINTER(V)],
        "sepconv5_pyramid_level": [V, c_int32, POINTER(c_int32), POINTER(c_int32), POINTER(c_int64)],
        "sepconv5_pyramid_run": [V, V, POINTER(c_void_p), POINTER(c_float), c_float, c_float, V],
        "sepconv5_pyramid_capture": [V, V, POINTER(c_void_p), POINTER(c_float), c_float, c_float],
        "sepconv5_pyramid_replay": [V, V],
        "sepconv5_pyramid_destroy": [V],
        "serve_create": [POINTER(ServeCfg), POINTER(V)],
        "serve_submit": [V, POINTER(Image), POINTER(c_uint64)],
        "serve_poll": [V, c_uint64, c_int32, POINTER(c_double)],
        "serve_get_stats": [V, POINTER(ServeStats)],
        "serve_destroy": [V],
        "sepconv5_empty_launches": [c_int32, V],
        "sepconv5_selftest_wait_timeout": [c_int32, V],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = c_int32
    lib.sepconv5_last_error.argtypes = []
    lib.sepconv5_last_error.restype = c_char_p
    lib.sepconv5_launch_count.argtypes = []
    lib.sepconv5_launch_count.restype = c_int64
    _lib = lib
    return lib


def header_symbols(path: str = HEADER) -> list[str]:
    """Names of the functions the public header declares."""
    text = open(path).read()
    return sorted(set(re.findall(r"^SC5_API\s+[\w\s\*]+?\b((?:sepconv5|serve)_\w+)\s*\(", text, re.M)))


def _check(status: int, func: str, ok=(OK,)) -> int:
    if status not in ok:
        msg = load().sepconv5_last_error()
        raise Sepconv5Error(status, func, msg.decode() if msg else "")
    return status


def _ptr(x) -> int | None:
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s) -> int | None:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def _taps(k, n=5):
    vals = [float(v) for v in k]
    if len(vals) != n:
        raise ValueError(f"k needs {n} taps")
    return (c_float * n)(*vals)


def _dt(d):
    return DTYPES[d] if isinstance(d, str) else int(d)


class Plan:
    """A plan for one image shape (sepconv5_plan)."""

    def __init__(self, planes: int, H: int, W: int, in_pitch: int | None = None, out_pitch: int | None = None,
                 in_dtype="f32", out_dtype=None, border="valid", algo="fused", tile_h=0, tile_w=0, stages=0,
                 ctas_per_sm=0, in_plane_stride=0, out_plane_stride=0, taps=5, layout="planar"):
        out_dtype = in_dtype if out_dtype is None else out_dtype
        taps = taps or 5  # 0 selects the default width, as in the C descriptor
        b = BORDERS[border] if isinstance(border, str) else int(border)
        d = PlanDesc()
        d.planes, d.H, d.W = planes, H, W
        d.in_pitch = W if in_pitch is None else in_pitch
        d.out_pitch = (W if b == 1 else W - (taps - 1)) if out_pitch is None else out_pitch
        d.in_dtype, d.out_dtype = _dt(in_dtype), _dt(out_dtype)
        d.border = b
        d.algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
        d.tile_h, d.tile_w, d.stages, d.ctas_per_sm = tile_h, tile_w, stages, ctas_per_sm
        d.in_plane_stride, d.out_plane_stride = in_plane_stride, out_plane_stride
        d.taps = taps
        d.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
        self.taps = taps
        self.desc = d
        h = c_void_p()
        _check(load().sepconv5_plan(byref(d), byref(h)), "sepconv5_plan")
        self._h = h

    @property
    def handle(self):
        return self._h

    def run(self, src, dst, k, in_scale=1.0, out_scale=1.0, stream=None):
        _check(load().sepconv5_run(self._h, _ptr(src), _ptr(dst), _taps(k, self.taps), in_scale, out_scale,
                                   _stream(stream)), "sepconv5_run")

    def run_K(self, src, dst, K, in_scale=1.0, out_scale=1.0, stream=None):
        """Direct form with a general 5x5 matrix K (25 values, row-major)."""
        vals = [float(v) for row in K for v in (row if hasattr(row, "__iter__") else [row])]
        if len(vals) != 25:
            raise ValueError("K needs 25 values")
        _check(load().sepconv5_run_K(self._h, _ptr(src), _ptr(dst), (c_float * 25)(*vals), in_scale, out_scale,
                                     _stream(stream)), "sepconv5_run_K")

    def run_inplace(self, img, k, scale=1.0, stream=None):
        _check(load().sepconv5_run_inplace(self._h, _ptr(img), _taps(k), scale, _stream(stream)),
               "sepconv5_run_inplace")

    def run_host(self, host_src, host_dst, k, in_scale=1.0, out_scale=1.0, stream=None):
        """host_src / host_dst: host addresses (or objects with data_ptr(), e.g.
        pinned CPU tensors)."""
        _check(load().sepconv5_run_host(self._h, _ptr(host_src), _ptr(host_dst), _taps(k), in_scale, out_scale,
                                        _stream(stream)), "sepconv5_run_host")

    def hpass(self, src, T, t_pitch, k, stream=None):
        _check(load().sepconv5_hpass(self._h, _ptr(src), _ptr(T), t_pitch, _taps(k), _stream(stream)),
               "sepconv5_hpass")

    def vpass(self, T, t_pitch, dst, k, in_scale=1.0, out_scale=1.0, stream=None):
        _check(load().sepconv5_vpass(self._h, _ptr(T), t_pitch, _ptr(dst), _taps(k), in_scale, out_scale,
                                     _stream(stream)), "sepconv5_vpass")

    def info(self) -> dict:
        """The launch configuration the plan chose (sepconv5_plan_info)."""
        th, tw, st, c = c_int32(), c_int32(), c_int32(), c_int32()
        _check(load().sepconv5_plan_info(self._h, byref(th), byref(tw), byref(st), byref(c)), "sepconv5_plan_info")
        return {"tile_h": th.value, "tile_w": tw.value, "stages": st.value, "ctas_per_sm": c.value}

    def run_batch(self, images, stream=None):
        arr = make_images(images)
        _check(load().sepconv5_run_batch(self._h, len(arr), arr, _stream(stream)), "sepconv5_run_batch")

    def close(self):
        if getattr(self, "_h", None):
            load().sepconv5_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_images(images) -> ctypes.Array:
    """images: iterable of dicts with keys in, out, H, W, in_pitch, out_pitch, k,
    in_scale (1), out_scale (1)."""
    images = list(images)
    arr = (Image * len(images))()
    for i, im in enumerate(images):
        a = arr[i]
        a.in_ = _ptr(im["in"])
        a.out = _ptr(im["out"])
        a.H, a.W = im["H"], im["W"]
        a.in_pitch = im.get("in_pitch", im["W"])
        a.out_pitch = im.get("out_pitch", im["W"] - 4)
        for t, v in enumerate(im["k"]):
            a.k[t] = float(v)
        a.in_scale = im.get("in_scale", 1.0)
        a.out_scale = im.get("out_scale", 1.0)
    return arr


class Batch:
    """A prepared batch replayed from a CUDA graph (sepconv5_batch_create)."""

    def __init__(self, plan: Plan, images):
        self._images = make_images(images)
        h = c_void_p()
        _check(load().sepconv5_batch_create(plan.handle, len(self._images), self._images, byref(h)),
               "sepconv5_batch_create")
        self._h = h

    def launch(self, stream=None):
        _check(load().sepconv5_batch_launch(self._h, _stream(stream)), "sepconv5_batch_launch")

    def info(self) -> dict:
        t, c, th, tw = c_int64(), c_int32(), c_int32(), c_int32()
        _check(load().sepconv5_batch_info(self._h, byref(t), byref(c), byref(th), byref(tw)), "sepconv5_batch_info")
        return {"tiles": t.value, "ctas": c.value, "tile_h": th.value, "tile_w": tw.value}

    def close(self):
        if getattr(self, "_h", None):
            load().sepconv5_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reduce_dims(H: int, W: int) -> tuple[int, int]:
    """Plane size (Ho, Wo) of one REDUCE step (algo="reduce") of an H x W plane."""
    return (H - 3) // 2, (W - 3) // 2


def device_status(stream=None) -> int:
    code = c_int32()
    st = load().sepconv5_device_status(_stream(stream), byref(code))
    _check(st, "sepconv5_device_status", ok=(OK, EDEVICE))
    return code.value


def fused_configs(in_dtype="f32", out_dtype=None) -> list[tuple[int, int, int]]:
    out_dtype = in_dtype if out_dtype is None else out_dtype
    buf = (c_int32 * 96)()
    n = c_int32()
    _check(load().sepconv5_fused_configs(_dt(in_dtype), _dt(out_dtype), buf, 32, byref(n)), "sepconv5_fused_configs")
    return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(n.value)]


def autotune(mode: int, pairs, path: str | None = None):
    flat = [v for a, b in pairs for v in (_dt(a), _dt(b))]
    arr = (c_int32 * max(1, len(flat)))(*flat)
    _check(load().sepconv5_autotune(mode, arr, len(pairs), path.encode() if path else None), "sepconv5_autotune")


def tune_load(path: str):
    _check(load().sepconv5_tune_load(path.encode()), "sepconv5_tune_load")


def tune_lookup(in_dtype, out_dtype, H, W, batch: bool = False) -> tuple[dict, bool]:
    """The tuned shape a plan (or, with batch=True, a batch) takes for an H x W
    plane, and whether the table had an entry."""
    th, tw, st, c = c_int32(), c_int32(), c_int32(), c_int32()
    name = "sepconv5_tune_lookup_batch" if batch else "sepconv5_tune_lookup"
    s = getattr(load(), name)(_dt(in_dtype), _dt(out_dtype), H, W, byref(th), byref(tw), byref(st), byref(c))
    _check(s, name, ok=(OK, ENOTFOUND))
    return {"tile_h": th.value, "tile_w": tw.value, "stages": st.value, "ctas_per_sm": c.value}, s == OK


def empty_launches(n: int, stream=None):
    _check(load().sepconv5_empty_launches(n, _stream(stream)), "sepconv5_empty_launches")


def selftest_wait_timeout(limit_us: int, stream=None):
    _check(load().sepconv5_selftest_wait_timeout(limit_us, _stream(stream)), "sepconv5_selftest_wait_timeout")


def launch_count() -> int:
    return load().sepconv5_launch_count()


class Pyramid:
    """`levels` chained REDUCE steps of a planar image (sepconv5_pyramid_*).
    level(l) gives (H, W, pitch) of level l (0 = the input); run() fills the
    caller's level buffers, levels[l-1] holding level l."""

    def __init__(self, planes: int, H: int, W: int, in_pitch: int | None = None, in_dtype="f32",
                 out_dtype=None, levels: int = 1):
        d = PyramidDesc()
        d.planes, d.H, d.W = planes, H, W
        d.in_pitch = W if in_pitch is None else in_pitch
        d.in_dtype = _dt(in_dtype)
        d.out_dtype = _dt(in_dtype if out_dtype is None else out_dtype)
        d.levels = levels
        h = c_void_p()
        _check(load().sepconv5_pyramid_create(byref(d), byref(h)), "sepconv5_pyramid_create")
        self._h = h
        self.levels = levels

    def level(self, level: int) -> tuple[int, int, int]:
        H, W, pitch = c_int32(), c_int32(), c_int64()
        _check(load().sepconv5_pyramid_level(self._h, level, byref(H), byref(W), byref(pitch)),
               "sepconv5_pyramid_level")
        return H.value, W.value, pitch.value

    def run(self, src, levels, k, in_scale=1.0, out_scale=1.0, stream=None):
        ptrs = (c_void_p * len(levels))(*[_ptr(t) for t in levels])
        _check(load().sepconv5_pyramid_run(self._h, _ptr(src), ptrs, _taps(k), in_scale, out_scale,
                                           _stream(stream)), "sepconv5_pyramid_run")

    def capture(self, src, levels, k, in_scale=1.0, out_scale=1.0):
        """Record run() for these buffers into a CUDA graph (sepconv5_pyramid_capture)."""
        self._keep = (src, list(levels))  # the graph holds their addresses
        ptrs = (c_void_p * len(levels))(*[_ptr(t) for t in levels])
        _check(load().sepconv5_pyramid_capture(self._h, _ptr(src), ptrs, _taps(k), in_scale, out_scale),
               "sepconv5_pyramid_capture")

    def replay(self, stream=None):
        _check(load().sepconv5_pyramid_replay(self._h, _stream(stream)), "sepconv5_pyramid_replay")

    def close(self):
        if getattr(self, "_h", None):
            load().sepconv5_pyramid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving runtime (serve_create / serve_submit / serve_poll / serve_destroy)."""

    def __init__(self, hbm_budget_bytes: int, dtype="bf16", planes=3, max_inflight=64, n_streams=2,
                 max_merge=8, merge=True, batch_window_us=0):
        cfg = ServeCfg()
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.max_inflight = max_inflight
        cfg.dtype = _dt(dtype)
        cfg.planes = planes
        cfg.n_streams = n_streams
        cfg.max_merge = max_merge
        cfg.merge = 1 if merge else 0
        cfg.batch_window_us = batch_window_us
        h = c_void_p()
        _check(load().serve_create(byref(cfg), byref(h)), "serve_create")
        self._h = h

    def submit(self, image: dict) -> int | None:
        """Queue a request (host pointers); None when the server pushes back (EAGAIN)."""
        arr = make_images([image])
        t = c_uint64()
        st = load().serve_submit(self._h, arr, byref(t))
        if st == EAGAIN:
            return None
        _check(st, "serve_submit")
        return t.value

    def submit_image(self, img) -> int | None:
        """Queue a request given as a prepared ``Image`` structure (e.g. one
        element of ``make_images``); None when the server pushes back."""
        t = c_uint64()
        st = load().serve_submit(self._h, byref(img), byref(t))
        if st == EAGAIN:
            return None
        _check(st, "serve_submit")
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1) -> float | None:
        """Latency in microseconds once done; None if not done within the timeout."""
        lat = c_double()
        st = load().serve_poll(self._h, ticket, timeout_us, byref(lat))
        if st in (EAGAIN, ETIMEDOUT):
            return None
        _check(st, "serve_poll")
        return lat.value

    def stats(self) -> dict:
        s = ServeStats()
        _check(load().serve_get_stats(self._h, byref(s)), "serve_get_stats")
        return {f: getattr(s, f) for f, _ in ServeStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _check(load().serve_destroy(self._h), "serve_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
