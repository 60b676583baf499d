"""Host-side logic that needs no GPU: the seeded generators, the stored-format
conversions (checked against the oracle's pinned decoders), the benchmark's
helpers, and the binding's argument checks."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1711_09791_gb300 import synth


def test_generators_are_seeded_and_in_range():
    a, b = synth.image(3, 17, 19), synth.image(3, 17, 19)
    assert np.array_equal(a, b) and a.dtype == np.float32 and a.shape == (3, 17, 19)
    assert a.min() >= 0.0 and a.max() < 255.0
    assert not np.array_equal(a, synth.image(4, 17, 19))
    p = synth.image(3, 5, 6, pitch=8)
    assert np.all(np.isnan(p[:, :, 6:])) and np.array_equal(p[:, :, :6], synth.image(3, 5, 6))
    k = synth.kernel_normalised(9)
    assert k.dtype == np.float32 and abs(float(k.astype(np.float64).sum()) - 1.0) < 1e-6 and np.all(k > 0)
    assert np.array_equal(synth.kernel_binomial() * 16, np.array([1, 4, 6, 4, 1], np.float32))


def test_batch_shapes_log_uniform():
    shapes = synth.batch_shapes(3, 256)
    assert len(shapes) == 256 and shapes == synth.batch_shapes(3, 256)
    hs = np.array([h for h, _ in shapes] + [w for _, w in shapes], np.float64)
    assert hs.min() >= 64 and hs.max() <= 4096
    # log-uniform on [64, 4096]: the mean of log2 is about 9, the spread covers the range
    assert abs(np.log2(hs).mean() - 9.0) < 0.4 and np.log2(hs).min() < 6.5 and np.log2(hs).max() > 11.5


@pytest.mark.parametrize("dtype", ["bf16", "f16", "fp8e4m3"])
def test_storage_rounding_is_nearest(dtype):
    x = synth.image(12, 16, 64)
    scale = synth.fp8_scale(x) if dtype == "fp8e4m3" else 1.0
    codes = synth.to_storage(x, dtype, scale)
    vals = oracle.decode(codes, dtype, scale)
    # the decoded value is within half an ulp of the format from the original
    mant = {"bf16": 7, "f16": 10, "fp8e4m3": 3}[dtype]
    e = np.floor(np.log2(np.maximum(np.abs(x.astype(np.float64)) * scale, 2.0 ** -6)))
    half_ulp = np.exp2(e - mant - 1) / scale
    assert np.all(np.abs(vals - x) <= half_ulp * (1 + 1e-12))
    if dtype == "fp8e4m3":
        assert float(np.max(np.abs(x))) * scale == pytest.approx(448.0)


def test_serve_stream_poisson():
    s = synth.serve_stream(5, 4000, 1000.0)
    t = np.array([a for a, _, _ in s])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 1e-3) < 1e-4
    classes = np.bincount([c for _, c, _ in s], minlength=3)
    assert np.all(classes > 1200)


def test_bench_helpers():
    import bench
    assert bench.algorithmic_bytes(8192, 8192) == 3 * 8192 * 8192 * 4 + 3 * 8188 * 8188 * 4 == 1609826496
    assert bench.whole_job_value(1, 8192 * 8192, 0.25) == pytest.approx(8192 * 8192 / 0.25e-3 / 1e6)
    assert bench.reduce_max(1.5, 1) == 1.5
    peaks = bench.measured_peaks()
    if peaks is not None:
        assert peaks["hbm_gbs"] > 1000
    # the committed profile is read only when it matches the kernel sources
    t = bench.profiled_traffic()
    assert t is None or 1.4e9 < t < 1.8e9


def test_clock_sampler_parsing():
    """Samples are time-stamped; the report covers the marked window plus the
    first sample after it, and names the throttle reasons seen there."""
    import bench
    cs = bench.ClockSampler("0")
    cs.PERIOD_MS = 0
    cs.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    cs.window = [10.0, 20.0]
    cs.lines = [(5.0, "0, 900, 2070, 300.0, 0x0, Not Active, Active, Not Active, Not Active"),   # before
                (11.0, "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active"),
                (15.0, "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"),
                (16.0, "garbage"),
                (21.0, "0, 2060, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active"),  # next
                (22.0, "0, 100, 2070, 80.0, 0x0, Active, Not Active, Not Active, Not Active")]        # later
    r = cs.stop()
    assert r["sm_max_mhz"] == 2070 and r["samples"] == 3 and r["samples_in_window"] == 3
    assert r["sm_mhz"] == 2060 and r["reasons"] == ["sw_power_cap"]
    empty = bench.ClockSampler("0")
    empty.proc = cs.proc
    empty.PERIOD_MS = 0
    assert empty.stop()["reasons"] == ["no samples"]


def test_binding_header_and_arguments():
    from paper_1711_09791_gb300 import sepconv5
    names = sepconv5.header_symbols()
    for n in ("sepconv5_plan", "sepconv5_run", "sepconv5_run_K", "sepconv5_run_inplace", "sepconv5_run_host",
              "sepconv5_run_batch", "serve_submit", "serve_poll", "sepconv5_autotune"):
        assert n in names
    assert sepconv5._taps([1, 2, 3, 4, 5])[4] == 5.0
    with pytest.raises(ValueError):
        sepconv5._taps([1, 2, 3])
    assert len(sepconv5._taps([1, 2, 3], 3)) == 3
    assert sepconv5._ptr(None) is None and sepconv5._ptr(1234) == 1234
    assert math.isclose(sepconv5.DTYPE_BYTES["fp8e4m3"], 1)


def test_reference_arm_line():
    """bench.py --impl reference on the host: one JSON line with the contract's
    keys, the same config object as the GPU arm, and the oracle as its CPU
    baseline."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "Mpix/s"
    assert d["config"] == bench.run_config(1)
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_oracle_is_test_infrastructure_only():
    """Static check of the oracle's isolation: no file of the product package
    (Python or CUDA/C++) names the oracle module or its C source, the oracle
    names nothing of the package's arithmetic (only the seeded generators are
    shared, through the tests), and bench.py imports it only in its two CPU
    baseline functions."""
    import ast
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1711_09791_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if not f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                continue
            text = open(os.path.join(dirpath, f)).read()
            if f.endswith(".py"):
                tree = ast.parse(text)
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert all(a.name.split(".")[0] != "oracle" for a in node.names), f
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", f
            else:
                assert "sepconv5_oracle" not in text and "sc5o_" not in text, f
    for f in os.listdir(os.path.join(root, "oracle")):
        if f.endswith((".py", ".c")):
            text = open(os.path.join(root, "oracle", f)).read()
            assert "import paper_1711_09791_gb300" not in text and "from paper_1711_09791_gb300" not in text, f
            assert "sepconv5.h" not in text and "sc5_internal" not in text, f
    tree = ast.parse(open(os.path.join(root, "bench.py")).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    users.add(fn.name)
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert not any(isinstance(n, ast.Import) and any(a.name == "oracle" for a in n.names) for n in top)
    assert users == {"oracle_sample", "run_reference"}, users


def test_device_waits_are_bounded_and_nothing_traps():
    """Static check of the failure-detection design: every mbarrier wait in
    the kernels goes through the bounded helper (global-timer limit, then an
    error status), the raw try-wait appears nowhere else, and no kernel traps
    or asserts."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_1711_09791_gb300", "csrc")
    raw_waits = {}
    for f in sorted(os.listdir(csrc)):
        if not f.endswith((".cu", ".cuh", ".h", ".cpp")):
            continue
        text = open(os.path.join(csrc, f)).read()
        assert "__trap" not in text and not re.search(r"asm[^;]*\btrap\b", text), f
        assert not re.search(r"(?<!static_)\bassert\s*\(", text), f
        assert text.count("mbarrier.try_wait") + text.count("mbarrier.test_wait") == (1 if f == "sc5_device.cuh" else 0), f
        n = len(re.findall(r"\bmbar_try_wait\s*\(", text))
        if n:
            raw_waits[f] = n
    # the definition and the two calls inside mbar_wait_bounded
    assert raw_waits == {"sc5_device.cuh": 3}, raw_waits
    dev = open(os.path.join(csrc, "sc5_device.cuh")).read()
    body = dev[dev.index("bool mbar_wait_bounded("):]
    body = body[:body.index("\n}\n")]
    assert "global_timer_ns()" in body and "return false" in body


def test_bench_case_parsing():
    """`bench.py --case` options: defaults (3 x 8192 x 8192 FP32 fused, width 5),
    integer keys parsed as integers, the output format defaulting to the
    input's, and unknown keys refused."""
    import bench
    c = bench.parse_case("")
    assert (c["dtype"], c["out"], c["algo"], c["H"], c["W"], c["taps"], c["batch"]) == \
        ("f32", "f32", "fused", 8192, 8192, 5, 0)
    c = bench.parse_case("dtype=bf16,tile=128x256x2,ctas=2,batch=256,taps=3,opitch=8196")
    assert c["out"] == "bf16" and c["tile"] == "128x256x2"
    assert (c["ctas"], c["batch"], c["taps"], c["opitch"]) == (2, 256, 3, 8196)
    with pytest.raises(SystemExit):
        bench.parse_case("colour=red")
