"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function the public header declares, and rejects bad
descriptors before touching the device."""
import ctypes
import os

import pytest

from paper_1711_09791_gb300 import build as sc5_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sc5():
    sc5_build.build()
    from paper_1711_09791_gb300 import sepconv5
    sepconv5.load()
    return sepconv5


def test_header_symbols_are_exported(sc5):
    names = sc5.header_symbols()
    assert len(names) >= 20
    lib = ctypes.CDLL(sc5.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared in include/sepconv5.h but not exported: {missing}"
    for required in ("sepconv5_plan", "sepconv5_run", "sepconv5_run_batch", "serve_submit", "serve_poll"):
        assert required in names


def test_fused_configs_listed(sc5):
    for pair in [("f32", "f32"), ("bf16", "bf16"), ("bf16", "f32"), ("f16", "f16"), ("f16", "f32"),
                 ("fp8e4m3", "fp8e4m3"), ("fp8e4m3", "f32")]:
        cfgs = sc5.fused_configs(*pair)
        assert cfgs and all(tw == 128 and th % 8 == 0 and 32 <= th + 4 <= 256 and st >= 2 for th, tw, st in cfgs)
        # a plan selects a shape by (tile_h, tile_w, stages): every triple must be unique
        assert len(set(cfgs)) == len(cfgs)
    with pytest.raises(sc5.Sepconv5Error):
        sc5.fused_configs("bf16", "f16")


@pytest.mark.parametrize("kw", [dict(H=4, W=64), dict(H=64, W=4), dict(planes=0, H=64, W=64),
                                dict(H=64, W=64, in_pitch=66), dict(H=64, W=64, out_pitch=50),
                                dict(H=64, W=64, in_dtype="bf16", out_dtype="f16")])
def test_bad_descriptors_rejected_on_host(sc5, kw):
    planes = kw.pop("planes", 3)
    H, W = kw.pop("H"), kw.pop("W")
    with pytest.raises(sc5.Sepconv5Error) as e:
        sc5.Plan(planes, H, W, **kw)
    assert e.value.status == sc5.EINVAL


def test_tune_lookup_defaults_without_table(sc5):
    cfg, found = sc5.tune_lookup("f32", "f32", 8192, 8192)
    assert not found and cfg["tile_w"] == 128


def test_header_compiles_as_c_and_cpp_alone(tmp_path):
    """include/sepconv5.h is self-contained: a translation unit that includes
    only it compiles as C11 and as C++17 (no CUDA headers needed)."""
    import subprocess
    inc = os.path.join(ROOT, "include")
    src_c = tmp_path / "h.c"
    src_c.write_text('#include "sepconv5.h"\nint main(void) { sc5_plan_desc d; (void)d; return (int)SC5_OK; }\n')
    src_cpp = tmp_path / "h.cpp"
    src_cpp.write_text('#include "sepconv5.h"\nint main() { sc5_pyramid_desc d{}; return d.levels; }\n')
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src_c)])
    subprocess.check_call(["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src_cpp)])
