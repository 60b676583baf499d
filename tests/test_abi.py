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
        # 128-wide tiles for every pair; 256-wide ones (8 columns per lane) for 8/16-bit inputs
        widths = (128,) if pair[0] == "f32" else (128, 256)
        assert cfgs and all(tw in widths and th % 8 == 0 and 32 <= th + 4 <= 256 and st >= 2 for th, tw, st in cfgs)
        assert cfgs[0][1] == 128 or pair[0] != "f32"
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


def test_tune_table_load_and_lookup(sc5, tmp_path):
    """A tuning table read by sepconv5_tune_load: entries are found by the size
    class of the plane area (one class per factor of 4 from 2^14 pixels) and by
    kernel kind, an entry naming a shape that is not compiled is dropped, and a
    table written for another GPU is refused.  Without a device the table key
    is the name "unknown"."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("the table key is the device's name; this test writes the no-device key")
    cfgs = sc5.fused_configs("f32", "f32")
    (th1, tw1, st1), (th2, tw2, st2) = cfgs[0], cfgs[1]

    def entry(kind, cls, th, tw, st, ctas):
        return (f' {{"in": 0, "out": 0, "kind": {kind}, "cls": {cls}, "tile_h": {th}, "tile_w": {tw}, '
                f'"stages": {st}, "ctas": {ctas}, "us": 1.000}}')

    def write(gpu, entries):
        p = tmp_path / f"{gpu.replace(' ', '_')}.json"
        p.write_text('{"gpu": "%s", "entries": [\n' % gpu + ",\n".join(entries) + "\n]}\n")
        return str(p)

    try:
        sc5.autotune(0, [])
        table = write("unknown", [entry(0, 2, th1, tw1, st1, 2), entry(1, 2, th2, tw2, st2, 1),
                                  entry(0, 4, 24, 128, 3, 1)])
        sc5.tune_load(table)
        # 256 x 256 = 2^16 and 300 x 300 (log2 = 16.5) are class 2; 64 x 64 is class 0
        for H, W in ((256, 256), (300, 300)):
            cfg, found = sc5.tune_lookup("f32", "f32", H, W)
            assert found and (cfg["tile_h"], cfg["tile_w"], cfg["stages"], cfg["ctas_per_sm"]) == (th1, tw1, st1, 2)
            cfg, found = sc5.tune_lookup("f32", "f32", H, W, batch=True)
            assert found and (cfg["tile_h"], cfg["tile_w"], cfg["stages"], cfg["ctas_per_sm"]) == (th2, tw2, st2, 1)
        assert not sc5.tune_lookup("f32", "f32", 64, 64)[1]
        assert not sc5.tune_lookup("bf16", "bf16", 256, 256)[1]
        # class 4 (2^20 .. 2^22 pixels) named a 24-row tile, which is not compiled
        cfg, found = sc5.tune_lookup("f32", "f32", 1024, 2048)
        assert not found and cfg["ctas_per_sm"] == 0
        with pytest.raises(sc5.Sepconv5Error) as e:
            sc5.tune_load(write("Another GPU", [entry(0, 0, th1, tw1, st1, 1)]))
        assert e.value.status == sc5.ENOTFOUND
        assert not sc5.tune_lookup("f32", "f32", 64, 64)[1]
    finally:
        sc5.autotune(0, [])
    assert not sc5.tune_lookup("f32", "f32", 256, 256)[1]


def test_binding_structs_match_header(tmp_path):
    """The binding's ctypes structures have the header's field names, offsets
    and sizes: a C program compiled against include/sepconv5.h prints
    offsetof/sizeof for every field the binding declares."""
    import ctypes
    import subprocess
    from paper_1711_09791_gb300 import sepconv5
    structs = {"sc5_plan_desc": sepconv5.PlanDesc, "sc5_image": sepconv5.Image,
               "sc5_pyramid_desc": sepconv5.PyramidDesc, "sc5_serve_cfg": sepconv5.ServeCfg,
               "sc5_serve_stats": sepconv5.ServeStats}
    rename = {"in_": "in"}  # a Python keyword in the binding
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sepconv5.h"', "int main(void) {"]
    expect = []
    for cname, py in structs.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        expect.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            lines.append(f'printf("%zu %zu\\n", offsetof({cname}, {rename.get(fname, fname)}), '
                         f'sizeof((({cname} *)0)->{rename.get(fname, fname)}));')
            f = getattr(py, fname)
            expect.append((f.offset, f.size))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                           str(src)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = [int(x) if " " not in x else tuple(int(v) for v in x.split()) for x in out if x]
    assert got == expect


def _c_param_kind(param: str) -> str:
    import re
    p = re.sub(r"\bconst\b", "", param).strip()
    if "*" in p or "[" in p or re.match(r"(sc5_plan|sc5_batch|sc5_server|sc5_pyramid)\b", p):
        return "ptr"
    base = p.split()[0]
    return {"int32_t": "i32", "int": "i32", "int64_t": "i64", "uint64_t": "u64", "float": "f32",
            "double": "f64", "size_t": "size"}[base]


def test_binding_signatures_match_header(sc5):
    """Every function the header declares is bound with the same number of
    parameters, each of the same kind (pointer, 32/64-bit integer, float,
    double), and returns a 32-bit status."""
    import ctypes
    import re
    text = open(sc5.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"^SC5_API\s+([\w\s\*]+?)\b((?:sepconv5|serve)_\w+)\s*\(([^)]*)\)\s*;", text, re.M)
    assert len(protos) == len(sc5.header_symbols())
    lib = sc5.load()
    kinds = {ctypes.c_int32: "i32", ctypes.c_int64: "i64", ctypes.c_uint64: "u64", ctypes.c_float: "f32",
             ctypes.c_double: "f64", ctypes.c_void_p: "ptr", ctypes.c_char_p: "ptr"}
    for ret, name, params in protos:
        params = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        want = [_c_param_kind(p) for p in params]
        f = getattr(lib, name)
        got = [kinds.get(a, "ptr" if issubclass(a, ctypes._Pointer) else "?") for a in (f.argtypes or [])]
        assert got == want, (name, got, want)
        if "sc5_status" in ret:
            assert f.restype is ctypes.c_int32, name
