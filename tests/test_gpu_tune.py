"""The autotuner: a quick tuning pass fills one entry per size class, the
table round-trips through its JSON file, and plans pick the tuned shape."""
import json

import pytest

pytestmark = pytest.mark.gpu


def test_autotune_table_roundtrip(tmp_path):
    import torch
    from paper_1711_09791_gb300 import sepconv5 as sc5
    sc5.load()
    path = str(tmp_path / "tune.json")
    sc5.autotune(0, [])  # start from an empty table (earlier tests may have tuned other pairs)
    sc5.autotune(1, [("f32", "f32"), ("bf16", "bf16")], path)
    table = json.load(open(path))
    assert table["gpu"] == torch.cuda.get_device_name(0)
    assert len(table["entries"]) == 2 * 7 * 2  # pairs x size classes x kernel kinds
    assert {e["kind"] for e in table["entries"]} == {0, 1}
    compiled = {p: set(sc5.fused_configs(*p)) for p in [("f32", "f32"), ("bf16", "bf16")]}
    for e in table["entries"]:
        pair = ({0: "f32", 1: "bf16"}[e["in"]], {0: "f32", 1: "bf16"}[e["out"]])
        assert (e["tile_h"], e["tile_w"], e["stages"]) in compiled[pair]
        assert e["ctas"] >= 1 and e["us"] > 0
    cfg, found = sc5.tune_lookup("f32", "f32", 8192, 8192)
    cfgb, foundb = sc5.tune_lookup("f32", "f32", 8192, 8192, batch=True)
    assert found and foundb
    sc5.autotune(0, [])  # clear
    assert not sc5.tune_lookup("f32", "f32", 8192, 8192)[1]
    assert not sc5.tune_lookup("f32", "f32", 8192, 8192, batch=True)[1]
    sc5.tune_load(path)
    cfg2, found2 = sc5.tune_lookup("f32", "f32", 8192, 8192)
    assert found2 and cfg2 == cfg
    assert sc5.tune_lookup("f32", "f32", 8192, 8192, batch=True) == (cfgb, True)
    # a plan takes the single-image entry of its size class
    plan1 = sc5.Plan(3, 8192, 8192)
    assert plan1.info() == cfg
    plan1.close()
    # a batch of large images takes the tuned shape of their size class
    A = torch.zeros((3, 3000, 3000), dtype=torch.float32, device="cuda")
    out = torch.zeros((3, 2996, 2996), dtype=torch.float32, device="cuda")
    plan = sc5.Plan(3, 64, 64)
    b = sc5.Batch(plan, [{"in": A, "out": out, "H": 3000, "W": 3000, "in_pitch": 3000, "out_pitch": 2996,
                          "k": [0, 0, 1, 0, 0]}])
    want, _ = sc5.tune_lookup("f32", "f32", 2048, 4096, batch=True)  # the dominant class of one 3000^2 image
    info = b.info()
    assert (info["tile_h"], info["tile_w"]) == (want["tile_h"], want["tile_w"])
    b.launch()
    torch.cuda.synchronize()
    assert sc5.device_status() == 0
    b.close()
    plan.close()
    sc5.autotune(0, [])


def _child(code, env_extra):
    import os
    import subprocess
    import sys
    import textwrap
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if not k.startswith("SEPCONV5_TUNE")}
    env.update(env_extra, PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], env=env, capture_output=True, text=True,
                       timeout=600, cwd=root)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout.strip().splitlines()[-1]


def test_tuning_from_the_environment(tmp_path):
    """SEPCONV5_TUNE=quick with SEPCONV5_TUNE_FILE: the first plan of a dtype
    pair tunes that pair and writes the table; a later process with only
    SEPCONV5_TUNE_FILE loads it, and its plans take the tuned entries."""
    path = str(tmp_path / "env_tune.json")
    code = """
        import json
        from paper_1711_09791_gb300 import sepconv5 as sc5
        sc5.load()
        p = sc5.Plan(3, 4096, 4096, 4096, 4092, "bf16")
        info = p.info()
        p.close()
        cfg, found = sc5.tune_lookup("bf16", "bf16", 4096, 4096)
        print(json.dumps({"info": info, "cfg": cfg, "found": found}))
    """
    first = json.loads(_child(code, {"SEPCONV5_TUNE": "quick", "SEPCONV5_TUNE_FILE": path}))
    table = json.load(open(path))
    pairs = {(e["in"], e["out"]) for e in table["entries"]}
    assert pairs == {(1, 1)} and len(table["entries"]) == 2 * 7
    assert first["found"]
    second = json.loads(_child(code, {"SEPCONV5_TUNE_FILE": path}))
    assert second["found"] and second["cfg"] == first["cfg"]
    for key in ("tile_h", "tile_w", "stages", "ctas_per_sm"):
        assert second["info"][key] == second["cfg"][key], key
    # without the variables a process keeps the built-in defaults
    third = json.loads(_child(code, {}))
    assert not third["found"]
