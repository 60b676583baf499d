"""Failure paths of the server, injected on the host (SC5_SERVE_FAULT): an
arena allocation that fails, and a slow scheduler that makes serve_poll time
out before the request completes normally.  Each case runs in a child
process so the environment variable is read fresh by serve_create."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(code, fault):
    env = dict(os.environ, SC5_SERVE_FAULT=fault, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", textwrap.dedent(code)], env=env, capture_output=True, text=True,
                       timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_arena_allocation_failure():
    out = _child("""
        import torch
        from paper_1711_09791_gb300 import sepconv5 as sc5
        sc5.load()
        try:
            sc5.Server(hbm_budget_bytes=1 << 26, dtype="bf16")
        except sc5.Sepconv5Error as e:
            assert e.status == sc5.ENOMEM, e
            print("ENOMEM")
    """, "arena_alloc")
    assert out.strip() == "ENOMEM"


def test_slow_scheduler_poll_times_out_then_completes():
    out = _child("""
        import numpy as np, torch
        from paper_1711_09791_gb300 import sepconv5 as sc5, synth
        sc5.load()
        srv = sc5.Server(hbm_budget_bytes=1 << 28, dtype="f32")
        A = torch.from_numpy(synth.image(1, 64, 68)).pin_memory()
        out = torch.zeros((3, 60, 64)).pin_memory()
        t = srv.submit({"in": A, "out": out, "H": 64, "W": 68, "in_pitch": 68, "out_pitch": 64,
                        "k": [0, 0, 1, 0, 0]})
        assert srv.poll(t, 1000) is None          # the scheduler sleeps 300 ms: 1 ms poll times out
        lat = srv.poll(t, -1)                     # then the request completes normally
        assert lat is not None and lat > 250e3, lat
        assert np.array_equal(out.numpy(), A.numpy()[:, 2:-2, 2:-2])
        srv.close()
        print("OK")
    """, "sched_delay_ms=300")
    assert out.strip() == "OK"
