"""The serving runtime's host-only parts without a GPU: tests/c/serve_host_check.cpp
compiles against the runtime's own header and checks the arena allocator
(first fit, alignment, no overlap, one free block per free run) against a
byte-level model under seeded random allocations and releases, and the phase
log's nearest-rank percentiles and ring."""
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1711_09791_gb300", "csrc")


def test_arena_and_phase_log():
    d = tempfile.mkdtemp(prefix="sc5_serve_host_")
    exe = os.path.join(d, "serve_host_check")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "c", "serve_host_check.cpp")])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
