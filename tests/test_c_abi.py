"""The C ABI from plain C: tests/c/abi_example.c includes only sepconv5.h
(and the CUDA runtime), is compiled with gcc and linked against
libsepconv5.so.  Host-only calls run without a GPU; the GPU variant checks
an identity convolution bit for bit, the plan's reported launch
configuration, and one pyramid REDUCE step (level sizes, pitch, values)."""
import os
import subprocess
import tempfile

import pytest

from paper_1711_09791_gb300 import build as sc5_build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def example():
    lib = sc5_build.build()
    d = tempfile.mkdtemp(prefix="sc5_cabi_")
    exe = os.path.join(d, "abi_example")
    cmd = ["gcc", "-std=c11", "-O1", "-o", exe, os.path.join(HERE, "c", "abi_example.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", os.path.dirname(lib), "-lsepconv5", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"]
    subprocess.check_call(cmd)
    return exe


def test_c_program_host_calls(example):
    r = subprocess.run([example, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "OK"


@pytest.mark.gpu
def test_c_program_on_gpu(example):
    r = subprocess.run([example, "gpu"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "OK"
