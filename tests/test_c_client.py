"""A plain C program uses the library through include/ftvote.h alone: it
compiles and links here (no GPU needed); on a GPU it votes and checks its
results against values it works out itself."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp):
    from paper_1405_2912_b300 import build
    lib = build.build()
    exe = os.path.join(tmp, "vote_from_c")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-o", exe, os.path.join(ROOT, "tests", "c_abi", "vote_from_c.c"),
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                           lib, "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-lm",
                           "-Wl,-rpath," + os.path.dirname(lib) + ":" + os.path.join(CUDA, "lib64")])
    return exe


def test_c_client_builds(tmp_path):
    assert os.path.exists(_build(str(tmp_path)))


@pytest.mark.gpu
def test_c_client_runs(tmp_path):
    r = subprocess.run([_build(str(tmp_path))], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "C ABI OK" in r.stdout, r.stdout + r.stderr
