"""The CRC32C tables and formulation of the CUDA kernels, checked on the CPU.

tests/host/crc_formulation.cu includes the kernels' own compile-time tables
(common.cuh) and digests bytes the way the kernels do: per-lane registers over
interleaved vectors with the shifted slicing tables and the per-lane combine
tables for full 4 KiB blocks, per-lane segments and the x^(8*2^j) shift
tables for a partial block.  Its block CRCs must equal the oracle's; the
multiplication by x^(8k) through the shift tables must equal the bit-serial
power.  The GPU parity tests check the kernels themselves."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("crc") / "crc_formulation")
    subprocess.check_call([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(ROOT, "paper_1405_2912_b300", "csrc"),
                           os.path.join(HERE, "host", "crc_formulation.cu"), "-o", exe])
    return exe


def _run(exe, data):
    out = subprocess.run([exe], input=data.tobytes(), capture_output=True, check=True).stdout.decode().split()
    assert out[-2:] == ["shift", "ok"], out[-2:]
    return np.array([int(x, 16) for x in out[:-2]], dtype=np.uint32)


@pytest.mark.parametrize("nbytes", [4096, 3 * 4096, 5 * 4096 + 1, 7 * 4096 + 2999, 4095, 1, 17])
def test_block_crcs_match_the_oracle(prog, nbytes):
    data = np.random.default_rng(nbytes).integers(0, 256, size=nbytes, dtype=np.uint8)
    got = _run(prog, data)
    ref = oracle.block_crc32c(data)
    assert np.array_equal(got, ref)


def test_zero_and_constant_blocks(prog):
    for fill in (0x00, 0xFF, 0x5A):
        data = np.full(2 * 4096 + 100, fill, dtype=np.uint8)
        assert np.array_equal(_run(prog, data), oracle.block_crc32c(data))
