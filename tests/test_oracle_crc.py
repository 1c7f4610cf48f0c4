"""Pins for the oracle's CRC32C (the per-4-KiB-block digest of the voted buffer).

The digest is CRC32C: Castagnoli polynomial, reflected, init and final XOR
0xFFFFFFFF.  The oracle's table form is checked against (a) published check
values (tests/golden/crc32c_vectors.txt: the standard "123456789" check value and
RFC 3720 Appendix B.4), (b) the x86 SSE4.2 CRC32 instruction, an implementation
in hardware that shares nothing with the oracle, and (c) the oracle's own
bit-at-a-time form.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _load_vectors():
    out = []
    with open(os.path.join(HERE, "golden", "crc32c_vectors.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            name, spec, crc = line.split()
            kind, _, arg = spec.partition(":")
            if kind == "ascii":
                data = arg.encode()
            elif kind == "hex":
                data = bytes.fromhex(arg)
            elif kind == "rep":
                b, k = arg.split(":")
                data = bytes([int(b, 16)]) * int(k)
            elif kind == "inc":
                b, k = arg.split(":")
                data = bytes(range(int(b, 16), int(b, 16) + int(k)))
            elif kind == "dec":
                b, k = arg.split(":")
                data = bytes(range(int(b, 16), int(b, 16) - int(k), -1))
            out.append((name, data, int(crc, 16)))
    return out


VECTORS = _load_vectors()


@pytest.mark.parametrize("name,data,crc", VECTORS, ids=[v[0] for v in VECTORS])
def test_published_vectors(name, data, crc):
    assert oracle.crc32c(data) == crc
    assert oracle.crc32c_bitwise(data) == crc


@pytest.fixture(scope="module")
def hw_crc(tmp_path_factory):
    with open("/proc/cpuinfo") as f:
        if "sse4_2" not in f.read():
            pytest.skip("host CPU has no SSE4.2")
    so = str(tmp_path_factory.mktemp("pin") / "libhwcrc.so")
    subprocess.check_call(["gcc", "-O2", "-msse4.2", "-fPIC", "-shared", "-o", so,
                           os.path.join(HERE, "pins", "crc32c_sse42.c")])
    L = ctypes.CDLL(so)
    L.hw_crc32c.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.hw_crc32c.restype = ctypes.c_uint32

    def f(b: np.ndarray) -> int:
        b = np.ascontiguousarray(b, dtype=np.uint8)
        return int(L.hw_crc32c(b.ctypes.data if b.size else None, b.size))
    return f


def test_hw_instruction_agrees_on_vectors(hw_crc):
    for name, data, crc in VECTORS:
        assert hw_crc(np.frombuffer(data, dtype=np.uint8)) == crc, name


@pytest.mark.parametrize("n", [1, 3, 15, 16, 17, 127, 128, 4095, 4096, 4097, 65536 + 13])
def test_oracle_matches_hw_random(hw_crc, n):
    rng = np.random.default_rng(n)
    b = rng.integers(0, 256, size=n, dtype=np.uint8)
    assert oracle.crc32c(b) == hw_crc(b)
    assert oracle.crc32c_bitwise(b) == hw_crc(b)


def test_block_crc_partitions(hw_crc):
    rng = np.random.default_rng(7)
    for nbytes in (0, 1, 4095, 4096, 4097, 3 * 4096 + 100):
        b = rng.integers(0, 256, size=nbytes, dtype=np.uint8)
        got = oracle.block_crc32c(b)
        assert got.size == (nbytes + 4095) // 4096
        for k in range(got.size):
            assert int(got[k]) == hw_crc(b[4096 * k: 4096 * (k + 1)])


def test_block_crc_zero_block_and_other_block_sizes(hw_crc):
    z = np.zeros(4096, dtype=np.uint8)
    assert int(oracle.block_crc32c(z)[0]) == hw_crc(z) == oracle.crc32c_bitwise(z)
    b = np.arange(10000, dtype=np.uint32).view(np.uint8)
    got = oracle.block_crc32c(b, 1000)
    assert [int(x) for x in got] == [hw_crc(b[i:i + 1000]) for i in range(0, b.size, 1000)]
