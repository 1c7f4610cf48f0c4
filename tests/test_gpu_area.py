"""Memory areas with a host and a device sibling (ft_area_*), after the
memory manager of Sec. IV.A and its Fig. 1 walk-through: versions, transfers
only when a sibling is older (and then only of the changed 4 KiB blocks), the
previous version kept in the other memory before a write, and a faulty run's
sibling dropped and rebuilt.  Contents are checked byte for byte."""
import ctypes
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def rt():
    L = ctypes.CDLL(os.path.join(CUDA, "lib64", "libcudart.so"))
    L.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    L.cudaMemcpy.restype = ctypes.c_int

    def to_dev(dst, arr):
        assert L.cudaMemcpy(dst, arr.ctypes.data, arr.nbytes, 1) == 0     # host to device

    def from_dev(src, n):
        out = np.empty(n, dtype=np.uint8)
        assert L.cudaMemcpy(out.ctypes.data, src, n, 2) == 0              # device to host
        return out
    return to_dev, from_dev


def test_fig1_walkthrough(rt):
    from paper_1405_2912_b300 import ftvote as fv
    to_dev, from_dev = rt
    nbytes = (4 << 20) + 1000
    nblocks = (nbytes + 4095) // 4096
    rng = np.random.default_rng(1)
    host = rng.integers(0, 256, size=nbytes, dtype=np.uint8)
    area = ctypes.c_void_p()
    fv.check(fv.ft_area_create(ctypes.byref(area), host.ctypes.data, nbytes), "ft_area_create")
    ptr, moved = ctypes.c_void_p(), ctypes.c_uint64()
    hv, dv = ctypes.c_uint64(), ctypes.c_uint64()
    sh = fv.stream_handle()

    def req(mem, acc):
        fv.check(fv.ft_area_request(area, mem, acc, ctypes.byref(ptr), sh, ctypes.byref(moved)), "request")
        return ptr.value, moved.value

    def versions():
        fv.ft_area_versions(area, ctypes.byref(hv), ctypes.byref(dv))
        return hv.value, dv.value

    def scribble(dptr, blocks, seed):
        buf = from_dev(dptr, nbytes)
        r = np.random.default_rng(seed)
        for b in blocks:
            buf[b * 4096 + int(r.integers(0, 4000))] ^= 0xA5
        to_dev(dptr, buf)
        return buf

    try:
        assert versions() == (1, 0)
        d, k = req(fv.FT_MEM_DEVICE, fv.FT_ACCESS_READ)          # first use: everything moves
        assert k == nblocks and versions() == (1, 1)
        assert from_dev(d, nbytes).tobytes() == host.tobytes()
        assert req(fv.FT_MEM_DEVICE, fv.FT_ACCESS_READ)[1] == 0   # up to date: nothing moves
        d, k = req(fv.FT_MEM_DEVICE, fv.FT_ACCESS_WRITE)          # host still holds version 1
        assert k == 0 and versions() == (1, 2)
        scribble(d, [3, 100, nblocks - 1], 5)                     # the run on the device faults ...
        fv.check(fv.ft_area_invalidate(area, fv.FT_MEM_DEVICE), "invalidate")
        assert versions() == (1, 0)
        d, k = req(fv.FT_MEM_DEVICE, fv.FT_ACCESS_WRITE)          # ... and is restarted from the host copy
        assert k == 3 and versions() == (1, 2)
        assert from_dev(d, nbytes).tobytes() == host.tobytes()
        good = scribble(d, [0, 7, 8, 9, 500], 6)                 # the restarted run succeeds
        h, k = req(fv.FT_MEM_HOST, fv.FT_ACCESS_READ)            # host reads the newest version
        assert k == 5 and versions() == (2, 2) and h == host.ctypes.data
        assert host.tobytes() == good.tobytes()
        req(fv.FT_MEM_HOST, fv.FT_ACCESS_WRITE)                  # the host writes
        assert versions() == (3, 2)
        host[[10, 20000]] ^= 1
        d, k = req(fv.FT_MEM_DEVICE, fv.FT_ACCESS_READ)          # unknown host digests: all blocks
        assert k == nblocks and versions() == (3, 3)
        assert from_dev(d, nbytes).tobytes() == host.tobytes()
        d, _ = req(fv.FT_MEM_DEVICE, fv.FT_ACCESS_WRITE)
        assert versions() == (3, 4)
        newest = scribble(d, [1, 2], 7)
        d, k = req(fv.FT_MEM_DEVICE, fv.FT_ACCESS_WRITE)         # writing the only copy of v4: back it up first
        assert k == 2 and versions() == (4, 5)
        assert host.tobytes() == newest.tobytes()
        fv.ft_area_invalidate(area, fv.FT_MEM_DEVICE)
        fv.ft_area_invalidate(area, fv.FT_MEM_HOST)
        assert fv.ft_area_request(area, fv.FT_MEM_HOST, fv.FT_ACCESS_READ, ctypes.byref(ptr), sh, None) == fv.FT_EINVAL
    finally:
        fv.ft_area_destroy(area)
