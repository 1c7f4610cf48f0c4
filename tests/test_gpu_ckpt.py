"""Digest-driven checkpoints (ft_ckpt_*): only blocks whose per-4-KiB CRC32C
changed cross PCIe, and the copies are exact, checked by comparing bytes."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ckpt(nbytes, stage=0):
    from paper_1405_2912_b300 import ftvote as fv
    c = ctypes.c_void_p()
    fv.check(fv.ft_ckpt_create(ctypes.byref(c), nbytes, stage), "ft_ckpt_create")
    return c


@pytest.mark.parametrize("nbytes,stage", [((64 << 20) + 123, 0), (4096 * 10, 4096 * 3), (5000, 0)])
def test_sync_moves_only_changed_blocks(nbytes, stage):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    rng = np.random.default_rng(nbytes)
    dev = torch.from_numpy(rng.integers(0, 256, size=nbytes, dtype=np.uint8)).cuda()
    host = np.zeros(nbytes, dtype=np.uint8)
    c = _ckpt(nbytes, stage)
    nblocks = (nbytes + 4095) // 4096
    moved = ctypes.c_uint64()
    sh = fv.stream_handle()
    try:
        fv.check(fv.ft_ckpt_sync(c, dev.data_ptr(), host.ctypes.data, sh, ctypes.byref(moved)), "sync")
        assert moved.value == nblocks
        assert host.tobytes() == dev.cpu().numpy().tobytes()
        fv.check(fv.ft_ckpt_sync(c, dev.data_ptr(), host.ctypes.data, sh, ctypes.byref(moved)), "sync")
        assert moved.value == 0
        # change a few bytes in some blocks (the last, partial one included)
        k = min(nblocks, 37)
        blocks = np.append(rng.choice(nblocks - 1, size=k - 1, replace=False), nblocks - 1)
        for b in blocks:
            off = int(b) * 4096 + int(rng.integers(0, min(4096, nbytes - int(b) * 4096)))
            dev[off] ^= 0x5A
        torch.cuda.synchronize()
        fv.check(fv.ft_ckpt_sync(c, dev.data_ptr(), host.ctypes.data, sh, ctypes.byref(moved)), "sync")
        assert moved.value == k
        assert host.tobytes() == dev.cpu().numpy().tobytes()
    finally:
        fv.ft_ckpt_destroy(c)


def test_restore_uploads_only_differing_blocks():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    nbytes = (8 << 20) + 7
    rng = np.random.default_rng(3)
    data = rng.integers(0, 256, size=nbytes, dtype=np.uint8)
    dev = torch.from_numpy(data).cuda()
    host = np.empty_like(data)
    c = _ckpt(nbytes)
    moved = ctypes.c_uint64()
    sh = fv.stream_handle()
    try:
        fv.check(fv.ft_ckpt_sync(c, dev.data_ptr(), host.ctypes.data, sh, ctypes.byref(moved)), "sync")
        # a faulty run scribbles over 11 blocks; roll back
        for b in rng.choice(nbytes // 4096, size=11, replace=False):
            dev[int(b) * 4096: int(b) * 4096 + 100] = 0
        torch.cuda.synchronize()
        fv.check(fv.ft_ckpt_restore(c, dev.data_ptr(), host.ctypes.data, sh, ctypes.byref(moved)), "restore")
        assert moved.value == 11
        assert dev.cpu().numpy().tobytes() == data.tobytes()
        fv.check(fv.ft_ckpt_restore(c, dev.data_ptr(), host.ctypes.data, sh, ctypes.byref(moved)), "restore")
        assert moved.value == 0
    finally:
        fv.ft_ckpt_destroy(c)
    # restore without a prior sync uploads everything
    c = _ckpt(nbytes)
    try:
        dev.zero_()
        fv.check(fv.ft_ckpt_restore(c, dev.data_ptr(), data.ctypes.data, sh, ctypes.byref(moved)), "restore")
        assert moved.value == (nbytes + 4095) // 4096
        assert dev.cpu().numpy().tobytes() == data.tobytes()
    finally:
        fv.ft_ckpt_destroy(c)


def test_dense_changes_copy_the_whole_buffer():
    """More than an eighth of a buffer of 64 MiB or more changed: sync and
    restore copy the whole buffer at once (all blocks reported moved); a
    sparse change still moves only its blocks.  Contents are checked each time."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    nbytes = (64 << 20) + 4096 * 3 + 100
    nblocks = (nbytes + 4095) // 4096
    rng = np.random.default_rng(4)
    dev = torch.from_numpy(rng.integers(0, 256, size=nbytes, dtype=np.uint8)).cuda()
    host = torch.zeros(nbytes, dtype=torch.uint8).pin_memory()
    c = _ckpt(nbytes)
    moved = ctypes.c_uint64()
    sh = fv.stream_handle()

    def sync():
        fv.check(fv.ft_ckpt_sync(c, dev.data_ptr(), host.data_ptr(), sh, ctypes.byref(moved)), "sync")
        assert torch.equal(host.cuda(), dev)
        return moved.value

    def damage(frac):
        idx = torch.from_numpy(rng.choice(nblocks - 1, size=int((nblocks - 1) * frac), replace=False)).cuda()
        dev[:(nblocks - 1) * 4096].view(nblocks - 1, 4096)[idx, 5] += 1
        return int(idx.numel())

    try:
        assert sync() == nblocks                      # first sync: every block, one copy
        damage(0.2)
        assert sync() == nblocks                      # dense: the whole buffer
        k = damage(0.01)
        assert sync() == k                            # sparse: only the changed blocks
        saved = host.clone()
        damage(0.3)
        fv.check(fv.ft_ckpt_restore(c, dev.data_ptr(), host.data_ptr(), sh, ctypes.byref(moved)), "restore")
        assert moved.value == nblocks and torch.equal(dev.cpu(), saved)
        k = damage(0.005)
        fv.check(fv.ft_ckpt_restore(c, dev.data_ptr(), host.data_ptr(), sh, ctypes.byref(moved)), "restore")
        assert moved.value == k and torch.equal(dev.cpu(), saved)
    finally:
        fv.ft_ckpt_destroy(c)
