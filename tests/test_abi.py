"""The C-ABI library loads, exports every entry point declared in
include/ftvote.h, and validates arguments on the host (no GPU needed: invalid
calls are rejected before any CUDA work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ftvote.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ft_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def fv():
    from paper_1405_2912_b300 import build
    build.build()
    from paper_1405_2912_b300 import ftvote
    return ftvote


def test_exports_every_declared_symbol(fv):
    names = _declared()
    assert "ft_vote" in names and "ft_poll" in names
    lib = ctypes.CDLL(fv.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version(fv):
    assert fv.ft_strerror(fv.FT_EINVAL) == b"invalid argument"
    assert fv.ft_version().startswith(b"ftvote")


def _desc(fv, **kw):
    d = fv.ft_vote_desc()
    d.R, d.dtype, d.n = 3, fv.DTYPE["f32"], 1024
    for r in range(3):
        d.replicas[r] = 0x10000 * (r + 1)
    d.out, d.stats, d.block_crc = 0x100000, 0x200000, 0x300000
    d.abs_tol, d.rel_tol = 1e-6, 1e-5
    for k, v in kw.items():
        if k == "rep1":
            d.replicas[1] = v
        else:
            setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [
    dict(R=1), dict(R=9), dict(dtype=7), dict(dtype=-1), dict(stats=None), dict(stats=0x200004),
    dict(out=None), dict(out=0x100008), dict(rep1=0x20008), dict(rep1=None),
    dict(abs_tol=-1.0), dict(rel_tol=float("nan")), dict(rel_tol=1.5), dict(abs_tol=1e300),
    dict(abs_tol=float("inf")), dict(block_crc=0x300002),
    dict(out=0x10000),            # out overlaps replica 0
    dict(block_crc=0x100000),     # digest overlaps out
])
def test_invalid_descriptors(fv, bad):
    d = _desc(fv, **bad)
    assert fv.ft_vote(ctypes.byref(d), None) == fv.FT_EINVAL
    assert fv.ft_vote(None, None) == fv.FT_EINVAL


def test_integer_types_ignore_tolerances_in_validation(fv):
    d = _desc(fv, dtype=fv.DTYPE["i32"], rel_tol=float("nan"), R=1)
    assert fv.ft_vote(ctypes.byref(d), None) == fv.FT_EINVAL   # R still checked


def test_digest_argument_checks(fv):
    assert fv.ft_digest(0x1000, 100, 4000, 0x2000, None) == fv.FT_EINVAL
    assert fv.ft_digest(0x1000, 100, 0, 0x2000, None) == fv.FT_EINVAL
    assert fv.ft_digest(0x1001, 100, 4096, 0x2000, None) == fv.FT_EINVAL
    assert fv.ft_digest(0x1000, 100, 4096, 0x2001, None) == fv.FT_EINVAL
    assert fv.ft_digest(0x1000, 0, 4096, 0x2000, None) == fv.FT_OK   # nothing to do


def test_server_config_validation(fv):
    srv = ctypes.c_void_p()
    for bad in [(0, 16, 2, 8, 0), (1 << 30, 0, 2, 8, 0), (1 << 30, 16, 0, 8, 0), (1 << 30, 16, 9, 8, 0),
                (1 << 30, 16, 2, 65, 0), (1 << 30, 16, 2, -1, 0), (1 << 30, 16, 2, 8, -1),
                (1 << 30, 16, 2, 8, 0, 0, -2)]:
        cfg = fv.ft_server_config(*bad)
        assert fv.ft_server_create(ctypes.byref(srv), ctypes.byref(cfg)) == fv.FT_EINVAL
    for resident in (-1, 3):
        cfg = fv.ft_server_config(1 << 30, 16, 2, 8, 0)
        cfg.resident = resident
        assert fv.ft_server_create(ctypes.byref(srv), ctypes.byref(cfg)) == fv.FT_EINVAL
    assert fv.ft_server_create(None, None) == fv.FT_EINVAL
    assert fv.ft_submit(None, None, None) == fv.FT_EINVAL
    assert fv.ft_poll(None, 1, 0, None) == fv.FT_EINVAL
    acc, nd = ctypes.c_int32(7), ctypes.c_int32(7)
    assert fv.ft_submit_many(None, None, 0, None, ctypes.byref(acc)) == fv.FT_EINVAL
    assert fv.ft_poll_many(None, None, 0, 0, None, ctypes.byref(nd)) == fv.FT_EINVAL
    assert fv.ft_server_info(None, None) == fv.FT_EINVAL
    assert fv.ft_server_destroy(None) == fv.FT_EINVAL
    assert fv.ft_plan_destroy(None) == fv.FT_EINVAL
    assert fv.ft_vote_batched(None, None) == fv.FT_EINVAL


def test_clock_is_monotonic(fv):
    import time
    a = fv.ft_clock_us()
    time.sleep(0.01)
    b = fv.ft_clock_us()
    assert b - a >= 9000


def test_ckpt_argument_checks(fv):
    c = ctypes.c_void_p()
    assert fv.ft_ckpt_create(ctypes.byref(c), 0, 0) == fv.FT_EINVAL
    assert fv.ft_ckpt_create(None, 100, 0) == fv.FT_EINVAL
    assert fv.ft_ckpt_sync(None, 0x1000, 0x2000, None, None) == fv.FT_EINVAL
    assert fv.ft_ckpt_restore(None, 0x1000, 0x2000, None, None) == fv.FT_EINVAL
    assert fv.ft_ckpt_destroy(None) == fv.FT_EINVAL


def test_area_argument_checks(fv):
    a = ctypes.c_void_p()
    p = ctypes.c_void_p()
    assert fv.ft_area_create(ctypes.byref(a), None, 100) == fv.FT_EINVAL
    assert fv.ft_area_create(ctypes.byref(a), 0x1000, 0) == fv.FT_EINVAL
    assert fv.ft_area_request(None, 0, 1, ctypes.byref(p), None, None) == fv.FT_EINVAL
    assert fv.ft_area_invalidate(None, 0) == fv.FT_EINVAL
    assert fv.ft_area_destroy(None) == fv.FT_EINVAL
    assert fv.ft_ckpt_forget(None) == fv.FT_EINVAL
