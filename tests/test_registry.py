"""The value-type registry (ft_register_data and friends, after the paper's
dls_register_data, Sec. IV.E): host-side bookkeeping, no GPU needed."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def fv():
    from paper_1405_2912_b300 import build
    build.build()
    from paper_1405_2912_b300 import ftvote
    return ftvote


def test_register_lookup_unregister(fv):
    base = 0x7000_0000_0000
    assert fv.ft_register_data(base, 4096 * 4, fv.DTYPE["f32"], 0.0, fv.FT_PAPER_F32_REL_TOL) == fv.FT_OK
    dt, at, rt, nb = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    args = [ctypes.byref(x) for x in (dt, at, rt, nb)]
    assert fv.ft_registered_type(base + 100, *args) == fv.FT_OK
    assert (dt.value, at.value, rt.value, nb.value) == (fv.DTYPE["f32"], 0.0, 1e-3, 4096 * 4 - 100)
    assert fv.ft_registered_type(base + 4096 * 4, *args) == fv.FT_ENOTFOUND
    assert fv.ft_registered_type(base - 1, *args) == fv.FT_ENOTFOUND
    # overlapping areas are refused, adjacent ones accepted
    assert fv.ft_register_data(base + 4096, 16, fv.DTYPE["i32"], 0, 0) == fv.FT_EINVAL
    assert fv.ft_register_data(base - 8, 16, fv.DTYPE["i32"], 0, 0) == fv.FT_EINVAL
    assert fv.ft_register_data(base + 4096 * 4, 16, fv.DTYPE["i32"], 0, 0) == fv.FT_OK
    assert fv.ft_unregister_data(base + 4096 * 4) == fv.FT_OK
    assert fv.ft_unregister_data(base) == fv.FT_OK
    assert fv.ft_unregister_data(base) == fv.FT_ENOTFOUND


@pytest.mark.parametrize("bad", [(0, 16, 5, 0, 0), (0x1000, 0, 5, 0, 0), (0x1000, 6, 5, 0, 0),
                                 (0x1000, 16, 9, 0, 0), (0x1000, 16, 5, -1.0, 0), (0x1000, 16, 5, 0, 2.0)])
def test_register_rejects(fv, bad):
    assert fv.ft_register_data(*bad) == fv.FT_EINVAL


def test_vote_registered_needs_a_registered_output(fv):
    reps = (ctypes.c_void_p * 3)(0x10000, 0x20000, 0x30000)
    assert fv.ft_vote_registered(reps, 3, 0x40000, None, 0x50000, None) == fv.FT_ENOTFOUND
    assert fv.ft_vote_registered(reps, 1, 0x40000, None, 0x50000, None) == fv.FT_EINVAL
    assert fv.ft_dmr_run(fv.ft_task_fn(lambda *a: 0), None, None, None) == fv.FT_EINVAL
