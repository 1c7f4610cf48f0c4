"""Task duplication followed by the vote (ft_dmr_run, Sec. IV.D) with the
paper's Listing 1 task (increase an array of floats), run heterogeneously:
replica 0 on the GPU, replica 1 on the CPU with a different operation order,
and (R = 3) a replica from a faulty kernel.  The CPU and GPU results differ in
the last bits; the paper's 0.1 % delta (FT_PAPER_F32_REL_TOL) accepts that, a
zero tolerance does not, and the faulty replica is outvoted.  Results are
compared with the oracle on the replicas the tasks produced.  Also
ft_vote_registered against ft_vote."""
import ctypes

import numpy as np
import pytest

import oracle

from _gpu import assert_same

pytestmark = pytest.mark.gpu

N = (1 << 20) + 3


def _make(R, faulty):
    import torch
    rng = np.random.default_rng(11)
    x = rng.uniform(-100, 100, size=N).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    reps = [torch.empty(N, dtype=torch.float32, device="cuda") for _ in range(R)]

    def task(user, r, out, stream):
        t = reps[r]
        assert out == t.data_ptr()
        if r == 0:                       # GPU kernel
            torch.mul(xd, 1.0009765625, out=t)
            t.add_(0.1)
        elif r == 1:                     # CPU kernel, other operation order, float64 then rounded
            t.copy_(torch.from_numpy(((x.astype(np.float64) + 0.1 / 1.0009765625) * 1.0009765625)
                                     .astype(np.float32)))
        else:                            # a faulty kernel: wrong on a stretch of elements
            torch.mul(xd, 1.0009765625, out=t)
            t.add_(0.1)
            t[1000:5000] += 1.0
        return 0

    return reps, task


@pytest.mark.parametrize("R,faulty", [(2, False), (3, True)])
def test_heterogeneous_dmr(R, faulty):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    reps, task = _make(R, faulty)
    cb = fv.ft_task_fn(task)
    for rel, expect_clean in ((fv.FT_PAPER_F32_REL_TOL, True), (0.0, False)):
        out = torch.empty(N, dtype=torch.float32, device="cuda")
        crc = torch.empty(fv.n_blocks(4 * N), dtype=torch.int32, device="cuda")
        st = fv.new_stats()
        d = fv.make_desc(reps, out, crc, st, 0.0, rel)
        fv.check(fv.ft_dmr_run(cb, None, ctypes.byref(d), fv.stream_handle()), "ft_dmr_run")
        torch.cuda.synchronize()
        host = [r.cpu().numpy() for r in reps]
        ref = oracle.vote(host, "f32", 0.0, rel)
        s = fv.parse_stats(st, R)
        got = {"out": out.cpu().numpy(), "block_crc": crc.cpu().numpy().view(np.uint32),
               "mismatch": np.array(s["mismatch"], dtype=np.uint64),
               "first_mismatch": np.array(s["first_mismatch"], dtype=np.int64),
               "no_majority": s["no_majority"], "first_no_majority": s["first_no_majority"],
               "raw_stats": st.cpu().numpy()}
        assert_same(got, ref, R)
        # the CPU and GPU kernels really differ in the last bits somewhere
        assert not np.array_equal(host[0], host[1])
        if expect_clean:
            assert s["mismatch"][0] == 0 and s["mismatch"][1] == 0
            if faulty:
                assert s["mismatch"][2] == 4000 and s["first_mismatch"][2] == 1000
                assert s["no_majority"] == 0
        else:
            assert s["mismatch"][1] > 0 or s["no_majority"] > 0


def test_vote_registered_equals_vote():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    rng = np.random.default_rng(4)
    a = torch.from_numpy(rng.standard_normal(100_003).astype(np.float64)).cuda()
    reps = [a, a.clone(), a.clone()]
    reps[2][7] += 1.0
    out1 = torch.empty_like(a)
    fv.check(fv.ft_register_data(out1.data_ptr(), out1.numel() * 8, fv.DTYPE["f64"], 0.0, 1e-12), "register")
    try:
        crc1 = torch.empty(fv.n_blocks(out1.numel() * 8), dtype=torch.int32, device="cuda")
        st1 = fv.new_stats()
        ptrs = (ctypes.c_void_p * 3)(*[r.data_ptr() for r in reps])
        fv.check(fv.ft_vote_registered(ptrs, 3, out1.data_ptr(), crc1.data_ptr(), st1.data_ptr(),
                                       fv.stream_handle()), "ft_vote_registered")
        out2, crc2, st2 = fv.vote(reps, 0.0, 1e-12)
        torch.cuda.synchronize()
        assert torch.equal(out1, out2) and torch.equal(crc1, crc2) and torch.equal(st1, st2)
        assert fv.parse_stats(st1, 3)["mismatch"] == [0, 0, 1]
    finally:
        fv.ft_unregister_data(out1.data_ptr())
