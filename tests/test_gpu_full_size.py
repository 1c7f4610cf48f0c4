"""Parity at the full sizes of the batched and serving workloads, and at an
element count beyond 2^32 (64-bit indices).

- batched, 4096 tasks (43 GB of replicas and outputs), in the launch
  configuration bench.py times: every task equals the oracle's vote of its
  replicas and its own ft_vote, bit for bit;
- serving, the 20 000 req/s Poisson stream over 64 resident payloads: every
  payload voted alone equals the oracle, and every request reports the
  statistics of its payload voted alone;
- a u8 vote of n = 2^32 + 4113 elements with faults planted above 2^32: counts,
  64-bit first indices and the digests of the blocks around the faults follow
  from the construction (and, for the digests, from the oracle's CRC of those
  blocks)."""
import collections
import concurrent.futures as cf
import ctypes

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

from _gpu import DevTask, assert_same, desc_array

pytestmark = pytest.mark.gpu


def _check_all_against_oracle(probs_of, tasks, threads=None):
    """Every task's device result against the oracle's vote of its replicas,
    regenerated from the seeded generator (probs_of(i)) in a thread pool so
    that only a few tasks' host replicas exist at a time."""
    import os
    threads = threads or max(2, min(32, len(os.sched_getaffinity(0))))

    def one(i):
        p = probs_of(i)
        assert_same(tasks[i].result(), oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol), p.R)
        return i

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        done = list(ex.map(one, range(len(tasks))))
    assert done == list(range(len(tasks)))


def test_batched_full_size():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    specs = synth.cfg4_specs()
    tasks = [DevTask(synth.task_problem(s)) for s in specs]
    plan = ctypes.c_void_p()
    fv.check(fv.ft_plan_create(ctypes.byref(plan), desc_array(tasks), len(tasks), None), "ft_plan_create")
    try:
        fv.check(fv.ft_vote_batched(plan, fv.stream_handle()), "ft_vote_batched")
        torch.cuda.synchronize()
        got = []
        for t in tasks:     # keep the batched results, then vote each task alone into the same buffers
            got.append((t.out[:t.nbytes].clone(), t.crc[:t.nb].clone(), t.stats.clone()))
    finally:
        fv.ft_plan_destroy(plan)
    # every task against the oracle (the batched results are still in place)
    _check_all_against_oracle(lambda i: synth.task_problem(specs[i]), tasks)
    for t in tasks:
        fv.check(fv.ft_vote(ctypes.byref(t.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    for i, (t, (o, c, s)) in enumerate(zip(tasks, got)):
        assert torch.equal(o, t.out[:t.nbytes]) and torch.equal(c, t.crc[:t.nb]) and torch.equal(s, t.stats), i


@pytest.mark.parametrize("resident", [0, 2])    # 2: small requests on the resident voter kernel
def test_serving_full_stream(resident):
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    from paper_1405_2912_b300 import serving
    reqs, specs = synth.cfg5_requests()
    probs = [synth.task_problem(s, config_id=5) for s in specs]
    tasks = [DevTask(p) for p in probs]
    for t in tasks:
        fv.check(fv.ft_vote(ctypes.byref(t.desc), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    alone = [t.result() for t in tasks]
    _check_all_against_oracle(lambda i: probs[i], tasks)
    descs = []
    for t in tasks:
        d = fv.ft_vote_desc.from_buffer_copy(t.desc)
        d.stats = None
        descs.append(d)
    cfg = fv.ft_server_config(int(40e9), 4096, 3, 0, 0)
    cfg.resident = resident
    srv = ctypes.c_void_p()
    fv.check(fv.ft_server_create(ctypes.byref(srv), ctypes.byref(cfg)), "ft_server_create")
    seen = []
    res = fv.ft_result()

    def collect(t, p):
        fv.check(fv.ft_poll(srv, t, 60_000_000, ctypes.byref(res)), "ft_poll")
        assert res.status == fv.FT_OK
        seen.append((p, list(res.stats.mismatch)[:probs[p].R], list(res.stats.first_mismatch)[:probs[p].R],
                     res.stats.no_majority, res.stats.first_no_majority))

    try:
        tk = ctypes.c_uint64()
        t0 = fv.ft_clock_us()
        pending = collections.deque()
        for r in reqs:
            while fv.ft_clock_us() < t0 + r.t_arrival * 1e6:
                pass
            while True:
                rc = fv.ft_submit(srv, ctypes.byref(descs[r.payload]), ctypes.byref(tk))
                if rc == fv.FT_OK:
                    break
                # over budget: collecting the oldest result releases its share
                assert rc == fv.FT_EAGAIN and pending
                collect(*pending.popleft())
            pending.append((tk.value, r.payload))
        while pending:
            collect(*pending.popleft())
    finally:
        fv.ft_server_destroy(srv)
    assert len(seen) == len(reqs) > 15_000
    for p, mism, first, nm, fnm in seen:
        a = alone[p]
        assert mism == [int(x) for x in a["mismatch"]] and first == [int(x) for x in a["first_mismatch"]]
        assert nm == a["no_majority"] and fnm == a["first_no_majority"]
    # concurrent requests of a payload write the same values into its output
    for t, a in zip(tasks, alone):
        assert t.out[:t.nbytes].cpu().numpy().tobytes() == a["out"].tobytes()


def test_beyond_2_to_32_elements():
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    n = (1 << 32) + 4113
    x = torch.empty(n, dtype=torch.uint8, device="cuda")
    x.random_(0, 256, generator=torch.Generator(device="cuda").manual_seed(5))
    y = x.clone()
    z = x.clone()
    far = [(1 << 32) + 7, (1 << 32) + 4100, n - 1]       # the last one is in the partial last block
    for i in far:
        y[i] ^= 0x10                                      # replica 1 wrong at three places
    z[(1 << 32) + 5000 - 4113] ^= 1                       # replica 2 wrong once (index < 2^32)
    out, crc, st = fv.vote([x, y, z])
    torch.cuda.synchronize()
    s = fv.parse_stats(st, 3)
    assert s["mismatch"] == [0, 3, 1]
    assert s["first_mismatch"] == [-1, far[0], (1 << 32) + 5000 - 4113]
    assert s["no_majority"] == 0
    assert torch.equal(out, x)
    nb = (n + 4095) // 4096
    assert crc.numel() == nb
    for b in sorted({far[0] // 4096, far[1] // 4096, nb - 1, 0, nb // 2}):
        blk = x[b * 4096: min(n, (b + 1) * 4096)].cpu().numpy()
        assert int(crc[b].item()) & 0xFFFFFFFF == oracle.crc32c(blk), b
