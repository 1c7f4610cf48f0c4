"""Benchmark of the majority voter on the 256M-element f32 workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload f32x3-256M|f32x3-1M|f64x5-64M|i32x5-64M]

One step = one ft_vote of the workload, by default R=3 replicas of 2^28 float32
(1 GiB per replica): the whole hot path (load, compare, vote, store,
statistics, CRC32C per 4 KiB block).  The metric is voter GB/s with bytes =
(R+1) * n * sizeof(element) (R reads + 1 write).  The default inputs (4 GiB)
exceed the 126 MB L2, so no flush is needed between steps.  The same line
carries the digest, batched, serving and size-sweep measurements.  Prints one
JSON line (rank 0).

--impl reference times the CPU oracle (the plain C voter under oracle/) on the
host cores over a bounded sample of the same workload.
Under torchrun each rank votes its own copy of the workload on its own GPU
(weak scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1405_2912_b300 import synth  # noqa: E402

METRIC = "voter input GB/s & % of HBM peak; batched tasks/s; p50/p99 vote latency"
WORKLOADS = {
    "f32x3-256M": "3 x 256M float32 replicas (lognormal sigma 2, random sign; +-1..4 ULP on 20% of replica 1; "
                  "bit flips at 1e-6/element in replica 2), abs_tol 1e-6, rel_tol 1e-5, CRC32C per 4 KiB block "
                  "of the voted buffer",
    "f32x3-1M": "3 x 1M float32 replicas (uniform [-1, 1]; +-1..2 ULP on 10% of replica 1; 100 bit flips in "
                "replica 2), abs_tol 1e-6, rel_tol 1e-5, CRC32C per 4 KiB block",
    "f64x5-64M": "5 x 64M float64 replicas (lognormal sigma 2; replica 3 wrong on a 1M-element block, bit flips "
                 "at 1e-5 in replicas 1 and 4, 1024 tie sites), rel_tol 1e-12, CRC32C per 4 KiB block",
    "i32x5-64M": "5 x 64M int32 replicas (uniform; replica 3 wrong on a 1M-element block, bit flips at 1e-5 in "
                 "replicas 1 and 4, 1024 tie sites), bit-wise, CRC32C per 4 KiB block",
}


def make_problem(args):
    """The workload of the timed step (the 256M-element f32 vote by default)."""
    if args.workload == "f32x3-256M":
        return synth.cfg2(n=args.n)
    if args.workload == "f32x3-1M":
        return synth.cfg1()
    f64, i32 = synth.cfg3()
    return f64 if args.workload == "f64x5-64M" else i32


FALLBACK_HBM_GBS = 6400.0
L2_BYTES = 126 << 20


KERNEL_SOURCES = ("paper_1405_2912_b300/csrc/common.cuh", "paper_1405_2912_b300/csrc/vote_kernel.cuh",
                  "paper_1405_2912_b300/csrc/vote.cu")
TRAFFIC_FILES = {"f32x3-256M": "profiles/vote_f32_r3_256M_dram.txt",
                 "f64x5-64M": "profiles/vote_f64_r5_64M_dram.txt",
                 "i32x5-64M": "profiles/vote_i32_r5_64M_dram.txt"}


def kernel_sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(workload="f32x3-256M"):
    """DRAM bytes (read + write) of one voter launch on the workload, from the
    ncu capture recorded in TRAFFIC_FILES, if the kernel sources are still the
    ones it was taken on; else None."""
    if workload not in TRAFFIC_FILES:
        return None
    path = os.path.join(ROOT, TRAFFIC_FILES[workload])
    if not os.path.exists(path):
        return None
    kv = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if "=" in line:
                k, v = (x.strip() for x in line.split("=", 1))
                kv[k] = v
    if kv.get("kernel_sources_sha256") != kernel_sources_hash():
        return None
    return float(kv["dram_bytes_read_per_launch"]) + float(kv["dram_bytes_write_per_launch"])


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def warm_up(steps, step, stream, min_seconds=0.2):
    """At least `steps` untimed steps, run right before the timed region and
    continued until `min_seconds` of wall time have passed (synchronising every
    16 steps), so that the GPU has left its idle clocks when timing starts.
    Without it, a short timed region after an idle pause (the clock sampler's
    start-up) ran ~16 ms slower in total."""
    t0 = time.perf_counter()
    k = 0
    while k < steps or time.perf_counter() - t0 < min_seconds:
        step()
        k += 1
        if k % 16 == 0:
            stream.synchronize()
    stream.synchronize()
    return k


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ftvote_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_run(problem, n_sample: int, threads: int) -> tuple:
    """Time the oracle on the first n_sample elements, split into 4 KiB-aligned
    chunks voted concurrently on `threads` host threads.  Returns (seconds,
    bytes)."""
    import oracle
    oracle.build()
    per = max(1024, (n_sample // threads) // 1024 * 1024)
    bounds = [(s, min(n_sample, s + per)) for s in range(0, n_sample, per)]

    def one(b):
        s, e = b
        oracle.vote([r[s:e] for r in problem.replicas], problem.dtype, problem.abs_tol, problem.rel_tol)

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, bounds))
    dt = time.perf_counter() - t0
    return dt, (problem.R + 1) * n_sample * problem.itemsize


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def config_of(problem, ws, workload):
    nb = problem.bytes_moved
    copies = max(2, -(-2 * L2_BYTES // nb))
    l2 = (f"inputs ({nb / 2**30:.2f} GiB per step) exceed the 126 MB L2; no flush" if nb > L2_BYTES
          else f"inputs ({nb / 2**20:.0f} MiB per step) fit in L2: {copies} copies of them "
               f"({copies * nb / 2**20:.0f} MiB) are voted in rotation, back to back, so that each vote reads "
               "replicas evicted from L2 by the votes since its copy's last turn")
    return {"workload": WORKLOADS[workload], "R": problem.R, "n": problem.n, "bytes_per_step": nb, "l2": l2,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}


def run_reference(args, problem):
    cores = host_cores()
    n_sample = min(problem.n, args.ref_sample)
    for _ in range(args.warmup if args.warmup < 2 else 1):
        oracle_run(problem, min(n_sample, 1 << 20), cores)
    times = []
    nbytes = 0
    for _ in range(args.steps):
        dt, nbytes = oracle_run(problem, n_sample, cores)
        times.append(dt)
    total = sum(times)
    gbs = nbytes * args.steps / total / 1e9
    sample = f"first {n_sample} of {problem.n} elements per step, 4 KiB-aligned chunks on {cores} threads"
    line = {"impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": problem.dtype, "data": "synthetic",
            "config": config_of(problem, 1, args.workload),
            "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args, problem, ws, rank, local):
    import torch
    from paper_1405_2912_b300 import ftvote as fv

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    sh = int(stream.cuda_stream)
    R, n = problem.R, problem.n
    nbytes = n * problem.itemsize
    reps = [torch.from_numpy(r.view(np.uint8)).to(dev) for r in problem.replicas]
    out = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    nblk = fv.n_blocks(nbytes)
    crc = torch.empty(nblk, dtype=torch.int32, device=dev)
    stats = fv.new_stats(dev)
    desc = fv.make_desc(reps, out, crc, stats, problem.abs_tol, problem.rel_tol, dtype=problem.dtype, n=n)
    pd = ctypes.byref(desc)
    # Inputs that fit in L2 are voted from several copies in rotation, whose
    # buffers together exceed twice the L2, so that each vote reads replicas
    # that later votes evicted from L2 (the timing rule's "inputs larger than
    # L2"), back to back as a stream of small votes runs.
    small = problem.bytes_moved <= L2_BYTES
    copies = max(2, -(-2 * L2_BYTES // problem.bytes_moved)) if small else 1
    sets = [(reps, out, crc, stats, desc)]
    for _ in range(copies - 1):
        r2 = [x.clone() for x in reps]
        o2, c2, s2 = torch.empty_like(out), torch.empty_like(crc), fv.new_stats(dev)
        sets.append((r2, o2, c2, s2, fv.make_desc(r2, o2, c2, s2, problem.abs_tol, problem.rel_tol,
                                                  dtype=problem.dtype, n=n)))
    pds = [ctypes.byref(x[4]) for x in sets]
    torch.cuda.synchronize()

    ev_start, ev_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    rot = [0]

    def one_vote():
        fv.check(fv.ft_vote(pds[rot[0] % copies], sh), "ft_vote")
        rot[0] += 1

    warm_steps = warm_up(args.warmup, one_vote, stream)
    launches0 = fv.ft_launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev_start.record(stream)
        for k in range(args.steps):
            fv.ft_vote(pds[k % copies], sh)
        ev_end.record(stream)
    torch.cuda.synchronize()
    elapsed = ev_start.elapsed_time(ev_end) / 1e3                      # s, whole timed region
    barrier(ws)
    launches = fv.ft_launch_count() - launches0
    clocks = sampler.stop()
    alone_us = None
    if small:
        # for context: one vote timed alone between two events right after a
        # write of four times the L2 (replicas and CRC tables come from HBM)
        scrub = torch.empty(4 * L2_BYTES, dtype=torch.uint8, device=dev)
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(30)]
        with torch.cuda.stream(stream):
            for k, (a, b) in enumerate(pairs):
                scrub.fill_(k & 0xFF)
                a.record(stream)
                fv.ft_vote(pd, sh)
                b.record(stream)
        torch.cuda.synchronize()
        alone_us = round(statistics.median(a.elapsed_time(b) * 1e3 for a, b in pairs), 2)
        del scrub
    del sets[1:]
    t_max = max_over_ranks(elapsed, ws)
    bytes_step = problem.bytes_moved
    value = bytes_step * args.steps * ws / t_max / 1e9
    launch_ms = 1e3 * elapsed / args.steps      # back-to-back launches on one stream: the mean per ft_vote
    peak, peak_kind = peaks()
    achieved = bytes_step / (launch_ms / 1e3) / 1e9

    # end to end through the host-buffer entry point: ft_vote_host uploads the
    # pinned replicas, votes and downloads the voted bytes, digests and
    # statistics in pipelined chunks, and returns when the host holds them
    e2e = None
    if args.e2e_steps > 0:
        host = [torch.from_numpy(r.view(np.uint8)).pin_memory() for r in problem.replicas]
        out_h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        crc_h = torch.empty(nblk, dtype=torch.int32).pin_memory()
        stats_h = fv.ft_stats()
        dh = fv.ft_vote_desc.from_buffer_copy(desc)
        for r, h in enumerate(host):
            dh.replicas[r] = h.data_ptr()
        dh.out, dh.block_crc, dh.stats = out_h.data_ptr(), crc_h.data_ptr(), ctypes.addressof(stats_h)
        chunk = 64 << 20
        fv.check(fv.ft_vote_host(ctypes.byref(dh), chunk), "ft_vote_host")      # staging allocated here
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            fv.check(fv.ft_vote_host(ctypes.byref(dh), chunk), "ft_vote_host")
        t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
        nchunks = (nbytes + chunk - 1) // chunk
        e2e = {"value": round(bytes_step * args.e2e_steps * ws / t_e2e / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": R * nbytes, "d2h_bytes_per_step": nbytes + 4 * nblk + 144 * nchunks,
               "steps": args.e2e_steps, "call": "ft_vote_host (pinned host buffers, 64 MiB chunks)",
               "matches_device_vote": bool(np.array_equal(crc_h.numpy(), crc.cpu().numpy()))}
        # the same copies alone, in the same chunks, uploads on one stream and
        # the download on another: the ceiling that the link sets for e2e (the
        # device replicas are overwritten with their own contents)
        up_s, down_s = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

        def copies():
            for off in range(0, nbytes, chunk):
                end = min(off + chunk, nbytes)
                with torch.cuda.stream(up_s):
                    for r in range(R):
                        reps[r][off:end].copy_(host[r][off:end], non_blocking=True)
                with torch.cuda.stream(down_s):
                    out_h[off:end].copy_(out[off:end], non_blocking=True)
            torch.cuda.synchronize()

        copies()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            copies()
        t_copy = max_over_ranks(time.perf_counter() - t0, ws)
        e2e["copy_only_gb_per_s"] = round(bytes_step * args.e2e_steps * ws / t_copy / 1e9, 3)
        e2e["frac_of_copy_only"] = round(e2e["value"] / e2e["copy_only_gb_per_s"], 3)
        del host, out_h

    s = fv.parse_stats(stats, R)
    digest = None
    if args.digest_reps > 0:
        # ft_digest alone over the voted buffer (n * 4 bytes read per call)
        dout = torch.empty_like(crc)
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for _ in range(3):
                fv.check(fv.ft_digest(out.data_ptr(), nbytes, 4096, dout.data_ptr(), sh), "ft_digest")
            d0.record(stream)
            for _ in range(args.digest_reps):
                fv.ft_digest(out.data_ptr(), nbytes, 4096, dout.data_ptr(), sh)
            d1.record(stream)
        torch.cuda.synchronize()
        t_d = d0.elapsed_time(d1) / 1e3 / args.digest_reps
        digest = {"bytes_per_call": nbytes, "gb_per_s": round(nbytes / t_d / 1e9, 1),
                  "us_per_call": round(t_d * 1e6, 1), "matches_fused_digest": bool(torch.equal(dout, crc))}
    del reps, out, crc, sets
    # the batched and serving forms are measured on a single-rank run (each is a
    # whole-GPU workload of its own; a scaling run times the vote step only)
    batched = run_batched(args, dev, stream) if args.batched_tasks > 0 and ws == 1 else None
    serving = run_serving(args, dev) if args.serve_seconds > 0 and ws == 1 else None
    size_sweep = run_size_sweep(args, dev) if args.size_sweep and ws == 1 else None
    next_rows = run_next_rows(args, dev) if args.next_rows and ws == 1 else None
    if rank != 0:
        return
    cpu = None
    if args.cpu_sample > 0 and ws == 1:
        cores = host_cores()
        n_s = min(n, args.cpu_sample)
        dt, b = oracle_run(problem, n_s, cores)
        cpu = {"value": round(b / dt / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"first {n_s} of {n} elements, 4 KiB-aligned chunks on {cores} threads, one pass"}
    # The detailed sections come first and the compact summaries of the
    # batched and serving forms last, so that the end of the line (what a
    # tail of the output shows) carries all three parts of the metric.
    line = {
        "size_sweep": size_sweep,
        "next_rows": next_rows,
        "digest": digest,
        "batched_detail": batched,
        "serving_detail": serving,
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "warmup_steps_run": warm_steps,
        "ms_per_step": round(1e3 * t_max / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": problem.dtype,
        "data": "synthetic",
        "config": config_of(problem, ws, args.workload),
        "hbm_frac_of_8tbs_spec": round(value / ws / 8000.0, 4),
        "us_per_vote": round(1e6 * t_max / args.steps, 2),
        "us_per_vote_alone_after_l2_flush": alone_us,
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": args.traffic if args.traffic is not None else (
                         measured_traffic(args.workload) if args.workload != "f32x3-256M" or n == 1 << 28
                         else None),
                     "kernel": f"vote_kernel<{problem.dtype},R={R}> (one ft_vote: one launch, statistics "
                               "through a library slot)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "result": {"mismatch": s["mismatch"], "no_majority": s["no_majority"]},
        "digest_gb_per_s": digest["gb_per_s"] if digest else None,
        "batched": batched_summary(batched),
        "serving": serving_summary(serving),
    }
    print(json.dumps(line), flush=True)


def batched_summary(b):
    """The batched figures that the end of the JSON line carries (the tuned
    launch shapes are in batched_detail: the batched and serving summaries
    together stay within the last 1500 characters of the line)."""
    if not b:
        return None
    out = {"tasks": b["tasks"], "tasks_per_s": b["tasks_per_s"], "gb_per_s": b["gb_per_s"],
           "per_task_launches_tasks_per_s": b["per_task_launches"]["tasks_per_s"],
           "speedup_vs_per_task": b["speedup_vs_per_task"],
           "noalloc_tasks_per_s": b["noalloc"]["tasks_per_s"] if b.get("noalloc") else None,
           "one_kernel_tasks_per_s": b["one_kernel_for_the_batch"]["tasks_per_s"],
           "launches_per_batch": b["launches_per_batch"]}
    return out


def _r(x):
    return None if x is None else round(x)


def serving_summary(sv):
    """p50 / p99 latency and throughput of each serving arm at each rate."""
    if not sv:
        return None
    out = {}
    for rate_key in ("at_20k_req_per_s", "at_60k_req_per_s"):
        r = sv.get(rate_key)
        if not r:
            continue
        arms = {}
        for arm in ("continuous_batching", "batch_launch", "unbatched", "plain_ft_vote"):
            a = r.get(arm)
            if not a:
                continue
            # to the microsecond and the request per second; every replay's
            # p99 beside the median for continuous batching and plain ft_vote
            # (the other arms' in serving_detail)
            reps = a.get("p99_us_replays")
            arms[arm] = {"p50_us": _r(a["p50_us"]), "p99_us": _r(a["p99_us"]), "req_per_s": _r(a["req_per_s"])}
            if arm in ("continuous_batching", "plain_ft_vote"):
                arms[arm]["p99_us_replays"] = [round(x) for x in reps] if reps else reps
            if arm == "continuous_batching" and "launch_host_us_per_batch" in a:
                arms[arm]["launch_host_us_per_batch"] = a["launch_host_us_per_batch"]
        out[rate_key] = arms
    return out


def device_tasks(specs, dev, config_id, threads, stats_ptr=True):
    """Generate each task's replicas with the seeded generator (a thread pool,
    in bounded chunks) and upload them; returns the device buffers and a
    ctypes array of descriptors."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    n = len(specs)
    keep = []
    descs = (fv.ft_vote_desc * n)()
    stats = torch.empty((n, 18), dtype=torch.int64, device=dev)
    nbytes_total = 0
    chunk = max(threads * 4, 16)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for c0 in range(0, n, chunk):
            probs = list(ex.map(lambda sp: synth.task_problem(sp, config_id=config_id), specs[c0:c0 + chunk]))
            for k, p in enumerate(probs):
                i = c0 + k
                reps = [torch.from_numpy(r.view(np.uint8)).to(dev, non_blocking=False) for r in p.replicas]
                nb = p.n * p.itemsize
                out = torch.empty(max(nb, 16), dtype=torch.uint8, device=dev)
                crc = torch.empty(max(1, fv.n_blocks(nb)), dtype=torch.int32, device=dev)
                descs[i] = fv.make_desc(reps, out, crc, stats[i] if stats_ptr else None, p.abs_tol, p.rel_tol,
                                        dtype=p.dtype, n=p.n)
                keep.append((reps, out, crc))
                nbytes_total += p.bytes_moved
    return keep, descs, stats, nbytes_total


def run_batched(args, dev, stream):
    """4096 tasks (n log-uniform 1K..4M, f32/f64/i32 40/30/30 %, R=3, one
    faulty replica in 5 % of the tasks): one graph-replayed batched vote
    against 4096 plain ft_vote calls (ft_vote_many) on the same buffers, and
    the same batch through ft_vote_batched_noalloc."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    specs = synth.cfg4_specs(ntasks=args.batched_tasks)
    t0 = time.perf_counter()
    keep, descs, stats, nbytes = device_tasks(specs, dev, 4, host_cores())
    gen_s = time.perf_counter() - t0
    sh = int(stream.cuda_stream)
    plan = ctypes.c_void_p()
    t0 = time.perf_counter()
    fv.check(fv.ft_plan_create(ctypes.byref(plan), descs, len(specs), None), "ft_plan_create")
    plan_s = time.perf_counter() - t0
    tune = fv.ft_tune()
    fv.ft_plan_tune(plan, ctypes.byref(tune))
    ng = ctypes.c_int32()
    fv.ft_plan_groups(plan, None, 0, ctypes.byref(ng))
    garr = (fv.ft_plan_group * max(1, ng.value))()
    fv.ft_plan_groups(plan, garr, ng.value, ctypes.byref(ng))
    dname = {v: k for k, v in fv.DTYPE.items()}
    groups = [{"dtype": dname[g.dtype], "R": g.R, "tasks": g.tasks, "warps": g.warps,
               "l2_prefetch": bool(g.l2_prefetch)} for g in list(garr)[:ng.value]]

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    l0 = fv.ft_launch_count()
    t_b = timed(lambda: fv.check(fv.ft_vote_batched(plan, sh), "batched"), args.batched_reps)
    launches_b = (fv.ft_launch_count() - l0) // (args.batched_reps + 3)
    t_p = timed(lambda: fv.check(fv.ft_vote_many(descs, len(specs), sh), "many"), max(2, args.batched_reps // 4))
    # the same batch through the entry point that allocates nothing (no plan,
    # no graph: the batch is laid out in static buffers on every call)
    noalloc = None
    if len(specs) <= fv.FT_NOALLOC_MAX_TASKS:
        t_n = timed(lambda: fv.check(fv.ft_vote_batched_noalloc(descs, len(specs), tune.tile_blocks, sh), "noalloc"),
                    args.batched_reps)
        noalloc = {"tasks_per_s": round(len(specs) / t_n, 1), "gb_per_s": round(nbytes / t_n / 1e9, 1),
                   "ms_per_batch": round(t_n * 1e3, 3)}
    fv.ft_plan_destroy(plan)
    # the same batch as one persistent kernel for all groups (the tuner's
    # other candidate), tile size as chosen above
    one = fv.ft_tune(tune.tile_blocks, 0, 0, 0, 1)
    plan1 = ctypes.c_void_p()
    fv.check(fv.ft_plan_create(ctypes.byref(plan1), descs, len(specs), ctypes.byref(one)), "ft_plan_create")
    t_1 = timed(lambda: fv.check(fv.ft_vote_batched(plan1, sh), "batched"), args.batched_reps)
    fv.ft_plan_destroy(plan1)
    del keep, stats
    torch.cuda.empty_cache()
    return {"workload": f"{len(specs)} tasks, n log-uniform [2^10, 2^22], f32/f64/i32 40/30/30 %, R=3, "
                        "one replica with bit flips (1e-4/element) in 5 % of tasks",
            "tasks": len(specs),
            "tasks_per_s": round(len(specs) / t_b, 1), "gb_per_s": round(nbytes / t_b / 1e9, 1),
            "ms_per_batch": round(t_b * 1e3, 3), "bytes_per_batch": nbytes,
            "launches_per_batch": int(launches_b),
            "tune": {"tile_blocks": tune.tile_blocks,
                     "kernels": "one for the batch" if tune.kernels == 1 else "one per (dtype, R) group",
                     "groups": [f"{g['dtype']} R={g['R']}: {g['warps']} warps"
                                f"{' + L2 prefetch' if g['l2_prefetch'] else ''}" for g in groups]},
            "per_task_launches": {"tasks_per_s": round(len(specs) / t_p, 1), "gb_per_s": round(nbytes / t_p / 1e9, 1),
                                  "ms_per_batch": round(t_p * 1e3, 3)},
            "speedup_vs_per_task": round(t_p / t_b, 2),
            "one_kernel_for_the_batch": {"tasks_per_s": round(len(specs) / t_1, 1),
                                         "gb_per_s": round(nbytes / t_1 / 1e9, 1)},
            "noalloc": noalloc,
            "setup_s": {"generate_upload": round(gen_s, 1), "plan_create_autotune": round(plan_s, 2)}}


# CUDA streams of every serving arm (batches or requests in flight at once).
# Continuous batching at 20k requests/s, p99 over two replays each: 3 streams
# 179-185 us, 4 streams 158-163 us, 6 streams 160-171 us; at 60k 4 streams
# keep the p99 of 3 (0.53-0.59 ms) and 6 raise it (0.80-0.88 ms).
SERVE_STREAMS = 4


def run_serving(args, dev):
    """Poisson arrivals of votes with n log-uniform 4K..16M, R in {3, 5},
    f32/f64, under a 40 GB budget, replicas resident: continuous batching
    (the server's shared mode: requests with fewer 4 KiB output blocks than
    the resident voter's warps to the resident voter on the 32 SMs that the
    batches leave free, the others in batches capped at 1 GB of request
    bytes) against the same server with every request batched and launched,
    against one-request batches on the same 4 streams, and against plain
    ft_vote calls issued at each arrival on 4 streams in turn (no server), at
    the workload's 20k requests/s and at three times that load."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    from paper_1405_2912_b300 import serving
    _, specs = synth.cfg5_requests(duration_s=args.serve_seconds, rate=args.serve_rate, pool=args.serve_pool)
    keep, descs, _, _ = device_tasks(specs, dev, 5, host_cores(), stats_ptr=False)
    # per-stream copies of the descriptors with statistics buffers, for the
    # plain per-request arm (ft_vote needs them; the server keeps its own)
    plain_stats = torch.empty((SERVE_STREAMS, len(specs), 18), dtype=torch.int64, device=dev)
    plain_descs = []
    for si in range(SERVE_STREAMS):
        row = []
        for p in range(len(specs)):
            d = fv.ft_vote_desc.from_buffer_copy(descs[p])
            d.stats = plain_stats[si, p].data_ptr()
            row.append(d)
        plain_descs.append(row)
    # one vote of every payload before any replay: with lazy module loading a
    # kernel's first launch costs 0.1-0.4 ms of host time, which the plain arm
    # would otherwise pay inside its stream (a server loads its kernels when it
    # is created)
    for p in range(len(specs)):
        fv.check(fv.ft_vote(ctypes.byref(plain_descs[0][p]), fv.stream_handle()), "ft_vote")
    torch.cuda.synchronize()
    out = {"workload": f"Poisson arrivals for {args.serve_seconds} s, n log-uniform [2^12, 2^24], R in {{3,5}}, "
                       f"f32/f64 50/50, 40 GB budget, {len(specs)} resident payloads, {SERVE_STREAMS} streams",
           "batch_cap_bytes": 1 << 30}
    for label, rate in (("at_20k_req_per_s", args.serve_rate), ("at_60k_req_per_s", 3 * args.serve_rate)):
        reqs, _ = synth.cfg5_requests(duration_s=args.serve_seconds, rate=rate, pool=args.serve_pool)
        arrivals = np.array([r.t_arrival for r in reqs])
        payload = np.array([r.payload for r in reqs])
        per_req = np.array([(specs[r.payload].R + 1) * r.n * (4 if r.dtype == "f32" else 8) for r in reqs])
        res = {"offered_gb_per_s": round(float(per_req.sum()) / args.serve_seconds / 1e9, 1)}
        # each arm replays the stream serve_reps times, the arms taking turns,
        # and reports the replay with the median p99 (every replay's p50 and
        # p99 are listed beside it): one replay's tail moves with the host's
        # scheduling
        warm = min(len(reqs), 300)
        runs = {"plain_ft_vote": [], "continuous_batching": [], "batch_launch": [], "unbatched": []}
        for _ in range(max(1, args.serve_reps)):
            # the plain arm: one ft_vote per request on the streams in turn, no server
            serving.replay_plain(plain_descs, arrivals[:warm] - arrivals[0], payload[:warm], nstreams=SERVE_STREAMS)
            r = serving.replay_plain(plain_descs, arrivals, payload, nstreams=SERVE_STREAMS)
            runs["plain_ft_vote"].append(serving.summarize(r, per_req))
            # continuous batching: small requests to the resident voter on the
            # SMs the batches leave free, the others batched and launched;
            # batch_launch: every request batched and launched
            for name, slots, cap, resident in (("continuous_batching", 4096, 1 << 30, 2),
                                               ("batch_launch", 4096, 1 << 30, 0), ("unbatched", 1, 0, 0)):
                cfg = fv.ft_server_config(int(40e9), slots, SERVE_STREAMS, 0, 0, cap)
                cfg.resident = resident
                srv = ctypes.c_void_p()
                fv.check(fv.ft_server_create(ctypes.byref(srv), ctypes.byref(cfg)), "ft_server_create")
                try:
                    serving.replay(srv, descs, arrivals[:warm] - arrivals[0], payload[:warm])
                    info0 = fv.ft_server_stats()
                    fv.ft_server_info(srv, ctypes.byref(info0))
                    r = serving.replay(srv, descs, arrivals, payload)
                    info = fv.ft_server_stats()
                    fv.ft_server_info(srv, ctypes.byref(info))
                finally:
                    fv.ft_server_destroy(srv)
                sm = serving.summarize(r, per_req)
                nb = info.batches - info0.batches
                sm.update({"batches": int(nb),
                           "mean_requests_per_batch": round((info.requests - info0.requests) / max(1, nb), 2),
                           "max_batches_in_flight": int(info.max_batches_in_flight),
                           # worker host time to lay out and launch a batch, and a
                           # batch's launch -> completion span, per batch
                           "launch_host_us_per_batch": round((info.launch_host_us - info0.launch_host_us)
                                                             / max(1, nb), 1),
                           "batch_span_us_mean": round((info.batch_span_us - info0.batch_span_us) / max(1, nb), 1)})
                runs[name].append(sm)
        for name, lst in runs.items():
            order = sorted(range(len(lst)), key=lambda k: lst[k]["p99_us"])
            res[name] = dict(lst[order[len(lst) // 2]])
            res[name]["p50_us_replays"] = [x["p50_us"] for x in lst]
            res[name]["p99_us_replays"] = [x["p99_us"] for x in lst]
        out[label] = res
    del keep, plain_stats
    torch.cuda.empty_cache()
    return out


def run_next_rows(args, dev):
    """The extension rows measured on their own workloads.

    checkpoint (Sec. IV.A, IV.C): a 1 GiB device buffer kept in sync with a
    pinned host copy by ft_ckpt_sync, which moves only the 4 KiB blocks whose
    digest changed: the first sync (every block), syncs after 1 % and after
    0 % of the blocks changed, and a restore of the 1 %, against one plain
    device-to-host copy of the whole buffer.  Synchronous calls, wall time.

    dmr (Sec. IV.D): the paper's Listing 1 task (increase an array of floats,
    here y = 1.0009765625 * x + 0.1 on 64M floats on the GPU) run once, against
    ft_dmr_run: the task twice, then the R = 2 vote with the paper's 0.1 %
    delta.  CUDA events, median of 20.

    rating (Sec. IV.B, V.C): the seeded simulation of the paper's injection
    experiment (rating_sim): mean time per result of the fault-aware choice
    and of avoiding the faulty unit after its first fault, across fault
    probabilities.

    hetdmr (Sec. IV.D, heterogeneous DMR): the task's GPU result resident on
    the device and its CPU result in pinned host memory (here the GPU result
    with 1-ULP differences on 10 % of the elements, standing in for CPU
    rounding), voted by ft_vote_host with the voted buffer and digests left on
    the device: only the host result crosses PCIe.  Against uploading the
    host result and then calling ft_vote.  Wall time of the synchronous
    calls, median of 10."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    out = {}
    # ---- checkpoint
    nbytes = 1 << 30
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    buf = torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device=dev, generator=g)
    host = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    ck = ctypes.c_void_p()
    fv.check(fv.ft_ckpt_create(ctypes.byref(ck), nbytes, 0), "ft_ckpt_create")
    blocks = ctypes.c_uint64()
    sh = fv.stream_handle()

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3

    try:
        full_copy = min(timed(lambda: host.copy_(buf)) for _ in range(3))
        first = timed(lambda: fv.check(fv.ft_ckpt_sync(ck, buf.data_ptr(), host.data_ptr(), sh,
                                                        ctypes.byref(blocks)), "ft_ckpt_sync"))
        first_blocks = blocks.value
        nblk = nbytes // 4096
        idx = torch.randperm(nblk, device=dev, generator=g)[: nblk // 100]
        view = buf.view(nblk, 4096)
        view[idx, 17] += 1
        changed = timed(lambda: fv.check(fv.ft_ckpt_sync(ck, buf.data_ptr(), host.data_ptr(), sh,
                                                          ctypes.byref(blocks)), "ft_ckpt_sync"))
        changed_blocks = blocks.value
        same = timed(lambda: fv.check(fv.ft_ckpt_sync(ck, buf.data_ptr(), host.data_ptr(), sh,
                                                       ctypes.byref(blocks)), "ft_ckpt_sync"))
        same_blocks = blocks.value
        ok = bool(torch.equal(host[: 1 << 20].to(dev), buf[: 1 << 20]))
        view[idx, 17] += 1              # a faulty run damages the same blocks; roll back
        restore = timed(lambda: fv.check(fv.ft_ckpt_restore(ck, buf.data_ptr(), host.data_ptr(), sh,
                                                             ctypes.byref(blocks)), "ft_ckpt_restore"))
        restore_blocks = blocks.value
        ok = ok and bool(torch.equal(view[idx[:64]].cpu(), host.view(nblk, 4096)[idx[:64].cpu()]))
    finally:
        fv.ft_ckpt_destroy(ck)
    out["checkpoint"] = {
        "workload": "1 GiB device buffer, pinned host copy, 4 KiB blocks; 1 % = random blocks with one byte changed",
        "full_copy_ms": round(full_copy, 2), "first_sync_ms": round(first, 2), "first_sync_blocks": first_blocks,
        "sync_1pct_ms": round(changed, 2), "sync_1pct_blocks": changed_blocks,
        "sync_unchanged_ms": round(same, 2), "sync_unchanged_blocks": same_blocks,
        "restore_1pct_ms": round(restore, 2), "restore_1pct_blocks": restore_blocks,
        "speedup_1pct_vs_full_copy": round(full_copy / changed, 1), "contents_match": ok}
    del buf, host
    torch.cuda.empty_cache()
    # ---- task duplication
    n = 1 << 26
    x = torch.rand(n, dtype=torch.float32, device=dev, generator=g) * 200 - 100
    reps = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    yv = torch.empty(n, dtype=torch.float32, device=dev)
    crc = torch.empty(fv.n_blocks(4 * n), dtype=torch.int32, device=dev)
    st = fv.new_stats(dev)

    def task(user, r, ptr, stream):
        torch.mul(x, 1.0009765625, out=reps[r])
        reps[r].add_(0.1)
        return 0

    cb = fv.ft_task_fn(task)
    d = fv.make_desc(reps, yv, crc, st, 0.0, fv.FT_PAPER_F32_REL_TOL)

    def ev_ms(fn, k=20):
        ts = []
        for _ in range(3):
            fn()
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    single = ev_ms(lambda: task(None, 0, 0, 0))
    dmr = ev_ms(lambda: fv.check(fv.ft_dmr_run(cb, None, ctypes.byref(d), fv.stream_handle()), "ft_dmr_run"))
    s = fv.parse_stats(st, 2)
    from paper_1405_2912_b300 import rating_sim
    qs = [0.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.65, 0.7, 0.8, 0.9]
    rows = rating_sim.sweep(qs, rounds=4000, seed=1)
    out["rating"] = {
        "workload": "Sec. V.C experiment, simulated: a CPU kernel 3x faster than the GPU kernel faults with "
                    "probability q; mean time per valid result (CPU runtime = 1), 4000 results per q",
        "rows": rows,
        "crossover_expected": round(1 - 1 / 3, 3),
        "paper": "expected crossover 66 %, observed 70 %; fault-aware > 2x faster than avoiding the CPU after "
                 "its first fault at q = 10 %",
        "speedup_at_q10": round(rows[1]["avoid_after_first_fault"] / rows[1]["fault_aware"], 2)}
    out["dmr"] = {"workload": "y = 1.0009765625 * x + 0.1 on 2^26 f32 (two GPU kernels per run), R = 2, rel_tol 1e-3",
                  "single_ms": round(single, 3), "dmr_ms": round(dmr, 3), "overhead": round(dmr / single, 2),
                  "mismatch": s["mismatch"], "paper_overhead_range": "x1 to x3 (Sec. V.B)"}
    # ---- heterogeneous DMR: one result on the device, one in host memory
    n_h = n
    gpu_y = reps[0]
    cpu_np = gpu_y.cpu().numpy().copy()
    idx = np.flatnonzero(np.random.default_rng(11).random(n_h) < 0.1)
    synth.ulp_perturb(cpu_np, idx, np.ones(idx.size, dtype=np.int64))
    cpu_y = torch.from_numpy(cpu_np).pin_memory()
    hst = fv.ft_stats()
    dh = fv.make_desc([gpu_y, cpu_y], yv, crc, None, 0.0, fv.FT_PAPER_F32_REL_TOL, dtype="f32", n=n_h)
    dh.stats = ctypes.addressof(hst)
    staged = torch.empty_like(gpu_y)
    dd = fv.make_desc([gpu_y, staged], yv, crc, st, 0.0, fv.FT_PAPER_F32_REL_TOL, dtype="f32", n=n_h)

    def wall_ms(fn, k=10):
        ts = []
        for _ in range(2):
            fn()
        for _ in range(k):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(ts)

    def upload_then_vote():
        staged.copy_(cpu_y, non_blocking=True)
        fv.check(fv.ft_vote(ctypes.byref(dd), fv.stream_handle()), "ft_vote")

    het = wall_ms(lambda: fv.check(fv.ft_vote_host(ctypes.byref(dh), 0), "ft_vote_host"))
    seq = wall_ms(upload_then_vote)
    hs = fv.parse_stats(st, 2)
    out["hetdmr"] = {"workload": "R = 2 f32, 2^26 elements: GPU result on the device, CPU result (1-ULP "
                                 "differences on 10 %) in pinned host memory, rel_tol 1e-3; voted buffer and "
                                 "digests left on the device",
                     "ft_vote_host_ms": round(het, 3), "upload_then_ft_vote_ms": round(seq, 3),
                     "voter_gb_per_s": round(3 * 4 * n_h / het / 1e6, 1),
                     "h2d_bytes": 4 * n_h, "mismatch": [int(hst.mismatch[0]), int(hst.mismatch[1])],
                     "same_as_device_vote": [int(hst.mismatch[r]) for r in range(2)] == hs["mismatch"]}
    del x, reps, yv, crc, cpu_y, staged
    torch.cuda.empty_cache()
    return out


def run_size_sweep(args, dev):
    """Voter time against result size, after the paper's comparison of its
    single-thread, OpenMP and GPU voter kernels (Sec. V.A): R = 2 (DMR) f32
    results of 1 KB to 256 MB, resident in each unit's memory (transfers
    excluded, as in the paper).  GPU: median wall time of one synchronous
    ft_vote.  CPU: the oracle on one thread and on all host cores (4 KiB-aligned
    chunks), up to 64 MB."""
    import torch
    from paper_1405_2912_b300 import ftvote as fv
    import oracle
    oracle.build()
    cores = host_cores()
    rng = np.random.default_rng(99)
    rows = []
    for kb in (1, 4, 16, 64, 256, 1024, 4096, 16384, 65536, 262144):
        n = kb * 256                          # f32 elements per replica
        a = rng.standard_normal(n).astype(np.float32)
        b = a.copy()
        b[::97] = np.nextafter(b[::97], np.float32(np.inf))
        p = synth.Problem([a, b], "f32", *synth.TOL["f32"])
        reps = [torch.from_numpy(x).to(dev) for x in (a, b)]
        out = torch.empty_like(reps[0])
        crc = torch.empty(fv.n_blocks(4 * n), dtype=torch.int32, device=dev)
        st = fv.new_stats(dev)
        d = fv.make_desc(reps, out, crc, st, p.abs_tol, p.rel_tol)
        pd = ctypes.byref(d)
        sh = fv.stream_handle()
        # the oracle runs between sizes leave the GPU idle: warm it up again
        warm_up(3, lambda: fv.ft_vote(pd, sh), torch.cuda.current_stream())
        ts = []
        for _ in range(21):
            t0 = time.perf_counter()
            fv.ft_vote(pd, sh)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        row = {"kb_per_result": kb, "gpu_us": round(statistics.median(ts) * 1e6, 1)}
        if kb <= 65536:
            c1 = []
            for _ in range(3 if kb <= 4096 else 1):
                t0 = time.perf_counter()
                oracle.vote([a, b], "f32", p.abs_tol, p.rel_tol)
                c1.append(time.perf_counter() - t0)
            row["cpu_1thread_us"] = round(min(c1) * 1e6, 1)
            cn = [oracle_run(p, n, cores)[0] for _ in range(3 if kb <= 4096 else 1)]
            row[f"cpu_{cores}threads_us"] = round(min(cn) * 1e6, 1)
        rows.append(row)
    fastest = []
    for r in rows:
        cand = {k[:-3]: v for k, v in r.items() if k.endswith("_us")}
        fastest.append((r["kb_per_result"], min(cand, key=cand.get)))
    return {"workload": "R=2 (DMR) f32 results with 1 ULP differences on 1 % of elements, resident in the "
                        "voting unit's memory", "rows": rows,
            "fastest_by_size_kb": fastest}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="f32x3-256M", choices=sorted(WORKLOADS),
                    help="the timed vote (default: the 256M-element f32 vote)")
    ap.add_argument("--n", type=int, default=1 << 28, help="elements per replica of the f32x3-256M workload")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=1 << 28, help="elements the oracle votes for cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=1 << 26, help="elements per reference step")
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per launch, if measured")
    ap.add_argument("--digest-reps", type=int, default=50, help="timed ft_digest calls on the voted buffer (0 = skip)")
    ap.add_argument("--size-sweep", type=int, default=1, help="voter time against result size, GPU vs CPU (0 = skip)")
    ap.add_argument("--next-rows", type=int, default=1, help="checkpoint and task-duplication measurements (0 = skip)")
    ap.add_argument("--batched-tasks", type=int, default=4096, help="tasks of the batched workload (0 = skip)")
    ap.add_argument("--batched-reps", type=int, default=20)
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="length of the request stream (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--serve-reps", type=int, default=7, help="replays of each serving arm (the median p99 is reported)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        if rank != 0:
            return 0
        problem = make_problem(args)
        run_reference(args, problem)
        return 0
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    problem = make_problem(args)
    run_ours(args, problem, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
