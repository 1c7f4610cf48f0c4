"""The end of bench.py's JSON line: the batched and serving summaries come
last and, with figures of the widest plausible size, fit within the last
1500 characters, so that a reader who keeps only the tail of the line still
sees all three parts of the metric."""
import json

import bench


def _arm(server, big):
    v = 123456.7 if big else 161.1
    a = {"p50_us": v, "p99_us": v, "req_per_s": 60166.6, "max_us": v, "submit_lag_p50_us": v,
         "p99_us_replays": [v] * 7}
    if server:
        a.update({"mean_requests_per_batch": 1.95, "launch_host_us_per_batch": 10.1, "batches": 30000})
    return a


def test_summaries_fit_the_tail():
    batched = {"tasks": 4096, "tasks_per_s": 625882.6, "gb_per_s": 6531.6,
               "per_task_launches": {"tasks_per_s": 55612.8}, "speedup_vs_per_task": 11.25,
               "noalloc": {"tasks_per_s": 615303.1}, "one_kernel_for_the_batch": {"tasks_per_s": 569204.5},
               "launches_per_batch": 4, "tune": {"groups": ["f32 R=3: 16 warps + L2 prefetch"] * 3}}
    serving = {rate: {"continuous_batching": _arm(True, True), "batch_launch": _arm(True, True),
                      "unbatched": _arm(True, True), "plain_ft_vote": _arm(False, True)}
               for rate in ("at_20k_req_per_s", "at_60k_req_per_s")}
    line = {"value": 6809.0, "batched": bench.batched_summary(batched), "serving": bench.serving_summary(serving)}
    text = json.dumps(line)
    tail = text[text.index('"batched"'):]
    assert len(tail) < 1500, len(tail)
    # every part of the metric is in the tail
    for key in ("tasks_per_s", "speedup_vs_per_task", "p50_us", "p99_us", "plain_ft_vote",
                "batch_launch", "continuous_batching", "unbatched", "at_60k_req_per_s"):
        assert key in tail
