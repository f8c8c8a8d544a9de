"""Latency statistics of the serving loop, on the CPU: the split into the wait for a worker and
the service time, and the median of the largest quarter of the jobs."""
from types import SimpleNamespace

import numpy as np


def _job(arrival, start, done, n_bases):
    return SimpleNamespace(arrival=arrival, t_start=start, t_done=done,
                           offsets=np.array([0, n_bases], dtype=np.uint64), n_bases=n_bases)


def test_latency_split_and_size_classes():
    from paper_1705_11147_gb300.serve import Server
    # 8 jobs: the four small ones wait 10 ms and take 10 ms, the four large ones wait 0 and take 90 ms
    done = [_job(1.0 * i, 1.0 * i + 0.010, 1.0 * i + 0.020, 1000) for i in range(4)]
    done += [_job(10.0 + i, 10.0 + i, 10.0 + i + 0.090, 10 ** 9) for i in range(4)]
    fake = SimpleNamespace(done=done, batches=8)
    st = Server.latency_stats(fake)
    assert st["jobs"] == 8 and st["batches"] == 8
    assert abs(st["p50_ms_largest_quarter"] - 90.0) < 1e-6
    assert abs(st["p50_ms_rest"] - 20.0) < 1e-6
    assert abs(st["p99_wait_ms"] - 10.0) < 1e-3
    assert abs(st["p99_service_ms"] - 90.0) < 0.1
    assert abs(st["mean_ms"] - 55.0) < 1e-6
    assert Server.latency_stats(SimpleNamespace(done=[], batches=0)) == {"jobs": 0}
