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


def test_job_parameters_take_the_tuning(tmp_path, monkeypatch):
    """A served job's counting parameters fill what the job leaves open from the autotuner's
    entry for its class; tuned=False keeps the library's automatic choices."""
    from paper_1705_11147_gb300 import autotune, build
    from paper_1705_11147_gb300.serve import Job
    build.build()
    n = 40_000_000
    job = Job(seq=np.zeros(0, np.uint8), qual=np.zeros(0, np.uint8),
              offsets=np.array([0, n], dtype=np.uint64), params={"k": 51, "min_depth": 2})
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("KMA_TUNE_CACHE", path)
    autotune.save_cache({autotune.cache_key(autotune._gpu_name(), 51, n): {"params": {"partitions": 6}}}, path)
    assert job.kma_params(True).partitions == 6
    assert job.kma_params(False).partitions == 0
