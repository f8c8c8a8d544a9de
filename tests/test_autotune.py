"""Autotuner: cache keys and persistence on the CPU; on the GPU, candidates are timed, must
give identical records, and the winner is cached and returned by best()."""
import numpy as np
import pytest

import synth


def test_cache_roundtrip_and_keys(tmp_path):
    from paper_1705_11147_gb300 import autotune
    path = str(tmp_path / "tune.json")
    assert autotune.load_cache(path) == {}
    assert autotune.size_class(6_000_000_000) == 32 and autotune.size_class(1) == 0
    k1 = autotune.cache_key("NVIDIA GB300", 31, 30_000_000)
    k2 = autotune.cache_key("NVIDIA GB300", 51, 30_000_000)
    assert k1 != k2 and "kw1" in k1 and "kw2" in k2
    autotune.save_cache({k2: {"params": {"partitions": 7}, "ms": 1.0}}, path)
    assert autotune.best(51, 31_000_000, gpu_name="NVIDIA GB300", path=path) == {"partitions": 7}
    assert autotune.best(31, 31_000_000, gpu_name="NVIDIA GB300", path=path) == {}


def test_relative_partition_candidates():
    from paper_1705_11147_gb300 import autotune, make_params, plan
    from paper_1705_11147_gb300 import build
    build.build()
    base = dict(k=51, max_bases=6_000_000_000, expected_distinct=2_100_000_000, expected_keys=300_000_000)
    auto = plan(make_params(**base)).partitions
    assert autotune.expand({"partitions": -2}, base)["partitions"] == min(4096, 2 * auto)
    assert autotune.expand({"partitions": 5}, base)["partitions"] == 5


@pytest.mark.gpu
def test_tune_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_11147_gb300 import autotune, build
    build.build()
    rs = synth.workload("plain_1m", scale=0.2)
    seq = torch.from_numpy(rs.seq).cuda()
    qual = torch.from_numpy(rs.qual).cuda()
    offs = torch.from_numpy(rs.offsets.astype(np.int64)).cuda()
    base = dict(k=31, min_depth=2, max_bases=rs.n_bases, max_reads=rs.n_reads, expected_distinct=rs.n_bases)
    path = str(tmp_path / "tune.json")
    cands = [dict(partitions=1, windows_per_thread=1), dict(partitions=1, windows_per_thread=2),
             dict(partitions=6), dict(partitions=-2, load_factor=0.7)]
    entry = autotune.tune(seq, qual, offs, base, candidates=cands, reps=1, path=path)
    assert entry["params"] in [autotune.expand(c, base) for c in cands]
    assert autotune.best(31, rs.n_bases, path=path) == entry["params"]
