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


def test_lookup_order_and_apply(tmp_path):
    """User cache first, then the shipped table; tuned keywords fill only what the job leaves
    open; relative partition counts resolve against the job's own automatic count, and a job
    the library keeps in one table is not partitioned by a scale."""
    from paper_1705_11147_gb300 import autotune, build, make_params, plan
    build.build()
    user = str(tmp_path / "user.json")
    shipped = str(tmp_path / "shipped.json")
    big = dict(k=51, max_bases=6_000_000_000, expected_distinct=2_100_000_000, expected_keys=300_000_000)
    key = autotune.cache_key("GPU X", 51, big["max_bases"])
    autotune.save_cache({key: {"params": {"partition_scale": 2.0, "load_factor": 0.6}}}, shipped)
    got, src = autotune.lookup(51, big["max_bases"], gpu_name="GPU X", path=user, shipped=shipped)
    assert src == "shipped" and got == {"partition_scale": 2.0, "load_factor": 0.6}
    auto = plan(make_params(**{**big, "load_factor": 0.6})).partitions
    kw, src = autotune.apply(dict(big), gpu_name="GPU X", path=user, shipped=shipped)
    assert src == "shipped" and kw["load_factor"] == 0.6 and kw["partitions"] == min(2048, 2 * auto)
    assert "partition_scale" not in kw
    kw, _ = autotune.apply({**big, "partitions": 7, "load_factor": 0.5}, gpu_name="GPU X", path=user,
                           shipped=shipped)
    assert kw["partitions"] == 7 and kw["load_factor"] == 0.5
    autotune.save_cache({key: {"params": {"windows_per_thread": 4}}}, user)
    got, src = autotune.lookup(51, big["max_bases"], gpu_name="GPU X", path=user, shipped=shipped)
    assert src == "cache" and got == {"windows_per_thread": 4}
    assert autotune.lookup(31, big["max_bases"], gpu_name="GPU X", path=user, shipped=shipped) == ({}, "none")
    # a one-table job stays one table under a partition scale
    small = dict(k=31, max_bases=1 << 20, expected_distinct=1 << 16)
    assert plan(make_params(**small)).partitions == 1
    assert autotune.expand({"partition_scale": 0.5}, small)["partitions"] == 1
    assert autotune.candidates_for(small) is autotune.DEFAULT_CANDIDATES
    assert autotune.candidates_for(big) is autotune.PARTITIONED_CANDIDATES


def test_shipped_table_is_valid():
    """Every entry of the table shipped with the package names only tunable keywords with
    values the library accepts."""
    from paper_1705_11147_gb300 import autotune, build, make_params, plan
    build.build()
    table = autotune.load_cache(autotune.SHIPPED_TABLE)
    for key, entry in table.items():
        gpu, kw, cls = key.split("|")
        assert kw in ("kw1", "kw2") and int(cls) >= 0 and gpu
        assert set(entry["params"]) <= set(autotune.TUNABLE), entry
        k = 51 if kw == "kw2" else 31
        n = 1 << int(cls)
        base = dict(k=k, max_bases=n, expected_distinct=n // 4)
        plan(make_params(**autotune.expand({**entry["params"]}, base) | base))


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
    assert entry["params"] in cands
    assert entry["resolved"] == autotune.expand(entry["params"], base)
    assert autotune.best(31, rs.n_bases, path=path) == entry["params"]
    # the choice reaches a handle through apply(): explicit keywords win
    kw, src = autotune.apply(dict(base), path=path, shipped=None)
    assert src == "cache" and kw == {**base, **entry["resolved"]}


def test_bench_handles_take_the_tuning(tmp_path, monkeypatch):
    """The bench's handle keywords come through apply(): an entry for the job's class in the
    user cache is used (source "cache"), explicit keywords win, and --no-tuned bypasses it."""
    import bench
    from paper_1705_11147_gb300 import autotune, build
    build.build()
    rs = synth.workload("plain_1m", scale=0.05)
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv("KMA_TUNE_CACHE", path)
    gpu = autotune._gpu_name()
    autotune.save_cache({autotune.cache_key(gpu, 31, rs.n_bases): {"params": {"load_factor": 0.6}}}, path)
    kw, src = bench.handle_kwargs(rs)
    assert src == "cache" and kw["load_factor"] == 0.6
    kw, src = bench.handle_kwargs(rs, load_factor=0.7)
    assert kw["load_factor"] == 0.7
    kw, src = bench.handle_kwargs(rs, tuned=False)
    assert src == "none" and "load_factor" not in kw
