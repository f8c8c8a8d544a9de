"""GPU parity: the CUDA path through the C ABI against the CPU oracle, record by record.

Every comparison is bit-exact (integer work): same k-mer set, counts, eight extension
counters and two side codes per k-mer, after sorting both by key (record order is
unspecified on the GPU)."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_11147_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def to_dev(torch, rs):
    return (torch.from_numpy(rs.seq).cuda(), torch.from_numpy(rs.qual).cuda(),
            torch.from_numpy(rs.offsets.astype(np.int64)).cuda())


def run_gpu(torch, rs, device_inputs=True, batches=1, **kw):
    from paper_1705_11147_gb300 import KmerAnalysis, make_params
    p = dict(rs.meta.get("params", {}))
    p.pop("bloom_fpr", None)
    p.update(kw)
    p.setdefault("max_bases", max(rs.n_bases, 1))
    p.setdefault("max_reads", max(rs.n_reads, 1))
    p.setdefault("expected_distinct", max(rs.n_bases, 1))
    with KmerAnalysis(make_params(**p)) as ka:
        cuts = np.linspace(0, rs.n_reads, batches + 1).astype(np.int64)
        if device_inputs:
            seq, qual, _ = to_dev(torch, rs)
        for b in range(batches):
            r0, r1 = int(cuts[b]), int(cuts[b + 1])
            offs = rs.offsets[r0:r1 + 1]
            if device_inputs:
                ka.count(seq, qual, torch.from_numpy(offs.astype(np.int64)).cuda())
            else:
                ka.count(rs.seq, rs.qual, offs)
        ka.finalize()
        return ka.copy_result().sorted()


def assert_same(got, want, what=""):
    assert len(got) == len(want), f"{what}: {len(got)} vs {len(want)} records"
    for f in ("keys", "counts", "ext", "codes"):
        a, b = getattr(got, f), getattr(want, f)
        if not np.array_equal(a, b):
            bad = np.nonzero((a != b).reshape(a.shape[0], -1).any(1))[0][:5]
            raise AssertionError(f"{what}: field {f} differs at rows {bad}: {a[bad]} vs {b[bad]}")


GPU_ONLY = ("use_bloom", "heavy_hitters", "partitions", "load_factor", "table_capacity", "block_threads", "windows_per_thread",
            "warp_aggregate", "ctas_per_sm", "expected_distinct", "expected_keys", "staging_bytes",
            "max_bases", "max_reads", "bloom_fpr")


def oracle_for(rs, **kw):
    p = dict(rs.meta.get("params", {}))
    p.update(kw)
    for key in GPU_ONLY:
        p.pop(key, None)
    return oracle.run(rs.seq, rs.qual, rs.offsets, **p)


def readset(reads, quals=None, **params):
    seq, qual, offs = oracle.reads_from_strings(reads, quals)
    rs = synth.ReadSet(seq, qual, offs)
    rs.meta["params"] = params
    return rs


# ------------------------------------------------------------------ paper examples

def test_chopping_example(gpu):
    rs = readset(["GATCTGAACCG"], k=3, min_depth=1, min_ext_count=1, canonical=False, use_bloom=False)
    got = run_gpu(gpu, rs)
    assert oracle.unpack(got.keys, 3) == sorted(["GAT", "ATC", "TCT", "CTG", "TGA", "GAA", "AAC", "ACC", "CCG"])
    assert got.valid_windows == 9
    rs.meta["params"]["canonical"] = True
    assert_same(run_gpu(gpu, rs), oracle_for(rs), "canonical example")


def test_contig_and_fork_examples(gpu):
    rs = readset(["GATCTGA", "GATCTGA"], k=3, min_depth=2, min_ext_count=2, canonical=False)
    got = run_gpu(gpu, rs)
    i = oracle.unpack(got.keys, 3).index("CTG")
    assert tuple(got.codes[i]) == (3, 0)  # left T, right A: value "AT" as [right][left]
    rs = readset(["GAAC", "GAAC", "GAAT", "GAAT"], k=3, min_depth=2, min_ext_count=2, canonical=False)
    got = run_gpu(gpu, rs)
    i = oracle.unpack(got.keys, 3).index("GAA")
    assert tuple(got.codes[i]) == (4, 5) and got.counts[i] == 4


# ------------------------------------------------------------------ tiny random / edge cases

@pytest.mark.parametrize("k", [1, 3, 5, 7, 21, 31, 33, 51, 63])
def test_random_reads_all_k(gpu, k):
    rs = synth.random_reads(seed=77 + k, n_reads=3000, min_len=0, max_len=200,
                            alphabet=b"ACGTACGTACGTACGTacgtNRY", q_lo=10, q_hi=30)
    for bloom, md in [(False, 1), (False, 2), (True, 2), (True, 3)]:
        for canonical in (True, False):
            if canonical and k % 2 == 0:
                continue
            params = dict(k=k, min_depth=md, min_ext_count=2, qual_threshold=20, canonical=canonical)
            rs.meta["params"] = params
            got = run_gpu(gpu, rs, use_bloom=bloom)
            assert_same(got, oracle_for(rs), f"k={k} bloom={bloom} md={md} canonical={canonical}")


def test_low_complexity_and_repeats(gpu):
    # the same k-mer many times inside one warp's windows (homopolymers, dinucleotide runs)
    reads = ["A" * 300, "AC" * 150, "ACGT" * 75, "GATTACA" * 40, "T" * 70 + "G" + "T" * 70] * 40
    quals = ["I" * len(r) for r in reads]
    for k in (3, 21, 31, 51):
        rs = readset(reads, quals, k=k, min_depth=2, min_ext_count=2, qual_threshold=20)
        want = oracle_for(rs)
        for agg in (False, True):
            for bloom in (False, True):
                assert_same(run_gpu(gpu, rs, warp_aggregate=agg, use_bloom=bloom), want,
                            f"k={k} agg={agg} bloom={bloom}")
        # partitioned: the repeated k-mers overfill their buckets and spill into the
        # overflow area
        for bloom in (False, True):
            for heavy in (False, True):
                assert_same(run_gpu(gpu, rs, partitions=5, use_bloom=bloom, heavy_hitters=heavy), want,
                            f"k={k} partitioned bloom={bloom} heavy_hitters={heavy}")


def test_edge_inputs(gpu):
    # no reads with windows: empty reads, reads shorter than k, all-N reads
    rs = readset(["", "ACG", "NNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNNN", ""],
                 k=31, min_depth=2, min_ext_count=2, qual_threshold=20)
    got = run_gpu(gpu, rs)
    assert len(got) == 0 and got.valid_windows == 0
    # a single read of exactly k bases, twice
    r = "ACGT" * 15 + "ACG"
    rs = readset([r, r], k=63, min_depth=2, min_ext_count=1)
    got = run_gpu(gpu, rs)
    assert_same(got, oracle_for(rs), "k=63 single window")
    assert got.counts.tolist() == [2]


def test_decreasing_host_offsets_rejected(gpu):
    """Host read offsets that decrease anywhere (checked by one thread, or by several for a
    million reads and more) are rejected before anything is copied; the handle stays usable."""
    from paper_1705_11147_gb300 import KMA_EINVAL, KmaError, KmerAnalysis, make_params
    good = readset(["ACGTTGCAAGGCTTAGCCATG" * 3] * 4, k=21, min_depth=1, min_ext_count=1, qual_threshold=20)
    with KmerAnalysis(make_params(k=21, min_depth=1, use_bloom=False, max_bases=4096, max_reads=64)) as ka:
        seq = np.full(64, ord("A"), np.uint8)
        for n in (3, (1 << 20) + 5):
            for at in (0, n // 2, n - 1):
                offs = np.full(n + 1, 8, np.uint64)
                offs[: at + 1] = 9                   # offsets[at] = 9 > offsets[at + 1] = 8
                with pytest.raises(KmaError) as e:
                    ka.count(seq, seq, offs)
                assert e.value.code == KMA_EINVAL, (n, at)
        ka.count(good.seq, good.qual, good.offsets)
        ka.finalize()
        assert_same(ka.copy_result().sorted(), oracle_for(good, use_bloom=False), "after rejected calls")


# ------------------------------------------------------------------ workloads

@pytest.fixture(scope="module")
def plain(gpu):
    rs = synth.workload("plain_1m")
    return rs, oracle.run_readset(rs)


def test_plain_1m_full(gpu, plain):
    rs, want = plain
    got = run_gpu(gpu, rs, use_bloom=True)
    assert_same(got, want, "plain_1m bloom")
    assert got.valid_windows == want.valid_windows
    assert got.n_uu == int(want.uu_mask().sum())


def test_plain_1m_without_bloom(gpu, plain):
    rs, want = plain
    assert_same(run_gpu(gpu, rs, use_bloom=False), want, "plain_1m no bloom")


def test_host_inputs_chunked(gpu, plain):
    rs, want = plain
    got = run_gpu(gpu, rs, device_inputs=False, staging_bytes=1 << 20)  # ~30 chunks
    assert_same(got, want, "host inputs")


def test_multiple_count_calls(gpu, plain):
    rs, want = plain
    assert_same(run_gpu(gpu, rs, batches=5), want, "5 count() calls")


@pytest.mark.parametrize("shape", [
    dict(block_threads=128, windows_per_thread=1),
    dict(block_threads=256, windows_per_thread=8, warp_aggregate=True),
    dict(block_threads=64, windows_per_thread=2, ctas_per_sm=1),
    dict(block_threads=224, windows_per_thread=4, slot_prefetch=2),
    dict(block_threads=160, windows_per_thread=8, table_capacity=1_300_000),  # load ~0.85
    dict(expected_distinct=50_000, bloom_fpr=0.3, table_capacity=9_000_000),  # saturated Bloom: ~all 4.4 M keys inserted
    dict(expected_distinct=200_000_000, bloom_fpr=0.001),  # huge filter
])
def test_results_independent_of_tuning(gpu, plain, shape):
    rs, want = plain
    assert_same(run_gpu(gpu, rs, **shape), want, str(shape))


@pytest.mark.parametrize("opts", [
    dict(partitions=7),
    dict(partitions=64, windows_per_thread=1),
    dict(partitions=4096),                      # many tiny partitions
    dict(partitions=5, use_bloom=False, min_depth=2),
    dict(partitions=3, expected_distinct=50_000, bloom_fpr=0.3, table_capacity=9_000_000),
    dict(partitions=9, heavy_hitters=True),
    dict(partitions=9, heavy_hitters=True, use_bloom=False, min_depth=2),
])
def test_partitioned_mode(gpu, plain, opts):
    """On-chip owner-computes partitions give the same records as one table."""
    rs, want = plain
    got = run_gpu(gpu, rs, **opts)
    assert_same(got, want, str(opts))
    assert got.valid_windows == want.valid_windows


def test_partitioned_batches_host_inputs_and_k63(gpu, plain):
    rs, want = plain
    assert_same(run_gpu(gpu, rs, partitions=16, batches=4), want, "4 count() calls")
    assert_same(run_gpu(gpu, rs, partitions=16, device_inputs=False, staging_bytes=4 << 20), want, "host")
    rr = synth.random_reads(seed=1234, n_reads=4000, min_len=50, max_len=200,
                            alphabet=b"ACGTACGTACGTacgtN", q_lo=10, q_hi=30)
    rr.seq[: rr.n_bases // 3] = np.frombuffer((b"ACGTTGCAGG" * (rr.n_bases // 30 + 1))[: rr.n_bases // 3], np.uint8)
    for k in (63, 21):
        rr.meta["params"] = dict(k=k, min_depth=2, min_ext_count=1, qual_threshold=20)
        assert_same(run_gpu(gpu, rr, partitions=9), oracle_for(rr), f"k={k} partitioned")


def test_bacterial_5m_full(gpu):
    rs = synth.workload("bacterial_5m")
    want = oracle.run_readset(rs)
    got = run_gpu(gpu, rs, expected_distinct=80_000_000, expected_keys=20_000_000)
    assert_same(got, want, "bacterial_5m")
    assert got.valid_windows == want.valid_windows


def test_table_full_is_reported(gpu, plain):
    from paper_1705_11147_gb300 import KMA_EFULL, KmaError, count_kmers
    rs, want = plain
    with pytest.raises(KmaError) as ei:
        run_gpu(gpu, rs, table_capacity=100_000)
    assert ei.value.code == KMA_EFULL
    # the convenience wrapper retries with a larger table; the result does not depend on it
    got = count_kmers(rs.seq, rs.qual, rs.offsets, k=31, table_capacity=300_000,
                      expected_distinct=rs.n_bases).sorted()
    assert_same(got, want, "after EFULL retry")


def test_bounded_wait_reports_timeout(gpu):
    """The packing kernel's wait for its staging copies is bounded: with fault injection the
    copies are never issued, the wait gives up, and the host sees KMA_ETIMEOUT; the context
    stays usable for the next handle."""
    from paper_1705_11147_gb300 import KMA_ETIMEOUT, KmaError
    rs = synth.workload("plain_1m", scale=0.05)
    with pytest.raises(KmaError) as ei:
        run_gpu(gpu, rs, fault_inject=1)
    assert ei.value.code == KMA_ETIMEOUT
    assert_same(run_gpu(gpu, rs), oracle.run_readset(rs), "after timeout")


def test_reset_and_reuse(gpu, plain):
    from paper_1705_11147_gb300 import KmerAnalysis, make_params
    rs, want = plain
    small = synth.workload("plain_1m", scale=0.1)
    seq, qual, offs = to_dev(gpu, rs)
    with KmerAnalysis(make_params(k=31, max_bases=rs.n_bases, max_reads=rs.n_reads,
                                  expected_distinct=rs.n_bases)) as ka:
        for rep in range(2):
            s2, q2, o2 = to_dev(gpu, small)
            ka.count(s2, q2, o2)
            ka.finalize()
            assert_same(ka.copy_result().sorted(), oracle.run_readset(small), "small")
            ka.reset()
            ka.count(seq, qual, offs)
            ka.finalize()
            assert_same(ka.copy_result().sorted(), want, f"rep {rep}")
            ka.reset()


def test_query_matches_oracle(gpu):
    from paper_1705_11147_gb300 import KmerAnalysis, make_params
    rs = synth.workload("bacterial_5m", scale=0.05)
    want = oracle.run_readset(rs, keep_table=True)
    rng = np.random.default_rng(9)
    present = want.keys[rng.integers(0, len(want), 3000)]
    # reverse-complement half of them through the oracle's own string helpers
    strs = oracle.unpack(present[:1500], 51)
    comp = str.maketrans("ACGT", "TGCA")
    rc = oracle.pack([s.translate(comp)[::-1] for s in strs])
    rand = oracle.pack(["".join("ACGT"[x] for x in rng.integers(0, 4, 51)) for _ in range(1000)])
    # low-count keys (below min_depth) must answer as absent
    low = oracle.run_readset(rs, min_depth=1)
    singles = low.keys[low.counts == 1][:500]
    q = np.concatenate([present, rc, rand, singles])
    p = rs.meta["params"]
    wc, we, wcd = want.query(q)
    for parts in (1, 11):
        with KmerAnalysis(make_params(k=51, max_bases=rs.n_bases, max_reads=rs.n_reads,
                                      expected_distinct=rs.n_bases, min_depth=p["min_depth"],
                                      partitions=parts)) as ka:
            seq, qual, offs = to_dev(gpu, rs)
            ka.count(seq, qual, offs)
            ka.finalize()
            c, e, cd = ka.query(q)
            qd = gpu.from_numpy(q.astype(np.int64)).cuda()
            c2, e2, cd2 = ka.query(qd)
            gpu.cuda.synchronize()
        np.testing.assert_array_equal(c, wc)
        np.testing.assert_array_equal(e, we)
        np.testing.assert_array_equal(cd, wcd)
        np.testing.assert_array_equal(c2.cpu().numpy().astype(np.uint32), wc)
        np.testing.assert_array_equal(e2.cpu().numpy().astype(np.uint32), we)
        assert (c[:3000] > 0).all() and (c[len(present) + 1500 + 1000:] == 0).all()


def test_count_batch_equals_solo_and_oracle(gpu):
    from paper_1705_11147_gb300 import KmerAnalysis, count_batch, finalize_batch, make_params
    specs = synth.batched_specs(6, scale=0.02)
    sets = [synth.sample_reads(s) for s in specs]
    handles, reads = [], []
    for i, rs in enumerate(sets):
        p = rs.meta["params"]
        handles.append(KmerAnalysis(make_params(k=p["k"], min_depth=p["min_depth"], max_bases=rs.n_bases,
                                                max_reads=rs.n_reads, expected_distinct=rs.n_bases,
                                                partitions=5 if i % 3 == 1 else 1)))
        reads.append(to_dev(gpu, rs))
    count_batch(handles, reads)
    finalize_batch(handles)
    for i, (h, rs) in enumerate(zip(handles, sets)):
        got = h.copy_result().sorted()
        assert_same(got, oracle.run_readset(rs), f"sample {i}")
        assert_same(got, run_gpu(gpu, rs), f"sample {i} solo")
        h.destroy()


def test_batch_graph_replay_equals_solo(gpu):
    """Batched samples of uneven size in one captured CUDA graph: every replay gives each
    sample exactly its solo result."""
    from paper_1705_11147_gb300 import BatchGraph, KmerAnalysis, make_params
    specs = synth.batched_specs(9, scale=0.01)
    sets = [synth.sample_reads(s) for s in specs]
    # one-table and partitioned handles mixed in one graph
    handles = [KmerAnalysis(make_params(k=51, min_depth=2, max_bases=rs.n_bases, max_reads=rs.n_reads,
                                        expected_distinct=rs.n_bases, partitions=1 if i % 3 else 7))
               for i, rs in enumerate(sets)]
    reads = [to_dev(gpu, rs) for rs in sets]
    g = BatchGraph(handles, reads)
    solo = [run_gpu(gpu, rs) for rs in sets]
    for rep in range(2):
        g.replay()
        infos = g.results()
        for i, h in enumerate(handles):
            assert infos[i].n == len(solo[i])
            assert_same(h.copy_result().sorted(), solo[i], f"replay {rep} sample {i}")
    for h in handles:
        h.destroy()


# ------------------------------------------------------------------ full-size sampled parity

def _owner_subset(res, k, n_parts, parts):
    """The records of `res` whose key belongs to one of the oracle's owner partitions `parts`
    (of n_parts, the oracle's own hash)."""
    sel = np.isin(oracle.partition_of(res.keys, k, n_parts), list(parts))
    return type(res)(res.keys[sel], res.counts[sel], res.ext[sel], res.codes[sel]).sorted()


@pytest.mark.slow
def test_large_200m_sampled_partitions(gpu):
    """6 Gbases, 4.8 G windows, in the bench's launch configuration: the whole GPU result is
    checked on the k-mers of 16 of 256 owner partitions (by the oracle's own hash), computed
    by the oracle in one scan of the reads. The set holds the partitions of the eight most
    frequent k-mers of the result (repeats, the keys with the most contended counters) and
    the first partitions up to 16. The total window count is checked too."""
    import bench
    rs = synth.workload("large_200m")
    got = bench.run_large_once(rs)
    n_parts = 256
    top = np.argsort(got.counts)[-8:]
    parts = set(int(x) for x in oracle.partition_of(got.keys[top], 51, n_parts))
    x = 0
    while len(parts) < 16:
        parts.add(x)
        x += 1
    want = oracle.run_readset(rs, n_parts=n_parts, parts=sorted(parts))
    assert len(want) > 10_000_000
    assert_same(_owner_subset(got, 51, n_parts, parts), want, f"large_200m partitions {sorted(parts)}/256")
    assert got.valid_windows == want.valid_windows


# ------------------------------------------------------------------ HyperLogLog sizing pass

def _distinct_keys(rs, k, canonical=True):
    """All distinct keys of the read set (the oracle with min_depth 1)."""
    return oracle.run(rs.seq, rs.qual, rs.offsets, k=k, min_depth=1, canonical=canonical,
                      min_ext_count=2, qual_threshold=20)


@pytest.mark.parametrize("k,canonical,p", [(31, True, 14), (21, False, 12), (51, True, 14), (63, True, 10),
                                           (5, True, 4)])
def test_hll_registers_match_oracle(gpu, k, canonical, p):
    """The GPU sketch equals the oracle's sketch of the exact distinct set, register by
    register; the estimate is within 4 relative standard errors of the exact count."""
    from paper_1705_11147_gb300 import estimate_distinct, hll_estimate
    rs = synth.random_reads(seed=500 + k, n_reads=6000, min_len=0, max_len=250,
                            alphabet=b"ACGTACGTACGTACGTacgtNRY", q_lo=10, q_hi=30)
    want = _distinct_keys(rs, k, canonical)
    est = estimate_distinct(rs.seq, rs.qual, rs.offsets, k=k, canonical=canonical, precision=p)
    ref = oracle.hll_registers(want.keys, p)
    assert np.array_equal(est.registers, ref), np.nonzero(est.registers != ref)[0][:10]
    assert est.valid_windows == want.valid_windows
    assert est.distinct == pytest.approx(oracle.hll_estimate(ref, p), rel=1e-12)
    assert est.distinct == pytest.approx(hll_estimate(est.registers, p), rel=1e-12)
    n = len(want)
    assert abs(est.distinct - n) <= 4 * est.rel_std_error * n + 2, (est.distinct, n)


def _check_heavy_summary(est, rs, k, canonical=True):
    """The merged Misra-Gries summaries of the cardinality pass against the exact sampled
    stream (oracle): the same sub-stream sizes, every key in its own sub-stream, and per
    sub-stream of n items the Misra-Gries bound: f - n/(m+1) <= c <= f for every key (c = 0
    if absent), every key with f > n/(m+1) present."""
    from paper_1705_11147_gb300 import capi
    stream = oracle.sampled_stream(rs.seq, rs.qual, rs.offsets, k=k, canonical=canonical)
    bucket = oracle.stream_bucket(stream, 5)
    assert est.sampled_windows == len(stream)
    np.testing.assert_array_equal(est.bucket_windows, np.bincount(bucket, minlength=capi.MG_BUCKETS))
    if len(est.summary_keys):
        np.testing.assert_array_equal(est.summary_bucket, oracle.stream_bucket(est.summary_keys, 5))
    got = {(int(a), int(b)): int(c) for (a, b), c in zip(est.summary_keys, est.summary_counts)}
    assert len(got) == len(est.summary_keys)
    keys, inv, freq = np.unique(stream.view([("lo", np.uint64), ("hi", np.uint64)]).ravel(), return_inverse=True,
                                return_counts=True)
    kb = np.zeros(len(keys), np.int64)
    kb[inv] = bucket
    for (lo_hi, f, b) in zip(keys, freq, kb):
        key = (int(lo_hi["lo"]), int(lo_hi["hi"]))
        eps = int(est.bucket_windows[b]) / (capi.MG_COUNTERS + 1)
        c = got.get(key, 0)
        assert f - eps <= c <= f, (key, f, c, eps)
        if f > eps:
            assert key in got
    assert set(got) <= {(int(x["lo"]), int(x["hi"])) for x in keys}
    return got, freq


def test_heavy_hitter_summaries(gpu):
    """Cardinality pass with the heavy-hitter summaries (Section 5.1): few distinct keys ->
    the summaries are the exact sampled frequencies; a satellite in a third of the reads ->
    its k-mers are found and heavy_hitters is recommended; uniform reads -> no heavy hitters.
    The read sets whose count runs with the recommended setting give the oracle's records."""
    from paper_1705_11147_gb300 import estimate_distinct
    rng = np.random.default_rng(31)
    # three reads repeated: at most a few dozen distinct sampled keys per sub-stream
    base = ["".join("ACGT"[i] for i in rng.integers(0, 4, 100)) for _ in range(3)]
    rs = readset([base[i % 3] for i in range(1500)], k=31, min_depth=2)
    est = estimate_distinct(rs.seq, rs.qual, rs.offsets, k=31)
    got, freq = _check_heavy_summary(est, rs, 31)
    stream = oracle.sampled_stream(rs.seq, rs.qual, rs.offsets, k=31)
    want = {(int(a), int(b)): 0 for a, b in stream}
    for a, b in stream:
        want[(int(a), int(b))] += 1
    assert got == want  # exact: no sub-stream ever exceeded its counters
    # satellite of period 171 in a third of the reads (as in the heavy-hitter grouping test)
    unit = "".join("ACGT"[i] for i in rng.integers(0, 4, 171))
    g = "".join("ACGT"[i] for i in rng.integers(0, 4, 200_000))
    sat, reads = unit * 60, []
    for i in range(6000):
        src = sat if i % 3 == 0 else g
        a = int(rng.integers(0, len(src) - 150))
        r = src[a:a + 150]
        reads.append(r if i % 2 else r.translate(str.maketrans("ACGT", "TGCA"))[::-1])
    rs = readset(reads, k=31, min_depth=2, min_ext_count=2, qual_threshold=20)
    for dev in (False, True):
        args = to_dev(gpu, rs) if dev else (rs.seq, rs.qual, rs.offsets)
        est = estimate_distinct(*args, k=31)
        _check_heavy_summary(est, rs, 31)
        assert est.heavy_hitters
    unit_keys = {min(w, w.translate(str.maketrans("ACGT", "TGCA"))[::-1])
                 for w in ((unit * 2)[i:i + 31] for i in range(171))}
    top = set(oracle.unpack(est.summary_keys[est.summary_counts >= est.heavy_threshold], 31))
    assert top and top <= unit_keys
    assert_same(run_gpu(gpu, rs, heavy_hitters=est.heavy_hitters, partitions=4), oracle_for(rs), "satellite")
    # uniform random genome: nothing frequent
    rp = synth.workload("plain_1m", scale=0.1)
    est = estimate_distinct(rp.seq, rp.qual, rp.offsets, k=31)
    _check_heavy_summary(est, rp, 31)
    assert not est.heavy_hitters


def test_hll_plain_1m_device_host_and_merge(gpu, plain):
    """Same sketch from host and device inputs; sketches of two halves merge (elementwise
    maximum) into the sketch of the whole; owner partitions of three 'GPUs' merge likewise."""
    from paper_1705_11147_gb300 import estimate_distinct
    rs, want = plain
    k = rs.meta["params"]["k"]
    allkeys = _distinct_keys(rs, k)
    full = estimate_distinct(rs.seq, rs.qual, rs.offsets, k=k)
    assert np.array_equal(full.registers, oracle.hll_registers(allkeys.keys, 14))
    seq, qual, offs = to_dev(gpu, rs)
    dev = estimate_distinct(seq, qual, offs, k=k)
    assert np.array_equal(dev.registers, full.registers) and dev.valid_windows == full.valid_windows
    half = rs.n_reads // 2
    a = estimate_distinct(rs.seq, rs.qual, rs.offsets[:half + 1], k=k)
    b = estimate_distinct(rs.seq, rs.qual, rs.offsets[half:], k=k, registers=a.registers)
    assert np.array_equal(b.registers, full.registers)
    assert a.valid_windows + b.valid_windows == full.valid_windows
    parts = [estimate_distinct(rs.seq, rs.qual, rs.offsets, k=k, n_parts=3, part=i) for i in range(3)]
    assert np.array_equal(np.maximum.reduce([e.registers for e in parts]), full.registers)
    assert sum(e.valid_windows for e in parts) == full.valid_windows
    assert abs(full.distinct - len(allkeys)) < 4 * full.rel_std_error * len(allkeys)


# ------------------------------------------------------------------ FASTQ parsing on the device

def _to_fastq(rs, crlf=False, final_newline=True):
    nl = b"\r\n" if crlf else b"\n"
    out = []
    for r in range(rs.n_reads):
        a, b = int(rs.offsets[r]), int(rs.offsets[r + 1])
        out += [b"@read%d" % r, rs.seq[a:b].tobytes(), b"+", rs.qual[a:b].tobytes()]
    text = nl.join(out)
    return text + nl if final_newline else text


def _parse_gpu(gpu, text, device=False):
    from paper_1705_11147_gb300 import parse_fastq
    if device:
        text = gpu.from_numpy(np.frombuffer(text, np.uint8).copy()).cuda()
    seq, qual, offs = parse_fastq(text)
    return seq.cpu().numpy(), qual.cpu().numpy(), offs.cpu().numpy().astype(np.uint64)


@pytest.mark.parametrize("crlf,final_newline,device", [(False, True, False), (True, True, True),
                                                       (False, False, True), (True, False, False)])
def test_fastq_parse_matches_oracle(gpu, crlf, final_newline, device):
    """Synthetic reads (empty and short reads, N/IUPAC/lowercase bases, qualities over the whole
    printable range, so quality lines start with '@' or '+') written as FASTQ: the device
    parser returns the reads exactly, as does the oracle's parser."""
    rs = synth.random_reads(seed=31, n_reads=5000, min_len=0, max_len=300,
                            alphabet=b"ACGTACGTACGTacgtNRY", q_lo=0, q_hi=60)
    text = _to_fastq(rs, crlf, final_newline)
    got = _parse_gpu(gpu, text, device)
    want = oracle.parse_fastq(text)
    for a, b, c in zip(got, want, (rs.seq, rs.qual, rs.offsets - rs.offsets[0])):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_fastq_golden_and_errors(gpu):
    from paper_1705_11147_gb300 import capi
    text = open(os.path.join(os.path.dirname(__file__), "golden", "fastq_records.fastq"), "rb").read()
    for t in (text, text + b"\n\n\r\n"):
        got, want = _parse_gpu(gpu, t), oracle.parse_fastq(t)
        assert all(np.array_equal(a, b) for a, b in zip(got, want))
    for bad in (b"@a\nAC\n-\nII\n", b"@a\nAC\n+\nI\n", b"@a\nAC\n+\nII\nX\n", b"a\nAC\n+\nII\n"):
        with pytest.raises(capi.KmaError) as e:
            _parse_gpu(gpu, bad)
        assert e.value.code == capi.KMA_EINVAL
    assert [len(x) for x in _parse_gpu(gpu, b"")] == [0, 0, 1]


def test_fastq_parse_then_count(gpu, plain):
    """FASTQ text of the 30 Mbase workload -> device parser -> counting: the same records as the
    oracle on the original reads."""
    from paper_1705_11147_gb300 import KmerAnalysis, make_params, parse_fastq
    rs, want = plain
    seq, qual, offs = parse_fastq(_to_fastq(rs))
    p = dict(rs.meta["params"])
    p.pop("bloom_fpr", None)
    with KmerAnalysis(make_params(max_bases=rs.n_bases, max_reads=rs.n_reads, expected_distinct=rs.n_bases,
                                  **p)) as ka:
        ka.count(seq, qual, offs)
        ka.finalize()
        assert_same(ka.copy_result().sorted(), want, "fastq")


# ------------------------------------------------------------------ contig generation

def _rc(s):
    return s.translate(str.maketrans("ACGT", "TGCA"))[::-1]


def _canon_sorted(contigs, canonical=True):
    return sorted(min(c, _rc(c)) for c in contigs) if canonical else sorted(contigs)


def _gpu_contigs(gpu, rs, **params):
    from paper_1705_11147_gb300 import KmerAnalysis, make_params
    p = dict(params)
    p.setdefault("max_bases", max(rs.n_bases, 1))
    p.setdefault("max_reads", max(rs.n_reads, 1))
    p.setdefault("expected_distinct", max(rs.n_bases, 1))
    with KmerAnalysis(make_params(**p)) as ka:
        ka.count(rs.seq, rs.qual, rs.offsets)
        ka.finalize()
        res = ka.copy_result()
        strings, info = ka.contigs()
        return strings, info, res


def _check_contigs(gpu, rs, k, canonical=True, min_depth=2, min_ext_count=2, **gpu_only):
    want_res = oracle.run(rs.seq, rs.qual, rs.offsets, k=k, min_depth=min_depth, min_ext_count=min_ext_count,
                          canonical=canonical, qual_threshold=20)
    want, want_cycles = oracle.contigs(want_res.keys, want_res.codes, k, canonical)
    gpu_only.setdefault("use_bloom", min_depth >= 2)  # the Bloom pass drops singletons
    got, info, _ = _gpu_contigs(gpu, rs, k=k, min_depth=min_depth, min_ext_count=min_ext_count,
                                canonical=canonical, qual_threshold=20, **gpu_only)
    assert info["n_cycles"] == want_cycles
    assert info["n_contigs"] == len(want) and info["n_bases"] == sum(len(c) for c in want)
    assert _canon_sorted(got, canonical) == _canon_sorted(want, canonical)
    return got, info


def test_contigs_golden_examples(gpu):
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "contigs_examples.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        reads, want = (x.strip() for x in line.split("|"))
        rs = readset(reads.split(","))
        got, info, _ = _gpu_contigs(gpu, rs, k=3, min_depth=2, min_ext_count=2, canonical=False, use_bloom=False)
        assert sorted(got) == want.split(","), (reads, got)


def test_contigs_linear_and_circular_genomes(gpu):
    rng = np.random.default_rng(9)
    g = "".join("ACGT"[i] for i in rng.integers(0, 4, 5000))
    for circular in (False, True):
        gg = g + g if circular else g
        reads = []
        for i in range(0, len(g) if circular else len(g) - 119, 6):
            reads += [gg[i:i + 120], _rc(gg[i:i + 120])]
        if not circular:
            reads += [g[-120:], _rc(g[-120:])]
        got, info = _check_contigs(gpu, readset(reads), 31)
        assert info["n_contigs"] == 1 and info["n_cycles"] == int(circular)
        assert len(got[0]) == len(g) + (30 if circular else 0)


@pytest.mark.parametrize("k,canonical", [(31, True), (21, False), (51, True)])
def test_contigs_random_reads(gpu, k, canonical):
    rs = synth.random_reads(seed=70 + k, n_reads=20000, min_len=60, max_len=200, alphabet=b"ACGT", q_lo=15, q_hi=40)
    _check_contigs(gpu, rs, k, canonical=canonical, min_depth=1, min_ext_count=1)


def test_contigs_plain_and_bacterial(gpu, plain):
    rs, _ = plain
    _check_contigs(gpu, rs, rs.meta["params"]["k"])
    rb = synth.workload("bacterial_5m", scale=0.2)
    _check_contigs(gpu, rb, rb.meta["params"]["k"], partitions=4)


def test_heavy_hitters_satellite(gpu):
    """A tandem satellite making up a third of the reads (its k-mers occur tens of thousands
    of times each): grouping equal keys in the warp (heavy_hitters) changes no record."""
    rng = np.random.default_rng(21)
    unit = "".join("ACGT"[i] for i in rng.integers(0, 4, 171))
    g = "".join("ACGT"[i] for i in rng.integers(0, 4, 200_000))
    sat = unit * 60
    reads = []
    for i in range(6000):
        src = sat if i % 3 == 0 else g
        a = int(rng.integers(0, len(src) - 150))
        r = src[a:a + 150]
        reads.append(r if i % 2 else r.translate(str.maketrans("ACGT", "TGCA"))[::-1])
    rs = readset(reads, k=31, min_depth=2, min_ext_count=2, qual_threshold=20)
    want = oracle_for(rs)
    for bloom in (True, False):
        for parts in (4, 1):
            got = run_gpu(gpu, rs, partitions=parts, use_bloom=bloom, heavy_hitters=True)
            assert_same(got, want, f"bloom={bloom} partitions={parts}")


# ------------------------------------------------------------------ finalize straight to host

def run_gpu_to_host(torch, rs, capacity=None, pinned=True, **kw):
    """count (device inputs) + kmer_analysis_finalize_to_host into host buffers; returns the
    sorted records and the handle's own finalize result for cross-checks."""
    from paper_1705_11147_gb300 import KmerAnalysis, host_result_buffers, make_params
    p = dict(rs.meta.get("params", {}))
    p.pop("bloom_fpr", None)
    p.update(kw)
    p.setdefault("max_bases", max(rs.n_bases, 1))
    p.setdefault("max_reads", max(rs.n_reads, 1))
    p.setdefault("expected_distinct", max(rs.n_bases, 1))
    cap = rs.n_bases + 1 if capacity is None else capacity
    with KmerAnalysis(make_params(**p)) as ka:
        ka.count(*to_dev(torch, rs))
        got = ka.finalize_to_host(host_result_buffers(cap, pinned=pinned))
        again = ka.copy_result()  # the device result stays valid
        return got.sorted(), again.sorted()


@pytest.mark.parametrize("opts", [
    dict(),
    dict(use_bloom=False, min_depth=1),
    dict(partitions=7),
    dict(partitions=64),
    dict(partitions=4096),
    dict(partitions=5, use_bloom=False, min_depth=2),
    dict(partitions=9, heavy_hitters=True),
])
def test_finalize_to_host(gpu, plain, opts):
    """The grouped recount + classification with overlapped copies gives finalize's records."""
    rs, want = plain
    got, again = run_gpu_to_host(gpu, rs, **opts)
    assert_same(again, got, f"copy_result after finalize_to_host {opts}")
    if opts.get("min_depth", 2) == 2:
        assert_same(got, want, str(opts))
    else:
        rs2 = synth.ReadSet(rs.seq, rs.qual, rs.offsets)
        rs2.meta["params"] = dict(rs.meta["params"], min_depth=opts["min_depth"])
        assert_same(got, oracle_for(rs2), str(opts))


def test_finalize_to_host_overflow_capacity_and_query(gpu):
    """Repeated k-mers spill into the overflow area (recounted before the groups); too small a
    host buffer gets the first `capacity` records and KMA_EFULL, with the handle finalized."""
    from paper_1705_11147_gb300 import KMA_EFULL, KmaError, KmerAnalysis, host_result_buffers, make_params
    reads = ["A" * 300, "AC" * 150, "ACGT" * 75, "GATTACA" * 40, "T" * 70 + "G" + "T" * 70] * 40
    rr = synth.random_reads(seed=99, n_reads=3000, min_len=60, max_len=200, alphabet=b"ACGT", q_lo=15, q_hi=40)
    strs = reads + [bytes(rr.seq[rr.offsets[i]:rr.offsets[i + 1]]).decode() for i in range(rr.n_reads)] * 2
    rs = readset(strs, k=31, min_depth=2, min_ext_count=2, qual_threshold=20)
    want = oracle_for(rs)
    for parts in (5, 1):
        got, _ = run_gpu_to_host(gpu, rs, partitions=parts, pinned=False)
        assert_same(got, want, f"partitions={parts}")
    n = len(want)
    p = dict(k=31, min_depth=2, min_ext_count=2, qual_threshold=20, max_bases=rs.n_bases, max_reads=rs.n_reads,
             expected_distinct=rs.n_bases, partitions=5)
    with KmerAnalysis(make_params(**p)) as ka:
        ka.count(*to_dev(gpu, rs))
        bufs = host_result_buffers(n // 3)
        with pytest.raises(KmaError) as ei:
            ka.finalize_to_host(bufs)
        assert ei.value.code == KMA_EFULL
        assert int(ka.result_info.n) == n
        keys = bufs[0]
        idx = {tuple(k): i for i, k in enumerate(want.keys.tolist())}
        for j in range(n // 3):  # every copied row is a correct record
            i = idx[tuple(keys[j].tolist())]
            assert bufs[1][j] == want.counts[i] and np.array_equal(bufs[2][j], want.ext[i])
            assert np.array_equal(bufs[3][j], want.codes[i])
        assert len({tuple(k) for k in keys.tolist()}) == n // 3
        assert_same(ka.copy_result().sorted(), want, "copy_result after a short buffer")
        counts, ext, codes = ka.query(want.keys[:100])
        assert np.array_equal(counts, want.counts[:100])


# ------------------------------------------------------------------ every batched sample, served subset

@pytest.mark.slow
def test_batched_64_every_sample_vs_oracle(gpu):
    """All 64 samples of the batched workload at the bench's size (12.7 Gbases), with the
    bench's per-sample parameters, through one captured graph replayed once: every sample's
    records equal the oracle's on one owner partition of 32 (by the oracle's own hash), and
    every sample's window count equals the oracle's."""
    import bench
    from paper_1705_11147_gb300 import BatchGraph, KmerAnalysis
    gpu.cuda.empty_cache()
    sets = [synth.sample_reads(s) for s in synth.batched_specs(64, scale=1.0)]
    handles = [KmerAnalysis(bench.make_handle_params(rs)) for rs in sets]
    g = BatchGraph(handles, [to_dev(gpu, rs) for rs in sets])
    g.replay()
    infos = g.results()
    results = []
    for h in handles:
        results.append(h.copy_result())
        h.destroy()
    del g, handles
    gpu.cuda.empty_cache()
    for i, (res, info, rs) in enumerate(zip(results, infos, sets)):
        want = oracle.run_readset(rs, n_parts=32, parts=[i % 32])
        assert_same(_owner_subset(res, 51, 32, [i % 32]), want, f"sample {i}")
        assert info.valid_windows == want.valid_windows


@pytest.mark.slow
def test_served_subset_vs_oracle(gpu):
    """30 jobs of the served workload at the bench's scale (genomes log-U[1, 50] Mbp x 0.05),
    the smallest and the largest of all 500 among them, through the batching server with the
    bench's per-job parameters: every job equals the oracle on 4 of 16 owner partitions (by
    the oracle's own hash); the window counts are checked whole."""
    import bench
    from paper_1705_11147_gb300.serve import Job, Server
    specs = synth.served_specs(500, scale=0.05)
    by_size = sorted(range(len(specs)), key=lambda j: specs[j]["G"])
    pick = {by_size[0], by_size[-1]}
    j = 0
    while len(pick) < 30:
        pick.add(j)
        j += 1
    pick = sorted(pick)
    jobs, sets = [], []
    for i in pick:
        rs = synth.sample_reads(specs[i])
        p = dict(rs.meta["params"])
        p.pop("bloom_fpr", None)
        p.update(bench.workload_sizing(rs))
        jobs.append(Job(rs.seq, rs.qual, rs.offsets, params=p, job_id=i))
        sets.append(rs)
    assert len(jobs) == 30 and {j.params["k"] for j in jobs} == {31, 51}
    with Server(max_batch=8, workers=2) as srv:
        got = [f.result(timeout=900) for f in [srv.submit(j) for j in jobs]]
    for i, (res, rs) in enumerate(zip(got, sets)):
        k = rs.meta["params"]["k"]
        parts = [(4 * i + d) % 16 for d in range(4)]
        want = oracle.run_readset(rs, n_parts=16, parts=parts)
        assert_same(_owner_subset(res, k, 16, parts), want, f"job {pick[i]}")
        assert res.valid_windows == want.valid_windows


@pytest.mark.slow
def test_served_quarter_scale_vs_oracle(gpu):
    """The served workload at the scale the served comparison runs (genomes log-U[1, 50] Mbp
    x 0.25, the first 250 jobs): the largest of those 250 jobs and nine of the first jobs, with
    three workers and the bench's per-job parameters, so that jobs above the host-count size
    are counted from host memory through the library's staged copies. Every job equals the
    oracle on 2 of 16 owner partitions (by the oracle's own hash); window counts whole."""
    import bench
    from paper_1705_11147_gb300.serve import Job, Server
    specs = synth.served_specs(250, scale=0.25)
    largest = max(range(len(specs)), key=lambda j: specs[j]["G"])
    pick = sorted({largest} | set(range(9)))
    jobs, sets = [], []
    for i in pick:
        rs = synth.sample_reads(specs[i])
        p = dict(rs.meta["params"])
        p.pop("bloom_fpr", None)
        p.update(bench.workload_sizing(rs))
        jobs.append(Job(rs.seq, rs.qual, rs.offsets, params=p, job_id=i))
        sets.append(rs)
    srv = Server(max_batch=8, workers=3)
    assert max(j.n_bases for j in jobs) >= srv.host_count_bases  # the host-memory path runs
    with srv:
        got = [f.result(timeout=1800) for f in [srv.submit(j) for j in jobs]]
    for i, (res, rs) in enumerate(zip(got, sets)):
        k = rs.meta["params"]["k"]
        parts = [(2 * i + d) % 16 for d in range(2)]
        want = oracle.run_readset(rs, n_parts=16, parts=parts)
        assert_same(_owner_subset(res, k, 16, parts), want, f"job {pick[i]}")
        assert res.valid_windows == want.valid_windows


# ------------------------------------------------------------------ multi-GPU owner shards

@pytest.mark.parametrize("n_parts", [2, 3])
@pytest.mark.parametrize("mode", ["one_table", "partitioned", "host_chunks", "one_table_no_bloom"])
def test_owner_shards_union_to_whole(gpu, plain, n_parts, mode):
    """Multi-GPU owner-computes (Section 5.1), one shard at a time on this GPU: each handle
    counts only the k-mers its n_parts/part selects. The shards are disjoint, their union is
    the oracle's whole result, and their window counts add up to the whole's."""
    rs, want = plain
    opts = {"one_table": dict(partitions=1),
            "partitioned": dict(partitions=7),
            "host_chunks": dict(partitions=5, device_inputs=False, staging_bytes=2 << 20),
            "one_table_no_bloom": dict(partitions=1, use_bloom=False)}[mode]
    shards = [run_gpu(gpu, rs, n_parts=n_parts, part=part, **opts) for part in range(n_parts)]
    assert all(len(s) > 0 for s in shards)
    keys = np.concatenate([s.keys for s in shards])
    assert len(np.unique(keys, axis=0)) == len(keys), "shards overlap"
    merged = type(shards[0])(keys, np.concatenate([s.counts for s in shards]),
                             np.concatenate([s.ext for s in shards]),
                             np.concatenate([s.codes for s in shards])).sorted()
    assert_same(merged, want, f"union of {n_parts} shards ({mode})")
    assert sum(s.valid_windows for s in shards) == want.valid_windows
