"""The continuous-batching server: every job's records are the same alone and in the mix,
admission never exceeds the memory budget, failures injected on the host fail only their
batch, and resident tables answer queries."""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jobs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_11147_gb300 import build
    from paper_1705_11147_gb300.serve import Job
    build.build()
    out = []
    for i, sp in enumerate(synth.served_specs(12, scale=0.004)):
        rs = synth.sample_reads(sp)
        p = dict(rs.meta["params"])
        p.pop("bloom_fpr")
        p["expected_distinct"] = rs.n_bases
        out.append(Job(rs.seq, rs.qual, rs.offsets, params=p, job_id=i))
    assert {j.params["k"] for j in out} == {31, 51}
    return out


def _same(a, b):
    a, b = a.sorted(), b.sorted()
    assert len(a) == len(b)
    for f in ("keys", "counts", "ext", "codes"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_served_results_equal_solo(jobs):
    from paper_1705_11147_gb300.serve import Server, run_plain
    solo = run_plain(jobs)
    with Server(max_batch=4, workers=2) as srv:
        futs = [srv.submit(j) for j in jobs]
        got = [f.result(timeout=300) for f in futs]
        assert srv.batches >= 3                    # batched, not one job per launch
    for g, s in zip(got, solo):
        _same(g, s)
    for i in (0, 7):                               # and against the oracle
        j = jobs[i]
        want = oracle.run(j.seq, j.qual, j.offsets, k=j.params["k"], min_depth=j.params["min_depth"],
                          qual_threshold=j.params["qual_threshold"])
        g = got[i].sorted()
        np.testing.assert_array_equal(g.keys, want.keys)
        np.testing.assert_array_equal(g.ext, want.ext)


def test_admission_respects_budget(jobs):
    from paper_1705_11147_gb300.serve import Server
    probe = Server(device_budget=1 << 50, workers=1)
    fps = [probe.footprint(j) for j in jobs]
    probe.close()
    budget = int(max(fps) * 1.5)
    seen = []
    lock = threading.Lock()
    with Server(device_budget=budget, max_batch=8, workers=3) as srv:
        def hook(job):
            with lock:
                seen.append(srv.used)
        srv.admit_hook = hook
        futs = [srv.submit(j) for j in jobs]
        for f in futs:
            f.result(timeout=300)
    assert seen and max(seen) <= budget
    assert len(seen) == len(jobs)


def test_failure_injection_fails_only_its_batch(jobs):
    from paper_1705_11147_gb300.serve import Server
    with Server(max_batch=1, workers=2) as srv:
        def hook(job):
            if job.job_id == 3:
                raise RuntimeError("injected allocation failure")
        srv.admit_hook = hook
        futs = [srv.submit(j) for j in jobs[:6]]
        for i, f in enumerate(futs):
            if i == 3:
                with pytest.raises(RuntimeError, match="injected"):
                    f.result(timeout=300)
            else:
                assert len(f.result(timeout=300)) > 0
        assert srv.used == 0 and len(srv.failures) == 1


def test_resident_tables_answer_queries(jobs):
    from paper_1705_11147_gb300.serve import Server
    with Server(max_batch=4, workers=1, keep_resident=True) as srv:
        futs = [srv.submit(j) for j in jobs[:3]]
        res = [f.result(timeout=300) for f in futs]
        for j, r in zip(jobs[:3], res):
            assert j.handle is not None
            c, e, cd = j.handle.query(r.keys[:100])
            np.testing.assert_array_equal(c, r.counts[:100])
            srv.release(j)
        assert srv.used == 0


def test_oversized_job_is_rejected(jobs):
    from paper_1705_11147_gb300.serve import Server
    with Server(device_budget=1024, workers=1) as srv:
        with pytest.raises(MemoryError):
            srv.submit(jobs[0]).result(timeout=10)
