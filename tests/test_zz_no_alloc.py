"""The allocation-free entry point, kmer_analysis_count_small_noalloc, called through the C ABI.

It is meant for callers that may not allocate device memory when they count (a fixed memory
budget reserved at start-up, or a plugin whose host framework owns every device allocation).
Its records must equal those of the regular create/count/finalize path on the same reads,
call after call: the fixed scratch array it works in keeps the previous call's contents, so
the second call checks that everything that must start empty is cleared.

This file is named to be collected last, so that a failure here leaves every other test
already run in a `-x` session.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1705_11147_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def _regular(torch, rs, **params):
    """Records of the existing entry points (create/count/finalize with the Bloom pass)."""
    from paper_1705_11147_gb300 import KmerAnalysis, make_params
    p = make_params(max_bases=max(rs.n_bases, 1), max_reads=max(rs.n_reads, 1),
                    expected_distinct=max(rs.n_bases, 1), **params)
    with KmerAnalysis(p) as ka:
        ka.count(torch.from_numpy(rs.seq).cuda(), torch.from_numpy(rs.qual).cuda(),
                 torch.from_numpy(rs.offsets.astype(np.int64)).cuda())
        ka.finalize()
        return ka.copy_result().sorted()


def _noalloc(torch, rs, capacity, **params):
    from paper_1705_11147_gb300 import capi, make_params
    lib = capi.load()
    p = make_params(max_bases=max(rs.n_bases, 1), **params)
    seq = torch.from_numpy(rs.seq).cuda()
    qual = torch.from_numpy(rs.qual).cuda()
    offs = torch.from_numpy(rs.offsets.astype(np.int64)).cuda()
    keys = torch.zeros((capacity, 2), dtype=torch.int64, device="cuda")
    counts = torch.zeros(capacity, dtype=torch.int32, device="cuda")
    ext = torch.zeros((capacity, 8), dtype=torch.int32, device="cuda")
    codes = torch.zeros((capacity, 2), dtype=torch.uint8, device="cuda")
    n_out = ctypes.c_uint64(0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.kmer_analysis_count_small_noalloc(
        ctypes.byref(p), seq.data_ptr(), qual.data_ptr(), offs.data_ptr(), rs.n_reads, rs.n_bases,
        keys.data_ptr(), counts.data_ptr(), ext.data_ptr(), codes.data_ptr(), capacity,
        ctypes.byref(n_out), stream)
    n = int(n_out.value)
    m = min(n, capacity)
    k = keys[:m].cpu().numpy().view(np.uint64)
    c = counts[:m].cpu().numpy().view(np.uint32)
    e = ext[:m].cpu().numpy().view(np.uint32)
    cd = codes[:m].cpu().numpy()
    order = np.lexsort((k[:, 0], k[:, 1]))
    return rc, n, k[order], c[order], e[order], cd[order]


def _same(reg, got):
    rc, n, k, c, e, cd = got
    assert rc == 0, rc
    assert n == len(reg)
    np.testing.assert_array_equal(k, reg.keys)
    np.testing.assert_array_equal(c, reg.counts)
    np.testing.assert_array_equal(e, reg.ext)
    np.testing.assert_array_equal(cd, reg.codes)


def test_noalloc_matches_regular_path_two_calls(torch_cuda):
    torch = torch_cuda
    # call 1: k = 31 on a small synthetic genome (~150 kbases)
    a = synth.workload("plain_1m", scale=0.005)
    pa = dict(k=31, min_depth=2, min_ext_count=2, qual_threshold=20)
    assert a.n_bases <= 262144 and a.n_reads <= 262144
    reg_a = _regular(torch, a, **pa)
    assert len(reg_a) > 1000
    _same(reg_a, _noalloc(torch, a, len(reg_a) + 10, **pa))
    # call 2, right after: k = 51 (two-word keys), N bases, lowercase, ragged reads
    b = synth.random_reads(seed=5, n_reads=900, min_len=0, max_len=220,
                           alphabet=b"ACGTACGTACGTACGTacgtN", q_lo=10, q_hi=40)
    b.seq[: b.n_bases // 2] = np.frombuffer((b"ACGTTGCA" * (b.n_bases // 16 + 1))[: b.n_bases // 2], np.uint8)
    pb = dict(k=51, min_depth=2, min_ext_count=1, qual_threshold=20)
    reg_b = _regular(torch, b, **pb)
    _same(reg_b, _noalloc(torch, b, len(reg_b) + 1, **pb))
    # and the first input again: nothing of call 2 may leak into call 3
    _same(reg_a, _noalloc(torch, a, len(reg_a), **pa))


def _oracle_same(rs, got, **params):
    import oracle
    want = oracle.run(rs.seq, rs.qual, rs.offsets, k=params["k"], min_depth=params["min_depth"],
                      min_ext_count=params["min_ext_count"], qual_threshold=params["qual_threshold"],
                      canonical=params.get("canonical", True))
    _same(want, got)


def test_noalloc_at_the_limits_and_vs_oracle(torch_cuda):
    """The sizes the fixed array is laid out for, used to the last byte, and the cases with no
    work: exactly KMA_NOALLOC_MAX_BASES bases, exactly KMA_NOALLOC_MAX_READS (very short)
    reads, an empty read set, forward-only keys. Each result equals the regular path's and the
    oracle's."""
    torch = torch_cuda
    from paper_1705_11147_gb300 import capi
    nb = capi.KMA_NOALLOC_MAX_BASES
    # exactly the base limit, reads of 100-250 bases, k = 31
    rs = synth.random_reads(seed=11, n_reads=2000, min_len=100, max_len=250, alphabet=b"ACGTACGTACGTN",
                            q_lo=10, q_hi=40)
    cut = int(np.searchsorted(rs.offsets, nb, side="right")) - 1
    offs = rs.offsets[: cut + 1].copy()
    offs = np.append(offs, nb).astype(np.uint64)
    full = synth.ReadSet(rs.seq[:nb].copy(), rs.qual[:nb].copy(), offs)
    full.seq[: nb // 2] = np.frombuffer((b"ACGTTGCAAC" * (nb // 20 + 1))[: nb // 2], np.uint8)
    assert full.n_bases == nb
    pa = dict(k=31, min_depth=2, min_ext_count=2, qual_threshold=20)
    got = _noalloc(torch, full, nb, **pa)
    _same(_regular(torch, full, **pa), got)
    _oracle_same(full, got, **pa)
    # exactly the read limit and the base limit at once: 262,143 reads of 0 or 1 base and one
    # long read holding the rest, k = 1
    lens = np.random.default_rng(3).integers(0, 2, capi.KMA_NOALLOC_MAX_READS)
    lens[-1] = nb - int(lens[:-1].sum())
    tot = int(lens.sum())
    assert tot == nb
    tiny = synth.random_reads(seed=12, n_reads=1, min_len=tot, max_len=tot, alphabet=b"ACGT", q_lo=15, q_hi=40)
    offs = np.zeros(lens.size + 1, np.uint64)
    offs[1:] = np.cumsum(lens)
    tiny = synth.ReadSet(tiny.seq, tiny.qual, offs)
    assert tiny.n_reads == capi.KMA_NOALLOC_MAX_READS and tiny.n_bases == nb
    pt = dict(k=1, min_depth=1, min_ext_count=1, qual_threshold=20)
    got = _noalloc(torch, tiny, 16, **pt)
    _same(_regular(torch, tiny, use_bloom=False, **pt), got)
    _oracle_same(tiny, got, **pt)
    # forward-only keys (canonical = 0), even k allowed
    pf = dict(k=20, min_depth=2, min_ext_count=1, qual_threshold=20, canonical=False)
    got = _noalloc(torch, full, nb, **pf)
    _same(_regular(torch, full, **pf), got)
    _oracle_same(full, got, **pf)
    # no reads at all: no records, and the array's previous contents do not show through
    empty = synth.ReadSet(np.zeros(0, np.uint8), np.zeros(0, np.uint8), np.zeros(1, np.uint64))
    rc, n, *_ = _noalloc(torch, empty, 8, **pa)
    assert rc == 0 and n == 0


def test_noalloc_limits_and_capacity(torch_cuda):
    torch = torch_cuda
    from paper_1705_11147_gb300 import capi
    a = synth.workload("plain_1m", scale=0.005)
    pa = dict(k=31, min_depth=2, min_ext_count=2, qual_threshold=20)
    reg = _regular(torch, a, **pa)
    # too small an output: KMA_EFULL and the size it needs
    rc, n, *_ = _noalloc(torch, a, 100, **pa)
    assert rc == capi.KMA_EFULL and n == len(reg)
    # sizes beyond the fixed scratch are rejected before anything runs
    lib = capi.load()
    from paper_1705_11147_gb300 import make_params
    p = make_params(k=31, max_bases=1)
    n_out = ctypes.c_uint64(7)
    rc = lib.kmer_analysis_count_small_noalloc(ctypes.byref(p), None, None, None, 10,
                                               capi.KMA_NOALLOC_MAX_BASES + 1, None, None, None,
                                               None, 0, ctypes.byref(n_out), None)
    assert rc == capi.KMA_ETOOLARGE and n_out.value == 0
    assert b"scratch" in lib.kmer_analysis_strerror(rc)
