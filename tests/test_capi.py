"""C ABI checks that need no GPU: the library loads, exports every declared entry point, and
its host-only sizing logic (kmer_analysis_plan) follows the Bloom-filter mathematics of
Section 5.1 and validates parameters."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1705_11147_gb300 import build, capi
    build.build()
    return capi.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(kmer_analysis_\w+)\s*\(", text, re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14, names
    for n in names:
        assert hasattr(lib, n), n
    from paper_1705_11147_gb300 import capi
    assert set(names) == set(capi._SIGS), set(names) ^ set(capi._SIGS)


def test_strerror(lib):
    for code in range(0, -8, -1):
        assert lib.kmer_analysis_strerror(code)
    assert b"unknown" in lib.kmer_analysis_strerror(-99)


def _plan(**kw):
    from paper_1705_11147_gb300 import capi, make_params, plan
    return plan(make_params(**kw))


def _plan_rc(**kw):
    from paper_1705_11147_gb300 import capi, make_params
    p = make_params(**kw)
    out = capi.kma_plan()
    return capi.load().kmer_analysis_plan(ctypes.byref(p), ctypes.byref(out))


def test_param_validation(lib):
    from paper_1705_11147_gb300 import capi
    assert _plan_rc(k=31, max_bases=1000) == 0
    assert _plan_rc(k=32, max_bases=1000) == capi.KMA_EINVAL          # even k, canonical
    assert _plan_rc(k=32, max_bases=1000, canonical=False) == 0       # forward mode allows it
    assert _plan_rc(k=0, max_bases=1000) == capi.KMA_EINVAL
    assert _plan_rc(k=65, max_bases=1000) == capi.KMA_EINVAL
    assert _plan_rc(k=63, max_bases=1000) == 0
    assert _plan_rc(k=31, max_bases=1000, min_depth=1) == capi.KMA_EINVAL   # Bloom needs >= 2
    assert _plan_rc(k=31, max_bases=1000, min_depth=1, use_bloom=False) == 0
    assert _plan_rc(k=31, max_bases=0) == capi.KMA_EINVAL
    assert _plan_rc(k=31, max_bases=1000, block_threads=100) == capi.KMA_EINVAL
    assert _plan_rc(k=31, max_bases=1000, block_threads=512) == capi.KMA_EINVAL
    assert _plan_rc(k=31, max_bases=1000, windows_per_thread=3) == capi.KMA_EINVAL
    assert _plan_rc(k=31, max_bases=1000, windows_per_thread=8) == 0
    assert _plan_rc(k=31, max_bases=1000, n_parts=4, part=4) == capi.KMA_EINVAL
    assert _plan_rc(k=31, max_bases=1000, load_factor=0.99) == capi.KMA_EINVAL


def _blocked_fpr_independent(m, words, h):
    """Same model as the library, evaluated differently: direct Poisson pmf via lgamma."""
    lam = m / words
    tot = 0.0
    for j in range(0, int(lam + 15 * math.sqrt(lam + 1) + 60)):
        pmf = math.exp(-lam + j * math.log(lam) - math.lgamma(j + 1)) if lam > 0 else (1.0 if j == 0 else 0.0)
        tot += pmf * (1 - (63 / 64) ** (h * j)) ** h
    return tot


@pytest.mark.parametrize("m,fpr", [(4_400_000, 0.01), (2_100_000_000, 0.01), (1_000_000, 0.05)])
def test_bloom_sizing(lib, m, fpr):
    pl = _plan(k=31, max_bases=10 * m, expected_distinct=m, bloom_fpr=fpr)
    bits_per_key = pl.bloom_words * 64 / m
    # estimate matches an independent evaluation of the blocked model and meets the target
    est = _blocked_fpr_independent(m, pl.bloom_words, pl.bloom_hashes)
    assert abs(est - pl.bloom_fpr_est) < 1e-6 + 1e-3 * est
    assert est <= fpr * 1.001
    # a slightly smaller filter would miss the target (the search is tight)
    assert _blocked_fpr_independent(m, pl.bloom_words * 0.97, pl.bloom_hashes) > fpr
    # the standard (unblocked) filter, (1 - e^{-h m/n})^h with h = ln2 n/m, needs
    # n/m = -ln(p)/ln(2)^2 bits per key; blocking into one word can only cost more
    std_bits = -math.log(fpr) / math.log(2) ** 2
    assert bits_per_key >= std_bits
    assert bits_per_key < 2.0 * std_bits
    # the standard formula itself at the optimum reproduces the target
    h_opt = math.log(2) * std_bits
    assert abs((1 - math.exp(-h_opt / std_bits)) ** h_opt - fpr) < 1e-9


def test_bloom_blocked_model_vs_simulation(lib):
    """Monte-Carlo check of the blocked-filter model used for sizing (small filter)."""
    m, fpr = 20000, 0.02
    pl = _plan(k=31, max_bases=10 * m, expected_distinct=m, bloom_fpr=fpr)
    rng = np.random.default_rng(3)
    W, h = int(pl.bloom_words), int(pl.bloom_hashes)
    words = np.zeros(W, np.uint64)
    idx = rng.integers(0, W, m)
    for i in range(m):
        mask = np.uint64(0)
        for b in rng.integers(0, 64, h):
            mask |= np.uint64(1) << np.uint64(b)
        words[idx[i]] |= mask
    trials = 40000
    qi = rng.integers(0, W, trials)
    hits = 0
    for t in range(trials):
        mask = np.uint64(0)
        for b in rng.integers(0, 64, h):
            mask |= np.uint64(1) << np.uint64(b)
        hits += int((words[qi[t]] & mask) == mask)
    measured = hits / trials
    assert abs(measured - pl.bloom_fpr_est) < 0.25 * pl.bloom_fpr_est + 0.002, (measured, pl.bloom_fpr_est)


def test_table_and_arena_sizing(lib):
    pl = _plan(k=51, max_bases=1_000_000, max_reads=10_000, expected_keys=100_000, load_factor=0.5)
    assert pl.table_slots >= 200_000
    assert pl.arena_positions >= 1_010_000 and pl.arena_positions % 64 == 0
    pl2 = _plan(k=51, max_bases=1_000_000, table_capacity=12345)
    assert pl2.table_slots == 12345
    assert pl2.device_bytes > 12345 * 64
    nb = _plan(k=51, max_bases=1_000_000, use_bloom=False, min_depth=1)
    assert nb.bloom_words == 0


def test_partition_sizing(lib):
    from paper_1705_11147_gb300 import capi
    tiny = _plan(k=31, max_bases=1_000_000, expected_distinct=100_000, expected_keys=50_000)
    assert tiny.partitions == 1                       # filter + table below 32 MB: one table
    small = _plan(k=51, max_bases=30_000_000, expected_distinct=4_400_000, expected_keys=1_100_000)
    per_small = (small.bloom_words * 8 + small.table_slots * 64) / small.partitions
    assert small.partitions >= 2 and per_small <= 64 * 2**20 * 1.01  # above 32 MB: at least two
    big = _plan(k=51, max_bases=6_000_000_000, expected_distinct=2_100_000_000,
                expected_keys=300_000_000)
    per_part = (big.bloom_words * 8 + big.table_slots * 64) / big.partitions
    assert big.partitions > 1 and per_part <= 64 * 2**20 * 1.01
    assert big.bloom_words % big.partitions == 0 and big.table_slots % big.partitions == 0
    forced = _plan(k=31, max_bases=1_000_000, partitions=7)
    assert forced.partitions == 7 and forced.table_slots % 7 == 0
    one = _plan(k=31, max_bases=6_000_000_000, expected_distinct=2_100_000_000, partitions=1)
    assert one.partitions == 1
    assert _plan_rc(k=31, max_bases=1000, partitions=5000) == capi.KMA_EINVAL
    # two-word keys stage larger scatter tiles: at most 2048 partitions
    assert _plan(k=31, max_bases=1_000_000, partitions=3000).partitions == 3000
    assert _plan_rc(k=51, max_bases=1_000_000, partitions=3000) == capi.KMA_EINVAL
    assert _plan(k=51, max_bases=1_000_000, partitions=2048).partitions == 2048


def test_missing_library_fails_loudly(tmp_path):
    from paper_1705_11147_gb300 import capi
    saved = capi._LIB
    capi._LIB = None
    try:
        with pytest.raises(RuntimeError, match="not been built"):
            capi.load(str(tmp_path / "nope.so"))
    finally:
        capi._LIB = saved


def test_hll_host_estimate_matches_oracle(lib):
    """kmer_analysis_hll_estimate (the library's host-side estimator, no GPU) against the
    oracle's estimator on the same sketches: empty, linear-counting range, raw range."""
    import oracle
    from paper_1705_11147_gb300 import capi, hll_estimate
    rng = np.random.default_rng(5)
    for n, p in ((0, 14), (1, 14), (3000, 14), (200_000, 14), (200_000, 8), (5000, 4)):
        keys = np.stack([rng.integers(0, 2**63, n, dtype=np.uint64),
                         rng.integers(0, 2**38, n, dtype=np.uint64)], 1)
        regs = oracle.hll_registers(keys, p)
        want = oracle.hll_estimate(regs, p)
        got = hll_estimate(regs, p)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-12), (n, p, got, want)
    out = ctypes.c_double()
    r = np.zeros(1 << 14, np.uint8)
    assert lib.kmer_analysis_hll_estimate(r.ctypes.data, 3, ctypes.byref(out)) == capi.KMA_EINVAL
    assert lib.kmer_analysis_hll_estimate(r.ctypes.data, 15, ctypes.byref(out)) == capi.KMA_EINVAL


def test_host_result_buffers_layout():
    """Host arrays for finalize_to_host have kma_result's layout (keys[c][2] u64, counts[c]
    u32, ext[c][8] u32, codes[c][2] u8), C-contiguous."""
    from paper_1705_11147_gb300 import host_result_buffers
    keys, counts, ext, codes = host_result_buffers(5)
    assert keys.shape == (5, 2) and keys.dtype == np.uint64
    assert counts.shape == (5,) and counts.dtype == np.uint32
    assert ext.shape == (5, 8) and ext.dtype == np.uint32
    assert codes.shape == (5, 2) and codes.dtype == np.uint8
    assert all(a.flags.c_contiguous for a in (keys, counts, ext, codes))


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets of the C header's
    (checked by compiling a small C program against include/kmer_analysis.h)."""
    import shutil
    import subprocess
    from paper_1705_11147_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [capi.kma_params, capi.kma_plan, capi.kma_result, capi.kma_timings, capi.kma_contigs,
               capi.kma_estimate, capi.kma_reads]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kmer_analysis.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("{st.__name__} size %zu\\n", sizeof({st.__name__}));')
        for name, *_ in st._fields_:
            lines.append(f'  printf("{st.__name__} {name} %zu\\n", offsetof({st.__name__}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", f"-I{os.path.join(ROOT, 'include')}", str(src), "-o", str(exe)])
    out = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for st in structs:
        assert int(out[f"{st.__name__} size"]) == ctypes.sizeof(st), st.__name__
        for name, *_ in st._fields_:
            assert int(out[f"{st.__name__} {name}"]) == getattr(st, name).offset, (st.__name__, name)
