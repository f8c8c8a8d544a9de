"""Pins for the CPU oracle against what the paper and plain mathematics fix.

- the paper's worked examples (Section 2 chopping figure, Section 2 fork, Section 5.2 CTG
  entry), stored as text fixtures under tests/golden/;
- a brute-force restatement on tiny inputs written independently here (Python strings,
  str.translate, collections.Counter);
- invariants: total count = valid windows, reverse-complement symmetry, read-order and
  partition independence, extension sums;
- a statistical check of the Section 2 coverage formula f = d (1 - (k-1)/L).
"""
import math
import os
import re
from collections import Counter

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
CODE = {"A": 0, "C": 1, "G": 2, "T": 3, "X": 4, "F": 5}


def _fixture(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _as_dict(res, k):
    strs = oracle.unpack(res.keys, k)
    return {s: (int(res.counts[i]), tuple(int(x) for x in res.ext[i]), tuple(int(x) for x in res.codes[i]))
            for i, s in enumerate(strs)}


# ------------------------------------------------------------------ paper worked examples

def test_chopping_example_forward():
    seq, qual, offs = oracle.reads_from_strings(["GATCTGAACCG"])
    res = oracle.run(seq, qual, offs, k=3, min_depth=1, min_ext_count=1, canonical=False)
    got = {s: int(c) for s, c in zip(oracle.unpack(res.keys, 3), res.counts)}
    want = {r[0]: int(r[1]) for r in _fixture("chop_GATCTGAACCG_k3.txt")}
    assert got == want
    assert res.valid_windows == 9


def test_chopping_example_canonical():
    seq, qual, offs = oracle.reads_from_strings(["GATCTGAACCG"])
    res = oracle.run(seq, qual, offs, k=3, min_depth=1, min_ext_count=1, canonical=True)
    got = _as_dict(res, 3)
    want = {}
    for key, cnt, left, right in _fixture("canonical_GATCTGAACCG_k3.txt"):
        want[key] = (int(cnt), tuple(int(x) for x in left.split(",")) + tuple(int(x) for x in right.split(",")))
    assert {s: (v[0], v[1]) for s, v in got.items()} == want
    assert int(res.counts.sum()) == 9


def test_contig_entry_ctg():
    seq, qual, offs = oracle.reads_from_strings(["GATCTGA", "GATCTGA"])
    res = oracle.run(seq, qual, offs, k=3, min_depth=2, min_ext_count=2, canonical=False)
    got = _as_dict(res, 3)
    for kmer, left, right in _fixture("contig_CTG_value.txt"):
        assert got[kmer][2] == (CODE[left], CODE[right]), kmer
    # the two-letter value of CTG rendered [right][left] is "AT"
    c = got["CTG"][2]
    assert "ACGT"[c[1]] + "ACGT"[c[0]] == "AT"


def test_fork_gaa():
    seq, qual, offs = oracle.reads_from_strings(["GAAC", "GAAC", "GAAT", "GAAT"])
    res = oracle.run(seq, qual, offs, k=3, min_depth=2, min_ext_count=2, canonical=False)
    got = _as_dict(res, 3)
    for kmer, cnt, left, right in _fixture("fork_GAA.txt"):
        assert got[kmer][0] == int(cnt)
        assert got[kmer][2] == (CODE[left], CODE[right]), kmer
    uu = res.uu_mask()
    assert not uu.any()  # no k-mer here has unique extensions on both sides


def test_quality_gate_boundary():
    seq, qual, offs = oracle.reads_from_strings(["ACGTA"], ["54II4"])
    res = oracle.run(seq, qual, offs, k=3, min_depth=1, min_ext_count=1, canonical=False,
                     qual_threshold=20)
    got = _as_dict(res, 3)
    for kmer, cnt, left, right in _fixture("quality_gate.txt"):
        e = tuple(int(x) for x in left.split(",")) + tuple(int(x) for x in right.split(","))
        assert got[kmer][:2] == (int(cnt), e), kmer


# ------------------------------------------------------------------ brute force

COMP = str.maketrans("ACGT", "TGCA")


def brute_force(reads, quals, k, min_depth, min_ext, Q, qoff=33, canonical=True):
    """Independent restatement: enumerate substrings, flip by string reversal."""
    table = {}
    for s, q in zip(reads, quals):
        s = s.upper()
        ok = [c in "ACGT" and ord(qc) - qoff >= Q for c, qc in zip(s, q)]
        for i in range(len(s) - k + 1):
            w = s[i:i + k]
            if re.fullmatch("[ACGT]+", w) is None:
                continue
            rc = w.translate(COMP)[::-1]
            before = s[i - 1] if i > 0 and ok[i - 1] else None
            after = s[i + k] if i + k < len(s) and ok[i + k] else None
            if canonical and rc < w:
                key, left, right = rc, (after.translate(COMP) if after else None), \
                    (before.translate(COMP) if before else None)
            else:
                key, left, right = w, before, after
            rec = table.setdefault(key, [0, Counter(), Counter()])
            rec[0] += 1
            if left:
                rec[1][left] += 1
            if right:
                rec[2][right] += 1
    out = {}
    for key, (cnt, lc, rc_) in table.items():
        if cnt < min_depth:
            continue
        ext = tuple(lc[b] for b in "ACGT") + tuple(rc_[b] for b in "ACGT")

        def code(cn):
            hq = [b for b in "ACGT" if cn[b] >= min_ext]
            return CODE["X"] if not hq else (CODE[hq[0]] if len(hq) == 1 else CODE["F"])
        out[key] = (cnt, ext, (code(lc), code(rc_)))
    return out


@pytest.mark.parametrize("k", [1, 3, 5, 7, 31, 33, 63])
@pytest.mark.parametrize("canonical", [True, False])
def test_brute_force_tiny(k, canonical):
    rs = synth.random_reads(seed=1000 + k, n_reads=60, min_len=0, max_len=90,
                            alphabet=b"ACGTACGTACGTacgtNR", q_lo=15, q_hi=25)
    reads = [bytes(rs.seq[int(rs.offsets[i]):int(rs.offsets[i + 1])]).decode() for i in range(rs.n_reads)]
    quals = [bytes(rs.qual[int(rs.offsets[i]):int(rs.offsets[i + 1])]).decode() for i in range(rs.n_reads)]
    for md, me in [(1, 1), (2, 2), (3, 1)]:
        res = oracle.run(rs.seq, rs.qual, rs.offsets, k=k, min_depth=md, min_ext_count=me,
                         qual_threshold=20, canonical=canonical)
        assert _as_dict(res, k) == brute_force(reads, quals, k, md, me, 20, canonical=canonical)


def test_brute_force_low_complexity():
    # repeats inside reads: same k-mer many times in one read, palindromic neighbourhoods
    reads = ["ACACACACACACACACAC", "TTTTTTTTTTTT", "AAAAAAAAAAAAAAAA", "ACGTACGTACGT", "GCGCGCGC" * 3]
    quals = ["I" * len(r) for r in reads]
    seq, qual, offs = oracle.reads_from_strings(reads, quals)
    for k in (3, 5, 7):
        res = oracle.run(seq, qual, offs, k=k, min_depth=1, min_ext_count=2)
        assert _as_dict(res, k) == brute_force(reads, quals, k, 1, 2, 20)


# ------------------------------------------------------------------ invariants

@pytest.fixture(scope="module")
def small_set():
    return synth.workload("bacterial_5m", scale=0.02)  # 100 kbp genome, N bases, repeats


def _valid_windows_python(rs, k):
    n = 0
    for i in range(rs.n_reads):
        s = bytes(rs.seq[int(rs.offsets[i]):int(rs.offsets[i + 1])]).decode().upper()
        for run in re.findall("[ACGT]+", s):
            n += max(len(run) - k + 1, 0)
    return n


def test_total_count_equals_valid_windows(small_set):
    k = 51
    res = oracle.run_readset(small_set, min_depth=1)
    assert int(res.counts.astype(np.int64).sum()) == res.valid_windows
    assert res.valid_windows == _valid_windows_python(small_set, k)


def test_extension_sums_bounded(small_set):
    res = oracle.run_readset(small_set, min_depth=1, min_ext_count=1)
    left = res.ext[:, :4].astype(np.int64).sum(1)
    right = res.ext[:, 4:].astype(np.int64).sum(1)
    assert (left <= res.counts).all() and (right <= res.counts).all()
    # every read has exactly one window without a left neighbour and one without a right
    # neighbour (if it has a valid window at its ends), so the deficits are positive overall
    assert left.sum() < res.counts.astype(np.int64).sum()


def _revcomp_readset(rs):
    comp = np.arange(256, dtype=np.uint8)
    for a, b in zip(b"ACGTacgt", b"TGCAtgca"):
        comp[a] = b
    seq = np.empty_like(rs.seq)
    qual = np.empty_like(rs.qual)
    for i in range(rs.n_reads):
        a, b = int(rs.offsets[i]), int(rs.offsets[i + 1])
        seq[a:b] = comp[rs.seq[a:b][::-1]]
        qual[a:b] = rs.qual[a:b][::-1]
    return seq, qual


def test_reverse_complement_invariance(small_set):
    res = oracle.run_readset(small_set)
    seq, qual = _revcomp_readset(small_set)
    res2 = oracle.run(seq, qual, small_set.offsets, **_params(small_set))
    for f in ("keys", "counts", "ext", "codes"):
        np.testing.assert_array_equal(getattr(res, f), getattr(res2, f))


def _params(rs):
    p = dict(rs.meta["params"])
    p.pop("bloom_fpr")
    return p


def test_read_order_invariance(small_set):
    res = oracle.run_readset(small_set)
    perm = np.random.default_rng(5).permutation(small_set.n_reads)
    lens = np.diff(small_set.offsets.astype(np.int64))[perm]
    offs = np.zeros(small_set.n_reads + 1, np.uint64)
    offs[1:] = np.cumsum(lens)
    seq = np.concatenate([small_set.seq[int(small_set.offsets[i]):int(small_set.offsets[i + 1])] for i in perm])
    qual = np.concatenate([small_set.qual[int(small_set.offsets[i]):int(small_set.offsets[i + 1])] for i in perm])
    res2 = oracle.run(seq, qual, offs, **_params(small_set))
    for f in ("keys", "counts", "ext", "codes"):
        np.testing.assert_array_equal(getattr(res, f), getattr(res2, f))


def test_partition_union_equals_whole(small_set):
    """Owner-computes (Section 5.1): the union of the per-owner results is the result."""
    whole = oracle.run_readset(small_set)
    parts = [oracle.run_readset(small_set, part=i, n_parts=5) for i in range(5)]
    keys = np.concatenate([p.keys for p in parts])
    order = np.lexsort((keys[:, 0], keys[:, 1]))
    np.testing.assert_array_equal(keys[order], whole.keys)
    np.testing.assert_array_equal(np.concatenate([p.counts for p in parts])[order], whole.counts)
    np.testing.assert_array_equal(np.concatenate([p.ext for p in parts])[order], whole.ext)
    for i, p in enumerate(parts):
        assert (oracle.partition_of(p.keys, 51, 5) == i).all()


def test_partition_set_equals_selected_parts(small_set):
    """A set of owner partitions in one scan (used to check full-size GPU runs on many
    partitions at once) keeps exactly the whole result's keys whose owner is in the set, with
    their records unchanged; the set and its complement are disjoint and cover the whole."""
    whole = oracle.run_readset(small_set)
    owner = oracle.partition_of(whole.keys, 51, 7)
    chosen = [0, 3, 4]
    got = oracle.run_readset(small_set, n_parts=7, parts=chosen)
    rest = oracle.run_readset(small_set, n_parts=7, parts=[1, 2, 5, 6])
    sel = np.isin(owner, chosen)
    assert 0 < len(got) < len(whole) and len(got) + len(rest) == len(whole)
    for f in ("keys", "counts", "ext", "codes"):
        np.testing.assert_array_equal(getattr(got, f), getattr(whole, f)[sel])
        np.testing.assert_array_equal(getattr(rest, f), getattr(whole, f)[~sel])
    assert got.valid_windows == whole.valid_windows
    # one part given as a set is that part
    one = oracle.run_readset(small_set, n_parts=7, parts=[5])
    np.testing.assert_array_equal(one.keys, oracle.run_readset(small_set, part=5, n_parts=7).keys)


def test_threads_do_not_change_result(small_set):
    a = oracle.run_readset(small_set, threads=1)
    b = oracle.run_readset(small_set, threads=7)
    for f in ("keys", "counts", "ext", "codes"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_query_reorients():
    seq, qual, offs = oracle.reads_from_strings(["GATCTGAACCG"])
    res = oracle.run(seq, qual, offs, k=3, min_depth=1, min_ext_count=1, keep_table=True)
    counts, ext, codes = res.query(oracle.pack(["ATC", "GAT", "TTT"]))
    assert list(counts) == [2, 2, 0]
    assert list(ext[0]) == [0, 0, 2, 0, 0, 0, 0, 1]      # left G x2, right T x1
    assert list(ext[1]) == [1, 0, 0, 0, 0, 2, 0, 0]      # seen as GAT: left A x1, right C x2
    assert list(codes[1]) == [0, 1] and list(codes[2]) == [4, 4]


def test_pack_roundtrip():
    kmers = ["A" * 63, "T" * 63, "ACGT" * 15 + "ACG", "C" * 31, "G"]
    for s in kmers:
        keys = oracle.pack([s])
        assert oracle.unpack(keys, len(s)) == [s]
    k = oracle.pack(["T" * 63])
    assert int(k[0, 1]) == 2**62 - 1 and int(k[0, 0]) == 2**64 - 1
    k = oracle.pack(["C" + "A" * 30])
    assert int(k[0, 0]) == 1 << 60 and int(k[0, 1]) == 0


# ------------------------------------------------------------------ statistics (Section 2)

def test_coverage_formula_peak():
    """Section 2: a true k-mer is expected f = d (1 - (k-1)/L) times; error-free occurrences
    scale that by (1 - e)^k. The count histogram of solid keys peaks near that value."""
    rs = synth.workload("plain_1m", scale=0.25)
    res = oracle.run_readset(rs)
    d, L, k, e = 30, 150, 31, 0.005
    f = d * (1 - (k - 1) / L) * (1 - e) ** k
    hist = np.bincount(res.counts[res.counts >= 5].astype(np.int64))
    mode = int(np.argmax(hist))
    assert abs(mode - f) <= 2.0, (mode, f)
    mean = float(res.counts[res.counts >= 8].mean())
    assert abs(mean - f) / f < 0.05, (mean, f)


# ---- HyperLogLog sketch (Section 5.1's cardinality pass) -----------------------------------

def _random_keys(n, seed, k=51):
    rng = np.random.default_rng(seed)
    hi_bits = max(2 * k - 64, 1)
    return np.stack([rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2)
                     + rng.integers(0, 2, n, dtype=np.uint64),
                     rng.integers(0, 2**hi_bits, n, dtype=np.uint64)], 1)


def test_hll_empty_and_single():
    # no key: every register empty, linear counting gives exactly 0
    for p in (4, 10, 14):
        r = oracle.hll_registers(np.zeros((0, 2), np.uint64), p)
        assert not r.any() and oracle.hll_estimate(r, p) == 0.0
    # one key: one register set; linear counting m ln(m / (m - 1)) = 1 + O(1/m)
    r = oracle.hll_registers(_random_keys(1, 7), 14)
    assert (r > 0).sum() == 1
    assert abs(oracle.hll_estimate(r, 14) - 1.0) < 1e-3


@pytest.mark.parametrize("n,p", [(1000, 14), (50_000, 12), (50_000, 14), (400_000, 14), (400_000, 10)])
def test_hll_error_bound(n, p):
    """Distinct random keys: the estimate is within 4 relative standard errors (1.04/sqrt(m),
    Section 5.1 / Flajolet et al.) of the true count, in the linear-counting and the raw range."""
    keys = _random_keys(n, 1000 + n + p)
    est = oracle.hll_estimate(oracle.hll_registers(keys, p), p)
    assert abs(est - n) / n < 4 * 1.04 / math.sqrt(2**p), (est, n)


def test_hll_duplicates_and_merge():
    a, b = _random_keys(20_000, 11), _random_keys(30_000, 12)
    ra, rb = oracle.hll_registers(a, 14), oracle.hll_registers(b, 14)
    # repeated keys change nothing: the sketch is a function of the distinct set
    assert np.array_equal(oracle.hll_registers(np.concatenate([a, a[::3]]), 14), ra)
    # union sketch = elementwise maximum (how sketches of read batches or GPUs merge)
    assert np.array_equal(oracle.hll_registers(np.concatenate([a, b]), 14), np.maximum(ra, rb))


def test_hll_rank_distribution():
    """Ranks are geometric: with n keys in one register class, a register reaches rank >= r
    with probability 1 - (1 - 2^-(r-1))^(n/m). Checked on the fraction of empty registers and
    of registers at rank 1 only (the two ends a shifted or reversed rank would break)."""
    p, n = 12, 8192
    m = 2**p
    r = oracle.hll_registers(_random_keys(n, 21), p)
    lam = n / m
    empty = (r == 0).mean()
    assert abs(empty - math.exp(-lam)) < 0.02
    # a register stays at rank 1 iff all its keys have rank 1 (prob 1/2 each)
    only1 = (r == 1).mean()
    want = sum(math.exp(-lam) * lam**j / math.factorial(j) * 0.5**j for j in range(1, 40))
    assert abs(only1 - want) < 0.02



# ---- FASTQ parsing (input side of the stage) ------------------------------------------------

def test_fastq_golden_records():
    text = open(os.path.join(GOLD, "fastq_records.fastq"), "rb").read()
    want = [ln.split() for ln in open(os.path.join(GOLD, "fastq_records_expected.txt"))
            if ln.strip() and not ln.startswith("#")]
    seq, qual, offs = oracle.parse_fastq(text)
    assert len(offs) == len(want) + 1
    for r, (b, q) in enumerate(want):
        b, q = ("" if b == "-" else b), ("" if q == "-" else q)
        assert bytes(seq[offs[r]:offs[r + 1]]).decode() == b
        assert bytes(qual[offs[r]:offs[r + 1]]).decode() == q
    # trailing empty lines change nothing; a missing '+' or a length mismatch is an error
    assert all(np.array_equal(a, b) for a, b in zip(oracle.parse_fastq(text + b"\n\n\r\n"), (seq, qual, offs)))
    with pytest.raises(ValueError):
        oracle.parse_fastq(b"@a\nAC\n-\nII\n")
    with pytest.raises(ValueError):
        oracle.parse_fastq(b"@a\nAC\n+\nI\n")
    with pytest.raises(ValueError):
        oracle.parse_fastq(b"@a\nAC\n+\nII\nX\n")


# ---- Contig generation (Section 5.2) --------------------------------------------------------

def _revcomp(s):
    return s.translate(str.maketrans("ACGT", "TGCA"))[::-1]


def _contigs_of(reads, k, canonical, min_depth=1, min_ext=1):
    seq, qual, offs = oracle.reads_from_strings(reads)
    r = oracle.run(seq, qual, offs, k=k, min_depth=min_depth, min_ext_count=min_ext, canonical=canonical)
    got, cycles = oracle.contigs(r.keys, r.codes, k, canonical)
    return got, cycles, r


def test_contig_golden_examples():
    for line in open(os.path.join(GOLD, "contigs_examples.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        reads, want = (x.strip() for x in line.split("|"))
        got, cycles, _ = _contigs_of(reads.split(","), 3, canonical=False, min_depth=2, min_ext=2)
        assert sorted(got) == want.split(",") and cycles == 0, (reads, got)


def _genome(n, seed):
    rng = np.random.default_rng(seed)
    return "".join("ACGT"[i] for i in rng.integers(0, 4, n))


def test_contig_linear_genome_is_one_contig():
    """Error-free reads from both strands tiling a random genome: one contig, the genome
    itself in one orientation."""
    g, k, L = _genome(3000, 5), 31, 120
    reads = []
    for i in range(0, len(g) - L + 1, 7):
        reads += [g[i:i + L], _revcomp(g[i:i + L])]
    reads += [g[-L:], _revcomp(g[-L:])]
    got, cycles, _ = _contigs_of(reads, k, canonical=True, min_depth=2)
    assert cycles == 0 and len(got) == 1 and got[0] in (g, _revcomp(g))


def test_contig_circular_genome_is_cut_cycle():
    """Reads around a circular genome: one cycle, cut at its smallest k-mer (left side), so
    the contig starts with that k-mer and is the whole circle plus k - 1 bases."""
    g, k, L = _genome(2000, 6), 31, 100
    gg = g + g
    reads = []
    for i in range(0, len(g), 5):
        reads += [gg[i:i + L], _revcomp(gg[i:i + L])]
    got, cycles, r = _contigs_of(reads, k, canonical=True, min_depth=2)
    assert cycles == 1 and len(got) == 1
    c = got[0]
    assert len(c) == len(g) + k - 1 and c[-(k - 1):] == c[:k - 1]
    assert c[:len(g)] in gg or c[:len(g)] in _revcomp(g) * 2      # a rotation, either strand
    kmers = [gg[i:i + k] for i in range(len(g))]
    smallest = min(min(x, _revcomp(x)) for x in kmers)
    # cut on the smallest k-mer's left side: it is an end of the contig, read forward from it
    assert c.startswith(smallest) or c.endswith(_revcomp(smallest))


def test_contig_vertices_used_once():
    """Synthetic reads with errors and repeats: every vertex (no fork on either side) lies in
    exactly one contig, and every k-mer of every contig is a vertex."""
    rs = synth.workload("plain_1m", scale=0.05)
    r = oracle.run(rs.seq, rs.qual, rs.offsets, k=31, min_depth=2, min_ext_count=2, canonical=True)
    got, cycles = oracle.contigs(r.keys, r.codes, 31, True)
    vertices = set(oracle.unpack(r.keys[(r.codes[:, 0] != 5) & (r.codes[:, 1] != 5)], 31))
    seen = []
    for c in got:
        for i in range(len(c) - 30):
            w = c[i:i + 31]
            seen.append(min(w, _revcomp(w)))
    assert len(seen) == len(set(seen)) == len(vertices) and set(seen) == vertices


# ------------------------------------------------------------------ heavy hitters (Misra-Gries)

def _exact_counts(stream):
    keys, counts = np.unique(np.ascontiguousarray(stream).view([("lo", np.uint64), ("hi", np.uint64)]).ravel(),
                             return_counts=True)
    return {(int(k["lo"]), int(k["hi"])): int(c) for k, c in zip(keys, counts)}


def test_misra_gries_worked_example():
    """By hand, m = 2: AAA CCC AAA GGG AAA -> {AAA:1, CCC:1} after three items' updates, GGG
    finds no free counter (both decrement: AAA 1, CCC 0), the last AAA raises AAA to 2."""
    keys, counts = oracle.misra_gries(oracle.pack(["AAA", "CCC", "AAA", "GGG", "AAA"]), 2)
    assert oracle.unpack(keys, 3) == ["AAA"] and list(counts) == [2]


def test_misra_gries_exact_with_few_keys_and_bound_otherwise():
    """With at most m distinct keys no decrement ever happens: the summary is the exact
    frequency table. With more, every key of frequency f > n/(m+1) is kept with a count c,
    f - n/(m+1) <= c <= f, and a key left out has f <= n/(m+1) (Misra and Gries 1982)."""
    rng = np.random.default_rng(7)
    for trial in range(30):
        m = int(rng.integers(2, 12))
        n_keys = int(rng.integers(1, m + 1))
        pool = rng.integers(0, 2**40, (n_keys, 2), dtype=np.uint64)
        stream = pool[rng.integers(0, n_keys, int(rng.integers(1, 400)))]
        keys, counts = oracle.misra_gries(stream, m)
        got = {(int(a), int(b)): int(c) for (a, b), c in zip(keys, counts)}
        assert got == _exact_counts(stream)
    for trial in range(40):
        m = int(rng.integers(2, 16))
        n = int(rng.integers(50, 3000))
        heavy = rng.integers(0, 2**40, (3, 2), dtype=np.uint64)
        noise = rng.integers(0, 2**40, (n, 2), dtype=np.uint64)
        pick = rng.random(n)
        stream = np.where((pick < 0.5)[:, None], heavy[rng.integers(0, 3, n)], noise)
        keys, counts = oracle.misra_gries(stream, m)
        got = {(int(a), int(b)): int(c) for (a, b), c in zip(keys, counts)}
        exact = _exact_counts(stream)
        eps = n / (m + 1)
        assert len(got) <= m
        for key, f in exact.items():
            c = got.get(key, 0)
            assert f - eps <= c <= f
            if f > eps:
                assert key in got


@pytest.mark.parametrize("sample", [16, 64])
def test_sampled_stream_by_brute_force(sample):
    """The sampled stream: windows starting at every `sample`-th position of the reads laid out
    with one separator per read, canonical keys, invalid windows skipped; brute force on
    strings."""
    rng = np.random.default_rng(11)
    reads = ["".join(rng.choice(list("ACGTACGTNacgt"), int(rng.integers(0, 70)))) for _ in range(300)]
    seq, qual, offs = oracle.reads_from_strings(reads)
    tr = str.maketrans("ACGT", "TGCA")
    for k, canonical in ((5, True), (21, True), (6, False)):
        want, pos = [], 0
        for r in reads:
            up = r.upper()
            for i in range(len(r) - k + 1):
                w = up[i:i + k]
                if (pos + i) % sample == 0 and set(w) <= set("ACGT"):
                    rc = w.translate(tr)[::-1]
                    want.append(min(w, rc) if canonical else w)
            pos += len(r) + 1
        got = oracle.unpack(oracle.sampled_stream(seq, qual, offs, k=k, canonical=canonical, sample=sample), k)
        assert got == want


def test_stream_bucket_is_the_sketch_register_prefix():
    """The sub-stream of a key is the top 5 bits of the sketch hash: the register index a
    one-key HyperLogLog sketch of precision 14 sets, shifted right by 9."""
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 2**62, (200, 2), dtype=np.uint64)
    b = oracle.stream_bucket(keys, 5)
    for i in range(keys.shape[0]):
        regs = oracle.hll_registers(keys[i:i + 1], 14)
        assert int(np.nonzero(regs)[0][0]) >> 9 == int(b[i])
    assert len(np.unique(oracle.stream_bucket(rng.integers(0, 2**62, (20000, 2), dtype=np.uint64), 5))) == 32
