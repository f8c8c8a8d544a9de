"""Seeded synthetic read sets, the single input source for both the oracle and the CUDA path.

The paper measures on human (NA12878, 2.9 G reads of 101 bp) and wheat (2.3 G reads of
150-250 bp) read sets (Section 6). Those are not available here, so every workload is a
synthetic stand-in with the same structure: a random genome (optionally with planted,
slightly diverged repeats), reads sampled uniformly from both strands at coverage d,
substitution errors with low Phred scores on erroneous bases, and rare N bases.

Nothing here does k-mer arithmetic; see synth.c for the generator definition.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        u64, u32, p = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p
        lib.synth_genome.argtypes = [u64, u64, p]
        lib.synth_plant_repeats.argtypes = [u64, p, u64, u64, u64, u32, u32, u64]
        lib.synth_plant_repeats.restype = u64
        lib.synth_reads.argtypes = [u64, p, u64, u64, u32, p, u64, u64, p, p, p, ctypes.c_int]
        lib.synth_draws.argtypes = [u64, u64, u64, u64, p]
        _LIB = lib
    return _LIB


def _thresh(p: float) -> int:
    """Probability -> 64-bit integer threshold (u < thresh happens with probability p)."""
    if p <= 0:
        return 0
    return min(int(p * 2.0 ** 64), 2 ** 64 - 1)


def _mix(seed: int, j: int) -> int:
    d = np.zeros(1, dtype=np.uint64)
    _lib().synth_draws(seed & (2**64 - 1), 7, j, 1, d.ctypes.data)
    return int(d[0])


def draws(seed: int, stream: int, n: int, ctr0: int = 0) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    if n:
        _lib().synth_draws(seed & (2**64 - 1), stream, ctr0, n, out.ctypes.data)
    return out


def _uniform(r) -> float:
    return (int(r) >> 11) * (1.0 / 9007199254740992.0)


@dataclass
class ReadSet:
    """Reads in the layout the library consumes: ASCII bases, Phred+33 qualities and
    read offsets (n_reads + 1 entries, read r = [offsets[r], offsets[r+1]))."""
    seq: np.ndarray
    qual: np.ndarray
    offsets: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_reads(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_bases(self) -> int:
        return int(self.offsets[-1])

    def windows_upper_bound(self, k: int) -> int:
        lens = np.diff(self.offsets.astype(np.int64))
        return int(np.maximum(lens - k + 1, 0).sum())


def genome(seed: int, G: int, repeat_copies: int = 0, repeat_frac: float = 0.0,
           repeat_len=(1000, 5000), divergence: float = 0.01) -> tuple[np.ndarray, int]:
    """Uniform random genome (codes 0..3) with planted repeats; returns (codes, pasted bases)."""
    g = np.empty(G, dtype=np.uint8)
    _lib().synth_genome(seed, G, g.ctypes.data)
    pasted = 0
    if repeat_copies or repeat_frac > 0:
        lo, hi = repeat_len
        hi = min(hi, G // 4)
        lo = min(lo, hi)
        pasted = _lib().synth_plant_repeats(seed ^ 0x52E9, g.ctypes.data, G, repeat_copies,
                                            int(repeat_frac * G), lo, hi, _thresh(divergence))
    return g, int(pasted)


def reads_from_genome(seed: int, g: np.ndarray, n_reads: int, L: int = 150, err: float = 0.01,
                      n_rate: float = 0.0, lens: np.ndarray | None = None,
                      threads: int | None = None) -> ReadSet:
    G = int(g.shape[0])
    if lens is not None:
        lens = np.ascontiguousarray(lens, dtype=np.uint32)
        assert lens.shape[0] == n_reads and int(lens.max(initial=0)) <= G
        total = int(lens.astype(np.uint64).sum())
    else:
        assert L <= G
        total = n_reads * L
    seq = np.empty(total, dtype=np.uint8)
    qual = np.empty(total, dtype=np.uint8)
    offs = np.empty(n_reads + 1, dtype=np.uint64)
    threads = threads or min(64, os.cpu_count() or 1)
    _lib().synth_reads(seed, g.ctypes.data, G, n_reads, L,
                       lens.ctypes.data if lens is not None else None,
                       _thresh(err), _thresh(n_rate), seq.ctypes.data, qual.ctypes.data,
                       offs.ctypes.data, threads)
    return ReadSet(seq, qual, offs)


def simulate(seed: int, G: int, coverage: float, L: int, err: float, n_rate: float = 0.0,
             repeat_copies: int = 0, repeat_frac: float = 0.0, threads: int | None = None,
             **meta) -> ReadSet:
    g, pasted = genome(seed, G, repeat_copies, repeat_frac)
    n_reads = int(round(coverage * G / L))
    rs = reads_from_genome(seed ^ 0xA5A5, g, n_reads, L, err, n_rate, threads=threads)
    rs.meta.update(dict(seed=seed, G=G, coverage=coverage, L=L, err=err, n_rate=n_rate,
                        repeat_bases=pasted, **meta))
    return rs


# --------------------------------------------------------------------------------------
# Named workloads. `params` are the counting parameters each workload is defined with.
# `scale` shrinks the genome (and so the read count) for test-sized variants.
# --------------------------------------------------------------------------------------

SEEDS = {"plain_1m": 0x5EED0001, "bacterial_5m": 0x5EED0002, "large_200m": 0x5EED0003,
         "batched_64": 0x5EED0004, "served_500": 0x5EED0005, "satellite_50m": 0x5EED0006}

WORKLOADS = {
    # 1 Mbp genome, 30x of 150 bp, 0.5 % errors, k=31, min depth 2, Q20
    "plain_1m": dict(G=1_000_000, coverage=30, L=150, err=0.005,
                     params=dict(k=31, min_depth=2, qual_threshold=20, bloom_fpr=0.01)),
    # 5 Mbp + 50 repeat copies of 1-5 kbp at 1 % divergence, 50x of 150 bp, 1 % errors,
    # 0.01 % N, k=51
    "bacterial_5m": dict(G=5_000_000, coverage=50, L=150, err=0.01, n_rate=1e-4,
                         repeat_copies=50,
                         params=dict(k=51, min_depth=2, qual_threshold=20, bloom_fpr=0.01)),
    # 200 Mbp with 5 % repeat content, 30x of 250 bp (24 M reads, 6 Gbases), 1 % errors,
    # k=51, Bloom pass sized at 1 % FPR, min depth 4
    "large_200m": dict(G=200_000_000, coverage=30, L=250, err=0.01, repeat_frac=0.05,
                       params=dict(k=51, min_depth=4, qual_threshold=20, bloom_fpr=0.01)),
}


def workload(name: str, scale: float = 1.0, threads: int | None = None) -> ReadSet:
    spec = dict(WORKLOADS[name])
    params = spec.pop("params")
    G = max(int(spec.pop("G") * scale), 4 * spec["L"])
    copies = spec.pop("repeat_copies", 0)
    if copies and scale < 1.0:
        copies = max(1, int(round(copies * scale)))
    rs = simulate(SEEDS[name], G, repeat_copies=copies, threads=threads, **spec)
    rs.meta["workload"] = name
    rs.meta["scale"] = scale
    rs.meta["params"] = dict(params)
    return rs


def concat(parts: list[ReadSet]) -> ReadSet:
    """Read sets one after the other (offsets rebased)."""
    seq = np.concatenate([p.seq for p in parts])
    qual = np.concatenate([p.qual for p in parts])
    offs = [np.zeros(1, np.uint64)]
    base = 0
    for p in parts:
        offs.append(p.offsets[1:] - p.offsets[0] + np.uint64(base))
        base += p.n_bases
    return ReadSet(seq, qual, np.concatenate(offs))


def satellite_workload(scale: float = 1.0, threads: int | None = None) -> ReadSet:
    """A genome with a tandem satellite (heavy hitters, Section 5.1: highly repetitive genomes
    have k-mers seen millions of times): a 50 Mbp random genome (x scale) read at 30x of 150 bp
    with 1 % errors, and as many reads again x 3/7 from a 100 kbp array of one 171-bp unit
    (an alpha-satellite-like period), so that 30 % of the reads are satellite; k = 31, min depth 2.
    Each of the unit's 171 k-mers then occurs in about 0.2 % of the windows."""
    seed = SEEDS["satellite_50m"]
    G = max(int(50_000_000 * scale), 4000)
    g, _ = genome(seed, G)
    n_main = int(round(30 * G / 150))
    main = reads_from_genome(seed ^ 0xA5A5, g, n_main, 150, 0.01, threads=threads)
    unit = genome(seed ^ 0x5A7, 171)[0]
    arr = np.ascontiguousarray(np.tile(unit, 100_000 // 171 + 1)[:100_000])
    sat = reads_from_genome(seed ^ 0x5A75, arr, int(round(n_main * 3 / 7)), 150, 0.01, threads=threads)
    rs = concat([main, sat])
    rs.meta.update(dict(seed=seed, G=G, coverage=30 / 0.7, L=150, err=0.01, workload="satellite_50m",
                        scale=scale, params=dict(k=31, min_depth=2, qual_threshold=20, bloom_fpr=0.01)))
    return rs


def batched_specs(n_samples: int = 64, seed: int = SEEDS["batched_64"], scale: float = 1.0):
    """Per-sample recipe of the batched workload: genome log-U[0.5, 20] Mbp, coverage
    U[20, 60], read length U{100..250}, error rate U[0.5 %, 2 %], k=51, min depth 2."""
    out = []
    for j in range(n_samples):
        d = draws(seed, 11, 4, 4 * j)
        G = int(round(math.exp(math.log(0.5e6) + _uniform(d[0]) * (math.log(20e6) - math.log(0.5e6)))
                      * scale / 1000.0)) * 1000
        L = 100 + int(d[2]) % 151
        out.append(dict(seed=_mix(seed, j), G=max(G, 4 * L), coverage=20 + 40 * _uniform(d[1]),
                        L=L, err=0.005 + 0.015 * _uniform(d[3]),
                        params=dict(k=51, min_depth=2, qual_threshold=20, bloom_fpr=0.01)))
    return out


def served_specs(n_jobs: int = 500, rate_per_s: float = 4.0, seed: int = SEEDS["served_500"],
                 scale: float = 1.0):
    """Per-job recipe of the served workload: Poisson arrivals at `rate_per_s`, genome
    log-U[1, 50] Mbp, 30x of 150 bp, 1 % errors, k drawn from {31, 51}, min depth 2."""
    out = []
    t = 0.0
    for j in range(n_jobs):
        d = draws(seed, 12, 4, 4 * j)
        t += -math.log(1.0 - _uniform(d[0])) / rate_per_s
        G = int(round(math.exp(math.log(1e6) + _uniform(d[1]) * (math.log(50e6) - math.log(1e6)))
                      * scale / 1000.0)) * 1000
        k = 31 if (int(d[2]) >> 63) == 0 else 51
        out.append(dict(seed=_mix(seed, j), arrival_s=t, G=max(G, 600), coverage=30, L=150,
                        err=0.01, params=dict(k=k, min_depth=2, qual_threshold=20, bloom_fpr=0.01)))
    return out


def sample_reads(spec: dict, threads: int | None = None) -> ReadSet:
    s = dict(spec)
    params = s.pop("params")
    s.pop("arrival_s", None)
    seed = s.pop("seed")
    rs = simulate(seed, threads=threads, **s)
    rs.meta["params"] = dict(params)
    return rs


def random_reads(seed: int, n_reads: int, min_len: int, max_len: int, alphabet: bytes = b"ACGT",
                 q_lo: int = 2, q_hi: int = 40) -> ReadSet:
    """Small unstructured read sets for edge-case tests: i.i.d. characters from `alphabet`
    (may include N or lowercase), lengths U{min_len..max_len}, Phred U{q_lo..q_hi}."""
    d = draws(seed, 13, 1 + n_reads, 0)
    lens = np.array([min_len + int(x) % (max_len - min_len + 1) for x in d[1:]], dtype=np.uint64)
    offs = np.zeros(n_reads + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    total = int(offs[-1])
    cd = draws(seed, 14, total, 0)
    qd = draws(seed, 15, total, 0)
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    seq = alpha[(cd % np.uint64(len(alphabet))).astype(np.int64)] if total else np.zeros(0, np.uint8)
    qual = (33 + q_lo + (qd % np.uint64(q_hi - q_lo + 1))).astype(np.uint8) if total else np.zeros(0, np.uint8)
    return ReadSet(np.ascontiguousarray(seq, dtype=np.uint8), qual, offs)
