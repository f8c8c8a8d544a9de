"""CPU oracle for k-mer analysis (HipMer, arXiv 1705.11147, Sections 2 and 5.1).

TEST INFRASTRUCTURE: only the tests, `__graft_entry__.smoke()` and the benchmark's
`cpu_baseline` / reference leg may import this package. The product library never does.
The computation lives in kmer_oracle.cpp (plain C++ on character strings, no Bloom filter);
this module only marshals numpy arrays.

Result layout (shared with the CUDA path's host copy, sorted by key here):
  keys   uint64[n, 2]  (lo, hi) words of the 2-bit key, A0 C1 G2 T3, first base most significant
  counts uint32[n]
  ext    uint32[n, 8]  left A C G T, right A C G T
  codes  uint8[n, 2]   left, right: 0..3 = A C G T, 4 = X (none), 5 = F (fork)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

CODE_X = 4
CODE_F = 5

_LIB = None


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("min_depth", ctypes.c_uint32),
                ("min_ext_count", ctypes.c_uint32), ("qual_threshold", ctypes.c_uint32),
                ("qual_offset", ctypes.c_uint32), ("canonical", ctypes.c_uint32)]


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        p, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        lib.oracle_run.argtypes = [p, p, p, u64, ctypes.POINTER(_Params), u32, u32, ctypes.c_int]
        lib.oracle_run.restype = p
        lib.oracle_run_parts.argtypes = [p, p, p, u64, ctypes.POINTER(_Params), p, u32, ctypes.c_int]
        lib.oracle_run_parts.restype = p
        lib.oracle_size.argtypes = [p]
        lib.oracle_size.restype = u64
        lib.oracle_valid_windows.argtypes = [p]
        lib.oracle_valid_windows.restype = u64
        lib.oracle_fetch.argtypes = [p, p, p, p, p]
        lib.oracle_query.argtypes = [p, p, u64, p, p, p]
        lib.oracle_free.argtypes = [p]
        lib.oracle_partition_of.argtypes = [p, u64, u32, u32, p]
        lib.oracle_pack_strings.argtypes = [ctypes.c_char_p, u64, u32, p]
        lib.oracle_unpack_keys.argtypes = [p, u64, u32, p]
        lib.oracle_hll_registers.argtypes = [p, u64, u32, p]
        lib.oracle_hll_estimate.argtypes = [p, u32]
        lib.oracle_hll_estimate.restype = ctypes.c_double
        lib.oracle_sampled_stream.argtypes = [p, p, p, u64, ctypes.POINTER(_Params), u32]
        lib.oracle_sampled_stream.restype = p
        lib.oracle_stream_size.argtypes = [p]
        lib.oracle_stream_size.restype = u64
        lib.oracle_stream_fetch.argtypes = [p, p]
        lib.oracle_stream_free.argtypes = [p]
        lib.oracle_stream_bucket.argtypes = [p, u64, u32, p]
        lib.oracle_misra_gries.argtypes = [p, u64, u32, p, p]
        lib.oracle_misra_gries.restype = u64
        lib.oracle_contigs.argtypes = [p, p, u64, u32, ctypes.c_int]
        lib.oracle_contigs.restype = p
        for fn in ("oracle_contigs_n", "oracle_contigs_bases", "oracle_contigs_cycles"):
            getattr(lib, fn).argtypes = [p]
            getattr(lib, fn).restype = u64
        lib.oracle_contigs_fetch.argtypes = [p, p, p]
        lib.oracle_contigs_free.argtypes = [p]
        _LIB = lib
    return _LIB


@dataclass
class OracleResult:
    keys: np.ndarray
    counts: np.ndarray
    ext: np.ndarray
    codes: np.ndarray
    valid_windows: int
    _handle: object = None

    def __len__(self):
        return int(self.counts.shape[0])

    def uu_mask(self) -> np.ndarray:
        return (self.codes[:, 0] < 4) & (self.codes[:, 1] < 4)

    def query(self, qkeys: np.ndarray):
        """Look up k-mers (uint64[n, 2], either orientation) in the full counted table."""
        if self._handle is None:
            raise RuntimeError("result was created with keep_table=False")
        q = np.ascontiguousarray(qkeys, dtype=np.uint64).reshape(-1, 2)
        n = q.shape[0]
        counts = np.zeros(n, np.uint32)
        ext = np.zeros((n, 8), np.uint32)
        codes = np.zeros((n, 2), np.uint8)
        _lib().oracle_query(self._handle.ptr, q.ctypes.data, n, counts.ctypes.data,
                            ext.ctypes.data, codes.ctypes.data)
        return counts, ext, codes


class _Handle:
    def __init__(self, ptr):
        self.ptr = ptr

    def __del__(self):
        if self.ptr and _LIB is not None:
            _LIB.oracle_free(self.ptr)
            self.ptr = None


def run(seq: np.ndarray, qual: np.ndarray, offsets: np.ndarray, k: int, min_depth: int = 2,
        min_ext_count: int = 2, qual_threshold: int = 20, qual_offset: int = 33,
        canonical: bool = True, part: int = 0, n_parts: int = 1, threads: int | None = None,
        keep_table: bool = False, parts=None) -> OracleResult:
    """Records of the read set. With n_parts > 1 only the keys of owner partition `part` are
    kept, or, if `parts` (an iterable of partition ids) is given, the keys of those partitions
    (one scan of the reads for the whole set)."""
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    qual = np.ascontiguousarray(qual, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n_reads = offsets.shape[0] - 1
    prm = _Params(k, min_depth, min_ext_count, qual_threshold, qual_offset, int(bool(canonical)))
    threads = threads or min(16, os.cpu_count() or 1)
    lib = _lib()
    if parts is not None and n_parts > 1:
        keep = np.zeros(n_parts, np.uint8)
        keep[np.asarray(list(parts), dtype=np.int64)] = 1
        h = lib.oracle_run_parts(seq.ctypes.data, qual.ctypes.data, offsets.ctypes.data, n_reads,
                                 ctypes.byref(prm), keep.ctypes.data, n_parts, threads)
    else:
        h = lib.oracle_run(seq.ctypes.data, qual.ctypes.data, offsets.ctypes.data, n_reads,
                           ctypes.byref(prm), part, n_parts, threads)
    handle = _Handle(h)
    n = lib.oracle_size(h)
    keys = np.zeros((n, 2), np.uint64)
    counts = np.zeros(n, np.uint32)
    ext = np.zeros((n, 8), np.uint32)
    codes = np.zeros((n, 2), np.uint8)
    lib.oracle_fetch(h, keys.ctypes.data, counts.ctypes.data, ext.ctypes.data, codes.ctypes.data)
    vw = int(lib.oracle_valid_windows(h))
    return OracleResult(keys, counts, ext, codes, vw, handle if keep_table else None)


def run_readset(rs, threads: int | None = None, part: int = 0, n_parts: int = 1,
                keep_table: bool = False, parts=None, **overrides) -> OracleResult:
    p = dict(rs.meta.get("params", {}))
    p.pop("bloom_fpr", None)
    p.update(overrides)
    return run(rs.seq, rs.qual, rs.offsets, threads=threads, part=part, n_parts=n_parts,
               keep_table=keep_table, parts=parts, **p)


def partition_of(keys: np.ndarray, k: int, n_parts: int) -> np.ndarray:
    q = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    out = np.zeros(q.shape[0], np.uint32)
    _lib().oracle_partition_of(q.ctypes.data, q.shape[0], k, n_parts, out.ctypes.data)
    return out


def pack(kmers: list[str]) -> np.ndarray:
    """k-mer strings (ACGT, equal length) -> uint64[n, 2] keys."""
    if not kmers:
        return np.zeros((0, 2), np.uint64)
    k = len(kmers[0])
    assert all(len(s) == k for s in kmers)
    out = np.zeros((len(kmers), 2), np.uint64)
    _lib().oracle_pack_strings("".join(kmers).encode(), len(kmers), k, out.ctypes.data)
    return out


def unpack(keys: np.ndarray, k: int) -> list[str]:
    q = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    buf = ctypes.create_string_buffer(q.shape[0] * k + 1)
    _lib().oracle_unpack_keys(q.ctypes.data, q.shape[0], k, buf)
    raw = buf.raw[: q.shape[0] * k].decode()
    return [raw[i * k:(i + 1) * k] for i in range(q.shape[0])]


def reads_from_strings(reads: list[str], quals: list[str] | None = None, default_q: int = 40):
    """Build (seq, qual, offsets) arrays from Python strings (qualities Phred+33)."""
    seq = np.frombuffer("".join(reads).encode(), dtype=np.uint8).copy()
    if quals is None:
        qual = np.full(seq.shape[0], 33 + default_q, np.uint8)
    else:
        qual = np.frombuffer("".join(quals).encode(), dtype=np.uint8).copy()
    offs = np.zeros(len(reads) + 1, np.uint64)
    offs[1:] = np.cumsum([len(r) for r in reads])
    return seq, qual, offs


def hll_registers(keys: np.ndarray, precision: int) -> np.ndarray:
    """HyperLogLog sketch (2^precision uint8 registers) of a set of distinct keys
    (Section 5.1's cardinality pass, written from its definition in kmer_oracle.cpp)."""
    q = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    out = np.zeros(1 << precision, np.uint8)
    _lib().oracle_hll_registers(q.ctypes.data, q.shape[0], precision, out.ctypes.data)
    return out


def hll_estimate(registers: np.ndarray, precision: int) -> float:
    """Flajolet et al.'s estimate (with linear counting in the small range) of a sketch."""
    r = np.ascontiguousarray(registers, dtype=np.uint8)
    assert r.shape == (1 << precision,)
    return float(_lib().oracle_hll_estimate(r.ctypes.data, precision))


def sampled_stream(seq: np.ndarray, qual: np.ndarray, offsets: np.ndarray, k: int, canonical: bool = True,
                   sample: int = 64, **_) -> np.ndarray:
    """Keys (uint64[n, 2]) of the valid windows starting at every `sample`-th position of the
    reads laid out back to back with one separator after each read, in read order (the
    stream the heavy-hitter summaries of the cardinality pass are defined on)."""
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    qual = np.ascontiguousarray(qual, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    prm = _Params(k, 1, 1, 0, 33, int(bool(canonical)))
    lib = _lib()
    h = lib.oracle_sampled_stream(seq.ctypes.data, qual.ctypes.data, offsets.ctypes.data, offsets.shape[0] - 1,
                                  ctypes.byref(prm), sample)
    try:
        n = lib.oracle_stream_size(h)
        out = np.zeros((n, 2), np.uint64)
        if n:
            lib.oracle_stream_fetch(h, out.ctypes.data)
        return out
    finally:
        lib.oracle_stream_free(h)


def stream_bucket(keys: np.ndarray, bits: int) -> np.ndarray:
    """Sub-stream of each key: the top `bits` bits of the sketch hash."""
    q = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    out = np.zeros(q.shape[0], np.uint32)
    _lib().oracle_stream_bucket(q.ctypes.data, q.shape[0], bits, out.ctypes.data)
    return out


def misra_gries(stream: np.ndarray, m: int):
    """Misra-Gries summary with m counters of a stream of keys (uint64[n, 2]): (keys, counts)
    of the keys left with a positive counter."""
    q = np.ascontiguousarray(stream, dtype=np.uint64).reshape(-1, 2)
    keys = np.zeros((m, 2), np.uint64)
    counts = np.zeros(m, np.uint64)
    n = _lib().oracle_misra_gries(q.ctypes.data, q.shape[0], m, keys.ctypes.data, counts.ctypes.data)
    return keys[:n], counts[:n]


def parse_fastq(text: bytes):
    """FASTQ text -> (seq, qual, offsets) numpy arrays, record by record in plain Python (small
    inputs only). A record is four lines: '@' name, bases, '+' line, qualities of the same
    length; '\r' before '\n' is dropped; the last line may lack '\n'; empty lines after the
    last record are ignored. Raises ValueError on anything else."""
    lines = text.split(b"\n")
    if lines and lines[-1] == b"":
        lines.pop()  # the text ended with a newline
    lines = [ln[:-1] if ln.endswith(b"\r") else ln for ln in lines]
    while len(lines) % 4 and lines and lines[-1] == b"":
        lines.pop()
    if len(lines) % 4:
        raise ValueError("line count is not a multiple of four")
    seqs, quals = [], []
    for r in range(len(lines) // 4):
        head, bases, plus, q = lines[4 * r: 4 * r + 4]
        if not head.startswith(b"@") or not plus.startswith(b"+") or len(bases) != len(q):
            raise ValueError(f"record {r} is malformed")
        seqs.append(bases)
        quals.append(q)
    seq = np.frombuffer(b"".join(seqs), dtype=np.uint8).copy()
    qual = np.frombuffer(b"".join(quals), dtype=np.uint8).copy()
    offs = np.zeros(len(seqs) + 1, np.uint64)
    offs[1:] = np.cumsum([len(s) for s in seqs]) if seqs else []
    return seq, qual, offs


def contigs(keys: np.ndarray, codes: np.ndarray, k: int, canonical: bool = True):
    """Contigs (Section 5.2) of a k-mer analysis result, walked k-mer by k-mer: a list of
    strings (each in the orientation its walk took) and the number of cycles that were cut."""
    q = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
    c = np.ascontiguousarray(codes, dtype=np.uint8).reshape(-1, 2)
    lib = _lib()
    h = lib.oracle_contigs(q.ctypes.data, c.ctypes.data, q.shape[0], k, int(canonical))
    try:
        n, nb = lib.oracle_contigs_n(h), lib.oracle_contigs_bases(h)
        buf = ctypes.create_string_buffer(nb + 1)
        offs = np.zeros(n + 1, np.uint64)
        lib.oracle_contigs_fetch(h, buf, offs.ctypes.data)
        raw = buf.raw[:nb].decode()
        return [raw[int(offs[i]):int(offs[i + 1])] for i in range(n)], int(lib.oracle_contigs_cycles(h))
    finally:
        lib.oracle_contigs_free(h)
