"""Python binding of the k-mer analysis library: the C ABI's calls under the same names,
taking numpy arrays (host) or torch CUDA tensors (device) and marshalling pointers.
PyTorch is used only for device memory and streams; all of the work runs in the library's
CUDA kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import capi
from .capi import check


def _torch():
    import torch
    return torch


def _is_cuda_tensor(x) -> bool:
    try:
        torch = _torch()
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            torch = _torch()
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(k: int, max_bases: int, min_depth: int = 2, min_ext_count: int = 2,
                qual_threshold: int = 20, qual_offset: int = 33, use_bloom: bool = True,
                canonical: bool = True, max_reads: int = 0, expected_distinct: int = 0,
                bloom_fpr: float = 0.01, table_capacity: int = 0, expected_keys: int = 0,
                load_factor: float = 0.0, staging_bytes: int = 0, block_threads: int = 0,
                windows_per_thread: int = 0, ctas_per_sm: int = 0,
                warp_aggregate: bool = False, n_parts: int = 1, part: int = 0,
                slot_prefetch: int = 0, fault_inject: int = 0,
                partitions: int = 0, heavy_hitters: bool = False) -> capi.kma_params:
    return capi.kma_params(k, min_depth, min_ext_count, qual_threshold, qual_offset,
                           int(bool(use_bloom)), int(bool(canonical)), max_bases, max_reads,
                           expected_distinct, bloom_fpr, table_capacity, expected_keys,
                           load_factor, staging_bytes, block_threads, windows_per_thread,
                           ctas_per_sm, int(bool(warp_aggregate)), n_parts, part, slot_prefetch,
                           fault_inject, partitions, int(bool(heavy_hitters)))


def plan(params: capi.kma_params) -> capi.kma_plan:
    """kmer_analysis_plan: sizes a handle with `params` would have (host only)."""
    out = capi.kma_plan()
    check(capi.load().kmer_analysis_plan(ctypes.byref(params), ctypes.byref(out)), "plan")
    return out


@dataclass
class Result:
    """Finalized records (order unspecified; see `sorted()`)."""
    keys: np.ndarray      # uint64[n, 2] (lo, hi)
    counts: np.ndarray    # uint32[n]
    ext: np.ndarray       # uint32[n, 8] left A C G T, right A C G T
    codes: np.ndarray     # uint8[n, 2]  0..3 A C G T, 4 X, 5 F
    n_uu: int = 0
    valid_windows: int = 0
    table_keys: int = 0
    meta: dict = field(default_factory=dict)

    def __len__(self):
        return int(self.counts.shape[0])

    def sorted(self) -> "Result":
        order = np.lexsort((self.keys[:, 0], self.keys[:, 1]))
        return Result(self.keys[order], self.counts[order], self.ext[order], self.codes[order],
                      self.n_uu, self.valid_windows, self.table_keys, dict(self.meta))


class KmerAnalysis:
    """One handle: kmer_analysis_create / count / finalize / copy_result / query / reset /
    destroy. Inputs are numpy arrays (host) or torch CUDA tensors (device)."""

    def __init__(self, params: capi.kma_params | None = None, stream=None, **kw):
        self._lib = capi.load()
        self.params = params if params is not None else make_params(**kw)
        self._h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        check(self._lib.kmer_analysis_create(ctypes.byref(self.params), self._stream,
                                             ctypes.byref(self._h)), "create")
        self.result_info: capi.kma_result | None = None

    # -------------------------------------------------------------- C ABI calls
    @property
    def handle(self):
        return self._h

    def count(self, seq, qual, offsets) -> None:
        if _is_cuda_tensor(seq):
            assert _is_cuda_tensor(qual) and _is_cuda_tensor(offsets)
            n_reads = offsets.numel() - 1
            check(self._lib.kmer_analysis_count(self._h, seq.data_ptr(), qual.data_ptr(),
                                                offsets.data_ptr(), n_reads, 1), "count")
            return
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        qual = np.ascontiguousarray(qual, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        check(self._lib.kmer_analysis_count(self._h, seq.ctypes.data, qual.ctypes.data,
                                            offsets.ctypes.data, offsets.shape[0] - 1, 0), "count")

    def finalize(self) -> capi.kma_result:
        r = capi.kma_result()
        check(self._lib.kmer_analysis_finalize(self._h, ctypes.byref(r)), "finalize")
        self.result_info = r
        return r

    def copy_result(self) -> Result:
        r = self.result_info
        if r is None:
            raise RuntimeError("finalize() first")
        n = int(r.n)
        keys = np.zeros((n, 2), np.uint64)
        counts = np.zeros(n, np.uint32)
        ext = np.zeros((n, 8), np.uint32)
        codes = np.zeros((n, 2), np.uint8)
        check(self._lib.kmer_analysis_copy_result(self._h, keys.ctypes.data, counts.ctypes.data,
                                                  ext.ctypes.data, codes.ctypes.data, n, 0),
              "copy_result")
        return Result(keys, counts, ext, codes, int(r.n_uu), int(r.valid_windows), int(r.table_keys))

    def finalize_to_host(self, out):
        """finalize + copy of the records to host arrays in one call, the copies of one group
        of partitions overlapping the recount of the next (kmer_analysis_finalize_to_host).
        `out` = (keys[c, 2] u64, counts[c] u32, ext[c, 8] u32, codes[c, 2] u8) host arrays of
        c rows (host_result_buffers; pinned memory copies fastest). Returns a Result viewing
        the first n rows; raises KmaError (KMA_EFULL) if n > c, the handle then finalized."""
        keys, counts, ext, codes = (np.asarray(a) for a in out)
        assert keys.dtype == np.uint64 and counts.dtype == np.uint32 and ext.dtype == np.uint32
        assert codes.dtype == np.uint8 and all(a.flags.c_contiguous for a in (keys, counts, ext, codes))
        cap = min(keys.shape[0], counts.shape[0], ext.shape[0], codes.shape[0])
        r = capi.kma_result()
        rc = self._lib.kmer_analysis_finalize_to_host(self._h, keys.ctypes.data, counts.ctypes.data,
                                                      ext.ctypes.data, codes.ctypes.data, cap,
                                                      ctypes.byref(r))
        if rc == 0 or (rc == capi.KMA_EFULL and int(r.n) > cap):
            self.result_info = r
        check(rc, "finalize_to_host")
        n = int(r.n)
        return Result(keys[:n], counts[:n], ext[:n], codes[:n], int(r.n_uu), int(r.valid_windows),
                      int(r.table_keys))

    def contigs(self):
        """Contigs of the finalized result (kmer_analysis_contigs, Section 5.2): (list of
        strings, info) with info = {n_contigs, n_bases, n_vertices, n_cycles}."""
        c = capi.kma_contigs()
        check(self._lib.kmer_analysis_contigs(self._h, ctypes.byref(c)), "contigs")
        seq = np.zeros(max(int(c.n_bases), 1), np.uint8)
        offs = np.zeros(int(c.n_contigs) + 1, np.uint64)
        check(self._lib.kmer_analysis_copy_contigs(self._h, seq.ctypes.data, offs.ctypes.data, 0), "copy_contigs")
        raw = seq[:int(c.n_bases)].tobytes().decode()
        strings = [raw[int(offs[i]):int(offs[i + 1])] for i in range(int(c.n_contigs))]
        info = {"n_contigs": int(c.n_contigs), "n_bases": int(c.n_bases), "n_vertices": int(c.n_vertices),
                "n_cycles": int(c.n_cycles)}
        return strings, info

    def copy_result_device(self):
        """Result arrays as torch CUDA tensors (copies of the handle-owned buffers)."""
        torch = _torch()
        r = self.result_info
        n = int(r.n)
        keys = torch.empty((n, 2), dtype=torch.int64, device="cuda")
        counts = torch.empty(n, dtype=torch.int32, device="cuda")
        ext = torch.empty((n, 8), dtype=torch.int32, device="cuda")
        codes = torch.empty((n, 2), dtype=torch.uint8, device="cuda")
        check(self._lib.kmer_analysis_copy_result(self._h, keys.data_ptr(), counts.data_ptr(),
                                                  ext.data_ptr(), codes.data_ptr(), n, 1),
              "copy_result")
        return keys, counts, ext, codes

    def query(self, keys, out=None):
        """Look up k-mers keys[n, 2] (either orientation). numpy in -> numpy out (synchronous);
        CUDA tensor in -> CUDA tensors out (enqueued on the handle's stream)."""
        if _is_cuda_tensor(keys):
            torch = _torch()
            n = keys.shape[0]
            counts, ext, codes = out if out is not None else (
                torch.empty(n, dtype=torch.int32, device=keys.device),
                torch.empty((n, 8), dtype=torch.int32, device=keys.device),
                torch.empty((n, 2), dtype=torch.uint8, device=keys.device))
            check(self._lib.kmer_analysis_query(self._h, keys.data_ptr(), n, counts.data_ptr(),
                                                ext.data_ptr(), codes.data_ptr(), 1), "query")
            return counts, ext, codes
        q = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, 2)
        n = q.shape[0]
        counts = np.zeros(n, np.uint32)
        ext = np.zeros((n, 8), np.uint32)
        codes = np.zeros((n, 2), np.uint8)
        check(self._lib.kmer_analysis_query(self._h, q.ctypes.data, n, counts.ctypes.data,
                                            ext.ctypes.data, codes.ctypes.data, 0), "query")
        return counts, ext, codes

    def reset(self) -> None:
        check(self._lib.kmer_analysis_reset(self._h), "reset")
        self.result_info = None

    def set_stream(self, stream) -> None:
        self._stream = _stream_handle(stream)
        check(self._lib.kmer_analysis_set_stream(self._h, self._stream), "set_stream")

    def status(self) -> int:
        return int(self._lib.kmer_analysis_status(self._h))

    def set_profiling(self, enable: bool = True) -> None:
        check(self._lib.kmer_analysis_set_profiling(self._h, int(bool(enable))), "set_profiling")

    def timings(self, reset: bool = False) -> dict:
        t = capi.kma_timings()
        check(self._lib.kmer_analysis_timings(self._h, ctypes.byref(t), int(bool(reset))), "timings")
        out = {f"ms_{k}": float(t.ms[i]) for i, k in enumerate(capi.KERNEL_KINDS)}
        out.update({f"n_{k}": int(t.launches[i]) for i, k in enumerate(capi.KERNEL_KINDS)})
        out["launches"] = int(t.total_launches)
        out["first_sightings"] = int(t.first_sightings)
        return out

    def device_bytes(self) -> int:
        return int(self._lib.kmer_analysis_device_bytes(self._h))

    def destroy(self) -> None:
        if self._h:
            self._lib.kmer_analysis_destroy(self._h)
            self._h = ctypes.c_void_p()

    close = destroy

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def host_result_buffers(capacity: int, pinned: bool = False):
    """Host arrays for `capacity` records in the layout of kma_result (keys, counts, ext,
    codes), optionally in pinned (page-locked) memory."""
    shapes = (((capacity, 2), np.uint64), ((capacity,), np.uint32), ((capacity, 8), np.uint32),
              ((capacity, 2), np.uint8))
    if not pinned:
        return tuple(np.zeros(sh, dt) for sh, dt in shapes)
    torch = _torch()
    tdt = {np.uint64: torch.int64, np.uint32: torch.int32, np.uint8: torch.uint8}
    return tuple(torch.empty(sh, dtype=tdt[dt]).pin_memory().numpy().view(dt) for sh, dt in shapes)


def count_batch(handles: list[KmerAnalysis], reads: list[tuple]) -> None:
    """kmer_analysis_count_batch: reads[i] = (seq, qual, offsets) CUDA tensors for handle i.
    Enqueued on handles[0]'s stream; does not synchronise."""
    n = len(handles)
    assert 0 < n <= capi.KMA_MAX_BATCH and len(reads) == n
    hs = (ctypes.c_void_p * n)(*[h.handle.value for h in handles])
    arr = (capi.kma_reads * n)()
    for i, (seq, qual, offs) in enumerate(reads):
        arr[i] = capi.kma_reads(seq.data_ptr(), qual.data_ptr(), offs.data_ptr(),
                                offs.numel() - 1, seq.numel())
    check(capi.load().kmer_analysis_count_batch(hs, arr, n), "count_batch")


def finalize_batch(handles: list[KmerAnalysis]) -> list[capi.kma_result]:
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.handle.value for h in handles])
    out = (capi.kma_result * n)()
    rc = capi.load().kmer_analysis_finalize_batch(hs, n, out)
    for i, h in enumerate(handles):
        h.result_info = out[i]
    check(rc, "finalize_batch")
    return list(out)


def reserve_output(h: KmerAnalysis, n_records: int) -> None:
    check(capi.load().kmer_analysis_reserve_output(h.handle, n_records), "reserve_output")


def finalize_batch_async(handles: list[KmerAnalysis]) -> None:
    """kmer_analysis_finalize_batch_async: no host synchronisation, capture-safe."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.handle.value for h in handles])
    check(capi.load().kmer_analysis_finalize_batch_async(hs, n), "finalize_batch_async")


def fetch_result(h: KmerAnalysis) -> capi.kma_result:
    r = capi.kma_result()
    check(capi.load().kmer_analysis_fetch_result(h.handle, ctypes.byref(r)), "fetch_result")
    h.result_info = r
    return r


class BatchGraph:
    """Many samples in one CUDA graph. Samples counted in one table are packed and counted
    together (one packing launch and one persistent counting launch), then recounted and
    classified together (kmer_analysis_finalize_batch_async). Samples large enough to be
    partitioned run their scatter/record passes one after another inside the same graph, each
    finalized before the next starts, so only one sample's record buckets exist at a time.
    Captured once, replayed per step. `reads[i]` = (seq, qual, offsets) CUDA tensors of
    handle i; all handles are moved to the capture stream."""

    def __init__(self, handles: list[KmerAnalysis], reads: list[tuple], headroom: float = 1.25):
        torch = _torch()
        assert len(handles) == len(reads) and handles
        self.handles, self.reads = handles, reads
        parts = [plan(h.params).partitions for h in handles]
        self.small = [i for i, p in enumerate(parts) if p <= 1]
        self.large = [i for i, p in enumerate(parts) if p > 1]
        self.stream = torch.cuda.Stream()
        for h in handles:
            h.set_stream(self.stream)
        # eager run: sizes the output buffers the captured finalize writes into
        with torch.cuda.stream(self.stream):
            self._step(finalize_batch)
        for h in handles:
            reserve_output(h, int(h.result_info.table_keys * headroom) + 1024)
        before = sum(h.timings()["launches"] for h in handles)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._step(finalize_batch_async)
        self.stream.synchronize()
        # library kernels in the graph (the host counters tick once, at capture)
        self.kernels_per_replay = sum(h.timings()["launches"] for h in handles) - before

    def _step(self, finalize):
        for h in self.handles:
            h.reset()
        for c0 in range(0, len(self.small), capi.KMA_MAX_BATCH):
            idx = self.small[c0:c0 + capi.KMA_MAX_BATCH]
            hs = [self.handles[i] for i in idx]
            count_batch(hs, [self.reads[i] for i in idx])
            finalize(hs)
        for i in self.large:
            count_batch([self.handles[i]], [self.reads[i]])
            finalize([self.handles[i]])

    def replay(self) -> None:
        """Launch the graph on the handles' stream (results are read from that stream)."""
        with _torch().cuda.stream(self.stream):
            self.graph.replay()

    def results(self) -> list[capi.kma_result]:
        return [fetch_result(h) for h in self.handles]


def count_kmers(seq, qual, offsets, k: int, min_depth: int = 2, min_ext_count: int = 2,
                qual_threshold: int = 20, use_bloom: bool = True, canonical: bool = True,
                expected_distinct: int = 0, expected_keys: int = 0, stream=None,
                retries: int = 4, **kw) -> Result:
    """One-shot convenience: create -> count -> finalize -> copy_result -> destroy.
    A full table (KMA_EFULL) is retried with twice the capacity; results never depend on the
    capacity."""
    n_bases = int(offsets[-1] - offsets[0]) if not _is_cuda_tensor(offsets) else int(seq.numel())
    n_reads = int(offsets.shape[0] - 1)
    table_capacity = kw.pop("table_capacity", 0)
    for attempt in range(retries + 1):
        p = make_params(k=k, max_bases=max(n_bases, 1), max_reads=max(n_reads, 1),
                        min_depth=min_depth, min_ext_count=min_ext_count,
                        qual_threshold=qual_threshold, use_bloom=use_bloom, canonical=canonical,
                        expected_distinct=expected_distinct, expected_keys=expected_keys,
                        table_capacity=table_capacity, **kw)
        ka = KmerAnalysis(p, stream=stream)
        try:
            ka.count(seq, qual, offsets)
            ka.finalize()
            res = ka.copy_result()
            res.meta["table_slots"] = plan(p).table_slots
            return res
        except capi.KmaError as e:
            if e.code != capi.KMA_EFULL or attempt == retries:
                raise
            table_capacity = 2 * plan(p).table_slots
        finally:
            ka.destroy()
    raise AssertionError("unreachable")


@dataclass
class Estimate:
    """The cardinality pass over a read set (Section 5.1): HyperLogLog estimate of the distinct
    canonical k-mers, and the heavy hitters found by the Misra-Gries summaries of the sampled
    window stream (every capi.MG_SAMPLE-th position, capi.MG_BUCKETS sub-streams by key hash,
    capi.MG_COUNTERS counters each)."""
    distinct: float
    rel_std_error: float
    valid_windows: int
    precision: int
    registers: np.ndarray  # uint8[2^precision]; merge sketches by np.maximum
    heavy_hitters: bool = False        # pass as make_params(heavy_hitters=...)
    sampled_windows: int = 0
    heavy_threshold: int = 0
    summary_keys: np.ndarray = None    # uint64[n, 2], by count descending
    summary_counts: np.ndarray = None  # uint64[n]
    summary_bucket: np.ndarray = None  # uint32[n]
    bucket_windows: np.ndarray = None  # uint64[MG_BUCKETS]: items of each sub-stream


def estimate_distinct(seq, qual, offsets, k: int, canonical: bool = True, precision: int = 14,
                      registers: np.ndarray | None = None, n_parts: int = 1, part: int = 0,
                      stream=None, **kw) -> Estimate:
    """One HyperLogLog pass over the reads (kmer_analysis_estimate). `registers` (optional) is
    a sketch to merge with; the returned sketch includes it."""
    lib = capi.load()
    on_dev = _is_cuda_tensor(seq)
    n_reads = int(offsets.shape[0] - 1) if not on_dev else int(offsets.numel() - 1)
    n_bases = int(seq.numel()) if on_dev else int(offsets[-1] - offsets[0])
    p = make_params(k=k, max_bases=max(n_bases, 1), max_reads=max(n_reads, 1), canonical=canonical,
                    use_bloom=False, n_parts=n_parts, part=part, **kw)
    regs = np.zeros(1 << precision, np.uint8) if registers is None else \
        np.ascontiguousarray(registers, dtype=np.uint8).copy()
    if regs.shape != (1 << precision,):
        raise ValueError("registers must hold 2^precision bytes")
    cap = capi.MG_BUCKETS * capi.MG_COUNTERS
    s_keys = np.zeros((cap, 2), np.uint64)
    s_counts = np.zeros(cap, np.uint64)
    s_bucket = np.zeros(cap, np.uint32)
    b_windows = np.zeros(capi.MG_BUCKETS, np.uint64)
    est = capi.kma_estimate(precision=precision, summary_capacity=cap, summary_keys=s_keys.ctypes.data,
                            summary_counts=s_counts.ctypes.data, summary_bucket=s_bucket.ctypes.data,
                            bucket_windows=b_windows.ctypes.data)
    if on_dev:
        args = (seq.data_ptr(), qual.data_ptr(), offsets.data_ptr(), n_reads, 1)
    else:
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        qual = np.ascontiguousarray(qual, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        args = (seq.ctypes.data, qual.ctypes.data, offsets.ctypes.data, n_reads, 0)
    check(lib.kmer_analysis_estimate(ctypes.byref(p), *args, _stream_handle(stream), ctypes.byref(est),
                                     regs.ctypes.data), "estimate")
    n = int(est.n_summary)
    return Estimate(float(est.distinct), float(est.rel_std_error), int(est.valid_windows),
                    int(est.precision), regs, bool(est.heavy_hitters), int(est.sampled_windows),
                    int(est.heavy_threshold), s_keys[:n], s_counts[:n], s_bucket[:n], b_windows)


def hll_estimate(registers: np.ndarray, precision: int) -> float:
    """Estimate of a (merged) sketch, on the host (kmer_analysis_hll_estimate)."""
    lib = capi.load()
    regs = np.ascontiguousarray(registers, dtype=np.uint8)
    out = ctypes.c_double()
    check(lib.kmer_analysis_hll_estimate(regs.ctypes.data, precision, ctypes.byref(out)), "hll_estimate")
    return float(out.value)


def parse_fastq(text, stream=None):
    """FASTQ text (bytes / numpy uint8 on the host, or a torch uint8 CUDA tensor) -> (seq, qual,
    offsets) as torch CUDA tensors (uint8, uint8, int64), ready for KmerAnalysis.count
    (kmer_analysis_parse_fastq). Capacities are bounded from the text size (a record takes at
    least six bytes and two per base), so one call suffices."""
    torch = _torch()
    lib = capi.load()
    if _is_cuda_tensor(text):
        ptr, n, on_dev = text.data_ptr(), int(text.numel()), 1
        keep = text
    else:
        keep = np.frombuffer(text, dtype=np.uint8) if isinstance(text, (bytes, bytearray)) else \
            np.ascontiguousarray(text, dtype=np.uint8)
        ptr, n, on_dev = keep.ctypes.data, int(keep.shape[0]), 0
    cap_bases, cap_reads = n // 2 + 1, n // 6 + 1
    seq = torch.empty(cap_bases, dtype=torch.uint8, device="cuda")
    qual = torch.empty(cap_bases, dtype=torch.uint8, device="cuda")
    offs = torch.empty(cap_reads + 1, dtype=torch.int64, device="cuda")
    nr, nb = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib.kmer_analysis_parse_fastq(ptr, n, on_dev, seq.data_ptr(), qual.data_ptr(), offs.data_ptr(),
                                        cap_bases, cap_reads, ctypes.byref(nr), ctypes.byref(nb),
                                        _stream_handle(stream)), "parse_fastq")
    del keep
    return seq[:nb.value], qual[:nb.value], offs[:nr.value + 1]
