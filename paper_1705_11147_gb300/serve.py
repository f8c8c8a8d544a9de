"""Serving loop for k-mer counting jobs on one GPU, with continuous batching.

Jobs (host reads + counting parameters) are submitted at any time and return futures. They
are admitted in arrival order while their device footprint (the handle's plan, the reads and
the result records) fits the memory budget. Each worker thread owns a CUDA stream; when it is
free it takes every admissible job that is waiting (up to `max_batch`) as one batch: the small
jobs' reads are copied in and packed and counted together (one launch each,
kmer_analysis_count_batch), the large jobs are counted from host memory (kmer_analysis_count:
staged copies overlapping the packing, in one call that releases the interpreter), and all are
finalized together (kmer_analysis_finalize_batch). While one
worker's batch is on the GPU the other workers copy in and launch the next jobs, so work of
jobs that arrive while others run overlaps on the device. A finished job's table can stay
resident for queries (`keep_resident`) until the caller releases it. Each job's counting
parameters take the autotuner's choices for its class (`tuned`, see autotune.apply), and
`latency_stats()` splits latency into the wait for a worker and the batch's service time.

All counting runs in the library's kernels; this module schedules, copies and bookkeeps.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import capi
from . import autotune
from .kmer_analysis import KmerAnalysis, Result, count_batch, finalize_batch, make_params, plan


@dataclass
class Job:
    seq: np.ndarray
    qual: np.ndarray
    offsets: np.ndarray
    params: dict                       # make_params keywords (k, min_depth, sizing, ...)
    job_id: int = 0
    arrival: float = 0.0               # set by submit()
    t_start: float = 0.0
    t_done: float = 0.0
    handle: KmerAnalysis | None = None  # resident table when keep_resident
    footprint: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_bases(self) -> int:
        return int(self.offsets[-1] - self.offsets[0])

    @property
    def n_reads(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def kma_params(self, tuned: bool = True) -> capi.kma_params:
        """Counting parameters of the job; the library chooses one table or on-chip partitions
        from the job's size (kmer_analysis_plan), as for any handle. With `tuned`, the
        autotuner's choice for the job's class fills in what the job's keywords leave open."""
        p = dict(self.params)
        p.setdefault("max_bases", max(self.n_bases, 1))
        p.setdefault("max_reads", max(self.n_reads, 1))
        if tuned:
            p, _ = autotune.apply(p)
        return make_params(**p)


class Server:
    """Continuous-batching server. `device_budget` bytes bound the device memory admitted
    jobs may hold (default: 80 % of the free memory at start)."""

    def __init__(self, device_budget: int | None = None, max_batch: int = 16, workers: int = 2,
                 keep_resident: bool = False, device: int = 0, host_count_bases: int = 32 << 20,
                 tuned: bool = True):
        import torch
        self.torch = torch
        self.device = device
        torch.cuda.set_device(device)
        if device_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            device_budget = int(free * 0.8)
        self.budget = device_budget
        self.max_batch = min(max_batch, capi.KMA_MAX_BATCH)
        self.keep_resident = keep_resident
        self.host_count_bases = host_count_bases  # jobs this large count from host memory
        self.tuned = tuned                        # autotuner's choices per job class
        self.used = 0
        self.pending: deque[tuple[Job, Future]] = deque()
        self.cv = threading.Condition()
        self.closed = False
        self.done: list[Job] = []
        self.failures: list[tuple[Job, BaseException]] = []
        self.batches = 0
        # host wall time of each phase of the batches, summed over the workers (ms)
        self.phase_ms = {"copy_in": 0.0, "create": 0.0, "count": 0.0, "finalize": 0.0, "copy_out": 0.0,
                         "release": 0.0}
        self.admit_hook = None  # testing: callable(job) that may raise to simulate failures
        self.threads = [threading.Thread(target=self._worker, daemon=True, name=f"kma-serve-{i}")
                        for i in range(workers)]
        for t in self.threads:
            t.start()

    # ------------------------------------------------------------------ client side
    def footprint(self, job: Job) -> int:
        pl = plan(job.kma_params(self.tuned))
        keys = int(job.params.get("expected_keys") or job.params.get("expected_distinct") or job.n_bases)
        return int(pl.device_bytes + 2 * job.n_bases + 8 * (job.n_reads + 1) + keys * 54)

    def submit(self, job: Job) -> Future:
        fut: Future = Future()
        job.footprint = self.footprint(job)
        if job.footprint > self.budget:
            fut.set_exception(MemoryError(f"job {job.job_id} needs {job.footprint} B > budget {self.budget} B"))
            return fut
        job.arrival = time.perf_counter()
        with self.cv:
            self.pending.append((job, fut))
            self.cv.notify_all()
        return fut

    def release(self, job: Job) -> None:
        """Free a resident job's table (keep_resident=True)."""
        if job.handle is not None:
            job.handle.destroy()
            job.handle = None
            with self.cv:
                self.used -= job.footprint
                self.cv.notify_all()

    def close(self, wait: bool = True) -> None:
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        if wait:
            for t in self.threads:
                t.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ scheduling
    def _admit(self) -> list[tuple[Job, Future]]:
        """Block until at least one job fits; take the admissible prefix of the queue."""
        with self.cv:
            while True:
                if self.pending and self.used + self.pending[0][0].footprint <= self.budget:
                    break
                if self.closed and not self.pending:
                    return []
                self.cv.wait(0.05)
            batch = []
            while (self.pending and len(batch) < self.max_batch
                   and self.used + self.pending[0][0].footprint <= self.budget):
                job, fut = self.pending.popleft()
                self.used += job.footprint
                batch.append((job, fut))
            return batch

    def _release_budget(self, jobs):
        with self.cv:
            for j in jobs:
                self.used -= j.footprint
            self.cv.notify_all()

    def _worker(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        dev = f"cuda:{self.device}"

        while True:
            batch = self._admit()
            if not batch:
                return
            jobs = [j for j, _ in batch]
            handles: list[KmerAnalysis] = []
            try:
                t0 = time.perf_counter()
                for j in jobs:
                    j.t_start = t0
                    if self.admit_hook is not None:
                        self.admit_hook(j)
                tp = [time.perf_counter()]
                with torch.cuda.stream(stream):
                    # small jobs: reads copied to the device and counted together (one packing
                    # and one counting launch); large jobs: counted from host memory through the
                    # library's staged copies (one call, so the copies of several workers overlap)
                    small = [i for i, j in enumerate(jobs) if j.n_bases < self.host_count_bases]
                    large = [i for i, j in enumerate(jobs) if j.n_bases >= self.host_count_bases]
                    reads = [(torch.from_numpy(jobs[i].seq).to(dev), torch.from_numpy(jobs[i].qual).to(dev),
                              torch.from_numpy(jobs[i].offsets.view(np.int64)).to(dev)) for i in small]
                    tp.append(time.perf_counter())
                    for j in jobs:
                        handles.append(KmerAnalysis(j.kma_params(self.tuned), stream=stream))
                    tp.append(time.perf_counter())
                    if small:
                        count_batch([handles[i] for i in small], reads)
                    for i in large:
                        handles[i].count(jobs[i].seq, jobs[i].qual, jobs[i].offsets)
                    tp.append(time.perf_counter())
                    finalize_batch(handles)
                    tp.append(time.perf_counter())
                    results = [h.copy_result() for h in handles]
                    tp.append(time.perf_counter())
                    del reads
                t1 = time.perf_counter()
                for name, a, b in zip(("copy_in", "create", "count", "finalize", "copy_out"), tp, tp[1:]):
                    self.phase_ms[name] += (b - a) * 1e3
                self.batches += 1
                for j, fut, h, r in zip(jobs, [f for _, f in batch], handles, results):
                    j.t_done = t1
                    if self.keep_resident:
                        j.handle = h
                    else:
                        h.destroy()
                    fut.set_result(r)
                    self.done.append(j)
                if not self.keep_resident:
                    self._release_budget(jobs)
                self.phase_ms["release"] += (time.perf_counter() - t1) * 1e3
            except BaseException as e:  # a failed batch fails its jobs, the server goes on
                for h in handles:
                    h.destroy()
                for j, fut in batch:
                    if not fut.done():
                        fut.set_exception(e)
                    self.failures.append((j, e))
                self._release_budget(jobs)

    # ------------------------------------------------------------------ statistics
    def latency_stats(self) -> dict:
        """Latency (arrival -> results) of the finished jobs: percentiles, split into the wait for
        a worker (arrival -> batch start) and the batch's service time, and p50 of the largest
        quarter of the jobs (by bases) against the rest."""
        lat = np.array([j.t_done - j.arrival for j in self.done])
        if lat.size == 0:
            return {"jobs": 0}
        wait = np.array([j.t_start - j.arrival for j in self.done])
        service = lat - wait
        size = np.array([j.n_bases for j in self.done])
        big = size >= np.percentile(size, 75)
        ms = lambda a, q: float(np.percentile(a, q) * 1e3) if a.size else 0.0  # noqa: E731
        return {"jobs": int(lat.size), "p50_ms": ms(lat, 50), "p99_ms": ms(lat, 99),
                "mean_ms": float(lat.mean() * 1e3), "batches": self.batches,
                "p99_wait_ms": ms(wait, 99), "p99_service_ms": ms(service, 99),
                "p50_ms_largest_quarter": ms(lat[big], 50), "p50_ms_rest": ms(lat[~big], 50)}


def run_plain(jobs: list[Job], device: int = 0, keep: bool = True, lazy: bool = False, tuned: bool = True):
    """The plain path: one job at a time, create -> count (host reads) -> finalize -> copy
    the records -> destroy. Returns the results (keep=False: the results without their
    records, only the sizes; lazy=True: a generator, one job's records in memory at a time)."""
    def one(j):
        with KmerAnalysis(j.kma_params(tuned)) as ka:
            ka.count(j.seq, j.qual, j.offsets)
            info = ka.finalize()
            r = ka.copy_result()
            if not keep:
                empty = np.zeros((0, 2), np.uint64)
                r = Result(empty, np.zeros(0, np.uint32), np.zeros((0, 8), np.uint32),
                           np.zeros((0, 2), np.uint8), int(info.n_uu), int(info.valid_windows),
                           int(info.table_keys))
            return r
    gen = (one(j) for j in jobs)
    return gen if lazy else list(gen)
