"""Autotuner for the counting launch shape, table load factor and on-chip partitioning.

Candidates are timed on a representative read set (device tensors) with the library's own
per-kernel CUDA events; every candidate must give identical records (same count and
checksum), otherwise tuning stops with an error. The fastest candidate is cached in a JSON
file keyed by (GPU name, key width: one or two 64-bit words, size class = floor(log2 bases)),
and `best()` returns it for later jobs of that class.

Cache file: $KMA_TUNE_CACHE, else ~/.cache/kmer_analysis_tune.json.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from .kmer_analysis import KmerAnalysis, make_params, plan

DEFAULT_CANDIDATES = [
    dict(partitions=1, windows_per_thread=1, block_threads=256),
    dict(partitions=1, windows_per_thread=2, block_threads=256),
    dict(partitions=1, windows_per_thread=2, block_threads=128),
    dict(partitions=1, windows_per_thread=2, load_factor=0.7),
    dict(partitions=0),                       # automatic partition count
    dict(partitions=0, load_factor=0.7),
    dict(partitions=-2),                      # twice the automatic count
    dict(partitions=-1, warp_aggregate=True),  # automatic count, warp aggregation
]


def cache_path() -> str:
    return os.environ.get("KMA_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                            "kmer_analysis_tune.json")


def size_class(n_bases: int) -> int:
    return int(math.floor(math.log2(max(n_bases, 1))))


def cache_key(gpu_name: str, k: int, n_bases: int) -> str:
    return f"{gpu_name}|kw{2 if k > 32 else 1}|{size_class(n_bases)}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def best(k: int, n_bases: int, gpu_name: str | None = None, path: str | None = None) -> dict:
    """Cached tuning for this class of job ({} if none): keyword arguments for make_params."""
    entry = load_cache(path).get(cache_key(gpu_name or _gpu_name(), k, n_bases))
    return dict(entry["params"]) if entry else {}


def expand(candidate: dict, base: dict) -> dict:
    """Resolve relative partition counts (-1 = automatic, -2 = twice automatic)."""
    c = dict(candidate)
    p = c.get("partitions", 0)
    if p < 0:
        auto = plan(make_params(**{**base, **{kk: v for kk, v in c.items() if kk != "partitions"},
                                   "partitions": 0})).partitions
        k = c.get("k", base.get("k", 31))
        c["partitions"] = max(1, min(2048 if k > 32 else 4096, auto * (-p)))
    return c


def _checksum(ka: KmerAnalysis) -> tuple:
    r = ka.copy_result()
    order = np.lexsort((r.keys[:, 0], r.keys[:, 1]))
    h = np.uint64(1469598103934665603)
    for arr in (r.keys[order], r.counts[order], r.ext[order]):
        h ^= np.bitwise_xor.reduce(arr.astype(np.uint64).ravel() * np.uint64(0x9E3779B97F4A7C15)
                                   + np.arange(arr.size, dtype=np.uint64), initial=np.uint64(0))
    return len(r), int(h), int(r.valid_windows)


def tune(seq, qual, offsets, base: dict, candidates: list[dict] | None = None, reps: int = 2,
         path: str | None = None, save: bool = True, log=None) -> dict:
    """Time every candidate on (seq, qual, offsets) with counting parameters `base` (k,
    min_depth, sizing, ...); return {"params": best, "ms": ..., "all": [...]} and cache it."""
    import torch
    candidates = candidates or DEFAULT_CANDIDATES
    n_bases = int(seq.numel())
    results = []
    ref = None
    for cand in candidates:
        c = expand(cand, base)
        prm = make_params(**{**base, **c})
        times = []
        with KmerAnalysis(prm) as ka:
            for rep in range(reps + 1):
                ka.reset()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ka.count(seq, qual, offsets)
                ka.finalize()
                torch.cuda.synchronize()
                if rep:  # first run warms the memory pool
                    times.append((time.perf_counter() - t0) * 1e3)
            chk = _checksum(ka)
        if ref is None:
            ref = chk
        elif chk != ref:
            raise RuntimeError(f"candidate {c} changed the result: {chk} != {ref}")
        ms = float(np.median(times))
        results.append({"params": c, "ms": ms})
        if log:
            log(f"  {c}: {ms:.2f} ms")
    win = min(results, key=lambda r: r["ms"])
    entry = {"params": win["params"], "ms": win["ms"], "n_bases": n_bases,
             "all": results, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if save:
        cache = load_cache(path)
        cache[cache_key(_gpu_name(), base["k"], n_bases)] = entry
        save_cache(cache, path)
    return entry
