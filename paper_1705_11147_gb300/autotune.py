"""Autotuner for the counting launch shape, table load factor and on-chip partitioning.

Candidates are timed on a representative read set (device tensors), count + finalize with
the device synchronised on both sides; every candidate must give identical records (same
number and an order-independent checksum computed on the device), otherwise tuning stops
with an error. The fastest candidate is cached in a JSON file keyed by (GPU name, key width:
one or two 64-bit words, size class = floor(log2 bases)), and `best()` returns it for later
jobs of that class.

Lookup order: the user cache ($KMA_TUNE_CACHE, else ~/.cache/kmer_analysis_tune.json), then
the table shipped with the package (tuned.json, written by tuning runs on GB300 with
`python bench.py --autotune`), else no tuning (the library's automatic choices).
`apply()` merges the choice under a job's own keywords; the bench, the batched handles and
the serving loop take their parameters through it.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from .kmer_analysis import KmerAnalysis, make_params, plan

SHIPPED_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")

# one table (jobs below the automatic partitioning threshold)
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

# on-chip partitions: partition count around the automatic one, sub-table load factor, records
# per thread of the record passes
PARTITIONED_CANDIDATES = [
    dict(),
    dict(partition_scale=0.5),
    dict(partition_scale=2.0),
    dict(load_factor=0.6),
    dict(load_factor=0.7),
    dict(windows_per_thread=4),
    dict(partition_scale=0.5, load_factor=0.7),
]

# keywords a tuning entry may set
TUNABLE = ("partitions", "partition_scale", "load_factor", "windows_per_thread", "block_threads", "ctas_per_sm",
           "warp_aggregate", "slot_prefetch")


def cache_path() -> str:
    return os.environ.get("KMA_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                            "kmer_analysis_tune.json")


def size_class(n_bases: int) -> int:
    return int(math.floor(math.log2(max(n_bases, 1))))


def cache_key(gpu_name: str, k: int, n_bases: int) -> str:
    return f"{gpu_name}|kw{2 if k > 32 else 1}|{size_class(n_bases)}"


_LOADED: dict[str, tuple[int, dict]] = {}


def load_cache(path: str | None = None) -> dict:
    """The tuning table at `path` ({} if absent or unreadable); re-read when its mtime changes."""
    path = path or cache_path()
    try:
        mtime = os.stat(path).st_mtime_ns
        hit = _LOADED.get(path)
        if hit and hit[0] == mtime:
            return dict(hit[1])
        with open(path) as f:
            table = json.load(f)
        _LOADED[path] = (mtime, table)
        return dict(table)
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
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "no-gpu"


def lookup(k: int, n_bases: int, gpu_name: str | None = None, path: str | None = None,
           shipped: str | None = SHIPPED_TABLE) -> tuple[dict, str]:
    """(tuning for this class of job, where it came from: "cache", "shipped" or "none")."""
    key = cache_key(gpu_name or _gpu_name(), k, n_bases)
    entry = load_cache(path).get(key)
    if entry:
        return dict(entry["params"]), "cache"
    if shipped:
        entry = load_cache(shipped).get(key)
        if entry:
            return dict(entry["params"]), "shipped"
    return {}, "none"


def best(k: int, n_bases: int, gpu_name: str | None = None, path: str | None = None,
         shipped: str | None = None) -> dict:
    """Cached tuning for this class of job ({} if none): keyword arguments for make_params."""
    return lookup(k, n_bases, gpu_name, path, shipped)[0]


def apply(kw: dict, gpu_name: str | None = None, path: str | None = None,
          shipped: str | None = SHIPPED_TABLE) -> tuple[dict, str]:
    """make_params keywords `kw` (k, max_bases, ...) with the tuned choices for their job class
    filled in where `kw` sets nothing (a keyword present in `kw` wins); returns (keywords,
    source of the tuning)."""
    tuned, src = lookup(kw["k"], int(kw["max_bases"]), gpu_name, path, shipped)
    out = dict(kw)
    for key, v in tuned.items():
        if key in TUNABLE and not out.get(key):
            out[key] = v
    if kw.get("partitions"):
        out.pop("partition_scale", None)
    return expand(out, {}), src


def expand(candidate: dict, base: dict) -> dict:
    """Resolve relative partition counts into absolute ones: partitions = -m is m times the
    automatic count, partition_scale = s is s times it (rounded, at least 2)."""
    c = dict(candidate)
    p = c.get("partitions", 0)
    scale = c.pop("partition_scale", None)
    if p < 0 or scale is not None:
        auto = plan(make_params(**{**base, **{kk: v for kk, v in c.items() if kk != "partitions"},
                                   "partitions": 0})).partitions
        k = c.get("k", base.get("k", 31))
        if p < 0:
            want = auto * (-p)
        else:  # a job the library keeps in one table stays in one table
            want = auto if auto == 1 else max(2, int(round(auto * scale)))
        c["partitions"] = max(1, min(2048 if k > 32 else 4096, want))
    return c


def candidates_for(base: dict) -> list[dict]:
    """The candidate list for a job: partitioned candidates when the library would partition it."""
    return PARTITIONED_CANDIDATES if plan(make_params(**base)).partitions > 1 else DEFAULT_CANDIDATES


_M31 = (1 << 31) - 1


def _checksum(ka: KmerAnalysis) -> tuple:
    """(records, valid windows, two order-independent sums): each record's 32-bit fields
    (key halves, count, extension counts, codes) are folded into a polynomial hash mod 2^31 - 1
    (every product stays below 2^63); the sums of the hashes and of their squares mod 2^31 - 1
    do not depend on the record order."""
    import torch
    keys, counts, ext, codes = ka.copy_result_device()
    n = int(counts.numel())
    if n == 0:
        return 0, int(ka.result_info.valid_windows), 0, 0
    lo32 = (1 << 32) - 1
    cols = [keys[:, 0] & lo32, (keys[:, 0] >> 32) & lo32, keys[:, 1] & lo32, (keys[:, 1] >> 32) & lo32,
            counts.to(torch.int64) & lo32]
    cols += [ext[:, j].to(torch.int64) & lo32 for j in range(ext.shape[1])]
    cols += [codes[:, j].to(torch.int64) for j in range(codes.shape[1])]
    h = torch.zeros(n, dtype=torch.int64, device=keys.device)
    for c in cols:
        h = (h * 1000003 + c % _M31) % _M31
    s1 = int(h.sum().item())
    s2 = int(((h * h) % _M31).sum().item())
    del keys, counts, ext, codes, cols, h
    return n, int(ka.result_info.valid_windows), s1, s2


def tune(seq, qual, offsets, base: dict, candidates: list[dict] | None = None, reps: int = 2,
         path: str | None = None, save: bool = True, log=None, label: str = "") -> dict:
    """Time every candidate on (seq, qual, offsets) with counting parameters `base` (k,
    min_depth, sizing, ...); return {"params": best candidate as given (relative partition
    counts stay relative), "resolved": its absolute keywords for this job, "ms": ..., "all":
    [...]} and cache it."""
    import torch
    candidates = candidates or candidates_for(base)
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
        torch.cuda.empty_cache()
        if ref is None:
            ref = chk
        elif chk != ref:
            raise RuntimeError(f"candidate {c} changed the result: {chk} != {ref}")
        ms = float(np.median(times))
        results.append({"params": dict(cand), "resolved": c, "ms": ms})
        if log:
            log(f"  {c}: {ms:.2f} ms")
    win = min(results, key=lambda r: r["ms"])
    entry = {"params": win["params"], "resolved": win["resolved"], "ms": win["ms"], "n_bases": n_bases,
             "all": results, "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if label:
        entry["workload"] = label
    if save:
        cache = load_cache(path)
        cache[cache_key(_gpu_name(), base["k"], n_bases)] = entry
        save_cache(cache, path)
    return entry
