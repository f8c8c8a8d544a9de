#!/usr/bin/env python
"""k-mer analysis throughput on GB300 (HipMer k-mer analysis stage, arXiv 1705.11147 Sec. 5.1).

One step = the whole hot path over the workload's reads, inputs resident in HBM:
  reset (Bloom filter, table) -> count (pack + Bloom pass) -> finalize (recount + classify
  and compaction) -> query (1 M present + 1 M random k-mers).
value = valid windows (k-mer occurrences) / step time, in G k-mers/s.

Default workload: the 200 Mbp genome with 5 % repeats, 30x of 250 bp reads (24 M reads,
6 Gbases, 4.8 G windows), k = 51, Bloom pass at 1 % FPR, min depth 4, Q20. The 12 GB of
reads are far larger than L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large_200m|bacterial_5m|plain_1m] [--no-e2e] [--no-cpu]

Under torchrun (N > 1) each rank owns 1/N of the k-mers (owner-computes, Section 5.1):
every rank scans all reads but counts only its own keys, no data-path collective; the time
is the max over ranks (strong scaling). --impl reference times the CPU oracle on a bounded
sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "k-mer analysis Gk-mers/s & HBM GB/s at 1 GB300; batched vs plain, bit-exact"
UNIT = "Gk-mers/s"


# ------------------------------------------------------------------ sizing

def workload_sizing(rs, n_parts: int = 1) -> dict:
    """Bloom and table sizes from the read set's recipe (genome size, coverage, error rate):
    what a user who knows the approximate genome size would pass. Results never depend on
    these; a table that turns out too small is reported (KMA_EFULL), not truncated."""
    m = rs.meta
    p = m["params"]
    k, G, e, L = p["k"], m["G"], m["err"], m["L"]
    W = rs.windows_upper_bound(k)
    p_err = 1.0 - (1.0 - e) ** k                 # windows holding at least one error
    distinct = G + W * p_err                      # true k-mers + (mostly unique) error k-mers
    f = m["coverage"] * (1.0 - (k - 1) / L)       # Section 2: expected occurrences of a k-mer
    lam = f * (e / 3.0) * (1.0 - e) ** (k - 1)    # reads sharing one specific error k-mer
    twice = G * k * 3 * (1.0 - math.exp(-lam) * (1.0 + lam))
    keys = G + twice + p.get("bloom_fpr", 0.01) * W * p_err
    return dict(expected_distinct=int(distinct * 1.05 / n_parts) + 1024,
                expected_keys=int(keys * 1.25 / n_parts) + 1024)


def handle_kwargs(rs, n_parts=1, part=0, tuned=True, **tuning):
    """make_params keywords of the bench's handles, and where their launch tuning came from:
    explicit keywords win, then the autotuner's choice for the job class (user cache, else the
    table shipped with the package), else the library's automatic choices."""
    from paper_1705_11147_gb300 import autotune
    p = rs.meta["params"]
    kw = dict(k=p["k"], min_depth=p["min_depth"], min_ext_count=2,
              qual_threshold=p["qual_threshold"], use_bloom=True,
              bloom_fpr=p.get("bloom_fpr", 0.01), max_bases=rs.n_bases,
              max_reads=rs.n_reads, n_parts=n_parts, part=part, **workload_sizing(rs, n_parts), **tuning)
    return autotune.apply(kw) if tuned else (kw, "none")


def make_handle_params(rs, n_parts=1, part=0, tuned=True, **tuning):
    from paper_1705_11147_gb300 import make_params
    return make_params(**handle_kwargs(rs, n_parts, part, tuned, **tuning)[0])


def run_large_once(rs, **tuning):
    """The bench's launch configuration, once, result copied to the host (used by the
    full-size sampled parity test)."""
    import torch
    from paper_1705_11147_gb300 import KmerAnalysis
    seq = torch.from_numpy(rs.seq).cuda()
    qual = torch.from_numpy(rs.qual).cuda()
    offs = torch.from_numpy(rs.offsets.astype(np.int64)).cuda()
    with KmerAnalysis(make_handle_params(rs, **tuning)) as ka:
        ka.count(seq, qual, offs)
        ka.finalize()
        res = ka.copy_result()
    del seq, qual, offs
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ distributed helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Barrier + max of a per-rank time (the only cross-rank operation: timing, not data)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ CPU baseline (oracle)

def cpu_baseline(rs, budget_s: float = 15.0, threads: int | None = None) -> dict:
    """The oracle as it stands, timed on a prefix of the workload's reads sized for about
    `budget_s` seconds of CPU work on all host cores."""
    import oracle
    threads = threads or os.cpu_count() or 1
    k = rs.meta["params"]["k"]
    p = dict(rs.meta["params"])
    p.pop("bloom_fpr", None)
    n = oracle_sample_reads(rs, budget_s, threads)
    offs = rs.offsets[: n + 1]
    t0 = time.perf_counter()
    r = oracle.run(rs.seq[: int(offs[-1])], rs.qual[: int(offs[-1])], offs, threads=threads, **p)
    dt = time.perf_counter() - t0
    return {"value": r.valid_windows / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} of {rs.n_reads} reads ({r.valid_windows} windows, k={k}), "
                      f"{dt:.1f} s wall on {threads} threads",
            "seconds": round(dt, 2), "windows": int(r.valid_windows), "reads": n}


# ------------------------------------------------------------------ GPU arm

PROFILE_DIR = os.path.join(ROOT, "profiles")


def kernel_source_digest(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1705_11147_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_values(summary: str, digest: str) -> dict:
    """Per-unit figures recorded by an ncu capture (profiles/<summary>: lines `name: value`),
    or {} when the kernel sources changed since the capture."""
    try:
        text = open(os.path.join(PROFILE_DIR, summary)).read()
    except OSError:
        return {}
    vals = {}
    for line in text.splitlines():
        if ":" in line and not line.startswith((" ", "|", "#")):
            key, val = line.split(":", 1)
            vals[key.strip()] = val.strip()
    if vals.get("kernel_source_digest", "").split(" ")[0] != digest:
        return {}
    out = {}
    for key in ("dram_bytes_per_unit", "l2_requests_per_unit", "l2_peak_requests_per_s"):
        try:
            out[key] = float(vals[key].split(" ")[0])
        except (KeyError, ValueError):
            pass
    return out


def roofline(timing: dict, res_info, positions: int, peak_gbs: float, plan_used, k: int) -> dict:
    """Dominant kernel (the counting pass), algorithmic DRAM bytes per launch.
    one table (pass_kernel, Bloom mode; filter and table far larger than L2, 32-byte sectors):
      64 B per valid window (Bloom word sector read + write-back), 128 B per window whose k-mer
      the filter had seen (slot key/count sector + extension sector, read + written back),
      0.625 B per arena position (codes, reverse codes... read, marks written).
    partitions (part_pass_kernel, Bloom mode), the partitioned model of the hot-path table:
      per record (one per valid window) its key + info byte read (17 B, 9 B for k <= 32), and
      per first sighting the record written back (compacted for the recount). A second figure
      adds each partition's Bloom sub-filter and sub-table brought from HBM once and written
      back once (2 x filter + table bytes).
    The partitioned pass keeps its random atomics in L2, so its ceiling is the L2 request
    rate: `l2` gives the L2 requests per record from the ncu capture times the records, over
    the live kernel time, against the L2's peak request rate (slices x L2 clock, from ncu)."""
    W = int(res_info.valid_windows)
    F = int(timing["first_sightings"])
    ms = timing["ms_pass"] / max(timing["n_pass"], 1)
    extra = {}
    if plan_used.partitions > 1:
        rec = (16 if k > 32 else 8) + 1
        struct_bytes = plan_used.bloom_words * 8 + plan_used.table_slots * 64
        algo = float(W) * rec + float(F) * rec
        kernel, files, summary = ("part_pass_kernel (Bloom mode)", ["kma_partition.cu", "kma_device.cuh"],
                                  "part_pass_kernel_large_200m.md")
        with_struct = algo + 2.0 * struct_bytes
        extra["with_partition_structures"] = {
            "algo_bytes_per_launch": int(with_struct),
            "achieved": round(with_struct / (ms * 1e-3) / 1e9, 1),
            "frac": round(with_struct / (ms * 1e-3) / 1e9 / peak_gbs, 4)}
    else:
        algo = 64.0 * W + 128.0 * (W - F) + 0.625 * positions
        kernel, files, summary = ("pass_kernel (Bloom mode)", ["kma_kernels.cu", "kma_device.cuh"],
                                  "pass_kernel_large_200m.md")
    achieved = algo / (ms * 1e-3) / 1e9
    prof = profiled_values(summary, kernel_source_digest(files))
    out = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak_gbs, "unit": "GB/s",
           "frac": round(achieved / peak_gbs, 4),
           "traffic": int(prof["dram_bytes_per_unit"] * W) if "dram_bytes_per_unit" in prof else None,
           "kernel": kernel, "ms_per_launch": round(ms, 3), "algo_bytes_per_launch": int(algo),
           "peak_source": "of measured (hbm_gbs)", **extra}
    if "l2_requests_per_unit" in prof and "l2_peak_requests_per_s" in prof:
        req = prof["l2_requests_per_unit"] * W
        l2_ach = req / (ms * 1e-3) / 1e9
        l2_peak = prof["l2_peak_requests_per_s"] / 1e9
        out["l2"] = {"achieved": round(l2_ach, 1), "peak": round(l2_peak, 1), "unit": "G L2 requests/s",
                     "frac": round(l2_ach / l2_peak, 4), "requests_per_launch": int(req),
                     "source": "ncu lts__t_requests per record x records / live kernel time; peak = "
                               "lts__t_requests.sum.peak_sustained x L2 clock (ncu)"}
    return out


def load_peak() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0  # fallback figure of the profiling recipe


def run_ours(args, ws, rank, local):
    import torch
    from paper_1705_11147_gb300 import KmerAnalysis

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    t_gen = time.perf_counter()
    rs = synth.workload(args.workload, scale=args.scale)
    t_gen = time.perf_counter() - t_gen
    k = rs.meta["params"]["k"]
    seq = torch.from_numpy(rs.seq).to(dev)
    qual = torch.from_numpy(rs.qual).to(dev)
    offs = torch.from_numpy(rs.offsets.astype(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)
    if args.autotune:
        autotune_workload(args, rs, seq, qual, offs, ws, rank)
    hkw, tuning_source = handle_kwargs(rs, n_parts=ws, part=rank, tuned=args.tuned, **args.tuning)
    from paper_1705_11147_gb300 import make_params
    prm = make_params(**hkw)
    from paper_1705_11147_gb300 import plan as _plan
    plan_used = _plan(prm)
    ka = KmerAnalysis(prm, stream=stream)

    # query set: 1 M k-mers present in the result + 1 M random k-mers (mostly absent)
    ka.count(seq, qual, offs)
    info = ka.finalize()
    n_res = int(info.n)
    keys_dev, _, _, _ = ka.copy_result_device()
    g = torch.Generator(device=dev).manual_seed(1234 + rank)
    nq = min(args.queries, max(n_res, 1))
    pick = torch.randint(0, max(n_res, 1), (nq,), device=dev, generator=g)
    present = keys_dev[pick] if n_res else torch.zeros((0, 2), dtype=torch.int64, device=dev)
    rnd = torch.randint(0, 2**62, (args.queries, 2), device=dev, generator=g, dtype=torch.int64)
    rnd[:, 1] &= (1 << max(2 * k - 64, 0)) - 1 if 2 * k > 64 else 0
    if 2 * k <= 64:
        rnd[:, 0] &= (1 << (2 * k)) - 1
    qkeys = torch.cat([present, rnd]).contiguous()
    del keys_dev
    q_out = (torch.empty(qkeys.shape[0], dtype=torch.int32, device=dev),
             torch.empty((qkeys.shape[0], 8), dtype=torch.int32, device=dev),
             torch.empty((qkeys.shape[0], 2), dtype=torch.uint8, device=dev))

    def step():
        ka.reset()
        ka.count(seq, qual, offs)
        r = ka.finalize()
        ka.query(qkeys, out=q_out)
        return r

    # Inputs + filter + table larger than 4x L2: nothing useful survives in L2 from one step to
    # the next. Smaller working sets: L2 is flushed (a buffer twice its size written) before
    # each timed step, and the steps are timed one by one.
    l2_bytes = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 128 << 20) or (128 << 20))
    reads_bytes = 2 * rs.n_bases + 8 * (rs.n_reads + 1)
    struct_bytes = int(plan_used.bloom_words) * 8 + int(plan_used.table_slots) * 64
    arena_bytes = (rs.n_bases + rs.n_reads) * 3 // 4   # codes, complemented codes, invalid, hq
    work_bytes = reads_bytes + struct_bytes + arena_bytes
    flush = work_bytes < 4 * l2_bytes
    scratch = torch.empty(2 * l2_bytes, dtype=torch.uint8, device=dev) if flush else None
    if flush:
        l2_note = (f"working set {work_bytes / 1e6:.0f} MB < 4x L2: L2 flushed before every timed step "
                   f"({2 * l2_bytes >> 20} MB written), steps timed one by one")
    else:
        l2_note = (f"inputs ({reads_bytes / 1e9:.1f} GB of reads) + filter/table/arena "
                   f"({(struct_bytes + arena_bytes) / 1e9:.1f} GB) far larger than L2; no flush")

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize(dev)
    ka.timings(reset=True)
    ka.set_profiling(True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if flush:
        ms_total = 0.0
        for i in range(args.steps):
            scratch.fill_(i & 0xFF)
            ev0.record(stream)
            info = step()
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            ms_total += ev0.elapsed_time(ev1)
    else:
        ev0.record(stream)
        for _ in range(args.steps):
            info = step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_total = ev0.elapsed_time(ev1)
    barrier(ws)
    clk = clocks.stop()
    del scratch
    ms_total = max_over_ranks(ms_total, ws, dev)
    timing = ka.timings(reset=True)
    ka.set_profiling(False)
    ms_step = ms_total / args.steps

    # whole-job units: every valid window of the read set counted once across the ranks
    W_total = rs.windows_upper_bound(k) if ws > 1 else int(info.valid_windows)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([int(info.valid_windows)], dtype=torch.int64, device=dev)
        dist.all_reduce(t)
        W_total = int(t.item())
    value = W_total / (ms_step * 1e-3) / 1e9
    positions = rs.n_bases + rs.n_reads
    roof = roofline(timing, info, positions, load_peak(), plan_used, k)
    kernel_ms = {k2[3:]: round(v / args.steps, 3) for k2, v in timing.items() if k2.startswith("ms_")}
    launches = int(timing["launches"])

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, ka, rs, dev, qkeys, ws)

    # Section 5.1's cardinality pass, timed once on the resident reads (not part of the step:
    # the step is sized from the workload recipe, as a user who knows the genome would)
    import ctypes
    from paper_1705_11147_gb300 import capi, estimate_distinct
    estimate_distinct(seq, qual, offs, k=k, canonical=bool(prm.canonical), stream=stream)  # warm
    torch.cuda.synchronize(dev)
    t_est = time.perf_counter()
    est = estimate_distinct(seq, qual, offs, k=k, canonical=bool(prm.canonical), stream=stream)
    t_est = time.perf_counter() - t_est
    sizing = {"ms": round(t_est * 1e3, 2), "distinct_estimate": round(est.distinct),
              "rel_std_error": round(est.rel_std_error, 5), "precision": est.precision,
              "recipe_expected_distinct": int(prm.expected_distinct),
              "what": "HyperLogLog pass (pack + sketch, temporary arena), host wall time"}

    # Section 5.2's next stage on the finalized result, timed once after the
    # measured steps (not part of the step; its temporaries do not share the pool with them)
    torch.cuda.synchronize(dev)
    t_cg = time.perf_counter()
    cg = capi.kma_contigs()
    capi.check(capi.load().kmer_analysis_contigs(ka.handle, ctypes.byref(cg)), "contigs")
    t_cg = time.perf_counter() - t_cg
    contigs = {"ms": round(t_cg * 1e3, 1), "n_contigs": int(cg.n_contigs), "n_bases": int(cg.n_bases),
               "n_vertices": int(cg.n_vertices), "n_cycles": int(cg.n_cycles),
               "what": "contig generation on the finalized k-mers (list ranking), host wall time"}


    ka.destroy()
    del seq, qual, offs

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
           "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic",
           "config": {"workload": args.workload, "genome_bp": rs.meta["G"], "reads": rs.n_reads,
                      "bases": rs.n_bases, "read_len": rs.meta["L"], "coverage": rs.meta["coverage"],
                      "k": k, "min_depth": rs.meta["params"]["min_depth"], "bloom_fpr": 0.01,
                      "valid_windows": int(info.valid_windows), "kmers_out": int(info.n),
                      "uu_kmers": int(info.n_uu), "table_keys": int(info.table_keys),
                      "queries_per_step": int(qkeys.shape[0]),
                      "parallelism": f"owner-computes x{ws}" if ws > 1 else "1 GPU",
                      "l2": l2_note},
           "roofline": roof, "kernel_ms_per_step": kernel_ms, "gpu_launches": launches,
           "tuning": {k2: getattr(prm, k2) for k2 in ("block_threads", "windows_per_thread", "ctas_per_sm",
                                                      "warp_aggregate", "slot_prefetch", "partitions")}
                     | {"partitions_used": int(plan_used.partitions), "load_factor": round(prm.load_factor, 3),
                        "source": tuning_source if not args.tuning else "command line"},
           "clocks": clk, "generation_s": round(t_gen, 1), "sizing_pass": sizing, "contigs": contigs}
    if e2e:
        out["e2e"] = e2e
    if rank == 0 and ws == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(rs, budget_s=args.cpu_budget)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out if rank == 0 else None


def run_e2e(args, ka, rs, dev, qkeys_dev, ws):
    """Same metric through the public API from pinned host buffers: host->device copies of the
    reads, the whole path, and device->host copies of the records (finalize_to_host) and of the
    query answers."""
    import torch
    seq_h = torch.from_numpy(rs.seq).pin_memory()
    qual_h = torch.from_numpy(rs.qual).pin_memory()
    offs_h = torch.from_numpy(rs.offsets.view(np.int64)).pin_memory()
    qk_h = qkeys_dev.cpu().pin_memory()
    qn = qk_h.shape[0]
    q_counts = torch.empty(qn, dtype=torch.int32).pin_memory()
    q_ext = torch.empty((qn, 8), dtype=torch.int32).pin_memory()
    q_codes = torch.empty((qn, 2), dtype=torch.uint8).pin_memory()
    import ctypes
    from paper_1705_11147_gb300 import capi
    lib = capi.load()
    out_cap = int(ka.result_info.table_keys) + 1
    r_keys = torch.empty((out_cap, 2), dtype=torch.int64).pin_memory()
    r_counts = torch.empty(out_cap, dtype=torch.int32).pin_memory()
    r_ext = torch.empty((out_cap, 8), dtype=torch.int32).pin_memory()
    r_codes = torch.empty((out_cap, 2), dtype=torch.uint8).pin_memory()
    seq_np, qual_np = seq_h.numpy(), qual_h.numpy()
    offs_np = offs_h.numpy().view(np.uint64)

    phases = {}
    step_ms = []

    def step():
        # host wall time of each call (count returns once its input copies are done;
        # finalize_to_host waits for the counting work still in flight, then recounts,
        # classifies and copies the records out, group by group)
        t = [time.perf_counter()]
        ka.reset()
        t.append(time.perf_counter())
        capi.check(lib.kmer_analysis_count(ka.handle, seq_np.ctypes.data, qual_np.ctypes.data,
                                           offs_np.ctypes.data, rs.n_reads, 0), "count")
        t.append(time.perf_counter())
        r = capi.kma_result()
        capi.check(lib.kmer_analysis_finalize_to_host(ka.handle, r_keys.data_ptr(), r_counts.data_ptr(),
                                                      r_ext.data_ptr(), r_codes.data_ptr(), out_cap,
                                                      ctypes.byref(r)), "finalize_to_host")
        t.append(time.perf_counter())
        capi.check(lib.kmer_analysis_query(ka.handle, qk_h.data_ptr(), qn, q_counts.data_ptr(),
                                           q_ext.data_ptr(), q_codes.data_ptr(), 0), "query")
        t.append(time.perf_counter())
        for name, a, b in zip(("reset", "count", "finalize_to_host", "query"), t, t[1:]):
            phases[name] = round((b - a) * 1e3, 2)
        step_ms.append(round((t[-1] - t[0]) * 1e3, 2))
        return r

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    torch.cuda.synchronize(dev)
    barrier(ws)
    step_ms.clear()
    t0 = time.perf_counter()
    steps = max(1, min(args.steps, 3))
    for _ in range(steps):
        info = step()
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t0) / steps
    dt = max_over_ranks(dt, ws, dev)
    n = int(info.n)
    h2d = rs.n_bases * 2 + (rs.n_reads + 1) * 8 + qn * 16
    d2h = n * (16 + 4 + 32 + 2) + qn * (4 + 32 + 2)
    return {"value": round(int(info.valid_windows) * (ws if ws > 1 else 1) / dt / 1e9, 3), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": steps,
            "ms_per_step": round(dt * 1e3, 2), "last_step_phases_ms": phases, "step_host_ms": step_ms}


# ------------------------------------------------------------------ batched (many samples)

def autotune_workload(args, rs, seq, qual, offs, ws, rank):
    """Tune the handle's launch shape, load factor and partition count on this workload (device
    tensors) and store the winner in `args.tune_out` (default: the user cache)."""
    from paper_1705_11147_gb300 import autotune
    base, _ = handle_kwargs(rs, n_parts=ws, part=rank, tuned=False)
    t0 = time.perf_counter()
    entry = autotune.tune(seq, qual, offs, base, reps=2, path=args.tune_out or None,
                          log=lambda m: print(m, file=sys.stderr, flush=True), label=args.workload)
    print(f"autotune: {entry['params']} {entry['ms']:.2f} ms ({time.perf_counter() - t0:.0f} s)",
          file=sys.stderr, flush=True)


def run_batched(args, ws, rank, local):
    """64 independent samples of uneven size: one captured CUDA graph per step (reset, one
    packing and one persistent counting launch for all samples, one recount and one
    classification launch), against the plain path that runs create -> count -> finalize ->
    destroy for one sample after another on the same device-resident reads."""
    import torch
    from paper_1705_11147_gb300 import BatchGraph, KmerAnalysis
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t_gen = time.perf_counter()
    specs = synth.batched_specs(args.samples, scale=args.scale)
    sets = [synth.sample_reads(sp) for sp in specs]
    t_gen = time.perf_counter() - t_gen
    reads = [(torch.from_numpy(rs.seq).to(dev), torch.from_numpy(rs.qual).to(dev),
              torch.from_numpy(rs.offsets.astype(np.int64)).to(dev)) for rs in sets]

    def params(rs):
        return make_handle_params(rs, tuned=args.tuned, **args.tuning)

    handles = [KmerAnalysis(params(rs)) for rs in sets]
    g = BatchGraph(handles, reads)
    for _ in range(args.warmup):
        g.replay()
    g.stream.synchronize()
    for h in handles:
        h.timings(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0.record(g.stream)
    for _ in range(args.steps):
        g.replay()
    ev1.record(g.stream)
    g.stream.synchronize()
    clk = clocks.stop()
    ms_batched = ev0.elapsed_time(ev1) / args.steps
    infos = g.results()
    windows = sum(int(r.valid_windows) for r in infos)
    launches = g.kernels_per_replay
    for h in handles:
        h.destroy()
    del g

    # plain: one job per launch sequence, sample after sample (parameters worked out before
    # the timed loop, as for the batched path: only library work is timed)
    stream = torch.cuda.current_stream(dev)
    plain_params = [params(rs) for rs in sets]

    def plain_once():
        n = 0
        for prm, (sq, ql, of) in zip(plain_params, reads):
            with KmerAnalysis(prm, stream=stream) as ka:
                ka.count(sq, ql, of)
                n += int(ka.finalize().valid_windows)
        return n

    plain_once()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    reps = max(1, min(args.steps, 3))
    for _ in range(reps):
        wp = plain_once()
    torch.cuda.synchronize(dev)
    ms_plain = (time.perf_counter() - t0) * 1e3 / reps
    assert wp == windows
    value = windows / (ms_batched * 1e-3) / 1e9
    plain_value = windows / (ms_plain * 1e-3) / 1e9
    return {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_batched, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched_64", "samples": len(sets),
                       "bases": int(sum(rs.n_bases for rs in sets)), "valid_windows": windows,
                       "k": 51, "scale": args.scale, "mode": "one CUDA graph per step",
                       "l2": "inputs (25 GB of reads) far larger than L2; no flush"},
            "plain": {"value": round(plain_value, 3), "unit": UNIT, "ms_per_step": round(ms_plain, 2),
                      "path": "create -> count -> finalize -> destroy per sample"},
            "batched_vs_plain": round(value / plain_value, 3), "gpu_launches": int(launches),
            "clocks": clk, "generation_s": round(t_gen, 1)}


# ------------------------------------------------------------------ served (job stream)

def records_digest(r) -> str:
    """Digest of a result's records (keys, counts, extension counters, side codes) sorted by
    key: two results hold the same records iff their digests are equal (up to SHA-256
    collisions), without keeping the records."""
    import hashlib
    s = r.sorted()
    h = hashlib.sha256()
    for f in ("keys", "counts", "ext", "codes"):
        h.update(np.ascontiguousarray(getattr(s, f)).tobytes())
    return h.hexdigest()


def run_served(args, ws, rank, local):
    """Counting jobs (genome log-U[1, 50] Mbp x scale, 30x of 150 bp, k in {31, 51}) through the
    continuous-batching server: saturation throughput with every job released at once against
    the plain one-job-at-a-time path, then p50/p99 latency with Poisson arrivals."""
    import torch
    from paper_1705_11147_gb300.serve import Job, Server, run_plain
    torch.cuda.set_device(local)
    t_gen = time.perf_counter()
    specs = synth.served_specs(args.jobs, scale=args.scale)
    jobs = []
    for i, sp in enumerate(specs):
        rs = synth.sample_reads(sp)
        p = dict(rs.meta["params"])
        p.pop("bloom_fpr", None)
        p.update(workload_sizing(rs))
        jobs.append(Job(rs.seq, rs.qual, rs.offsets, params=p, job_id=i,
                        meta={"arrival_s": sp["arrival_s"], "windows": rs.windows_upper_bound(p["k"])}))
    t_gen = time.perf_counter() - t_gen

    def saturate():
        # results are reduced to their window counts as they complete (the records of all
        # jobs would not fit in host memory at the larger scales); digests are taken after
        # the timed region
        with Server(max_batch=args.max_batch, workers=args.workers, tuned=args.tuned) as srv:
            t0 = time.perf_counter()
            futs = [srv.submit(j) for j in jobs]
            windows = []
            for i in range(len(futs)):
                windows.append(int(futs[i].result().valid_windows))
                futs[i] = None  # the records are not kept
            dt = time.perf_counter() - t0
        return dt, windows, srv.batches, {k2: round(v, 1) for k2, v in srv.phase_ms.items()}

    saturate()  # warm-up (pools, module load)
    t_srv, win_srv, batches, phases = saturate()
    t0 = time.perf_counter()
    win_plain = [int(r.valid_windows) for r in run_plain(jobs, keep=False, tuned=args.tuned)]
    t_plain = time.perf_counter() - t0
    windows = sum(win_srv)
    assert win_srv == win_plain
    # every served job's records against its plain run, job by job (outside the timed region)
    n_check = min(len(jobs), args.check_jobs)
    with Server(max_batch=args.max_batch, workers=args.workers, tuned=args.tuned) as srv:
        futs = [srv.submit(j) for j in jobs[:n_check]]
        dig_srv = []
        for i in range(len(futs)):
            dig_srv.append(records_digest(futs[i].result()))
            futs[i] = None
    dig_plain = [records_digest(r) for r in run_plain(jobs[:n_check], keep=True, lazy=True, tuned=args.tuned)]
    same = dig_srv == dig_plain
    # latency under Poisson arrivals (arrival times of the first jobs, in real time)
    n_lat = min(len(jobs), args.latency_jobs)
    with Server(max_batch=args.max_batch, workers=args.workers, tuned=args.tuned) as srv:
        start = time.perf_counter()
        futs = []
        for j in jobs[:n_lat]:
            delay = j.meta["arrival_s"] - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            futs.append(srv.submit(j))
        for f in futs:
            f.result()
        lat = srv.latency_stats()
    value = windows / t_srv / 1e9
    plain_value = windows / t_plain / 1e9
    return {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": 1,
            "warmup": 1, "ms_per_step": round(t_srv * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "served_500", "jobs": len(jobs), "scale": args.scale,
                       "bases": int(sum(j.n_bases for j in jobs)), "valid_windows": windows,
                       "max_batch": args.max_batch, "workers": args.workers,
                       "tuned": bool(args.tuned), "saturation": "all jobs released at t=0"},
            "plain": {"value": round(plain_value, 3), "unit": UNIT, "seconds": round(t_plain, 3),
                      "path": "create -> count (host reads) -> finalize -> copy -> destroy, one job at a time"},
            "served_vs_plain": round(value / plain_value, 3), "batches": batches,
            "records_match_plain": bool(same), "records_checked_jobs": n_check,
            "server_phase_ms": phases,
            "latency": {"jobs": n_lat, "rate_per_s": 4.0, **lat}, "generation_s": round(t_gen, 1)}


# ------------------------------------------------------------------ heavy hitters (satellite)

def run_satellite(args, ws, rank, local):
    """Heavy hitters (Section 5.1): a read set with a tandem satellite in 30 % of its reads.
    The cardinality pass (HyperLogLog + Misra-Gries summaries) runs first, as the paper's
    sizing pass does; its heavy-hitter recommendation chooses the counting mode (warp-level
    grouping of equal keys). Both modes are timed over the same steps (count + finalize)."""
    import torch
    from paper_1705_11147_gb300 import KmerAnalysis, estimate_distinct
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rs = synth.satellite_workload(args.scale)
    seq = torch.from_numpy(rs.seq).to(dev)
    qual = torch.from_numpy(rs.qual).to(dev)
    offs = torch.from_numpy(rs.offsets.astype(np.int64)).to(dev)
    k = rs.meta["params"]["k"]
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    est = estimate_distinct(seq, qual, offs, k=k, stream=stream)
    t_est = time.perf_counter() - t0

    def timed(heavy):
        with KmerAnalysis(make_handle_params(rs, heavy_hitters=heavy, tuned=args.tuned), stream=stream) as ka:
            def step():
                ka.reset()
                ka.count(seq, qual, offs)
                return ka.finalize()
            for _ in range(args.warmup):
                step()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            ev0.record(stream)
            for _ in range(args.steps):
                info = step()
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            return ev0.elapsed_time(ev1) / args.steps, info

    clocks = ClockSampler(local)
    clocks.start()
    ms_rec, info = timed(bool(est.heavy_hitters))
    ms_other, info2 = timed(not est.heavy_hitters)
    clk = clocks.stop()
    assert int(info.n) == int(info2.n) and int(info.valid_windows) == int(info2.valid_windows)
    W = int(info.valid_windows)
    return {"metric": METRIC, "value": round(W / (ms_rec * 1e-3) / 1e9, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_rec, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": "satellite_50m", "scale": args.scale, "bases": rs.n_bases,
                       "reads": rs.n_reads, "valid_windows": W, "k": k, "kmers_out": int(info.n),
                       "step": "reset -> count -> finalize (device-resident reads)"},
            "sizing_pass": {"ms": round(t_est * 1e3, 2), "heavy_hitters": bool(est.heavy_hitters),
                            "sampled_windows": est.sampled_windows, "heavy_threshold": est.heavy_threshold,
                            "top_counts": [int(x) for x in est.summary_counts[:8]]},
            "grouping": {"recommended": bool(est.heavy_hitters), "ms_recommended": round(ms_rec, 3),
                         "ms_other": round(ms_other, 3), "speedup": round(ms_other / ms_rec, 3)},
            "clocks": clk}


# ------------------------------------------------------------------ reference arm

def oracle_sample_reads(rs, budget_s: float, threads: int) -> int:
    """Reads of a prefix that takes the oracle about `budget_s` seconds (from a short
    calibration on the first 20000 reads)."""
    import oracle
    p = dict(rs.meta["params"])
    p.pop("bloom_fpr", None)
    n = min(20000, rs.n_reads)
    offs = rs.offsets[: n + 1]
    t0 = time.perf_counter()
    oracle.run(rs.seq[: int(offs[-1])], rs.qual[: int(offs[-1])], offs, threads=threads, **p)
    dt = max(time.perf_counter() - t0, 1e-6)
    return int(min(rs.n_reads, max(n, n * budget_s / dt)))


def run_reference(args, ws, rank):
    """The CPU oracle on the same workload, metric and unit; each step a bounded prefix of
    the reads, sized so that warm-up + steps take about two minutes (rank 0 only)."""
    if rank != 0:
        return None
    import oracle
    rs = synth.workload(args.workload if args.workload in synth.WORKLOADS else "large_200m", scale=args.scale)
    threads = os.cpu_count() or 1
    p = dict(rs.meta["params"])
    p.pop("bloom_fpr", None)
    budget = max(3.0, min(15.0, 110.0 / max(args.steps + args.warmup, 1)))
    n = oracle_sample_reads(rs, budget, threads)
    offs = rs.offsets[: n + 1]
    s, q = rs.seq[: int(offs[-1])], rs.qual[: int(offs[-1])]
    for _ in range(args.warmup):
        oracle.run(s, q, offs, threads=threads, **p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.run(s, q, offs, threads=threads, **p)
    dt = (time.perf_counter() - t0) / args.steps
    value = r.valid_windows / dt / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt * 1e3, 1), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": rs.meta["workload"], "k": p["k"], "sample_reads": n,
                       "sample_windows": int(r.valid_windows)},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": threads,
                             "kind": "oracle", "sample": f"first {n} of {rs.n_reads} reads per step"},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_200m",
                    choices=list(synth.WORKLOADS) + ["batched_64", "served_500", "satellite_50m"])
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--jobs", type=int, default=500)
    ap.add_argument("--latency-jobs", type=int, default=60)
    ap.add_argument("--check-jobs", type=int, default=500)
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--workers", type=int, default=3)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--queries", type=int, default=1_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--tune", action="append", default=[],
                    help="launch-shape override key=value (block_threads, windows_per_thread, "
                         "ctas_per_sm, warp_aggregate, slot_prefetch, load_factor)")
    ap.add_argument("--no-tuned", dest="tuned", action="store_false",
                    help="library defaults instead of the autotuner's choices for every handle")
    ap.add_argument("--autotune", action="store_true",
                    help="time the autotuner's candidates on the workload first and store the winner "
                         "(measure in a separate run: the timing that follows in the same process "
                         "can be perturbed)")
    ap.add_argument("--tune-out", default="",
                    help="tuning table to write with --autotune (default: the user cache)")
    args = ap.parse_args()
    args.tuning = {}
    for kv in args.tune:
        key, val = kv.split("=", 1)
        args.tuning[key] = float(val) if key == "load_factor" else int(val)
    args.tuning = {k: v for k, v in args.tuning.items()}
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
    else:
        from paper_1705_11147_gb300 import build
        build.build()
        if args.workload == "batched_64":
            out = run_batched(args, ws, rank, local)
        elif args.workload == "served_500":
            out = run_served(args, ws, rank, local)
        elif args.workload == "satellite_50m":
            out = run_satellite(args, ws, rank, local)
        else:
            out = run_ours(args, ws, rank, local)
    if out is not None and rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
