"""ctypes declarations of the C ABI in include/kmer_analysis.h.

Loading fails loudly when libkmer_analysis.so has not been built: there is no fallback
implementation of any step of the path in Python.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkmer_analysis.so")

KMA_OK = 0
KMA_EINVAL = -1
KMA_ENOMEM = -2
KMA_EFULL = -3
KMA_ESTATE = -4
KMA_ETIMEOUT = -5
KMA_EOVERFLOW = -6
KMA_ECUDA = -7
KMA_ETOOLARGE = -8
KMA_NOALLOC_MAX_BASES = 262144
KMA_NOALLOC_MAX_READS = 262144
KMA_CODE_X = 4
KMA_CODE_F = 5
KMA_MAX_BATCH = 64

u8, u32, u64, dbl, vp = ctypes.c_uint8, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class kma_params(ctypes.Structure):
    _fields_ = [("k", u32), ("min_depth", u32), ("min_ext_count", u32),
                ("qual_threshold", u8), ("qual_offset", u8), ("use_bloom", u8), ("canonical", u8),
                ("max_bases", u64), ("max_reads", u64), ("expected_distinct", u64),
                ("bloom_fpr", dbl), ("table_capacity", u64), ("expected_keys", u64),
                ("load_factor", dbl), ("staging_bytes", u64),
                ("block_threads", u32), ("windows_per_thread", u32), ("ctas_per_sm", u32),
                ("warp_aggregate", u32), ("n_parts", u32), ("part", u32),
                ("slot_prefetch", u32), ("fault_inject", u32), ("partitions", u32),
                ("heavy_hitters", u32)]


class kma_plan(ctypes.Structure):
    _fields_ = [("bloom_words", u64), ("bloom_hashes", u32), ("partitions", u32),
                ("bloom_fpr_est", dbl), ("table_slots", u64), ("arena_positions", u64),
                ("device_bytes", u64)]


class kma_result(ctypes.Structure):
    _fields_ = [("n", u64), ("n_uu", u64), ("valid_windows", u64), ("table_keys", u64),
                ("keys", vp), ("counts", vp), ("ext", vp), ("codes", vp)]


class kma_timings(ctypes.Structure):
    _fields_ = [("ms", dbl * 8), ("launches", u64 * 8), ("total_launches", u64),
                ("first_sightings", u64)]


KERNEL_KINDS = ("pack", "pass", "recount", "classify", "query", "init", "unused", "scatter")


class kma_contigs(ctypes.Structure):
    _fields_ = [("n_contigs", u64), ("n_bases", u64), ("n_vertices", u64), ("n_cycles", u64),
                ("seq", vp), ("offsets", vp)]


class kma_estimate(ctypes.Structure):
    _fields_ = [("precision", u32), ("heavy_hitters", u32), ("distinct", dbl), ("rel_std_error", dbl),
                ("valid_windows", u64), ("sampled_windows", u64), ("heavy_threshold", u64),
                ("n_summary", u64), ("summary_capacity", u64), ("summary_keys", vp),
                ("summary_counts", vp), ("summary_bucket", vp), ("bucket_windows", vp)]


HLL_MIN_PRECISION, HLL_MAX_PRECISION = 4, 14
MG_SAMPLE, MG_BUCKETS, MG_COUNTERS = 64, 32, 32


class kma_reads(ctypes.Structure):
    _fields_ = [("seq", vp), ("qual", vp), ("offsets", vp), ("n_reads", u64), ("n_bases", u64)]


_SIGS = {
    "kmer_analysis_plan": ([ctypes.POINTER(kma_params), ctypes.POINTER(kma_plan)], ctypes.c_int),
    "kmer_analysis_create": ([ctypes.POINTER(kma_params), vp, ctypes.POINTER(vp)], ctypes.c_int),
    "kmer_analysis_count": ([vp, vp, vp, vp, u64, ctypes.c_int], ctypes.c_int),
    "kmer_analysis_finalize": ([vp, ctypes.POINTER(kma_result)], ctypes.c_int),
    "kmer_analysis_copy_result": ([vp, vp, vp, vp, vp, u64, ctypes.c_int], ctypes.c_int),
    "kmer_analysis_finalize_to_host": ([vp, vp, vp, vp, vp, u64, ctypes.POINTER(kma_result)], ctypes.c_int),
    "kmer_analysis_query": ([vp, vp, u64, vp, vp, vp, ctypes.c_int], ctypes.c_int),
    "kmer_analysis_reset": ([vp], ctypes.c_int),
    "kmer_analysis_set_stream": ([vp, vp], ctypes.c_int),
    "kmer_analysis_status": ([vp], ctypes.c_int),
    "kmer_analysis_device_bytes": ([vp], u64),
    "kmer_analysis_set_profiling": ([vp, ctypes.c_int], ctypes.c_int),
    "kmer_analysis_timings": ([vp, ctypes.POINTER(kma_timings), ctypes.c_int], ctypes.c_int),
    "kmer_analysis_destroy": ([vp], None),
    "kmer_analysis_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "kmer_analysis_count_batch": ([ctypes.POINTER(vp), ctypes.POINTER(kma_reads), u32], ctypes.c_int),
    "kmer_analysis_finalize_batch": ([ctypes.POINTER(vp), u32, ctypes.POINTER(kma_result)], ctypes.c_int),
    "kmer_analysis_reserve_output": ([vp, u64], ctypes.c_int),
    "kmer_analysis_finalize_batch_async": ([ctypes.POINTER(vp), u32], ctypes.c_int),
    "kmer_analysis_fetch_result": ([vp, ctypes.POINTER(kma_result)], ctypes.c_int),
    "kmer_analysis_count_small_noalloc": ([ctypes.POINTER(kma_params), vp, vp, vp, u64, u64, vp, vp,
                                           vp, vp, u64, ctypes.POINTER(u64), vp], ctypes.c_int),
    "kmer_analysis_estimate": ([ctypes.POINTER(kma_params), vp, vp, vp, u64, ctypes.c_int, vp,
                                ctypes.POINTER(kma_estimate), vp], ctypes.c_int),
    "kmer_analysis_hll_estimate": ([vp, u32, ctypes.POINTER(dbl)], ctypes.c_int),
    "kmer_analysis_contigs": ([vp, ctypes.POINTER(kma_contigs)], ctypes.c_int),
    "kmer_analysis_copy_contigs": ([vp, vp, vp, ctypes.c_int], ctypes.c_int),
    "kmer_analysis_parse_fastq": ([vp, u64, ctypes.c_int, vp, vp, vp, u64, u64, ctypes.POINTER(u64),
                                   ctypes.POINTER(u64), vp], ctypes.c_int),
}

_LIB = None


def load(path: str = LIB_PATH):
    """Load the built library (build it with `__graft_entry__.build()` or
    `python paper_1705_11147_gb300/build.py`)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: the CUDA library has not been built "
                               "(no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = lib
    return _LIB


class KmaError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load().kmer_analysis_strerror(code).decode()
        super().__init__(f"{what}: {msg} ({code})")


def check(code: int, what: str) -> None:
    if code != KMA_OK:
        raise KmaError(code, what)
