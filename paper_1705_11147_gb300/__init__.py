"""GB300-native k-mer analysis (HipMer / Meraculous, arXiv 1705.11147, Sections 2 and 5.1).

The work runs in libkmer_analysis.so (CUDA, sm_103a), reached through the C ABI declared in
include/kmer_analysis.h. This package is the thin Python binding over it.
"""
from .capi import (KMA_CODE_F, KMA_CODE_X, KMA_EFULL, KMA_EINVAL, KMA_ESTATE, KMA_ETIMEOUT, KMA_OK,
                   KmaError, load)
from .kmer_analysis import (BatchGraph, Estimate, KmerAnalysis, Result, count_batch, count_kmers,
                            estimate_distinct, fetch_result, finalize_batch, finalize_batch_async,
                            hll_estimate, host_result_buffers, make_params, parse_fastq, plan,
                            reserve_output)

__all__ = ["BatchGraph", "Estimate", "KmerAnalysis", "Result", "count_batch", "count_kmers",
           "estimate_distinct", "hll_estimate", "host_result_buffers", "parse_fastq", "fetch_result",
           "finalize_batch", "finalize_batch_async", "reserve_output",
           "make_params", "plan", "load", "KmaError", "KMA_OK", "KMA_EINVAL", "KMA_EFULL",
           "KMA_ESTATE", "KMA_ETIMEOUT", "KMA_CODE_X", "KMA_CODE_F"]
