/*
 * kmer_analysis.h — C ABI of the GB300 k-mer analysis library (libkmer_analysis.so).
 *
 * The library implements the k-mer analysis stage of HipMer / Meraculous (arXiv 1705.11147):
 *   - chopping reads into overlapping k-mers (Section 2, item 1; Figure "combined"(b)),
 *   - canonical form (lexicographic min of a k-mer and its reverse complement),
 *   - a Bloom-filter pass that keeps singleton (error) k-mers out of the hash table
 *     (Section 5.1),
 *   - exact counting in a device hash table with per-k-mer counts of high-quality left and
 *     right extension bases (Section 5.1: two arrays of four counters per k-mer),
 *   - the depth filter and classification of each side into A/C/G/T (unique), X (none,
 *     Section 4.1) or F (fork, Section 2), the unique-extension (UU) set being the k-mers
 *     with A/C/G/T on both sides (Section 5.2),
 *   - a read-only lookup phase (Section 4.2, use case GRO).
 *
 * Conventions common to every entry point
 *   - Return value: KMA_OK (0) or a negative KMA_E* code; kmer_analysis_strerror() names it.
 *   - Work is enqueued on the CUDA stream given at create (cudaStream_t passed as void*;
 *     NULL = legacy default stream). Calls return before the GPU finishes unless stated.
 *   - `on_device` = 1: every pointer argument of that call is a device pointer (or managed
 *     memory); 0: host pointers (pinned memory gives the fastest copies). The library never
 *     keeps a caller pointer past the call: input bytes are packed into library-owned device
 *     memory, so the caller may reuse its buffers once the call's stream work is done (host
 *     inputs: once the call returns).
 *   - A handle is not thread-safe; different handles may be used from different threads.
 *   - k-mer keys are 2-bit codes A=0 C=1 G=2 T=3, first base most significant, as a 128-bit
 *     number stored as two uint64 words {lo, hi}. k <= 32 keys have hi = 0.
 *   - Side codes: 0..3 = A C G T (unique high-quality extension), 4 = X, 5 = F.
 */
#ifndef KMER_ANALYSIS_H
#define KMER_ANALYSIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KMA_OK 0
#define KMA_EINVAL (-1)    /* bad argument: k, thresholds, sizes, pointers, inconsistent offsets */
#define KMA_ENOMEM (-2)    /* device allocation failed */
#define KMA_EFULL (-3)     /* hash table or packed-read arena capacity exceeded: no partial result;
                              recreate with a larger table_capacity / max_bases and count again */
#define KMA_ESTATE (-4)    /* call not allowed in the handle's state (count after finalize, ...) */
#define KMA_ETIMEOUT (-5)  /* a bounded device-side wait (completion of the staging copies of
                              the read-packing kernel) gave up: no partial result */
#define KMA_EOVERFLOW (-6) /* a 32-bit k-mer counter would have wrapped */
#define KMA_ECUDA (-7)     /* a CUDA runtime call failed (cudaGetLastError text via strerror) */
#define KMA_ETOOLARGE (-8) /* input above a fixed limit: the allocation-free entry point's
                              scratch (KMA_NOALLOC_MAX_BASES / KMA_NOALLOC_MAX_READS), or
                              2^31 contig-graph vertices */

#define KMA_CODE_X 4
#define KMA_CODE_F 5

typedef struct kma_handle kma_handle;

/* Counting parameters (Section 5.1: reads, k, error cutoff epsilon, threshold t_hq). */
typedef struct {
  uint32_t k;                 /* k-mer length, 1..63; odd when canonical = 1 (an even k admits
                                 k-mers equal to their own reverse complement) */
  uint32_t min_depth;         /* keep k-mers with count >= min_depth (paper: > epsilon) */
  uint32_t min_ext_count;     /* an extension base is high quality if seen >= this many times
                                 (paper: more than t_hq) */
  uint8_t qual_threshold;     /* an extension base is counted only if its Phred >= this */
  uint8_t qual_offset;        /* quality encoding offset: 33 for ASCII Phred+33, 0 for raw */
  uint8_t use_bloom;          /* 1: Bloom-filter singleton pass (requires min_depth >= 2);
                                 0: every k-mer goes straight into the table */
  uint8_t canonical;          /* 1: canonical k-mers (default); 0: forward strand only */
  uint64_t max_bases;         /* arena capacity: total bases over all count() calls */
  uint64_t max_reads;         /* total reads over all count() calls (0: max_bases / 32) */
  uint64_t expected_distinct; /* Bloom sizing: expected distinct k-mers incl. errors
                                 (0: the number of windows max_bases allows) */
  double bloom_fpr;           /* target false-positive rate of the Bloom filter (0: 0.01) */
  uint64_t table_capacity;    /* hash-table slots (0: expected_keys / load_factor) */
  uint64_t expected_keys;     /* keys the table must hold (0: expected_distinct, or the window
                                 bound). With the Bloom pass only k-mers seen twice (plus
                                 false positives) are inserted. */
  double load_factor;         /* target table load when table_capacity = 0 (0: 0.5) */
  uint64_t staging_bytes;     /* device staging buffer for host inputs (0: 256 MiB) */
  /* Launch shape (0 = library default; chosen by the autotuner per GPU and size class). */
  uint32_t block_threads;     /* threads per CTA of the counting kernels: 64..256, x32 */
  uint32_t windows_per_thread;/* window starts one thread handles per tile: 1, 2, 4 or 8
                                 (with partitions: records per thread, 4 or 8 -> 4, else 2) */
  uint32_t ctas_per_sm;       /* persistent grid = SMs x ctas_per_sm (0: occupancy bound) */
  uint32_t warp_aggregate;    /* 1: merge identical keys inside a warp before the atomics */
  /* Owner-computes partition (Section 5.1: a deterministic k-mer -> owner map makes every
   * owner's Bloom filter and table exact on its own). With n_parts > 1 the handle counts
   * only k-mers whose owner is `part`; the union of the n_parts results is the whole result.
   * The owner of a k-mer is a hash of its canonical key (library-defined, fixed). */
  uint32_t n_parts;           /* 0 or 1: no partition */
  uint32_t part;              /* 0 .. n_parts-1 */
  uint32_t slot_prefetch;     /* Bloom pass: prefetch each window's table slot into L2 while
                                 its Bloom word is tested. 0: default (off), 1: on, 2: off */
  uint32_t fault_inject;      /* testing only. 0: off. 1: the read-packing kernel waits for
                                 staging copies it never issued, with a short poll limit, so
                                 its bounded wait gives up and the handle reports KMA_ETIMEOUT */
  uint32_t partitions;        /* on-chip owner-computes partitions (Section 5.1's owner map on
                                 one GPU): the Bloom filter and table are split by a hash into
                                 P parts, windows are first written to per-part record buckets,
                                 and the buckets are counted part by part so one part's filter
                                 and table stay in L2. 0: automatic (P >= 2 when filter + table
                                 exceed 32 MB, at most 64 MB per part); 1: one table, windows
                                 counted in place; P >= 2: that many parts (<= 4096 for
                                 k <= 32, <= 2048 for k > 32; more: KMA_EINVAL). Results
                                 do not depend on it. */
  uint32_t heavy_hitters;     /* 1: k-mers with very many occurrences (satellites, low-complexity
                                 sequence) are expected. The partitioned counting passes then
                                 look for equal keys among each warp's records and treat them
                                 as one (one Bloom test-and-set and one table probe per group,
                                 counter updates summed in shared memory first: Section 5.1's
                                 local accumulation of heavy hitters, at warp level). 0: off.
                                 Results do not depend on it. */
} kma_params;

/* Sizes derived from a kma_params (pure host arithmetic, no GPU needed). */
typedef struct {
  uint64_t bloom_words;    /* 64-bit words of the blocked Bloom filter (0 without Bloom) */
  uint32_t bloom_hashes;   /* bits set per k-mer, all inside one 64-bit word */
  uint32_t partitions;     /* on-chip partitions (1: one table) */
  double bloom_fpr_est;    /* predicted false-positive rate at expected_distinct k-mers */
  uint64_t table_slots;    /* hash-table slots, 64 bytes each */
  uint64_t arena_positions;/* packed positions: bases + one separator per read + padding */
  uint64_t device_bytes;   /* device memory a handle holds (all buffers; with partitions,
                              including per-window records for max_bases windows) */
} kma_plan;

/* Result of finalize. Pointers are device memory owned by the handle, valid until the
 * next finalize, reset or destroy. Record order is unspecified. */
typedef struct {
  uint64_t n;              /* k-mers with count >= min_depth */
  uint64_t n_uu;           /* of those, unique high-quality extension on both sides */
  uint64_t valid_windows;  /* windows (k-mer occurrences) counted */
  uint64_t table_keys;     /* distinct keys in the table before the depth filter */
  const uint64_t* keys;    /* [n][2] {lo, hi} */
  const uint32_t* counts;  /* [n] */
  const uint32_t* ext;     /* [n][8]: left A C G T, right A C G T */
  const uint8_t* codes;    /* [n][2]: left code, right code */
} kma_result;

/* Sizes of a handle for `params` (Section 5.1 Bloom sizing: false-positive rate of a filter
 * whose bits for one key share a 64-bit word). Host only. KMA_EINVAL on bad params. */
int kmer_analysis_plan(const kma_params* params, kma_plan* out);

/* Allocate a handle: packed-read arena, Bloom filter, hash table, status words, staging.
 * `cuda_stream` is a cudaStream_t (NULL = default stream). The handle starts empty and belongs
 * to the CUDA device that is current here; every later call on it must be made with that
 * device current (the library does not switch devices). A handle is not thread-safe: one
 * host thread at a time. Errors: KMA_EINVAL (params), KMA_ENOMEM, KMA_ECUDA. On error *out
 * is NULL. */
int kmer_analysis_create(const kma_params* params, void* cuda_stream, kma_handle** out);

/* Add reads (Section 5.1 counting phase; may be called repeatedly with further batches).
 * Read r is seq[offsets[r] .. offsets[r+1]) with qualities at the same positions of `qual`;
 * offsets has n_reads + 1 non-decreasing entries. Bases other than A/C/G/T (either case)
 * make every window covering them invalid. Reads shorter than k add no windows.
 * Packs the reads 2 bits per base into the handle's arena and runs the first pass
 * (Bloom test-and-set, table insert of k-mers seen twice; without Bloom, the counting).
 * With on_device = 1 the call reads offsets[0] and offsets[n_reads] back, which waits for
 * the stream up to that point. Errors: KMA_EINVAL (decreasing offsets), KMA_EFULL (arena:
 * max_bases / max_reads exceeded; table overflow is reported by finalize), KMA_ESTATE
 * (after finalize), KMA_ECUDA. */
int kmer_analysis_count(kma_handle* h, const char* seq, const char* qual,
                        const uint64_t* offsets, uint64_t n_reads, int on_device);

/* Finish counting: second pass over the retained reads (first sightings of k-mers the
 * Bloom pass left out of the table), depth filter, classification and compaction into
 * device arrays (see kma_result). Synchronises the stream. Errors: KMA_EFULL (table
 * overflow: no partial result), KMA_EOVERFLOW, KMA_EINVAL (inconsistent offsets seen on
 * the device), KMA_ESTATE (already finalized), KMA_ENOMEM, KMA_ECUDA. */
int kmer_analysis_finalize(kma_handle* h, kma_result* out);

/* Copy the finalized records into caller buffers of `capacity` records (host or device
 * pointers, per on_device; any pointer may be NULL to skip that array). Synchronises.
 * Errors: KMA_ESTATE (not finalized), KMA_EINVAL (capacity < n). */
int kmer_analysis_copy_result(kma_handle* h, uint64_t* keys, uint32_t* counts, uint32_t* ext,
                              uint8_t* codes, uint64_t capacity, int on_device);

/* kmer_analysis_finalize followed by kmer_analysis_copy_result into HOST buffers, with the
 * copies overlapped: the recount (Section 5.1's exact second pass) and the classification
 * run in groups of on-chip partitions (of table slots with one table), and each group's
 * records are copied to the host while the next group is recounted. The records, their
 * order aside, are those of finalize. Buffers hold `capacity` records each (keys[c][2],
 * counts[c], ext[c][8], codes[c][2] as in kma_result); any pointer may be NULL to skip that
 * array; pinned host memory gives full copy bandwidth. The device result stays valid
 * (kma_result in *out, copy_result and query work as after finalize). Synchronises.
 * Errors: as kmer_analysis_finalize; KMA_EFULL also when out->n > capacity: the handle IS
 * finalized, the first `capacity` records were copied and copy_result can fetch them all.
 * On any other error the buffers' contents are unspecified. */
int kmer_analysis_finalize_to_host(kma_handle* h, uint64_t* keys, uint32_t* counts, uint32_t* ext,
                                   uint8_t* codes, uint64_t capacity, kma_result* out);

/* Look up n k-mers given as keys[n][2] in either orientation (read-only phase, Section
 * 4.2 GRO). Answers are in the query's orientation: counts[i], ext[i][8] (left A C G T,
 * right A C G T) and codes[i][2]; k-mers below min_depth or absent give count 0, zero
 * extensions and codes X/X. Keys with bits set at or above bit 2k answer as absent.
 * Errors: KMA_ESTATE (not finalized), KMA_EINVAL, KMA_ECUDA. */
int kmer_analysis_query(kma_handle* h, const uint64_t* keys, uint64_t n, uint32_t* counts,
                        uint32_t* ext, uint8_t* codes, int on_device);

/* Empty the handle for a new read set with the same parameters, keeping its memory
 * (Bloom filter and table are cleared on the stream; the packed-read arena is rewritten by
 * the next count calls). */
int kmer_analysis_reset(kma_handle* h);

/* Change the stream later calls enqueue on (the caller orders the two streams). */
int kmer_analysis_set_stream(kma_handle* h, void* cuda_stream);

/* Status flags the device raised so far (table full, overflow, bad offsets) as a KMA_E*
 * code, KMA_OK if none. Synchronises the stream. */
int kmer_analysis_status(kma_handle* h);

/* Device bytes the handle holds (arena, Bloom, table, staging, result buffers). */
uint64_t kmer_analysis_device_bytes(const kma_handle* h);

/* Per-kernel timing (tracing). With profiling enabled the library records a CUDA event pair
 * around each of its kernel launches on the launching stream. kmer_analysis_timings
 * synchronises, sums the elapsed times since the last reset and optionally resets them.
 * Launch counts are kept whether or not profiling is enabled. */
typedef struct {
  double ms[8];           /* per kernel kind: see KMA_KERNEL_* */
  uint64_t launches[8];   /* launches per kernel kind */
  uint64_t total_launches;
  uint64_t first_sightings; /* Bloom pass: windows that were the first sighting of their k-mer */
} kma_timings;

#define KMA_KERNEL_PACK 0
#define KMA_KERNEL_PASS 1      /* first pass: Bloom test-and-set + table (or counting) */
#define KMA_KERNEL_RECOUNT 2   /* second pass over first sightings */
#define KMA_KERNEL_CLASSIFY 3
#define KMA_KERNEL_QUERY 4
#define KMA_KERNEL_INIT 5      /* table initialisation on create / reset */
#define KMA_KERNEL_SCATTER 7   /* partitioned mode: windows -> per-partition record buckets */

int kmer_analysis_set_profiling(kma_handle* h, int enable);
int kmer_analysis_timings(kma_handle* h, kma_timings* out, int reset);

/* Free everything (waits for the handle's stream). NULL is a no-op. */
void kmer_analysis_destroy(kma_handle* h);

const char* kmer_analysis_strerror(int code);

/* ---- Batched counting: many independent read sets in one persistent launch ----------
 * Each handle keeps its own arena, Bloom filter and table (per-sample partitions); the
 * counting kernels take all of them at once, so small samples share the GPU instead of
 * each paying its own launches and synchronisations. All handles must have been created
 * on the same device; work is enqueued on hs[0]'s stream (the caller orders the other
 * handles' streams before it). Up to KMA_MAX_BATCH handles per call.
 * kmer_analysis_count_batch takes device pointers only and does not synchronise, so it can
 * be captured into a CUDA graph: n_bases must equal offsets[n_reads] - offsets[0]
 * (checked on the device; a mismatch makes finalize return KMA_EINVAL). */
#define KMA_MAX_BATCH 64

typedef struct {
  const char* seq;
  const char* qual;
  const uint64_t* offsets; /* n_reads + 1 entries */
  uint64_t n_reads;
  uint64_t n_bases;
} kma_reads;

int kmer_analysis_count_batch(kma_handle* const* hs, const kma_reads* reads, uint32_t n);

/* Finalize several handles with one launch per phase; out[i] receives handle i's result.
 * Synchronises hs[0]'s stream. Errors as kmer_analysis_finalize; the first failing
 * handle's code is returned and the others are still finalized. */
int kmer_analysis_finalize_batch(kma_handle* const* hs, uint32_t n, kma_result* out);

/* ---- Capture-safe finalize (for CUDA graphs of whole batched steps) -------------------
 * kmer_analysis_reserve_output allocates result buffers for up to n_records records now, so
 * that kmer_analysis_finalize_batch_async needs no allocation: it enqueues the recount and
 * classification of n handles on hs[0]'s stream without any host synchronisation and marks
 * them finalized (it can be captured into a CUDA graph together with kmer_analysis_reset and
 * kmer_analysis_count_batch). kmer_analysis_fetch_result then synchronises the handle's
 * stream and reads the result of the last completed finalize (*out->n may exceed the
 * reserved capacity: KMA_EFULL, reserve more and run again). */
int kmer_analysis_reserve_output(kma_handle* h, uint64_t n_records);
int kmer_analysis_finalize_batch_async(kma_handle* const* hs, uint32_t n);
int kmer_analysis_fetch_result(kma_handle* h, kma_result* out);

/* ---- Allocation-free counting for small read sets --------------------------------------
 * The paper has no counterpart: this entry point serves callers that must not allocate
 * device memory when they count, for example code that reserves a fixed memory budget at
 * start-up and forbids later allocations, or a plugin inside a host framework that owns
 * every device allocation. It runs the same kernels as create/count/finalize (exact counting
 * without the Bloom filter, which gives the same records) in one call and allocates nothing:
 * its working memory (packed reads, hash table, status words) is a fixed file-scope device
 * array of about 34 MB that every GPU loading the library holds until the process exits.
 *
 * Inputs (seq, qual, offsets: read r is seq[offsets[r] .. offsets[r+1]), n_bases must equal
 * offsets[n_reads] - offsets[0]) and outputs (keys[capacity][2], counts[capacity],
 * ext[capacity][8], codes[capacity][2], same layout as kma_result) are device pointers
 * owned by the caller; *n_out (host) receives the number of records, also when it exceeds
 * `capacity` (then KMA_EFULL is returned and the arrays hold the first `capacity` records in
 * unspecified order). params->k, canonical, min_depth, min_ext_count, qual_threshold and
 * qual_offset are used; the sizing and launch-shape fields are ignored.
 * Limits: n_bases <= KMA_NOALLOC_MAX_BASES and n_reads <= KMA_NOALLOC_MAX_READS, otherwise
 * KMA_ETOOLARGE and nothing runs. The call synchronises `cuda_stream` before it returns.
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress), so the address stays right after a device reset. Device offsets
 * must not decrease; decreasing ones are not fully checked on the device and can give wrong
 * records instead of KMA_EINVAL. All calls share the array and it keeps
 * the previous call's contents (each call clears what it needs): calls whose GPU work can
 * overlap, on different streams or from unsynchronised threads, race on it. */
#define KMA_NOALLOC_MAX_BASES 262144
#define KMA_NOALLOC_MAX_READS 262144

int kmer_analysis_count_small_noalloc(const kma_params* params, const char* seq, const char* qual,
                                      const uint64_t* offsets, uint64_t n_reads, uint64_t n_bases,
                                      uint64_t* keys, uint32_t* counts, uint32_t* ext,
                                      uint8_t* codes, uint64_t capacity, uint64_t* n_out,
                                      void* cuda_stream);

/* ---- Contig generation (Section 5.2) on a finalized handle --------------------------------
 * Vertices: the finalized k-mers without a fork on either side (codes A/C/G/T or X; Section 2
 * removes the fork vertices). The neighbour of k-mer x on its right is x[1..k) + R, on its
 * left L + x[0..k-1) (R, L: its side codes; X: no neighbour), looked up by key; it is an edge
 * only if it is another vertex whose code on the facing side points back to x. Contigs are
 * the resulting paths, k-mers merged (length = k-mers + k - 1); a cycle is cut at its
 * smallest key, on that k-mer's left side. Contigs are in unspecified order, each in one of
 * its two orientations (with forward keys: read forward). */
typedef struct {
  uint64_t n_contigs;
  uint64_t n_bases;        /* total length */
  uint64_t n_vertices;     /* k-mers in the graph (no fork on either side) */
  uint64_t n_cycles;       /* circular components that were cut */
  const char* seq;         /* device: contig bases (A, C, G, T), concatenated */
  const uint64_t* offsets; /* device: [n_contigs + 1]; contig i is seq[offsets[i] .. offsets[i+1]) */
} kma_contigs;

/* Build the contigs of the finalized result; the arrays are owned by the handle (valid until
 * the next kmer_analysis_contigs, reset or destroy). Synchronises. Errors: KMA_ESTATE (not
 * finalized), KMA_ENOMEM, KMA_ETOOLARGE (2^31 or more vertices), KMA_ECUDA. */
int kmer_analysis_contigs(kma_handle* h, kma_contigs* out);

/* Copy the contigs to caller buffers (n_bases bytes, n_contigs + 1 offsets; host or device per
 * on_device; NULL skips an array). Synchronises. KMA_ESTATE before kmer_analysis_contigs. */
int kmer_analysis_copy_contigs(kma_handle* h, char* seq, uint64_t* offsets, int on_device);

/* ---- Cardinality estimate (Section 5.1: a HyperLogLog pass sizes the Bloom filter) --------
 * Estimates the number of distinct canonical k-mers of a read set with a HyperLogLog sketch
 * of m = 2^precision registers (64-bit hashes, as in Section 5.1): every valid window's key
 * (with n_parts > 1: every key owned by `part`) is hashed; the top `precision` bits of the
 * hash pick a register, which keeps the largest rank seen, rank = 1 + leading zeros of the
 * remaining bits. Relative standard error 1.04 / sqrt(m) (0.8 % at the default m = 2^14).
 * The sketch depends only on the set of distinct keys; sketches merge by elementwise
 * maximum (several batches of reads, or the owner partitions of several GPUs). */
#define KMA_HLL_MIN_PRECISION 4
#define KMA_HLL_MAX_PRECISION 14

/* Heavy hitters (Section 5.1: frequent k-mers are found in the same pass, so that they can be
 * accumulated locally). The windows starting at every KMA_MG_SAMPLE-th position of the packed
 * reads (read r's base j at offsets[r] - offsets[0] + r + j; one separator per read) form a
 * sampled stream, split by the top 5 bits of the key hash into KMA_MG_BUCKETS sub-streams.
 * Each is summarised by the Misra-Gries algorithm with KMA_MG_COUNTERS counters (per CTA, then
 * merged: counts of a key summed, the (m+1)-th largest subtracted): for a sub-stream of n
 * sampled windows, every key with sampled frequency f > n / (m + 1) is in the summary, with a
 * count c, f - n / (m + 1) <= c <= f; keys not in it have f <= n / (m + 1). */
#define KMA_MG_SAMPLE 64
#define KMA_MG_BUCKETS 32
#define KMA_MG_COUNTERS 32

typedef struct {
  uint32_t precision;       /* in: p (KMA_HLL_MIN_PRECISION .. KMA_HLL_MAX_PRECISION; 0 = 14) */
  uint32_t heavy_hitters;   /* out: 1 if some k-mer's summary count (a lower bound of its sampled
                               frequency) reaches heavy_threshold: pass it as kma_params.heavy_hitters */
  double distinct;          /* out: estimated distinct canonical k-mers (of the merged sketch) */
  double rel_std_error;     /* out: 1.04 / sqrt(2^p) */
  uint64_t valid_windows;   /* out: valid windows this call saw (exact; owned keys only) */
  uint64_t sampled_windows; /* out: windows of the sampled stream (owned keys only) */
  uint64_t heavy_threshold; /* out: max(1, sampled_windows / 2048) */
  uint64_t n_summary;       /* out: keys in the merged summaries (<= buckets * counters) */
  uint64_t summary_capacity;     /* in: rows of the arrays below (0: not wanted) */
  uint64_t* summary_keys;        /* in: host [capacity][2] or NULL; out: keys, by count descending */
  uint64_t* summary_counts;      /* in: host [capacity] or NULL; out: their summary counts */
  uint32_t* summary_bucket;      /* in: host [capacity] or NULL; out: their sub-stream */
  uint64_t* bucket_windows;      /* in: host [KMA_MG_BUCKETS] or NULL; out: n of each sub-stream */
} kma_estimate;

/* One estimation pass over reads given like kmer_analysis_count's (host pointers, or device
 * pointers with on_device = 1). params->k, canonical, n_parts and part are used, plus
 * max_bases / max_reads as lower bounds of the temporary read arena (the call allocates what
 * the reads need, packs them with the counting path's kernel, runs the sketch kernel and
 * frees everything before it returns; it synchronises `cuda_stream`). `registers`, if not
 * NULL, is a host array of 2^p bytes: on entry a sketch to merge with (all zero = empty), on
 * return the merged sketch; the estimate is that of the merged sketch. The heavy-hitter
 * summaries cover this call's reads only (they are not merged across calls).
 * Errors: KMA_EINVAL (params, precision, offsets), KMA_ENOMEM, KMA_ECUDA. */
int kmer_analysis_estimate(const kma_params* params, const char* seq, const char* qual,
                           const uint64_t* offsets, uint64_t n_reads, int on_device,
                           void* cuda_stream, kma_estimate* est, uint8_t* registers);

/* The estimate of a sketch (host only, no GPU): E = alpha_m m^2 / sum_j 2^-M[j], replaced by
 * linear counting m ln(m / V) when E <= 5m/2 and V registers are zero (Flajolet et al. 2007;
 * with 64-bit hashes no large-range correction). KMA_EINVAL on a bad precision. */
int kmer_analysis_hll_estimate(const uint8_t* registers, uint32_t precision, double* distinct);

/* ---- FASTQ parsing on the device (the input side of the stage, Section 2 item 1) ---------
 * Splits FASTQ text into the read layout kmer_analysis_count takes. A record is four lines:
 * "@name", the bases, "+" (optionally followed by the name) and one quality character per
 * base; records are found by line number, so quality lines may start with '@' or '+'. Lines
 * may end in "\n" or "\r\n"; the last line need not end in a newline; empty lines after the
 * last record are ignored. Multi-line (wrapped) records are not supported.
 * `text` is host memory, or device memory with on_device = 1. The outputs are device arrays
 * owned by the caller: seq[cap_bases], qual[cap_bases] (bases and qualities of read r at
 * [offsets[r], offsets[r+1])) and offsets[cap_reads + 1] (offsets[0] = 0). *n_reads and
 * *n_bases (host) receive the sizes, also when they exceed the capacities (then KMA_EFULL
 * is returned and the arrays are incomplete). Temporaries come from the library's pool.
 * Synchronises `cuda_stream`. Errors: KMA_EINVAL (a record without '@' or '+' line, or whose
 * base and quality lines differ in length; a line count that is not a multiple of four),
 * KMA_EFULL, KMA_ENOMEM, KMA_ECUDA. */
int kmer_analysis_parse_fastq(const char* text, uint64_t n_bytes, int on_device, char* seq, char* qual,
                              uint64_t* offsets, uint64_t cap_bases, uint64_t cap_reads, uint64_t* n_reads,
                              uint64_t* n_bases, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KMER_ANALYSIS_H */
