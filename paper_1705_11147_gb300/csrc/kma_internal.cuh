// Internal layout shared by the library's CUDA translation units (not part of the C ABI).
//
// Device data of one handle ("sample"):
//   packed-read arena  positions q = 0 .. arena_positions-1. Each count() batch starts at a
//                      multiple of 64; read r of a batch occupies [ps_r, ps_r + len_r) and is
//                      followed by one separator position (invalid), so no window can span
//                      two reads and the bases before/after a read are never usable.
//     codes  u64[arena/32]  2 bits per position, first position in the two most significant
//                           bits (A0 C1 G2 T3; 0 for invalid positions)
//     rcodes u64[arena/32]  complemented codes (3 - code), first position in the two LEAST
//                           significant bits: bits [2i, 2i+2k) of consecutive words read as
//                           one number are the reverse complement of the window at i
//     inv    u64[arena/64]  1 = position is not A/C/G/T (separator, N, padding), MSB first
//     hq     u64[arena/64]  1 = A/C/G/T with Phred >= qual_threshold, MSB first
//     marks  u32[arena/32]  Bloom pass: 1 = this window was the first sighting of its k-mer
//   bloom    u64[bloom_words]  blocked Bloom filter: all bits of a k-mer in one word
//   table    Slot[slots]       open addressing, linear probing, 64-byte slots
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kma {

constexpr uint64_t kEmpty = ~0ull;          // both key words of an empty slot
constexpr uint32_t kMaxProbe = 1u << 14;    // probe limit before reporting a full table
constexpr int kMaxBatch = 64;

// Bounded device waits (bulk-copy staging): polls of an mbarrier before giving up, each poll
// suspending the thread for at most kWaitHintNs (about 1.3 s in all), and the short limit of
// the fault-injection test.
constexpr unsigned kWaitHintNs = 10000;
constexpr unsigned kWaitPolls = 1u << 17;
constexpr unsigned kWaitPollsInjected = 1u << 6;

// Status flags raised on the device.
constexpr uint32_t kFlagFull = 1u;
constexpr uint32_t kFlagOverflow = 2u;
constexpr uint32_t kFlagBadOffsets = 4u;
constexpr uint32_t kFlagTimeout = 8u;     // a bounded device wait gave up

// One hash-table slot. Every occurrence has exactly one left outcome (a usable base A/C/G/T
// or none) and one right outcome, so the slot keeps five counters per side and no separate
// count: count = none[0] + ext[0..3] = none[1] + ext[4..7]. An occurrence costs two
// counter updates. The key and the two "none" counters share the first 32-byte sector, the
// eight extension counters fill the second.
struct __align__(64) Slot {
  unsigned long long lo, hi;
  unsigned int none[2];  // occurrences without a usable left / right extension base
  unsigned int pad[2];
  unsigned int ext[8];   // left A C G T, right A C G T
};
static_assert(sizeof(Slot) == 64, "slot must be 64 bytes");

struct DevStatus {
  unsigned int flags;
  unsigned int pad;
  unsigned long long valid_windows;
  unsigned long long table_keys;
  unsigned long long n_out;
  unsigned long long n_uu;
  unsigned long long first_sightings;  // Bloom pass: windows marked as first sightings
  unsigned long long reserved[2];
};

// Per-sample view the pass kernels need. Passed by value inside kernel parameters.
struct PassDesc {
  const unsigned long long* codes;
  const unsigned long long* rcodes;
  const unsigned long long* inv;
  const unsigned long long* hq;
  unsigned int* marks;
  unsigned long long* bloom;
  Slot* table;
  DevStatus* status;
  unsigned long long bloom_words;
  unsigned long long slots;
  unsigned long long q0;          // first window start of this launch (multiple of 64)
  unsigned long long q1;          // one past the last window start
  unsigned long long tile_begin;  // first global tile index of this sample
  unsigned int k;
  unsigned int bloom_h;
  unsigned int canonical;
  unsigned int mode;              // kModeBloom / kModeCount / kModeRecount
  unsigned int n_parts;           // owner-computes partition: count only keys owned by `part`
  unsigned int part;
  unsigned int no_overflow;       // 1: no count can reach 2^32 (host bound), counts use red.add
  unsigned int pad;
};

struct PassBatch {
  unsigned int n;
  unsigned int prefetch;          // 1: L2-prefetch each window's first table slot in the Bloom pass
  unsigned long long total_tiles;
  PassDesc d[kMaxBatch];
};

constexpr unsigned int kModeBloom = 0;    // Bloom test-and-set; "seen" -> insert + count; else mark
constexpr unsigned int kModeCount = 1;    // no Bloom: insert + count every window
constexpr unsigned int kModeRecount = 2;  // marked windows: count if the key is in the table

// Pack kernel per-sample input.
struct PackDesc {
  const unsigned char* seq;
  const unsigned char* qual;
  const unsigned long long* offsets;  // n_reads + 1 entries
  long long delta;                    // seq/qual index of base b is offsets-relative b - delta
  unsigned long long n_reads;
  unsigned long long n_bases;         // offsets[n_reads] - offsets[0] as the host believes
  unsigned long long q0;              // arena start (multiple of 64)
  unsigned long long n_pos;           // n_bases + n_reads, rounded up to a multiple of 64
  unsigned long long chunk_begin;     // prefix of 256-word pack chunks over the batch
  unsigned long long* codes;
  unsigned long long* rcodes;
  unsigned long long* inv;
  unsigned long long* hq;
  DevStatus* status;
  unsigned int qual_min;              // qual byte >= qual_min <=> Phred >= threshold
  unsigned int pad;
};

constexpr unsigned long long kPackChunkWords = 256;  // 64-position words per pack CTA chunk

struct PackBatch {
  unsigned int n;
  unsigned int skip_copy;             // testing: wait for staging copies that were never issued
  unsigned int wait_limit;            // polls of the staging barrier before giving up
  unsigned int pad;
  unsigned long long total_chunks;
  PackDesc d[kMaxBatch];
};

struct ClassDesc {
  const Slot* table;
  DevStatus* status;
  unsigned long long slots;
  unsigned long long* out_keys;
  unsigned int* out_counts;
  unsigned int* out_ext;
  unsigned char* out_codes;
  unsigned long long out_cap;
  unsigned long long block_begin;
  unsigned int min_depth;
  unsigned int min_ext;
};

struct ClassBatch {
  unsigned int n;
  unsigned int write;   // 0: count survivors only; 1: compact into out_*
  unsigned long long total_blocks;
  ClassDesc d[kMaxBatch];
};

// ---- Partitioned mode ("owner-computes on chip", Section 5.1's k-mer -> owner map) -------
// The k-mer space is split by a hash into P partitions; partition p owns Bloom words
// [p*Wp, (p+1)*Wp) and table slots [p*Sp, (p+1)*Sp). Windows are first scattered into
// per-partition record buckets (streaming writes), then the buckets are processed in order,
// so the random Bloom/table traffic of one partition stays in L2.
constexpr unsigned kMaxPartitions = 4096;      // k <= 32 (one-word keys)
constexpr unsigned kMaxPartitionsWide = 2048;  // k > 32: the scatter's staged tile is larger

// Record info byte: bits 0-1 left base, bit 2 left usable, bits 3-4 right base,
// bit 5 right usable, bit 7 first sighting (set by the Bloom pass).
constexpr unsigned char kInfoFirst = 0x80;

struct PartGeom {
  unsigned long long* bloom;
  Slot* table;
  DevStatus* status;
  unsigned long long* keyfilter;  // Bloom mode: blocked Bloom filter of the keys in the table
  unsigned long long Wp;        // Bloom words per partition
  unsigned long long Sp;        // table slots per partition
  unsigned long long Wk;        // key-filter words per partition (0: no key filter)
  unsigned int P;
  unsigned int bloom_h;
  unsigned int k;
  unsigned int canonical;
  unsigned int n_parts;         // multi-GPU owner filter (as PassDesc)
  unsigned int part;
  unsigned int rpt;             // records per thread in flight in the record passes (2 or 4)
  unsigned int wait_limit;      // polls of the bounded wait for a staged record tile
  unsigned int no_overflow;     // 1: no count can reach 2^32 (host bound), counts use red.add
  unsigned int group;           // 1: group equal keys within a warp (heavy hitters)
};

struct PartWindows {
  const unsigned long long* codes;
  const unsigned long long* rcodes;
  const unsigned long long* inv;
  const unsigned long long* hq;
  unsigned long long q0, q1;    // window starts of one count() batch (multiples of 64)
};

// Record buckets of one count() batch: P buckets of `cap` records (bucket p starts at p*cap),
// then an overflow area of `ocap` records for partitions whose bucket filled up. cap and ocap
// are multiples of 16 and both arrays 16-byte aligned, so every tile of the record passes
// starts on a 16-byte boundary and may be staged with 1-D bulk copies rounded up to 16
// records without leaving its bucket (or the overflow area). fill[p]
// counts the records that were assigned to bucket p (those beyond cap went to the overflow
// area); fill[P] counts the overflow records.
// The record passes hand out their tiles (32 * rpt records, in bucket order) from a queue:
// `queue` counts the chunks of tiles taken so far and is zeroed before every launch.
struct PartRecords {
  void* keys;                   // unsigned long long[] (k <= 32) or ulonglong2[]
  unsigned char* info;
  unsigned long long cap;       // records per bucket
  unsigned long long ocap;      // overflow records
  unsigned long long* fill;     // [P + 1]
  unsigned* queue;              // record passes: chunks of tiles handed out so far
  // record passes: the buckets of partitions [p_begin, p_end), then the overflow area if
  // `overflow` (the whole batch: 0, P, 1); the scatter ignores these
  unsigned int p_begin, p_end;
  unsigned int overflow, pad;
};

cudaError_t launch_part_scatter(const PartGeom& g, const PartWindows& w, const PartRecords& r,
                                cudaStream_t stream, int num_sms);
cudaError_t launch_part_pass(const PartGeom& g, const PartRecords& r, unsigned mode,
                             cudaStream_t stream, int num_sms);
// Key filter of the recount: set by every key in the table (after the Bloom pass).
cudaError_t launch_keyfilter_build(const PartGeom& g, cudaStream_t stream, int num_sms);

// FASTQ parsing (kma_fastq.cu) and the device-wide exclusive scan it uses.
unsigned long long scan_scratch_items(unsigned long long n);
cudaError_t scan_exclusive(unsigned long long* data, unsigned long long n, unsigned long long* tmp,
                           cudaStream_t stream);
unsigned long long fastq_chunks(unsigned long long n_bytes);
cudaError_t launch_fastq_count(const unsigned char* text, unsigned long long n, unsigned long long* chunk_counts,
                               cudaStream_t stream);
cudaError_t launch_fastq_lines(const unsigned char* text, unsigned long long n,
                               const unsigned long long* chunk_offsets, unsigned long long* line_end,
                               cudaStream_t stream);
cudaError_t launch_fastq_records(const unsigned char* text, const unsigned long long* line_end,
                                 unsigned long long n_reads, unsigned long long* seq_len,
                                 unsigned long long* bad, cudaStream_t stream);
cudaError_t launch_fastq_copy(const unsigned char* text, const unsigned long long* line_end,
                              unsigned long long n_reads, const unsigned long long* offsets, unsigned char* seq,
                              unsigned char* qual, cudaStream_t stream);

// Contig generation over finalized records (kma_contig.cu). Returns 0, a negative KMA_E*
// code (-7 = CUDA error in *err), and on success pool allocations in *seq_out / *offsets_out.
int contig_pass(const unsigned long long* keys, const unsigned char* codes, unsigned long long n, unsigned k,
                unsigned canonical, cudaMemPool_t pool, cudaStream_t st, char** seq_out,
                unsigned long long** offsets_out, unsigned long long* n_contigs, unsigned long long* n_bases,
                unsigned long long* n_vertices, unsigned long long* n_cycles, unsigned* dev_flags, cudaError_t* err);

// Heavy-hitter summaries of the cardinality pass (kma_hll.cu): the windows at every
// 2^kMgSampleShift-th arena position, split by the top kMgBucketBits bits of the key hash into
// kMgBuckets sub-streams, one Misra-Gries summary of kMgCounters counters per sub-stream and CTA.
constexpr unsigned kMgSampleShift = 6;
constexpr unsigned kMgBucketBits = 5;
constexpr unsigned kMgBuckets = 1u << kMgBucketBits;
constexpr unsigned kMgCounters = 32;

// Where the CTAs leave their summaries: entry [cta][bucket][counter] (lo, hi, count; count 0
// = unused), items[cta][bucket] = sampled windows of that bucket the CTA saw. lo == nullptr:
// no summaries.
struct MgOut {
  unsigned long long* lo;
  unsigned long long* hi;
  unsigned* count;
  unsigned long long* items;
};

// Lets `fn` launch with up to the device's opt-in shared memory per block (less its static
// shared memory) and checks that `need` dynamic bytes fit. The limit is a property of the
// kernel, shared by every host thread: handles counting on several threads launch the same
// kernel with different sizes, and a limit set to one launch's own size could be lowered by
// another thread between that thread's set and its launch. So it is only ever set to the
// maximum (once per kernel and device).
cudaError_t allow_dynamic_smem(const void* fn, size_t need);

// HyperLogLog registers (2^p, 32-bit each) of the windows [w.q0, w.q1), and the heavy-hitter
// summaries of `grid` CTAs (kma_hll.cu); hll_grid gives the number of resident CTAs.
unsigned hll_grid(unsigned p, int num_sms);
cudaError_t launch_hll(const PartWindows& w, unsigned k, unsigned canonical, unsigned n_parts, unsigned part,
                       unsigned p, unsigned* regs, DevStatus* st, const MgOut& mg, unsigned grid,
                       cudaStream_t stream);

struct LaunchShape {
  int block_threads;
  int windows_per_thread;
  int grid;
};

// Launchers (kma_kernels.cu). All enqueue on `stream`.
cudaError_t launch_pack(const PackBatch& b, cudaStream_t stream, int num_sms);
cudaError_t launch_pass(const PassBatch& b, const LaunchShape& shape, bool warp_aggregate,
                        cudaStream_t stream);
cudaError_t launch_classify(const ClassBatch& b, cudaStream_t stream, int num_sms);
cudaError_t launch_table_init(Slot* table, unsigned long long slots, cudaStream_t stream);
cudaError_t launch_query(const Slot* table, unsigned long long slots, unsigned int parts,
                         unsigned int k,
                         unsigned int canonical, unsigned int min_depth, unsigned int min_ext,
                         const unsigned long long* keys, unsigned long long n,
                         unsigned int* counts, unsigned int* ext, unsigned char* codes,
                         DevStatus* status, cudaStream_t stream);
int pass_max_ctas_per_sm(int block_threads, int windows_per_thread, bool warp_aggregate);

}  // namespace kma
