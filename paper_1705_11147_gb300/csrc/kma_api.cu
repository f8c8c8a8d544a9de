// Host side of the C ABI declared in include/kmer_analysis.h: parameter checks, sizing
// (Bloom filter, table, arena), device memory, staging of host inputs, launch sequencing
// and status reporting. Every computation on reads and k-mers runs in kma_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/kmer_analysis.h"
#include "kma_internal.cuh"

using namespace kma;
typedef unsigned long long u64;

namespace {

thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e, const char* what) {
  g_last_cuda_error = std::string(what) + ": " + cudaGetErrorString(e);
  return KMA_ECUDA;
}

#define KMA_CUDA(call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
  } while (0)

constexpr u64 kArenaSlack = 64ull * 4096;  // padding positions for per-batch 64-alignment
constexpr u64 kBatchSlack = 256;            // invalid positions kept behind the last batch
constexpr u64 kDefaultStaging = 256ull << 20;

// ------------------------------------------------------------------ Bloom sizing
//
// Section 5.1 sizes the filter from the number of distinct k-mers m, the filter size n and
// h hash functions with Pr(e) = (1 - e^{-h m / n})^h, optimal h = ln 2 * n / m (the printed
// version swaps m and n in the exponent and in h; this is the standard form). Here all h
// bits of a k-mer lie in one 64-bit word (so one atomicOr is a linearisable test-and-set),
// which raises the rate: a word receives j other k-mers with j ~ Poisson(m / W) for W words,
// and given j the probability that one bit is set is 1 - (63/64)^{h j}. The estimate is the
// Poisson mixture of (1 - (63/64)^{h j})^h.
double blocked_fpr(double m, double words, unsigned h) {
  if (words <= 0) return 1.0;
  const double lam = m / words;
  const double q = std::log(63.0 / 64.0);
  // sum the Poisson(lam) pmf over lam +- 12 sd (+40); the mass outside counts as certain
  // false positives, which only makes the estimate conservative
  const double sd = std::sqrt(lam);
  const long j0 = (long)std::max(0.0, std::floor(lam - 12.0 * sd - 40.0));
  const long j1 = (long)std::ceil(lam + 12.0 * sd + 40.0);
  double fpr = 0.0, mass = 0.0;
  for (long j = j0; j <= j1; ++j) {
    const double pmf = lam > 0 ? std::exp(-lam + (double)j * std::log(lam) - std::lgamma((double)j + 1.0))
                               : (j == 0 ? 1.0 : 0.0);
    mass += pmf;
    fpr += pmf * std::pow(1.0 - std::exp(q * h * (double)j), (double)h);
  }
  return std::min(1.0, fpr + std::max(0.0, 1.0 - mass));
}

void size_bloom(double m, double target, uint64_t& words, uint32_t& hbits, double& est) {
  words = 0;
  hbits = 0;
  est = 1.0;
  if (m < 1) m = 1;
  for (unsigned h = 1; h <= 10; ++h) {
    // smallest W with blocked_fpr <= target (monotone in W)
    double lo = 1, hi = std::max(1.0, m / 64.0);  // start at one bit per key
    while (blocked_fpr(m, hi, h) > target && hi < 1e15) hi *= 2;
    if (blocked_fpr(m, hi, h) > target) continue;
    lo = std::max(1.0, hi / 2);
    while (hi - lo > std::max(1.0, hi * 1e-4)) {
      const double mid = std::floor((lo + hi) / 2);
      if (blocked_fpr(m, mid, h) <= target) hi = mid; else lo = mid;
    }
    const uint64_t w = (uint64_t)std::ceil(hi);
    if (words == 0 || w < words) {
      words = w;
      hbits = h;
      est = blocked_fpr(m, (double)w, h);
    }
  }
}

struct Derived {
  kma_plan plan;
  u64 codes_words, bit_words, mark_words;
  u64 staging;
  unsigned P;      // on-chip partitions (1: one table)
  u64 Wp, Sp;      // Bloom words / table slots per partition
  u64 Wt;          // key filter words per partition (partitioned Bloom mode, else 0)
  u64 rec_bytes;   // bytes per record in partitioned mode
};

// Key filter of the partitioned recount: a second blocked Bloom filter that records the keys
// inserted into the table, sized at this many bits per key the table is built for.
constexpr double kKeyFilterBitsPerKey = 12.0;

// Partitioned above 32 MB of filter + table: from 45 MB (7.5 Mbases, k = 31) up, two L2-sized
// partitions beat one table (0.62 -> 0.57 ms; 1.87 -> 1.41 ms at 30 Mbases).
constexpr u64 kAutoPartitionAbove = 32ull << 20;   // filter + table bytes
constexpr u64 kPartitionTarget = 64ull << 20;      // filter + table bytes per partition

int check_params(const kma_params* p) {
  if (!p) return KMA_EINVAL;
  if (p->k < 1 || p->k > 63) return KMA_EINVAL;
  if (p->canonical && (p->k % 2 == 0)) return KMA_EINVAL;
  if (p->min_depth < 1) return KMA_EINVAL;
  if (p->use_bloom && p->min_depth < 2) return KMA_EINVAL;
  if (p->bloom_fpr < 0 || p->bloom_fpr >= 1) return KMA_EINVAL;
  if (p->load_factor < 0 || p->load_factor > 0.95) return KMA_EINVAL;
  if (p->max_bases == 0) return KMA_EINVAL;
  if (p->block_threads && (p->block_threads < 64 || p->block_threads > 256 || p->block_threads % 32))
    return KMA_EINVAL;
  if (p->windows_per_thread && p->windows_per_thread != 1 && p->windows_per_thread != 2 &&
      p->windows_per_thread != 4 && p->windows_per_thread != 8)
    return KMA_EINVAL;
  if (p->slot_prefetch > 2) return KMA_EINVAL;
  if (p->fault_inject > 1) return KMA_EINVAL;
  if (p->heavy_hitters > 1) return KMA_EINVAL;
  if (p->partitions > (p->k > 32 ? kMaxPartitionsWide : kMaxPartitions)) return KMA_EINVAL;
  if (p->n_parts > 1 && p->part >= p->n_parts) return KMA_EINVAL;
  return KMA_OK;
}

int derive(const kma_params* p, Derived& d) {
  int rc = check_params(p);
  if (rc) return rc;
  std::memset(&d, 0, sizeof(d));
  const u64 windows_bound = p->max_bases;
  const double distinct = p->expected_distinct ? (double)p->expected_distinct : (double)windows_bound;
  if (p->use_bloom) {
    const double target = p->bloom_fpr > 0 ? p->bloom_fpr : 0.01;
    size_bloom(distinct, target, d.plan.bloom_words, d.plan.bloom_hashes, d.plan.bloom_fpr_est);
    if (d.plan.bloom_words == 0) return KMA_EINVAL;
  }
  if (p->table_capacity) {
    d.plan.table_slots = p->table_capacity;
  } else {
    const double keys = p->expected_keys ? (double)p->expected_keys : distinct;
    const double lf = p->load_factor > 0 ? p->load_factor : 0.5;
    d.plan.table_slots = (u64)std::ceil(keys / lf) + 64;
  }
  // on-chip partitions: each part's Bloom sub-filter and sub-table sized for L2
  {
    const u64 W = d.plan.bloom_words, S = d.plan.table_slots;
    const u64 bytes = W * 8 + S * sizeof(Slot);
    u64 P = p->partitions;
    if (P == 0) P = bytes > kAutoPartitionAbove ? std::max<u64>(2, (bytes + kPartitionTarget - 1) / kPartitionTarget) : 1;
    const u64 max_parts = p->k > 32 ? kMaxPartitionsWide : kMaxPartitions;
    if (P > max_parts) P = max_parts;
    if (P < 1) P = 1;
    d.P = (unsigned)P;
    d.Wp = (W + P - 1) / P;
    d.Sp = (S + P - 1) / P;
    if (P > 1) {
      if (d.Sp < 64) d.Sp = 64;
      d.plan.bloom_words = W ? d.Wp * P : 0;
      d.plan.table_slots = d.Sp * P;
    } else {
      d.Wp = W;
      d.Sp = S;
    }
    d.plan.partitions = d.P;
    d.rec_bytes = (p->k > 32 ? 16 : 8) + 1;
    if (P > 1 && p->use_bloom) {
      const double lf = p->load_factor > 0 ? p->load_factor : 0.5;
      const double keys = (double)d.plan.table_slots * lf;
      d.Wt = std::max<u64>((u64)std::ceil(keys * kKeyFilterBitsPerKey / 64.0 / (double)P), 64);
    }
  }
  // bit slices of the key hash address at most 2^32 Bloom words and 2^32 slots per partition
  if (d.plan.bloom_words >= (1ull << 32) || d.Sp >= (1ull << 32)) return KMA_EINVAL;
  const u64 reads = p->max_reads ? p->max_reads : p->max_bases / 32 + 1;
  const u64 pos = ((p->max_bases + reads + kArenaSlack + 63) / 64) * 64;
  d.plan.arena_positions = pos;
  d.codes_words = pos / 32 + 4;
  d.bit_words = pos / 64 + 4;
  d.mark_words = pos / 32 + 4;
  d.staging = p->staging_bytes ? p->staging_bytes : kDefaultStaging;
  d.plan.device_bytes = 2 * d.codes_words * 8 + 2 * d.bit_words * 8 + d.mark_words * 4 +
                        d.plan.bloom_words * 8 + d.plan.table_slots * sizeof(Slot) +
                        sizeof(DevStatus) + 2 * (2 * d.staging + (d.staging / 16 + 2) * 8);
  if (d.P > 1)  // record buckets and the key filter
    d.plan.device_bytes += (p->max_bases + p->max_bases / 16) * d.rec_bytes + d.Wt * d.P * 8;
  return KMA_OK;
}

// Library-private stream-ordered pool per device: handles of a serving loop come and go,
// and freed blocks are reused instead of going back to the driver.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64];
bool g_pool_init[64];

int get_pool(int dev, cudaMemPool_t* out) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (dev < 0 || dev >= 64) return KMA_EINVAL;
  if (!g_pool_init[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    KMA_CUDA(cudaMemPoolCreate(&g_pools[dev], &props));
    u64 thr = ~0ull;
    KMA_CUDA(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thr));
    g_pool_init[dev] = true;
  }
  *out = g_pools[dev];
  return KMA_OK;
}

// Heavy hitters: the CTAs' Misra-Gries summaries of one sub-stream merged into one (mergeable
// summaries, Agarwal et al. 2012): the counts of each key are summed; if more than m keys
// remain, the (m+1)-th largest count is subtracted from every count and the keys left at zero
// or below are dropped. The merged summary keeps the bound of its parts: for a sub-stream of n
// items, every key with frequency f > n / (m + 1) is present with f - n / (m + 1) <= c <= f.
struct MgEntry {
  u64 lo, hi, count;
  unsigned bucket;
};

void mg_merge(const std::vector<u64>& lo, const std::vector<u64>& hi, const std::vector<unsigned>& cnt,
              unsigned grid, std::vector<MgEntry>& out) {
  out.clear();
  for (unsigned b = 0; b < kMgBuckets; ++b) {
    std::vector<MgEntry> e;
    for (unsigned c = 0; c < grid; ++c)
      for (unsigned i = 0; i < kMgCounters; ++i) {
        const u64 o = ((u64)c * kMgBuckets + b) * kMgCounters + i;
        if (cnt[o]) e.push_back({lo[o], hi[o], cnt[o], b});
      }
    std::sort(e.begin(), e.end(), [](const MgEntry& x, const MgEntry& y) {
      return x.hi != y.hi ? x.hi < y.hi : x.lo < y.lo;
    });
    std::vector<MgEntry> sum;  // one entry per key
    for (const MgEntry& x : e) {
      if (!sum.empty() && sum.back().lo == x.lo && sum.back().hi == x.hi) sum.back().count += x.count;
      else sum.push_back(x);
    }
    std::sort(sum.begin(), sum.end(), [](const MgEntry& x, const MgEntry& y) { return x.count > y.count; });
    const u64 delta = sum.size() > kMgCounters ? sum[kMgCounters].count : 0;
    for (MgEntry& x : sum)
      if (x.count > delta) {
        x.count -= delta;
        out.push_back(x);
      }
  }
  std::stable_sort(out.begin(), out.end(), [](const MgEntry& x, const MgEntry& y) { return x.count > y.count; });
}

// Small pinned host blocks (a handle's status word and group counts), kept in a free list
// for the life of the process: cudaFreeHost synchronises the whole device, so a handle
// destroyed in one thread would otherwise stall the GPU work other threads have queued.
constexpr size_t kPinnedBlock = 256;
std::mutex g_pinned_mu;
std::vector<void*> g_pinned_free;

void* pinned_take() {
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  if (g_pinned_free.empty()) {
    char* page = nullptr;
    constexpr size_t kPerPage = 64;
    if (cudaMallocHost((void**)&page, kPinnedBlock * kPerPage) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (size_t i = 0; i < kPerPage; ++i) g_pinned_free.push_back(page + i * kPinnedBlock);
  }
  void* b = g_pinned_free.back();
  g_pinned_free.pop_back();
  return b;
}

void pinned_give(void* b) {
  if (!b) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  g_pinned_free.push_back(b);
}

}  // namespace

// finalize_to_host splits the recount and classification into this many groups of
// partitions (of table slots with one table), so that each group's records are copied to the
// host while the next group is still being recounted.
constexpr unsigned kFinalizeGroups = 8;

struct kma_handle {
  kma_params p;
  Derived d;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr};
  cudaEvent_t consumed[2] = {nullptr, nullptr};
  int device = 0;
  int num_sms = 0;
  cudaMemPool_t pool = nullptr;
  LaunchShape shape{256, 4, 0};
  bool agg = false;
  unsigned prefetch = 1;

  u64* codes = nullptr;
  u64* rcodes = nullptr;
  u64* inv = nullptr;
  u64* hq = nullptr;
  unsigned* marks = nullptr;
  u64* bloom = nullptr;
  u64* keyfilter = nullptr;  // partitioned Bloom mode: keys inserted into the table
  Slot* table = nullptr;
  DevStatus* status = nullptr;
  DevStatus* host_status = nullptr;  // pinned
  unsigned char* stage_seq[2] = {nullptr, nullptr};
  unsigned char* stage_qual[2] = {nullptr, nullptr};
  u64* stage_offs[2] = {nullptr, nullptr};
  u64 stage_offs_cap = 0;
  int stage_next = 0;

  u64 q_used = 0, reads_used = 0, bases_used = 0;
  // Upper bound on the occurrences any one key can have collected since the last reset
  // (windows counted in one table; bucket + overflow records per batch in partitioned
  // mode). Below 2^32 no counter can wrap and the passes count with plain reductions.
  u64 count_bound = 0;
  bool finalized = false;
  bool failed = false;
  bool pack_only = false;  // estimation handles: count() packs the reads, no counting pass

  // partitioned mode: per-partition histogram / cursors and the record buckets of each
  // count() batch (kept until finalize has recounted them)
  struct RecBatch { void* keys; unsigned char* info; u64* fill; u64 cap, ocap; };
  std::vector<RecBatch> rec_batches;

  // contigs of the finalized result (kmer_analysis_contigs), freed by reset / destroy
  char* contig_seq = nullptr;
  u64* contig_offsets = nullptr;
  u64 contig_n = 0, contig_bases = 0, contig_vertices = 0, contig_cycles = 0;
  u64* out_keys = nullptr;
  unsigned* out_counts = nullptr;
  unsigned* out_ext = nullptr;
  unsigned char* out_codes = nullptr;
  u64 out_cap = 0;
  kma_result res;
  // finalize_to_host: per-group record counts (pinned) and the events that publish them
  u64* host_groups = nullptr;
  cudaEvent_t group_ev[kFinalizeGroups] = {};

  // tracing
  bool profiling = false;
  struct ProfRec { int kind; cudaEvent_t a, b; };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> event_pool;
  double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  u64 launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

template <typename T>
int dalloc(kma_handle* h, T** ptr, u64 count) {
  *ptr = nullptr;
  if (count == 0) return KMA_OK;
  cudaError_t e = cudaMallocFromPoolAsync((void**)ptr, count * sizeof(T), h->pool, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return e == cudaErrorMemoryAllocation ? KMA_ENOMEM : cuda_fail(e, "cudaMallocFromPoolAsync");
  }
  return KMA_OK;
}

template <typename T>
void dfree(kma_handle* h, T*& ptr) {
  if (ptr) cudaFreeAsync(ptr, h->stream);
  ptr = nullptr;
}

cudaEvent_t take_event(kma_handle* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch one library kernel on `stream`, counting it and (when profiling) bracketing it
// with a pair of CUDA events on that stream.
template <typename F>
int timed_launch(kma_handle* h, int kind, cudaStream_t stream, bool has_work, F&& launch) {
  if (!has_work) return KMA_OK;
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->profiling) {
    a = take_event(h);
    b = take_event(h);
    if (a) cudaEventRecord(a, stream);
  }
  cudaError_t e = launch();
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  h->launches[kind]++;
  if (h->profiling && a && b) {
    cudaEventRecord(b, stream);
    h->prof.push_back({kind, a, b});
  }
  return KMA_OK;
}

void free_records(kma_handle* h) {
  for (auto& b : h->rec_batches) {
    if (b.keys) cudaFreeAsync(b.keys, h->stream);
    if (b.info) cudaFreeAsync(b.info, h->stream);
    if (b.fill) cudaFreeAsync(b.fill, h->stream);
  }
  h->rec_batches.clear();
}

void free_contigs(kma_handle* h) {
  if (h->contig_seq) cudaFreeAsync(h->contig_seq, h->stream);
  if (h->contig_offsets) cudaFreeAsync(h->contig_offsets, h->stream);
  h->contig_seq = nullptr;
  h->contig_offsets = nullptr;
  h->contig_n = h->contig_bases = h->contig_vertices = h->contig_cycles = 0;
}

void free_all(kma_handle* h) {
  free_records(h);
  dfree(h, h->codes); dfree(h, h->rcodes); dfree(h, h->inv); dfree(h, h->hq); dfree(h, h->marks);
  dfree(h, h->bloom); dfree(h, h->keyfilter); dfree(h, h->table); dfree(h, h->status);
  for (int i = 0; i < 2; ++i) { dfree(h, h->stage_seq[i]); dfree(h, h->stage_qual[i]); dfree(h, h->stage_offs[i]); }
  dfree(h, h->out_keys); dfree(h, h->out_counts); dfree(h, h->out_ext); dfree(h, h->out_codes);
  free_contigs(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  pinned_give(h->host_status);
  h->host_status = nullptr;
  pinned_give(h->host_groups);
  h->host_groups = nullptr;
  for (auto& e : h->group_ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  for (int i = 0; i < 2; ++i) {
    if (h->copied[i]) cudaEventDestroy(h->copied[i]);
    if (h->consumed[i]) cudaEventDestroy(h->consumed[i]);
    h->copied[i] = h->consumed[i] = nullptr;
  }
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  h->copy_stream = nullptr;
  for (auto& r : h->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  h->prof.clear();
  for (auto e : h->event_pool) cudaEventDestroy(e);
  h->event_pool.clear();
}

// Back to the empty state: status, Bloom filter, key filter and table cleared on the handle's
// stream. The arena is not cleared: every count() rewrites the words of its batch and sets the
// slack words behind it invalid (reserve_batch).
int clear_state(kma_handle* h) {
  free_records(h);
  free_contigs(h);
  KMA_CUDA(cudaMemsetAsync(h->status, 0, sizeof(DevStatus), h->stream));
  if (h->bloom) KMA_CUDA(cudaMemsetAsync(h->bloom, 0, h->d.plan.bloom_words * 8, h->stream));
  if (h->keyfilter) KMA_CUDA(cudaMemsetAsync(h->keyfilter, 0, h->d.Wt * h->d.P * 8, h->stream));
  int rc = timed_launch(h, KMA_KERNEL_INIT, h->stream, h->d.plan.table_slots > 0,
                        [&] { return launch_table_init(h->table, h->d.plan.table_slots, h->stream); });
  if (rc) return rc;
  h->q_used = h->reads_used = h->bases_used = 0;
  h->count_bound = 0;
  h->finalized = false;
  h->failed = false;
  std::memset(&h->res, 0, sizeof(h->res));
  return KMA_OK;
}

void choose_shape(kma_handle* h) {
  h->shape.block_threads = h->p.block_threads ? (int)h->p.block_threads : 256;
  h->shape.windows_per_thread = h->p.windows_per_thread ? (int)h->p.windows_per_thread : 2;
  h->agg = h->p.warp_aggregate != 0;
  h->prefetch = h->p.slot_prefetch == 1 ? 1u : 0u;
  int per_sm = h->p.ctas_per_sm ? (int)h->p.ctas_per_sm
                                : pass_max_ctas_per_sm(h->shape.block_threads, h->shape.windows_per_thread, h->agg);
  if (per_sm < 1) per_sm = 1;
  h->shape.grid = h->num_sms * per_sm;
}

int flags_to_code(unsigned flags) {
  if (flags & kFlagTimeout) return KMA_ETIMEOUT;
  if (flags & kFlagBadOffsets) return KMA_EINVAL;
  if (flags & kFlagFull) return KMA_EFULL;
  if (flags & kFlagOverflow) return KMA_EOVERFLOW;
  return KMA_OK;
}

int read_status(kma_handle* h) {
  KMA_CUDA(cudaMemcpyAsync(h->host_status, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
  KMA_CUDA(cudaStreamSynchronize(h->stream));
  return KMA_OK;
}

PassDesc pass_desc(kma_handle* h, unsigned mode, u64 q0, u64 q1) {
  PassDesc d;
  std::memset(&d, 0, sizeof(d));
  d.codes = h->codes; d.rcodes = h->rcodes; d.inv = h->inv; d.hq = h->hq; d.marks = h->marks;
  d.bloom = h->bloom; d.table = h->table; d.status = h->status;
  d.bloom_words = h->d.plan.bloom_words; d.slots = h->d.plan.table_slots;
  d.q0 = q0; d.q1 = q1;
  d.k = h->p.k; d.bloom_h = h->d.plan.bloom_hashes; d.canonical = h->p.canonical;
  d.mode = mode;
  d.n_parts = h->p.n_parts > 1 ? h->p.n_parts : 1;
  d.part = h->p.n_parts > 1 ? h->p.part : 0;
  d.no_overflow = h->count_bound < (1ull << 32) ? 1u : 0u;
  return d;
}

// Staging-copy wait policy of the pack kernel: a generous poll limit, or (fault injection
// for tests) copies that are never issued and a short limit, which must end in KMA_ETIMEOUT.
void set_pack_waits(kma_handle* h, PackBatch& pb) {
  pb.skip_copy = h->p.fault_inject == 1 ? 1u : 0u;
  pb.wait_limit = h->p.fault_inject == 1 ? kWaitPollsInjected : kWaitPolls;
}

// Reserve arena positions for a batch of n_reads reads (n_bases bases), packed on stream `st`,
// and describe it for the pack kernel. The windows of the batch read up to 192 positions past
// its end; the 256 positions behind it are set invalid here (ordered before the packing on
// `st`), and the next batch's packing overwrites them.
int reserve_batch(kma_handle* h, u64 n_reads, u64 n_bases, PackDesc& pd, u64& q0, u64& n_pos, cudaStream_t st) {
  n_pos = ((n_bases + n_reads + 63) / 64) * 64;
  if (n_pos == 0) n_pos = 64;
  if (h->q_used + n_pos + kBatchSlack > h->d.plan.arena_positions) return KMA_EFULL;
  if (h->bases_used + n_bases > h->p.max_bases) return KMA_EFULL;
  q0 = h->q_used;
  {
    const u64 e = q0 + n_pos;  // a multiple of 64
    KMA_CUDA(cudaMemsetAsync(h->inv + e / 64, 0xFF, kBatchSlack / 64 * 8, st));
    KMA_CUDA(cudaMemsetAsync(h->hq + e / 64, 0, kBatchSlack / 64 * 8, st));
    KMA_CUDA(cudaMemsetAsync(h->codes + e / 32, 0, kBatchSlack / 32 * 8, st));
    KMA_CUDA(cudaMemsetAsync(h->rcodes + e / 32, 0xFF, kBatchSlack / 32 * 8, st));
  }
  std::memset(&pd, 0, sizeof(pd));
  pd.n_reads = n_reads; pd.n_bases = n_bases; pd.q0 = q0; pd.n_pos = n_pos;
  pd.codes = h->codes; pd.rcodes = h->rcodes; pd.inv = h->inv; pd.hq = h->hq; pd.status = h->status;
  pd.qual_min = (unsigned)h->p.qual_offset + (unsigned)h->p.qual_threshold;
  h->q_used += n_pos;
  h->reads_used += n_reads;
  h->bases_used += n_bases;
  return KMA_OK;
}

PartGeom part_geom(kma_handle* h) {
  PartGeom g;
  std::memset(&g, 0, sizeof(g));
  g.bloom = h->bloom;
  g.keyfilter = h->keyfilter;
  g.Wk = h->d.Wt;
  g.table = h->table;
  g.status = h->status;
  g.Wp = h->d.Wp;
  g.Sp = h->d.Sp;
  g.P = h->d.P;
  g.bloom_h = h->d.plan.bloom_hashes;
  g.k = h->p.k;
  g.canonical = h->p.canonical;
  g.n_parts = h->p.n_parts > 1 ? h->p.n_parts : 1;
  g.part = h->p.n_parts > 1 ? h->p.part : 0;
  g.rpt = h->p.windows_per_thread >= 4 ? 4 : 2;
  g.wait_limit = kWaitPolls;
  g.no_overflow = h->count_bound < (1ull << 32) ? 1u : 0u;
  g.group = h->p.heavy_hitters ? 1u : 0u;
  return g;
}

// First pass over the windows [q0, q0 + n_pos) of one packed batch (n_reads reads, n_bases
// bases) on stream `st`. One table: Bloom test-and-set (or counting) in place. Partitions:
// scatter into per-partition record buckets, then the record pass part by part; the buckets
// are kept for the recount in finalize. Nothing here waits for the GPU.
// Partitioned mode: record buckets for a count() call of n_pos arena positions (n_reads reads,
// n_bases bases), appended to the handle's record batches (kept for the recount).
int prepare_records(kma_handle* h, u64 n_pos, u64 n_reads, u64 n_bases, cudaStream_t st, size_t& index) {
  const u64 P = h->d.P, k = h->p.k;
  // Bucket capacity from the window count of reads of length >= k (exact for such reads);
  // shorter reads, hash imbalance and repeated k-mers spill into the overflow area. Both are
  // multiples of 16 records (the record passes stage 16-byte aligned tiles).
  const u64 w_est = n_bases > (k - 1) * n_reads ? n_bases - (k - 1) * n_reads : 0;
  u64 cap = ((u64)((double)w_est / (double)P * 1.05) + 64 + 15) & ~15ull;
  u64 ocap = n_pos / 16 + 65536;
  if (P * cap < n_bases) ocap = std::max(ocap, n_bases - P * cap + n_pos / 64);
  ocap = (ocap + 15) & ~15ull;
  // the kernels hold in-bucket and overflow positions, and tile numbers, in 32 bits
  const u64 tile_recs = 32ull * part_geom(h).rpt;
  if (cap >= (1ull << 32) || ocap >= (1ull << 32) ||
      P * ((cap + tile_recs - 1) / tile_recs) + (ocap + tile_recs - 1) / tile_recs >= (1ull << 31))
    return KMA_EINVAL;  // more partitions, or smaller count() batches, are needed
  h->count_bound += cap + ocap;
  const u64 total = P * cap + ocap;
  kma_handle::RecBatch rb{nullptr, nullptr, nullptr, cap, ocap};
  const size_t kb = (size_t)total * (k > 32 ? 16 : 8);
  cudaError_t e = cudaMallocFromPoolAsync(&rb.keys, kb, h->pool, st);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&rb.info, (size_t)total, h->pool, st);
  // fill[0..P], then one word for the record passes' tile queue
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&rb.fill, (size_t)(P + 2) * 8, h->pool, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (rb.keys) cudaFreeAsync(rb.keys, st);
    if (rb.info) cudaFreeAsync(rb.info, st);
    if (rb.fill) cudaFreeAsync(rb.fill, st);
    return e == cudaErrorMemoryAllocation ? KMA_ENOMEM : cuda_fail(e, "record buckets");
  }
  h->rec_batches.push_back(rb);
  index = h->rec_batches.size() - 1;
  KMA_CUDA(cudaMemsetAsync(rb.fill, 0, (size_t)(P + 2) * 8, st));
  return KMA_OK;
}

// Record batch `rb` of a handle with P partitions, all of it (every bucket, then the
// overflow area).
PartRecords records_of(const kma_handle::RecBatch& rb, u64 P) {
  PartRecords r;
  r.keys = rb.keys; r.info = rb.info; r.cap = rb.cap; r.ocap = rb.ocap; r.fill = rb.fill;
  r.queue = reinterpret_cast<unsigned*>(rb.fill + P + 1);
  r.p_begin = 0; r.p_end = (unsigned)P; r.overflow = 1; r.pad = 0;
  return r;
}

// Partitioned mode: the windows [q0, q0 + n_pos) into record batch `index`.
int scatter_windows(kma_handle* h, size_t index, u64 q0, u64 n_pos, cudaStream_t st) {
  const PartGeom g = part_geom(h);
  PartWindows w;
  w.codes = h->codes; w.rcodes = h->rcodes; w.inv = h->inv; w.hq = h->hq;
  w.q0 = q0; w.q1 = q0 + n_pos;
  const PartRecords r = records_of(h->rec_batches[index], h->d.P);
  return timed_launch(h, KMA_KERNEL_SCATTER, st, n_pos > 0,
                      [&] { return launch_part_scatter(g, w, r, st, h->num_sms); });
}

// Partitioned mode: the record pass (Bloom test-and-set, or counting) over batch `index`.
int record_pass(kma_handle* h, size_t index, cudaStream_t st) {
  const unsigned mode = h->p.use_bloom ? kModeBloom : kModeCount;
  const PartGeom g = part_geom(h);
  const PartRecords r = records_of(h->rec_batches[index], h->d.P);
  return timed_launch(h, KMA_KERNEL_PASS, st, true, [&] { return launch_part_pass(g, r, mode, st, h->num_sms); });
}

// First pass over the windows [q0, q0 + n_pos) of one packed batch (n_reads reads, n_bases
// bases) on stream `st`. One table: Bloom test-and-set (or counting) in place. Partitions:
// scatter into per-partition record buckets, then the record pass part by part; the buckets
// are kept for the recount in finalize. Nothing here waits for the GPU.
int first_pass(kma_handle* h, u64 q0, u64 n_pos, u64 n_reads, u64 n_bases, cudaStream_t st) {
  const unsigned mode = h->p.use_bloom ? kModeBloom : kModeCount;
  if (h->d.P <= 1) {
    h->count_bound += n_pos;
    PassBatch b;
    std::memset(&b, 0, offsetof(PassBatch, d) + sizeof(PassDesc));
    b.n = 1;
    b.prefetch = h->prefetch;
    b.d[0] = pass_desc(h, mode, q0, q0 + n_pos);
    const u64 tile = (u64)h->shape.block_threads * h->shape.windows_per_thread;
    b.d[0].tile_begin = 0;
    b.total_tiles = (n_pos + tile - 1) / tile;
    return timed_launch(h, KMA_KERNEL_PASS, st, b.total_tiles > 0,
                        [&] { return launch_pass(b, h->shape, h->agg, st); });
  }
  size_t index = 0;
  int rc = prepare_records(h, n_pos, n_reads, n_bases, st, index);
  if (rc || (rc = scatter_windows(h, index, q0, n_pos, st))) return rc;
  return n_pos ? record_pass(h, index, st) : KMA_OK;
}

int run_pack_and_pass(kma_handle* h, const PackDesc& pd) {
  PackBatch pb;
  std::memset(&pb, 0, offsetof(PackBatch, d) + sizeof(PackDesc));
  pb.n = 1;
  set_pack_waits(h, pb);
  pb.d[0] = pd;
  pb.d[0].chunk_begin = 0;
  pb.total_chunks = (pd.n_pos / 64 + kPackChunkWords - 1) / kPackChunkWords;
  int rc = timed_launch(h, KMA_KERNEL_PACK, h->stream, pb.total_chunks > 0,
                        [&] { return launch_pack(pb, h->stream, h->num_sms); });
  if (rc) return rc;
  if (h->pack_only) return KMA_OK;
  return first_pass(h, pd.q0, pd.n_pos, pd.n_reads, pd.n_bases, h->stream);
}

int ensure_output(kma_handle* h, u64 need) {
  if (need <= h->out_cap && h->out_keys) return KMA_OK;
  dfree(h, h->out_keys); dfree(h, h->out_counts); dfree(h, h->out_ext); dfree(h, h->out_codes);
  h->out_cap = 0;
  u64 cap = std::max<u64>(need + need / 8, 1024);
  int rc;
  if ((rc = dalloc(h, &h->out_keys, 2 * cap))) return rc;
  if ((rc = dalloc(h, &h->out_counts, cap))) return rc;
  if ((rc = dalloc(h, &h->out_ext, 8 * cap))) return rc;
  if ((rc = dalloc(h, &h->out_codes, 2 * cap))) return rc;
  h->out_cap = cap;
  return KMA_OK;
}

ClassDesc class_desc(kma_handle* h) {
  ClassDesc c;
  std::memset(&c, 0, sizeof(c));
  c.table = h->table; c.status = h->status; c.slots = h->d.plan.table_slots;
  c.out_keys = h->out_keys; c.out_counts = h->out_counts; c.out_ext = h->out_ext;
  c.out_codes = h->out_codes; c.out_cap = h->out_cap;
  c.min_depth = h->p.min_depth;
  c.min_ext = h->p.min_ext_count ? h->p.min_ext_count : 1;
  return c;
}

constexpr u64 kClassTile = 256 * 4;  // slots per classify block tile (kernel constants)

void fill_result(kma_handle* h) {
  kma_result& r = h->res;
  r.n = h->host_status->n_out;
  r.n_uu = h->host_status->n_uu;
  r.valid_windows = h->host_status->valid_windows;
  r.table_keys = h->host_status->table_keys;
  r.keys = (const uint64_t*)h->out_keys;
  r.counts = h->out_counts;
  r.ext = h->out_ext;
  r.codes = h->out_codes;
}

// HyperLogLog estimate of 2^p registers (Flajolet, Fusy, Gandouet, Meunier 2007): the raw
// estimate alpha_m m^2 / sum 2^-M[j], replaced by linear counting m ln(m / V) in the small
// range (raw <= 5m/2 with V > 0 empty registers). 64-bit hashes need no large-range
// correction.
double hll_estimate(const uint8_t* regs, unsigned p) {
  const double m = (double)(1u << p);
  double sum = 0.0;
  u64 zeros = 0;
  for (u64 j = 0; j < (1ull << p); ++j) {
    sum += std::ldexp(1.0, -(int)regs[j]);
    zeros += regs[j] == 0;
  }
  const double alpha = p == 4 ? 0.673 : p == 5 ? 0.697 : p == 6 ? 0.709 : 0.7213 / (1.0 + 1.079 / m);
  const double raw = alpha * m * m / sum;
  if (raw <= 2.5 * m && zeros > 0) return m * std::log(m / (double)zeros);
  return raw;
}

}  // namespace

extern "C" {

int kmer_analysis_plan(const kma_params* params, kma_plan* out) {
  if (!out) return KMA_EINVAL;
  Derived d;
  int rc = derive(params, d);
  if (rc) return rc;
  *out = d.plan;
  return KMA_OK;
}

int kmer_analysis_create(const kma_params* params, void* cuda_stream, kma_handle** out) {
  if (!out) return KMA_EINVAL;
  *out = nullptr;
  Derived d;
  int rc = derive(params, d);
  if (rc) return rc;
  kma_handle* h = new kma_handle();
  h->p = *params;
  h->d = d;
  h->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaGetDevice"); }
  if ((rc = get_pool(h->device, &h->pool))) { delete h; return rc; }
  choose_shape(h);
  h->stage_offs_cap = d.staging / 16 + 2;
  if ((rc = dalloc(h, &h->codes, d.codes_words)) || (rc = dalloc(h, &h->rcodes, d.codes_words)) ||
      (rc = dalloc(h, &h->inv, d.bit_words)) ||
      (rc = dalloc(h, &h->hq, d.bit_words)) || (rc = dalloc(h, &h->marks, d.mark_words)) ||
      (rc = dalloc(h, &h->bloom, d.plan.bloom_words)) || (rc = dalloc(h, &h->keyfilter, d.Wt * d.P)) ||
      (rc = dalloc(h, &h->table, d.plan.table_slots)) || (rc = dalloc(h, &h->status, 1))) {
    free_all(h);
    delete h;
    return rc;
  }
  static_assert(sizeof(DevStatus) <= kPinnedBlock && kFinalizeGroups * sizeof(u64) <= kPinnedBlock,
                "pinned blocks hold a status word and the group counts");
  h->host_status = static_cast<DevStatus*>(pinned_take());
  if (!h->host_status) { free_all(h); delete h; return KMA_ENOMEM; }

  std::memset(h->host_status, 0, sizeof(DevStatus));
  if ((rc = clear_state(h))) { free_all(h); delete h; return rc; }
  *out = h;
  return KMA_OK;
}

// offsets[0..n] non-decreasing? Large read sets are checked by several host threads (the
// check is a stream over 8 bytes per read, done before any input is copied).
static bool offsets_nondecreasing(const uint64_t* offsets, u64 n) {
  auto check = [offsets](u64 a, u64 b) {
    unsigned bad = 0;
    for (u64 r = a; r < b; ++r) bad |= offsets[r + 1] < offsets[r];
    return bad == 0;
  };
  const unsigned hw = std::thread::hardware_concurrency();
  const unsigned T = n < (1u << 20) ? 1u : std::max(1u, std::min(8u, hw));
  if (T == 1) return check(0, n);
  std::vector<char> ok(T, 0);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < T; ++t)
    th.emplace_back([&, t] { ok[t] = check(n * t / T, n * (t + 1) / T); });
  for (auto& x : th) x.join();
  return std::all_of(ok.begin(), ok.end(), [](char v) { return v != 0; });
}

static int setup_staging(kma_handle* h) {
  if (h->stage_seq[0]) return KMA_OK;
  int rc;
  for (int i = 0; i < 2; ++i) {
    if ((rc = dalloc(h, &h->stage_seq[i], h->d.staging)) || (rc = dalloc(h, &h->stage_qual[i], h->d.staging)) ||
        (rc = dalloc(h, &h->stage_offs[i], h->stage_offs_cap)))
      return rc;
    KMA_CUDA(cudaEventCreateWithFlags(&h->copied[i], cudaEventDisableTiming));
    KMA_CUDA(cudaEventCreateWithFlags(&h->consumed[i], cudaEventDisableTiming));
  }
  KMA_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  // the staging buffers were allocated on h->stream: make the copy stream wait for that
  KMA_CUDA(cudaEventRecord(h->consumed[0], h->stream));
  KMA_CUDA(cudaEventRecord(h->consumed[1], h->stream));
  return KMA_OK;
}

int kmer_analysis_count(kma_handle* h, const char* seq, const char* qual, const uint64_t* offsets,
                        uint64_t n_reads, int on_device) {
  if (!h) return KMA_EINVAL;
  if (h->finalized || h->failed) return KMA_ESTATE;
  if (!offsets) return KMA_EINVAL;
  if (n_reads == 0) return KMA_OK;
  if (!seq || !qual) return KMA_EINVAL;
  int rc;
  if (on_device) {
    u64 ends[2];
    KMA_CUDA(cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, h->stream));
    KMA_CUDA(cudaMemcpyAsync(&ends[1], offsets + n_reads, 8, cudaMemcpyDeviceToHost, h->stream));
    KMA_CUDA(cudaStreamSynchronize(h->stream));
    if (ends[1] < ends[0]) return KMA_EINVAL;
    PackDesc pd;
    u64 q0, n_pos;
    if ((rc = reserve_batch(h, n_reads, ends[1] - ends[0], pd, q0, n_pos, h->stream))) return rc;
    pd.seq = (const unsigned char*)seq;
    pd.qual = (const unsigned char*)qual;
    pd.offsets = (const unsigned long long*)offsets;
    pd.delta = 0;
    return run_pack_and_pass(h, pd);
  }
  // Host input: validate offsets, then stream chunks through two staging buffers; the copy
  // of chunk i+1 overlaps the packing and first pass of chunk i.
  if (!offsets_nondecreasing(offsets, n_reads)) return KMA_EINVAL;
  if (offsets[n_reads] - offsets[0] + h->bases_used > h->p.max_bases) return KMA_EFULL;
  if ((rc = setup_staging(h))) return rc;
  // With partitions, every staged chunk is packed and scattered into one set of record buckets
  // (so the copy of the next chunk overlaps both), and the record pass runs once over all of
  // them: a pass per chunk would bring every partition's filter and table back into L2 once
  // per chunk.
  const bool parts = h->d.P > 1 && !h->pack_only;
  size_t rec_index = 0;
  if (parts) {
    // positions of the whole call: every chunk is rounded up to 64 positions, and a chunk
    // ends only when the next read would overflow the staged bases or read offsets
    const u64 nb_all = offsets[n_reads] - offsets[0];
    const u64 chunks = 2 * (nb_all / h->d.staging + n_reads / (h->stage_offs_cap - 1) + 1);
    if ((rc = prepare_records(h, nb_all + n_reads + 64 * chunks, n_reads, nb_all, h->stream, rec_index))) return rc;
  }
  u64 r0 = 0;
  while (r0 < n_reads) {
    u64 r1 = r0;
    while (r1 < n_reads && offsets[r1 + 1] - offsets[r0] <= h->d.staging && r1 - r0 + 1 < h->stage_offs_cap) ++r1;
    if (r1 == r0) return KMA_EINVAL;  // a single read longer than the staging buffer
    const u64 nb = offsets[r1] - offsets[r0];
    PackDesc pd;
    u64 q0, n_pos;
    if ((rc = reserve_batch(h, r1 - r0, nb, pd, q0, n_pos, h->stream))) return rc;
    const int b = h->stage_next;
    h->stage_next ^= 1;
    KMA_CUDA(cudaStreamWaitEvent(h->copy_stream, h->consumed[b], 0));
    KMA_CUDA(cudaMemcpyAsync(h->stage_seq[b], seq + offsets[r0], nb, cudaMemcpyHostToDevice, h->copy_stream));
    KMA_CUDA(cudaMemcpyAsync(h->stage_qual[b], qual + offsets[r0], nb, cudaMemcpyHostToDevice, h->copy_stream));
    KMA_CUDA(cudaMemcpyAsync(h->stage_offs[b], offsets + r0, (r1 - r0 + 1) * 8, cudaMemcpyHostToDevice, h->copy_stream));
    KMA_CUDA(cudaEventRecord(h->copied[b], h->copy_stream));
    KMA_CUDA(cudaStreamWaitEvent(h->stream, h->copied[b], 0));
    pd.seq = h->stage_seq[b];
    pd.qual = h->stage_qual[b];
    pd.offsets = h->stage_offs[b];
    pd.delta = (long long)offsets[r0];
    PackBatch pb;
    std::memset(&pb, 0, offsetof(PackBatch, d) + sizeof(PackDesc));
    pb.n = 1;
    set_pack_waits(h, pb);
    pb.d[0] = pd;
    pb.total_chunks = (n_pos / 64 + kPackChunkWords - 1) / kPackChunkWords;
    if ((rc = timed_launch(h, KMA_KERNEL_PACK, h->stream, true,
                           [&] { return launch_pack(pb, h->stream, h->num_sms); })))
      return rc;
    KMA_CUDA(cudaEventRecord(h->consumed[b], h->stream));
    if (parts) {
      if ((rc = scatter_windows(h, rec_index, q0, n_pos, h->stream))) return rc;
    } else if (!h->pack_only && (rc = first_pass(h, q0, n_pos, r1 - r0, nb, h->stream))) {
      return rc;
    }
    r0 = r1;
  }
  if (parts && (rc = record_pass(h, rec_index, h->stream))) return rc;
  // Host buffers may be reused once the call returns: wait for the copies.
  KMA_CUDA(cudaStreamSynchronize(h->copy_stream));
  return KMA_OK;
}

// Recount pass (first sightings) of the Bloom handles: one launch for all one-table handles,
// one per record batch of the partitioned ones. Enqueued on h0's stream.
static int enqueue_recount(kma_handle* const* hs, uint32_t n) {
  kma_handle* h0 = hs[0];
  PassBatch pb;
  std::memset(&pb, 0, sizeof(pb));
  pb.prefetch = h0->prefetch;
  const u64 tile = (u64)h0->shape.block_threads * h0->shape.windows_per_thread;
  u64 tiles = 0;
  for (uint32_t i = 0; i < n; ++i) {
    kma_handle* h = hs[i];
    if (!h->p.use_bloom || h->q_used == 0 || h->d.P > 1) continue;
    PassDesc d = pass_desc(h, kModeRecount, 0, h->q_used);
    d.tile_begin = tiles;
    tiles += (h->q_used + tile - 1) / tile;
    pb.d[pb.n++] = d;
  }
  pb.total_tiles = tiles;
  int rc = timed_launch(h0, KMA_KERNEL_RECOUNT, h0->stream, pb.n > 0 && tiles > 0,
                        [&] { return launch_pass(pb, h0->shape, h0->agg, h0->stream); });
  if (rc) return rc;
  for (uint32_t i = 0; i < n; ++i) {  // partitioned handles: recount their record buckets
    kma_handle* h = hs[i];
    if (!h->p.use_bloom || h->d.P <= 1) continue;
    const PartGeom g = part_geom(h);
    rc = timed_launch(h0, KMA_KERNEL_RECOUNT, h0->stream, g.Wk > 0,
                      [&] { return launch_keyfilter_build(g, h0->stream, h0->num_sms); });
    if (rc) return rc;
    for (auto& rb : h->rec_batches) {
      const PartRecords r = records_of(rb, h->d.P);
      rc = timed_launch(h0, KMA_KERNEL_RECOUNT, h0->stream, true,
                        [&] { return launch_part_pass(g, r, kModeRecount, h0->stream, h0->num_sms); });
      if (rc) return rc;
    }
  }
  return KMA_OK;
}

// Classification + compaction of the handles with ok[i] into their current output buffers,
// one launch; then their record buckets are released. Enqueued on h0's stream.
static int enqueue_classify(kma_handle* const* hs, uint32_t n, const std::vector<int>& ok) {
  kma_handle* h0 = hs[0];
  for (uint32_t i = 0; i < n; ++i)
    if (ok[i]) KMA_CUDA(cudaMemsetAsync(&hs[i]->status->n_out, 0, 2 * sizeof(u64), h0->stream));
  ClassBatch cb;
  std::memset(&cb, 0, sizeof(cb));
  cb.write = 1;
  u64 blocks = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (!ok[i]) continue;
    ClassDesc c = class_desc(hs[i]);
    c.block_begin = blocks;
    blocks += (c.slots + kClassTile - 1) / kClassTile;
    cb.d[cb.n++] = c;
  }
  cb.total_blocks = blocks;
  int rc = timed_launch(h0, KMA_KERNEL_CLASSIFY, h0->stream, cb.n > 0 && blocks > 0,
                        [&] { return launch_classify(cb, h0->stream, h0->num_sms); });
  if (rc) return rc;
  for (uint32_t i = 0; i < n; ++i) {  // the record buckets are not needed after the recount
    cudaStream_t saved = hs[i]->stream;
    hs[i]->stream = h0->stream;
    free_records(hs[i]);
    hs[i]->stream = saved;
  }
  return KMA_OK;
}

static int check_batch(kma_handle* const* hs, uint32_t n) {
  if (!hs || n == 0 || n > KMA_MAX_BATCH) return KMA_EINVAL;
  for (uint32_t i = 0; i < n; ++i) {
    if (!hs[i]) return KMA_EINVAL;
    if (hs[i]->finalized || hs[i]->failed) return KMA_ESTATE;
    for (uint32_t j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return KMA_EINVAL;
  }
  return KMA_OK;
}

static int finalize_many(kma_handle* const* hs, uint32_t n, kma_result* out) {
  int rc = check_batch(hs, n);
  if (rc) return rc;
  kma_handle* h0 = hs[0];
  // make every handle's stream work visible to h0's stream
  for (uint32_t i = 1; i < n; ++i) {
    if (hs[i]->stream != h0->stream) {
      cudaEvent_t ev;
      KMA_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      cudaError_t e = cudaEventRecord(ev, hs[i]->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h0->stream, ev, 0);
      cudaEventDestroy(ev);
      if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    }
  }
  if ((rc = enqueue_recount(hs, n))) return rc;
  // statuses -> output capacities (table_keys bounds the records)
  for (uint32_t i = 0; i < n; ++i)
    KMA_CUDA(cudaMemcpyAsync(hs[i]->host_status, hs[i]->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, h0->stream));
  KMA_CUDA(cudaStreamSynchronize(h0->stream));
  int first_err = KMA_OK;
  std::vector<int> ok(n, 0);
  for (uint32_t i = 0; i < n; ++i) {
    kma_handle* h = hs[i];
    int e = flags_to_code(h->host_status->flags);
    if (e) { h->failed = true; if (!first_err) first_err = e; continue; }
    cudaStream_t saved = h->stream;
    h->stream = h0->stream;
    e = ensure_output(h, h->host_status->table_keys);
    h->stream = saved;
    if (e) { h->failed = true; if (!first_err) first_err = e; continue; }
    ok[i] = 1;
  }
  if ((rc = enqueue_classify(hs, n, ok))) return rc;
  for (uint32_t i = 0; i < n; ++i)
    if (ok[i]) KMA_CUDA(cudaMemcpyAsync(hs[i]->host_status, hs[i]->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, h0->stream));
  KMA_CUDA(cudaStreamSynchronize(h0->stream));
  for (uint32_t i = 0; i < n; ++i) {
    kma_handle* h = hs[i];
    if (!ok[i]) { if (out) std::memset(&out[i], 0, sizeof(kma_result)); continue; }
    int e = flags_to_code(h->host_status->flags);
    if (e) { h->failed = true; if (!first_err) first_err = e; if (out) std::memset(&out[i], 0, sizeof(kma_result)); continue; }
    fill_result(h);
    h->finalized = true;
    if (out) out[i] = h->res;
  }
  return first_err;
}

int kmer_analysis_finalize(kma_handle* h, kma_result* out) {
  if (!h) return KMA_EINVAL;
  kma_handle* hs[1] = {h};
  return finalize_many(hs, 1, out);
}

int kmer_analysis_finalize_batch(kma_handle* const* hs, uint32_t n, kma_result* out) {
  return finalize_many(hs, n, out);
}

int kmer_analysis_reserve_output(kma_handle* h, uint64_t n_records) {
  if (!h) return KMA_EINVAL;
  return ensure_output(h, n_records);
}

int kmer_analysis_finalize_batch_async(kma_handle* const* hs, uint32_t n) {
  int rc = check_batch(hs, n);
  if (rc) return rc;
  for (uint32_t i = 0; i < n; ++i)
    if (!hs[i]->out_keys) return KMA_ESTATE;  // kmer_analysis_reserve_output first
  if ((rc = enqueue_recount(hs, n))) return rc;
  std::vector<int> ok(n, 1);
  if ((rc = enqueue_classify(hs, n, ok))) return rc;
  for (uint32_t i = 0; i < n; ++i) hs[i]->finalized = true;
  return KMA_OK;
}

int kmer_analysis_fetch_result(kma_handle* h, kma_result* out) {
  if (!h) return KMA_EINVAL;
  if (!h->finalized) return KMA_ESTATE;
  int rc = read_status(h);
  if (rc) return rc;
  fill_result(h);
  if (out) *out = h->res;
  rc = flags_to_code(h->host_status->flags);
  if (!rc && h->host_status->n_out > h->out_cap) rc = KMA_EFULL;
  return rc;
}

int kmer_analysis_count_batch(kma_handle* const* hs, const kma_reads* reads, uint32_t n) {
  if (!hs || !reads || n == 0 || n > KMA_MAX_BATCH) return KMA_EINVAL;
  kma_handle* h0 = hs[0];
  for (uint32_t i = 0; i < n; ++i) {
    if (!hs[i]) return KMA_EINVAL;
    if (hs[i]->finalized || hs[i]->failed) return KMA_ESTATE;
    if (hs[i]->device != h0->device) return KMA_EINVAL;
    for (uint32_t j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return KMA_EINVAL;
    if (reads[i].n_reads && (!reads[i].seq || !reads[i].qual || !reads[i].offsets)) return KMA_EINVAL;
  }
  PackBatch pk;
  std::memset(&pk, 0, sizeof(pk));
  set_pack_waits(h0, pk);
  struct Later { kma_handle* h; u64 q0, n_pos, n_reads, n_bases; };
  std::vector<Later> part_later;
  PassBatch ps;
  std::memset(&ps, 0, sizeof(ps));
  ps.prefetch = h0->prefetch;
  const u64 tile = (u64)h0->shape.block_threads * h0->shape.windows_per_thread;
  u64 words = 0, tiles = 0;
  for (uint32_t i = 0; i < n; ++i) {
    kma_handle* h = hs[i];
    if (reads[i].n_reads == 0) continue;
    PackDesc pd;
    u64 q0, n_pos;
    int rc = reserve_batch(h, reads[i].n_reads, reads[i].n_bases, pd, q0, n_pos, h0->stream);
    if (rc) return rc;
    pd.seq = (const unsigned char*)reads[i].seq;
    pd.qual = (const unsigned char*)reads[i].qual;
    pd.offsets = (const unsigned long long*)reads[i].offsets;
    pd.delta = 0;
    pd.chunk_begin = words;
    words += (n_pos / 64 + kPackChunkWords - 1) / kPackChunkWords;
    pk.d[pk.n++] = pd;
    if (h->d.P > 1) {  // partitioned: its own histogram/scatter/record pass after the packing
      part_later.push_back({h, q0, n_pos, reads[i].n_reads, reads[i].n_bases});
      continue;
    }
    h->count_bound += n_pos;
    PassDesc d = pass_desc(h, h->p.use_bloom ? kModeBloom : kModeCount, q0, q0 + n_pos);
    d.tile_begin = tiles;
    tiles += (n_pos + tile - 1) / tile;
    ps.d[ps.n++] = d;
  }
  pk.total_chunks = words;
  ps.total_tiles = tiles;
  int rc = timed_launch(h0, KMA_KERNEL_PACK, h0->stream, pk.n > 0 && words > 0,
                        [&] { return launch_pack(pk, h0->stream, h0->num_sms); });
  if (rc) return rc;
  rc = timed_launch(h0, KMA_KERNEL_PASS, h0->stream, ps.n > 0 && tiles > 0,
                    [&] { return launch_pass(ps, h0->shape, h0->agg, h0->stream); });
  if (rc) return rc;
  for (auto& l : part_later)
    if ((rc = first_pass(l.h, l.q0, l.n_pos, l.n_reads, l.n_bases, h0->stream))) return rc;
  return KMA_OK;
}

int kmer_analysis_copy_result(kma_handle* h, uint64_t* keys, uint32_t* counts, uint32_t* ext,
                              uint8_t* codes, uint64_t capacity, int on_device) {
  if (!h) return KMA_EINVAL;
  if (!h->finalized) return KMA_ESTATE;
  const u64 n = h->res.n;
  if (capacity < n) return KMA_EINVAL;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (n) {
    if (keys) KMA_CUDA(cudaMemcpyAsync(keys, h->out_keys, n * 16, kind, h->stream));
    if (counts) KMA_CUDA(cudaMemcpyAsync(counts, h->out_counts, n * 4, kind, h->stream));
    if (ext) KMA_CUDA(cudaMemcpyAsync(ext, h->out_ext, n * 32, kind, h->stream));
    if (codes) KMA_CUDA(cudaMemcpyAsync(codes, h->out_codes, n * 2, kind, h->stream));
  }
  KMA_CUDA(cudaStreamSynchronize(h->stream));
  return KMA_OK;
}

int kmer_analysis_finalize_to_host(kma_handle* h, uint64_t* keys, uint32_t* counts, uint32_t* ext,
                                   uint8_t* codes, uint64_t capacity, kma_result* out) {
  if (!h) return KMA_EINVAL;
  if (h->finalized || h->failed) return KMA_ESTATE;
  if (!h->host_groups) {
    h->host_groups = static_cast<u64*>(pinned_take());
    if (!h->host_groups) return KMA_ENOMEM;
    for (auto& e : h->group_ev) KMA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (!h->copy_stream) KMA_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  // Everything counted so far: the keys in the table bound the records.
  int rc = read_status(h);
  if (rc) return rc;
  if ((rc = flags_to_code(h->host_status->flags))) { h->failed = true; return rc; }
  if ((rc = ensure_output(h, h->host_status->table_keys))) { h->failed = true; return rc; }
  KMA_CUDA(cudaMemsetAsync(&h->status->n_out, 0, 2 * sizeof(u64), h->stream));
  const bool parts = h->d.P > 1;
  const bool recount_parts = parts && h->p.use_bloom;
  const u64 S = h->d.plan.table_slots;
  const unsigned G = (unsigned)std::max<u64>(1, std::min<u64>(kFinalizeGroups, parts ? h->d.P : S / kClassTile));
  const PartGeom g = part_geom(h);
  // What the groups do not split: the one-table recount (a pass over the windows), or the
  // overflow records of every partition.
  if (h->p.use_bloom && !parts) {
    kma_handle* hs[1] = {h};
    if ((rc = enqueue_recount(hs, 1))) return rc;
  }
  if (recount_parts) {
    if ((rc = timed_launch(h, KMA_KERNEL_RECOUNT, h->stream, g.Wk > 0,
                           [&] { return launch_keyfilter_build(g, h->stream, h->num_sms); })))
      return rc;
    for (auto& rb : h->rec_batches) {
      PartRecords r = records_of(rb, h->d.P);
      r.p_end = 0;  // overflow area only
      if ((rc = timed_launch(h, KMA_KERNEL_RECOUNT, h->stream, true,
                             [&] { return launch_part_pass(g, r, kModeRecount, h->stream, h->num_sms); })))
        return rc;
    }
  }
  // Per group: recount its partitions, classify its slots (the records append to the output),
  // publish the record count so far.
  for (unsigned i = 0; i < G; ++i) {
    u64 s0, s1;
    if (parts) {
      const u64 p0 = h->d.P * i / G, p1 = h->d.P * (i + 1) / G;
      s0 = p0 * h->d.Sp;
      s1 = p1 * h->d.Sp;
      if (recount_parts) {
        for (auto& rb : h->rec_batches) {
          PartRecords r = records_of(rb, h->d.P);
          r.p_begin = (unsigned)p0;
          r.p_end = (unsigned)p1;
          r.overflow = 0;
          if ((rc = timed_launch(h, KMA_KERNEL_RECOUNT, h->stream, p1 > p0,
                                 [&] { return launch_part_pass(g, r, kModeRecount, h->stream, h->num_sms); })))
            return rc;
        }
      }
    } else {
      s0 = S * i / G;
      s1 = S * (i + 1) / G;
    }
    ClassBatch cb;
    std::memset(&cb, 0, sizeof(cb));
    cb.write = 1;
    cb.n = 1;
    cb.d[0] = class_desc(h);
    cb.d[0].table = h->table + s0;
    cb.d[0].slots = s1 - s0;
    cb.total_blocks = (s1 - s0 + kClassTile - 1) / kClassTile;
    if ((rc = timed_launch(h, KMA_KERNEL_CLASSIFY, h->stream, cb.total_blocks > 0,
                           [&] { return launch_classify(cb, h->stream, h->num_sms); })))
      return rc;
    KMA_CUDA(cudaMemcpyAsync(&h->host_groups[i], &h->status->n_out, sizeof(u64), cudaMemcpyDeviceToHost, h->stream));
    KMA_CUDA(cudaEventRecord(h->group_ev[i], h->stream));
  }
  KMA_CUDA(cudaMemcpyAsync(h->host_status, h->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
  // As each group completes, its records go to the host on the copy stream while the GPU
  // recounts the next group.
  const u64 cap = std::min<u64>(capacity, h->out_cap);
  u64 done = 0;
  for (unsigned i = 0; i < G; ++i) {
    KMA_CUDA(cudaEventSynchronize(h->group_ev[i]));
    const u64 upto = std::min<u64>(h->host_groups[i], cap);
    if (upto <= done) continue;
    const u64 n = upto - done;
    KMA_CUDA(cudaStreamWaitEvent(h->copy_stream, h->group_ev[i], 0));
    if (keys) KMA_CUDA(cudaMemcpyAsync(keys + 2 * done, h->out_keys + 2 * done, n * 16, cudaMemcpyDeviceToHost, h->copy_stream));
    if (counts) KMA_CUDA(cudaMemcpyAsync(counts + done, h->out_counts + done, n * 4, cudaMemcpyDeviceToHost, h->copy_stream));
    if (ext) KMA_CUDA(cudaMemcpyAsync(ext + 8 * done, h->out_ext + 8 * done, n * 32, cudaMemcpyDeviceToHost, h->copy_stream));
    if (codes) KMA_CUDA(cudaMemcpyAsync(codes + 2 * done, h->out_codes + 2 * done, n * 2, cudaMemcpyDeviceToHost, h->copy_stream));
    done = upto;
  }
  free_records(h);
  KMA_CUDA(cudaStreamSynchronize(h->stream));
  KMA_CUDA(cudaStreamSynchronize(h->copy_stream));
  if ((rc = flags_to_code(h->host_status->flags))) {
    h->failed = true;
    if (out) std::memset(out, 0, sizeof(kma_result));
    return rc;
  }
  fill_result(h);
  h->finalized = true;
  if (out) *out = h->res;
  return h->res.n > capacity ? KMA_EFULL : KMA_OK;
}

int kmer_analysis_query(kma_handle* h, const uint64_t* keys, uint64_t n, uint32_t* counts,
                        uint32_t* ext, uint8_t* codes, int on_device) {
  if (!h) return KMA_EINVAL;
  if (!h->finalized) return KMA_ESTATE;
  if (n == 0) return KMA_OK;
  if (!keys || !counts || !ext || !codes) return KMA_EINVAL;
  const unsigned min_ext = h->p.min_ext_count ? h->p.min_ext_count : 1;
  if (on_device) {
    return timed_launch(h, KMA_KERNEL_QUERY, h->stream, true, [&] {
      return launch_query(h->table, h->d.Sp, h->d.P, h->p.k, h->p.canonical, h->p.min_depth,
                          min_ext, (const u64*)keys, n, counts, ext, codes, h->status, h->stream);
    });
  }
  u64* dk = nullptr;
  unsigned *dc = nullptr, *de = nullptr;
  unsigned char* dcode = nullptr;
  int rc;
  if ((rc = dalloc(h, &dk, 2 * n)) || (rc = dalloc(h, &dc, n)) || (rc = dalloc(h, &de, 8 * n)) ||
      (rc = dalloc(h, &dcode, 2 * n))) {
    dfree(h, dk); dfree(h, dc); dfree(h, de); dfree(h, dcode);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(dk, keys, n * 16, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    rc = timed_launch(h, KMA_KERNEL_QUERY, h->stream, true, [&] {
      return launch_query(h->table, h->d.Sp, h->d.P, h->p.k, h->p.canonical, h->p.min_depth,
                          min_ext, dk, n, dc, de, dcode, h->status, h->stream);
    });
    if (rc) { dfree(h, dk); dfree(h, dc); dfree(h, de); dfree(h, dcode); return rc; }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dc, n * 4, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ext, de, n * 32, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(codes, dcode, n * 2, cudaMemcpyDeviceToHost, h->stream);
  dfree(h, dk); dfree(h, dc); dfree(h, de); dfree(h, dcode);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "query");
  return KMA_OK;
}

int kmer_analysis_reset(kma_handle* h) {
  if (!h) return KMA_EINVAL;
  return clear_state(h);
}

int kmer_analysis_set_stream(kma_handle* h, void* cuda_stream) {
  if (!h) return KMA_EINVAL;
  h->stream = (cudaStream_t)cuda_stream;
  return KMA_OK;
}

int kmer_analysis_status(kma_handle* h) {
  if (!h) return KMA_EINVAL;
  int rc = read_status(h);
  if (rc) return rc;
  return flags_to_code(h->host_status->flags);
}

uint64_t kmer_analysis_device_bytes(const kma_handle* h) {
  if (!h) return 0;
  return h->d.plan.device_bytes + h->out_cap * (16 + 4 + 32 + 2);
}

int kmer_analysis_set_profiling(kma_handle* h, int enable) {
  if (!h) return KMA_EINVAL;
  h->profiling = enable != 0;
  return KMA_OK;
}

int kmer_analysis_timings(kma_handle* h, kma_timings* out, int reset) {
  if (!h || !out) return KMA_EINVAL;
  KMA_CUDA(cudaStreamSynchronize(h->stream));
  for (auto& r : h->prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && r.kind >= 0 && r.kind < 8) h->ms[r.kind] += ms;
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->prof.clear();
  cudaGetLastError();
  std::memset(out, 0, sizeof(*out));
  for (int i = 0; i < 8; ++i) {
    out->ms[i] = h->ms[i];
    out->launches[i] = h->launches[i];
    out->total_launches += h->launches[i];
  }
  int rc = read_status(h);
  if (rc) return rc;
  out->first_sightings = h->host_status->first_sightings;
  if (reset) {
    for (int i = 0; i < 8; ++i) { h->ms[i] = 0; h->launches[i] = 0; }
  }
  return KMA_OK;
}

int kmer_analysis_contigs(kma_handle* h, kma_contigs* out) {
  if (!h || !out) return KMA_EINVAL;
  if (!h->finalized) return KMA_ESTATE;
  free_contigs(h);
  cudaError_t err = cudaSuccess;
  const int rc = contig_pass(h->out_keys, h->out_codes, h->res.n, h->p.k, h->p.canonical, h->pool, h->stream,
                             &h->contig_seq, &h->contig_offsets, &h->contig_n, &h->contig_bases,
                             &h->contig_vertices, &h->contig_cycles, &h->status->flags, &err);
  if (rc == KMA_ECUDA) return cuda_fail(err, "contig generation");
  if (rc) return rc;
  int st = read_status(h);
  if (st) return st;
  if (h->host_status->flags & kFlagFull) return KMA_EFULL;
  out->n_contigs = h->contig_n;
  out->n_bases = h->contig_bases;
  out->n_vertices = h->contig_vertices;
  out->n_cycles = h->contig_cycles;
  out->seq = h->contig_seq;
  out->offsets = (const uint64_t*)h->contig_offsets;
  return KMA_OK;
}

int kmer_analysis_copy_contigs(kma_handle* h, char* seq, uint64_t* offsets, int on_device) {
  if (!h) return KMA_EINVAL;
  if (!h->contig_offsets) return KMA_ESTATE;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (seq && h->contig_bases) KMA_CUDA(cudaMemcpyAsync(seq, h->contig_seq, h->contig_bases, kind, h->stream));
  if (offsets) KMA_CUDA(cudaMemcpyAsync(offsets, h->contig_offsets, (h->contig_n + 1) * 8, kind, h->stream));
  KMA_CUDA(cudaStreamSynchronize(h->stream));
  return KMA_OK;
}

int kmer_analysis_hll_estimate(const uint8_t* registers, uint32_t precision, double* distinct) {
  if (!registers || !distinct || precision < KMA_HLL_MIN_PRECISION || precision > KMA_HLL_MAX_PRECISION)
    return KMA_EINVAL;
  *distinct = hll_estimate(registers, precision);
  return KMA_OK;
}

int kmer_analysis_estimate(const kma_params* params, const char* seq, const char* qual,
                           const uint64_t* offsets, uint64_t n_reads, int on_device, void* cuda_stream,
                           kma_estimate* est, uint8_t* registers) {
  if (!params || !est || !offsets) return KMA_EINVAL;
  const unsigned p = est->precision ? est->precision : 14;
  if (p < KMA_HLL_MIN_PRECISION || p > KMA_HLL_MAX_PRECISION) return KMA_EINVAL;
  if (n_reads && (!seq || !qual)) return KMA_EINVAL;
  int rc = check_params(params);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // bases of the read set (device offsets: read back the two ends)
  u64 ends[2] = {0, 0};
  if (n_reads) {
    if (on_device) {
      KMA_CUDA(cudaMemcpyAsync(&ends[0], offsets, 8, cudaMemcpyDeviceToHost, stream));
      KMA_CUDA(cudaMemcpyAsync(&ends[1], offsets + n_reads, 8, cudaMemcpyDeviceToHost, stream));
      KMA_CUDA(cudaStreamSynchronize(stream));
    } else {
      ends[0] = offsets[0];
      ends[1] = offsets[n_reads];
    }
    if (ends[1] < ends[0]) return KMA_EINVAL;
  }
  // a handle that only packs: the read arena, no Bloom filter, a token table
  kma_params q = *params;
  q.use_bloom = 0;
  q.table_capacity = 64;
  q.expected_keys = 0;
  q.expected_distinct = 0;
  q.partitions = 1;
  q.fault_inject = 0;
  q.max_bases = std::max<u64>(q.max_bases, std::max<u64>(ends[1] - ends[0], 1));
  q.max_reads = std::max<u64>(q.max_reads, std::max<u64>(n_reads, 1));
  kma_handle* h = nullptr;
  if ((rc = kmer_analysis_create(&q, cuda_stream, &h))) return rc;
  h->pack_only = true;
  const u64 m = 1ull << p;
  std::vector<unsigned> regs32(m, 0);
  if (registers)
    for (u64 j = 0; j < m; ++j) regs32[j] = registers[j];
  // device temporaries: sketch registers, the CTAs' heavy-hitter summaries, and (host input)
  // the reads, copied whole so that they are packed as one batch (the sampled stream is
  // defined on the positions of one packed batch)
  const unsigned grid = hll_grid(p, h->num_sms);
  const u64 mg_n = (u64)grid * kMgBuckets * kMgCounters;
  std::vector<void*> temps;
  auto finish = [&](int code) {
    for (void* t : temps) cudaFreeAsync(t, h->stream);
    kmer_analysis_destroy(h);
    return code;
  };
  auto temp = [&](void** ptr, u64 bytes) -> int {
    cudaError_t e = cudaMallocFromPoolAsync(ptr, std::max<u64>(bytes, 16), h->pool, h->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *ptr = nullptr;
      return e == cudaErrorMemoryAllocation ? KMA_ENOMEM : cuda_fail(e, "estimate temporaries");
    }
    temps.push_back(*ptr);
    return KMA_OK;
  };
  unsigned* d_regs = nullptr;
  MgOut mg{nullptr, nullptr, nullptr, nullptr};
  if ((rc = temp((void**)&d_regs, m * 4)) || (rc = temp((void**)&mg.lo, mg_n * 8)) ||
      (rc = temp((void**)&mg.hi, mg_n * 8)) || (rc = temp((void**)&mg.count, mg_n * 4)) ||
      (rc = temp((void**)&mg.items, (u64)grid * kMgBuckets * 8)))
    return finish(rc);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_regs, regs32.data(), m * 4, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
    return finish(cuda_fail(e, "sketch registers in"));
  if (n_reads) {
    const char *s_in = seq, *q_in = qual;
    const uint64_t* o_in = offsets;
    if (!on_device) {
      const u64 nb = ends[1] - ends[0];
      void *ds = nullptr, *dq = nullptr, *dof = nullptr;
      if ((rc = temp(&ds, nb)) || (rc = temp(&dq, nb)) || (rc = temp(&dof, (n_reads + 1) * 8))) return finish(rc);
      if ((e = cudaMemcpyAsync(ds, seq + ends[0], nb, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
          (e = cudaMemcpyAsync(dq, qual + ends[0], nb, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
          (e = cudaMemcpyAsync(dof, offsets, (n_reads + 1) * 8, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
        return finish(cuda_fail(e, "estimate reads in"));
      // the device copy of the bases starts at offsets[0]
      s_in = (const char*)ds - ends[0];
      q_in = (const char*)dq - ends[0];
      o_in = (const uint64_t*)dof;
    }
    if ((rc = kmer_analysis_count(h, s_in, q_in, o_in, n_reads, 1))) return finish(rc);
  }
  PartWindows w;
  w.codes = h->codes; w.rcodes = h->rcodes; w.inv = h->inv; w.hq = h->hq;
  w.q0 = 0; w.q1 = h->q_used;
  const unsigned n_parts = params->n_parts > 1 ? params->n_parts : 1;
  const unsigned part = params->n_parts > 1 ? params->part : 0;
  if ((e = launch_hll(w, params->k, params->canonical, n_parts, part, p, d_regs, h->status, mg, grid,
                      h->stream)) != cudaSuccess)
    return finish(cuda_fail(e, "hll_kernel"));
  std::vector<u64> mlo(mg_n), mhi(mg_n), items((u64)grid * kMgBuckets);
  std::vector<unsigned> mcnt(mg_n);
  if ((e = cudaMemcpyAsync(regs32.data(), d_regs, m * 4, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(mlo.data(), mg.lo, mg_n * 8, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(mhi.data(), mg.hi, mg_n * 8, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(mcnt.data(), mg.count, mg_n * 4, cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(items.data(), mg.items, items.size() * 8, cudaMemcpyDeviceToHost, h->stream)) !=
          cudaSuccess)
    return finish(cuda_fail(e, "estimate results out"));
  if ((rc = read_status(h))) return finish(rc);
  if ((rc = flags_to_code(h->host_status->flags))) return finish(rc);
  std::vector<uint8_t> regs8(m);
  for (u64 j = 0; j < m; ++j) regs8[j] = (uint8_t)regs32[j];
  if (registers) std::memcpy(registers, regs8.data(), m);
  est->precision = p;
  est->distinct = hll_estimate(regs8.data(), p);
  est->rel_std_error = 1.04 / std::sqrt((double)m);
  est->valid_windows = h->host_status->valid_windows;
  // heavy hitters: merge the summaries, report the keys by count
  std::vector<u64> bucket_n(kMgBuckets, 0);
  for (unsigned c = 0; c < grid; ++c)
    for (unsigned b = 0; b < kMgBuckets; ++b) bucket_n[b] += items[(u64)c * kMgBuckets + b];
  std::vector<MgEntry> merged;
  mg_merge(mlo, mhi, mcnt, grid, merged);
  u64 sampled = 0;
  for (u64 x : bucket_n) sampled += x;
  est->sampled_windows = sampled;
  est->heavy_threshold = std::max<u64>(1, sampled / 2048);
  est->heavy_hitters = !merged.empty() && merged[0].count >= est->heavy_threshold ? 1u : 0u;
  est->n_summary = merged.size();
  const u64 rows = std::min<u64>(est->summary_capacity, merged.size());
  for (u64 i = 0; i < rows; ++i) {
    if (est->summary_keys) { est->summary_keys[2 * i] = merged[i].lo; est->summary_keys[2 * i + 1] = merged[i].hi; }
    if (est->summary_counts) est->summary_counts[i] = merged[i].count;
    if (est->summary_bucket) est->summary_bucket[i] = merged[i].bucket;
  }
  if (est->bucket_windows)
    for (unsigned b = 0; b < kMgBuckets; ++b) est->bucket_windows[b] = bucket_n[b];
  return finish(KMA_OK);
}

int kmer_analysis_parse_fastq(const char* text, uint64_t n_bytes, int on_device, char* seq, char* qual,
                              uint64_t* offsets, uint64_t cap_bases, uint64_t cap_reads, uint64_t* n_reads,
                              uint64_t* n_bases, void* cuda_stream) {
  if (!n_reads || !n_bases || !offsets || (n_bytes && !text)) return KMA_EINVAL;
  *n_reads = *n_bases = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, rc;
  KMA_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  if ((rc = get_pool(dev, &pool))) return rc;
  std::vector<void*> temps;
  auto alloc = [&](void** p, u64 bytes) -> int {
    cudaError_t e = cudaMallocFromPoolAsync(p, std::max<u64>(bytes, 8), pool, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? KMA_ENOMEM : cuda_fail(e, "fastq temporaries");
    }
    temps.push_back(*p);
    return KMA_OK;
  };
  auto done = [&](int code) {
    for (void* p : temps) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
    return code;
  };
#define FQ_CUDA(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return done(cuda_fail(e_, #call));      \
  } while (0)
  if (n_bytes == 0) {
    FQ_CUDA(cudaMemsetAsync(offsets, 0, 8, st));
    return done(KMA_OK);
  }
  const unsigned char* d_text = (const unsigned char*)text;
  if (!on_device) {
    void* t = nullptr;
    if ((rc = alloc(&t, n_bytes))) return done(rc);
    FQ_CUDA(cudaMemcpyAsync(t, text, n_bytes, cudaMemcpyHostToDevice, st));
    d_text = (const unsigned char*)t;
  }
  // 1-2: newlines per chunk, scanned (one extra element receives the total)
  const u64 chunks = fastq_chunks(n_bytes);
  u64 *cc = nullptr, *tmp = nullptr;
  if ((rc = alloc((void**)&cc, (chunks + 1) * 8)) ||
      (rc = alloc((void**)&tmp, scan_scratch_items(std::max<u64>(chunks + 1, 1)) * 8)))
    return done(rc);
  FQ_CUDA(launch_fastq_count(d_text, n_bytes, cc, st));
  FQ_CUDA(cudaMemsetAsync(cc + chunks, 0, 8, st));
  FQ_CUDA(scan_exclusive(cc, chunks + 1, tmp, st));
  u64 n_lines = 0;
  FQ_CUDA(cudaMemcpyAsync(&n_lines, cc + chunks, 8, cudaMemcpyDeviceToHost, st));
  FQ_CUDA(cudaStreamSynchronize(st));
  // 3: line ends
  u64* line_end = nullptr;
  if ((rc = alloc((void**)&line_end, n_lines * 8))) return done(rc);
  FQ_CUDA(launch_fastq_lines(d_text, n_bytes, cc, line_end, st));
  // lines after the last complete record must be empty
  const u64 extra = n_lines % 4;
  if (extra) {
    const u64 first = n_lines - extra;  // first extra line
    u64 ends[4] = {0, 0, 0, 0};
    const u64 from = first ? first - 1 : 0, cnt = first ? extra + 1 : extra;
    FQ_CUDA(cudaMemcpyAsync(ends, line_end + from, cnt * 8, cudaMemcpyDeviceToHost, st));
    FQ_CUDA(cudaStreamSynchronize(st));
    u64 prev_end = first ? ends[0] : (u64)-1;  // (u64)-1 + 1 == 0: the text's first byte
    for (u64 i = 0; i < extra; ++i) {
      const u64 e = ends[first ? i + 1 : i];
      const u64 len = e - (prev_end + 1);
      if (len > 1) return done(KMA_EINVAL);
      if (len == 1) {  // a lone '\r' is an empty line too
        char c = 0;
        FQ_CUDA(cudaMemcpyAsync(&c, d_text + prev_end + 1, 1, cudaMemcpyDeviceToHost, st));
        FQ_CUDA(cudaStreamSynchronize(st));
        if (c != '\r') return done(KMA_EINVAL);
      }
      prev_end = e;
    }
  }
  const u64 nr = (n_lines - extra) / 4;
  *n_reads = nr;
  if (nr > cap_reads) return done(KMA_EFULL);
  // 4-5: record checks, bases per record, scanned into the offsets
  unsigned long long* bad = nullptr;
  if ((rc = alloc((void**)&bad, 8))) return done(rc);
  u64* scan_tmp = nullptr;
  if ((rc = alloc((void**)&scan_tmp, scan_scratch_items(nr + 1) * 8))) return done(rc);
  FQ_CUDA(cudaMemsetAsync(bad, 0xFF, 8, st));
  FQ_CUDA(launch_fastq_records(d_text, line_end, nr, (u64*)offsets, bad, st));
  FQ_CUDA(cudaMemsetAsync(offsets + nr, 0, 8, st));
  FQ_CUDA(scan_exclusive((u64*)offsets, nr + 1, scan_tmp, st));
  u64 back[2] = {0, 0};
  FQ_CUDA(cudaMemcpyAsync(&back[0], offsets + nr, 8, cudaMemcpyDeviceToHost, st));
  FQ_CUDA(cudaMemcpyAsync(&back[1], bad, 8, cudaMemcpyDeviceToHost, st));
  FQ_CUDA(cudaStreamSynchronize(st));
  if (back[1] != ~0ull) return done(KMA_EINVAL);
  *n_bases = back[0];
  if (back[0] > cap_bases) return done(KMA_EFULL);
  if (nr && (!seq || !qual)) return done(KMA_EINVAL);
  // 6: bases and qualities
  FQ_CUDA(launch_fastq_copy(d_text, line_end, nr, (const u64*)offsets, (unsigned char*)seq,
                            (unsigned char*)qual, st));
  return done(KMA_OK);
#undef FQ_CUDA
}

void kmer_analysis_destroy(kma_handle* h) {
  if (!h) return;
  free_all(h);
  delete h;
}

const char* kmer_analysis_strerror(int code) {
  switch (code) {
    case KMA_OK: return "ok";
    case KMA_EINVAL: return "invalid argument";
    case KMA_ENOMEM: return "out of device memory";
    case KMA_EFULL: return "capacity exceeded (hash table or read arena)";
    case KMA_ESTATE: return "call not allowed in this state";
    case KMA_ETIMEOUT: return "device wait timed out";
    case KMA_EOVERFLOW: return "k-mer counter overflow";
    case KMA_ECUDA: return g_last_cuda_error.empty() ? "CUDA error" : g_last_cuda_error.c_str();
    case KMA_ETOOLARGE: return "input exceeds a fixed limit (allocation-free scratch, or 2^31 contig vertices)";
    default: return "unknown error";
  }
}

}  // extern "C"
