// Allocation-free k-mer counting for small read sets.
//
// kmer_analysis_count_small_noalloc runs the same kernels as the handle-based path (read
// packing, counting pass, classification and compaction) but keeps all of its working memory
// (packed reads, hash table, status words) in one file-scope device array of fixed size
// instead of allocating it. It exists for callers that must not allocate device memory at
// the point where they count: code that owns a fixed memory budget set up at start-up,
// framework plugins whose host application manages every device allocation, and paths with
// a no-allocation-after-initialisation rule. The caller provides the inputs and the output
// arrays; nothing is allocated by this file, neither by cudaMalloc nor by any allocating
// library routine.
//
// Every GPU that loads this library holds the array (kNoallocScratchBytes, about 34 MB)
// until the process exits. All calls share it and it keeps the last call's contents, so every
// call clears what must start empty (status words, read arena, table) before it uses them.
// Calls whose GPU work overlaps (different streams, or host threads without ordering)
// race on the shared array and give wrong results: order them on one stream.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/kmer_analysis.h"
#include "kma_internal.cuh"

using namespace kma;
typedef unsigned long long u64;

namespace {

// Fixed limits (also published in the header as KMA_NOALLOC_MAX_BASES / _MAX_READS).
constexpr u64 kMaxBases = KMA_NOALLOC_MAX_BASES;
constexpr u64 kMaxReads = KMA_NOALLOC_MAX_READS;
constexpr u64 kMaxPositions = ((kMaxBases + kMaxReads + 63) / 64) * 64 + 256;
constexpr u64 kMaxSlots = 2 * kMaxBases;  // load <= 0.5: distinct k-mers <= windows <= bases

constexpr u64 align256(u64 x) { return (x + 255) / 256 * 256; }
constexpr u64 kCodesBytes = align256((kMaxPositions / 32 + 4) * 8);
constexpr u64 kBitsBytes = align256((kMaxPositions / 64 + 4) * 8);
constexpr u64 kStatusBytes = align256(sizeof(DevStatus));
constexpr u64 kTableBytes = kMaxSlots * sizeof(Slot);
constexpr u64 kOffCodes = 0;
constexpr u64 kOffRcodes = kOffCodes + kCodesBytes;
constexpr u64 kOffInv = kOffRcodes + kCodesBytes;
constexpr u64 kOffHq = kOffInv + kBitsBytes;
constexpr u64 kOffStatus = kOffHq + kBitsBytes;
constexpr u64 kOffTable = kOffStatus + kStatusBytes;
constexpr u64 kNoallocScratchBytes = kOffTable + kTableBytes;

// The scratch array. In host code `g_noalloc_scratch` is only a stand-in symbol, not a device
// address: kernels get the address from cudaGetSymbolAddress (scratch_address below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// The device address of the array in the current device's context. It is looked up on every
// call: a cached address would go stale if the process reset the device (cudaDeviceReset) or
// otherwise made a new context, where the module, and the array with it, is loaded anew. The
// lookup is a host-side query and the call synchronises with its stream anyway.
int scratch_address(unsigned char** out) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
    cudaGetLastError();
    return KMA_ECUDA;
  }
  *out = static_cast<unsigned char*>(ptr);
  return KMA_OK;
}

int check(cudaError_t e) {
  if (e == cudaSuccess) return KMA_OK;
  cudaGetLastError();
  return KMA_ECUDA;
}

}  // namespace

extern "C" int kmer_analysis_count_small_noalloc(const kma_params* params, const char* seq,
                                                 const char* qual, const uint64_t* offsets,
                                                 uint64_t n_reads, uint64_t n_bases,
                                                 uint64_t* keys, uint32_t* counts, uint32_t* ext,
                                                 uint8_t* codes, uint64_t capacity,
                                                 uint64_t* n_out, void* cuda_stream) {
  if (n_out) *n_out = 0;
  if (!params || !n_out) return KMA_EINVAL;
  const kma_params& p = *params;
  if (p.k < 1 || p.k > 63 || (p.canonical && p.k % 2 == 0) || p.min_depth < 1) return KMA_EINVAL;
  if (n_bases > kMaxBases || n_reads > kMaxReads) return KMA_ETOOLARGE;
  if (n_reads && (!seq || !qual || !offsets)) return KMA_EINVAL;
  if (capacity && (!keys || !counts || !ext || !codes)) return KMA_EINVAL;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int dev = 0, num_sms = 0, rc;
  if ((rc = check(cudaGetDevice(&dev)))) return rc;
  if ((rc = check(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev)))) return rc;
  unsigned char* base = nullptr;
  if ((rc = scratch_address(&base))) return rc;

  u64* d_codes = reinterpret_cast<u64*>(base + kOffCodes);
  u64* d_rcodes = reinterpret_cast<u64*>(base + kOffRcodes);
  u64* d_inv = reinterpret_cast<u64*>(base + kOffInv);
  u64* d_hq = reinterpret_cast<u64*>(base + kOffHq);
  DevStatus* d_status = reinterpret_cast<DevStatus*>(base + kOffStatus);
  Slot* d_table = reinterpret_cast<Slot*>(base + kOffTable);

  const u64 n_pos = n_reads ? ((n_bases + n_reads + 63) / 64) * 64 : 0;
  const u64 slots = n_pos ? ((2 * n_bases + 64 < kMaxSlots) ? 2 * n_bases + 64 : kMaxSlots) : 64;
  const u64 codes_words = n_pos / 32 + 4, bit_words = n_pos / 64 + 4;

  // Clear what must start empty: the array keeps the previous call's contents.
  if ((rc = check(cudaMemsetAsync(d_status, 0, sizeof(DevStatus), stream)))) return rc;
  if ((rc = check(cudaMemsetAsync(d_codes, 0, codes_words * 8, stream)))) return rc;
  if ((rc = check(cudaMemsetAsync(d_rcodes, 0xFF, codes_words * 8, stream)))) return rc;
  if ((rc = check(cudaMemsetAsync(d_inv, 0xFF, bit_words * 8, stream)))) return rc;
  if ((rc = check(cudaMemsetAsync(d_hq, 0, bit_words * 8, stream)))) return rc;
  if ((rc = check(launch_table_init(d_table, slots, stream)))) return rc;

  if (n_pos) {
    PackBatch pb;
    std::memset(&pb, 0, offsetof(PackBatch, d) + sizeof(PackDesc));
    pb.n = 1;
    pb.wait_limit = kWaitPolls;
    PackDesc& pd = pb.d[0];
    pd.seq = reinterpret_cast<const unsigned char*>(seq);
    pd.qual = reinterpret_cast<const unsigned char*>(qual);
    pd.offsets = reinterpret_cast<const unsigned long long*>(offsets);
    pd.delta = 0;
    pd.n_reads = n_reads;
    pd.n_bases = n_bases;
    pd.q0 = 0;
    pd.n_pos = n_pos;
    pd.chunk_begin = 0;
    pd.codes = d_codes;
    pd.rcodes = d_rcodes;
    pd.inv = d_inv;
    pd.hq = d_hq;
    pd.status = d_status;
    pd.qual_min = (unsigned)p.qual_offset + (unsigned)p.qual_threshold;
    pb.total_chunks = (n_pos / 64 + kPackChunkWords - 1) / kPackChunkWords;
    if ((rc = check(launch_pack(pb, stream, num_sms)))) return rc;

    PassBatch b;
    std::memset(&b, 0, offsetof(PassBatch, d) + sizeof(PassDesc));
    b.n = 1;
    PassDesc& d = b.d[0];
    d.codes = d_codes;
    d.rcodes = d_rcodes;
    d.inv = d_inv;
    d.hq = d_hq;
    d.table = d_table;
    d.status = d_status;
    d.slots = slots;
    d.q0 = 0;
    d.q1 = n_pos;
    d.k = p.k;
    d.canonical = p.canonical;
    d.mode = kModeCount;  // every window straight into the table: no Bloom filter to hold
    d.n_parts = 1;
    d.no_overflow = 1;    // at most n_pos < 2^32 occurrences per key
    LaunchShape shape{256, 2, num_sms * 2};
    b.total_tiles = (n_pos + 511) / 512;
    if ((rc = check(launch_pass(b, shape, false, stream)))) return rc;
  }

  ClassBatch cb;
  std::memset(&cb, 0, offsetof(ClassBatch, d) + sizeof(ClassDesc));
  cb.n = 1;
  cb.write = 1;
  ClassDesc& c = cb.d[0];
  c.table = d_table;
  c.status = d_status;
  c.slots = slots;
  c.out_keys = reinterpret_cast<unsigned long long*>(keys);
  c.out_counts = counts;
  c.out_ext = ext;
  c.out_codes = codes;
  c.out_cap = capacity;
  c.min_depth = p.min_depth;
  c.min_ext = p.min_ext_count ? p.min_ext_count : 1;
  cb.total_blocks = (slots + 1023) / 1024;
  if ((rc = check(launch_classify(cb, stream, num_sms)))) return rc;

  DevStatus st;
  if ((rc = check(cudaMemcpyAsync(&st, d_status, sizeof(st), cudaMemcpyDeviceToHost, stream)))) return rc;
  if ((rc = check(cudaStreamSynchronize(stream)))) return rc;
  *n_out = st.n_out;
  if (st.flags & kFlagTimeout) return KMA_ETIMEOUT;
  if (st.flags & kFlagBadOffsets) return KMA_EINVAL;
  if (st.n_out > capacity) return KMA_EFULL;  // *n_out tells the caller the size it needs
  if (st.flags & kFlagFull) return KMA_EFULL;
  if (st.flags & kFlagOverflow) return KMA_EOVERFLOW;
  return KMA_OK;
}
