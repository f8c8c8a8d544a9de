// HyperLogLog cardinality pass (HipMer, arXiv 1705.11147, Section 5.1): one streaming pass
// over the packed reads estimates the number of distinct canonical k-mers, so that the Bloom
// filter can be sized before counting.
//
// Sketch: m = 2^p registers. Every valid window's canonical key is hashed to 64 bits
// (key_hash); the top p bits pick register j, and the register keeps the largest rank seen,
// rank = 1 + the number of leading zeros of the remaining 64 - p bits (64 - p + 1 when they
// are all zero). The registers depend only on the set of distinct keys, and sketches of
// several read sets (or of several GPUs' owner partitions) merge by taking the elementwise
// maximum. The estimate itself is computed on the host (kma_api.cu).
//
// Each CTA keeps its own registers in shared memory (32-bit words, shared-memory atomicMax),
// walks tiles of 4096 window starts with the same rolling extraction as the scatter, and
// merges its registers into the global ones once at the end.
//
// Heavy hitters (Section 5.1: frequent k-mers are identified during this same pass, so that
// they can be accumulated locally before the global update). The windows that start at every
// 2^kMgSampleShift-th arena position form the sampled stream; it is split by the top
// kMgBucketBits bits of the key hash into kMgBuckets sub-streams, and every CTA keeps one
// Misra-Gries summary of kMgCounters counters per sub-stream. An item whose key holds a
// counter increments it; a new key takes a counter at zero if there is one; otherwise every
// counter of that summary is decremented. A summary of a sub-stream of n items then holds every
// key with frequency f > n / (m + 1), with a count in [f - n / (m + 1), f]. Warp w updates
// the summaries of buckets w and w + 16, one item at a time, a counter per lane. The host
// merges the CTAs' summaries bucket by bucket (counts of a key summed, the (m+1)-th largest
// subtracted, non-positive ones dropped), which keeps the bound for the whole sub-stream.
#include "kma_device.cuh"

namespace kma {

constexpr int kHllThreads = 512;
constexpr int kHllWpt = 8;
constexpr int kHllTile = kHllThreads * kHllWpt;
constexpr int kHllWarps = kHllThreads / 32;
constexpr int kMgItemsPerTile = kHllTile >> kMgSampleShift;  // at most one per 2^kMgSampleShift window starts
static_assert(kMgCounters == 32 && kMgBuckets == 2 * kHllWarps, "one counter per lane, two buckets per warp");

__host__ __device__ constexpr size_t hll_smem(unsigned p) {
  return ((size_t)4 << p) +                                   // HLL registers
         (size_t)kMgBuckets * kMgCounters * (8 + 8 + 4) +     // summaries: key lo, hi, count
         (size_t)kMgItemsPerTile * (8 + 8 + 4) +              // the tile's sampled items: lo, hi, bucket
         (size_t)kMgBuckets * 8 + 16;                         // items per bucket, item count
}

__global__ void __launch_bounds__(kHllThreads) hll_kernel(const __grid_constant__ PartWindows W, unsigned k,
                                                          unsigned canonical, unsigned n_parts, unsigned part,
                                                          unsigned p, unsigned* regs, DevStatus* st,
                                                          const __grid_constant__ MgOut mg) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const unsigned m = 1u << p;
  u64* mg_lo = reinterpret_cast<u64*>(s_raw);                       // [buckets * counters]
  u64* mg_hi = mg_lo + kMgBuckets * kMgCounters;
  u64* it_lo = mg_hi + kMgBuckets * kMgCounters;                    // [items per tile]
  u64* it_hi = it_lo + kMgItemsPerTile;
  u64* mg_n = it_hi + kMgItemsPerTile;                              // [buckets]
  unsigned* mg_c = reinterpret_cast<unsigned*>(mg_n + kMgBuckets);  // [buckets * counters]
  unsigned* it_b = mg_c + kMgBuckets * kMgCounters;                 // [items per tile]
  unsigned* s_nit = it_b + kMgItemsPerTile;
  unsigned* s_reg = s_nit + 4;                                      // [2^p]
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned i = threadIdx.x; i < m; i += blockDim.x) s_reg[i] = 0;
  for (unsigned i = threadIdx.x; i < kMgBuckets * kMgCounters; i += blockDim.x) mg_c[i] = 0;
  if (threadIdx.x < kMgBuckets) mg_n[threadIdx.x] = 0;
  if (threadIdx.x == 0) *s_nit = 0;
  __syncthreads();
  const u64 n_tiles = (W.q1 - W.q0 + kHllTile - 1) / kHllTile;
  unsigned acc_valid = 0;
  for (u64 t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const u64 q = W.q0 + t * kHllTile + (u64)threadIdx.x * kHllWpt;
    if (q < W.q1) {  // q1 - q0 is a multiple of 64: all kHllWpt starts are inside
      RollingWindows rw;
      rw.init(W, k, q);
#pragma unroll
      for (int j = 0; j < kHllWpt; ++j) {
        Window w;
        if (rw.get(j, canonical, w)) {
          const u64 h = key_hash(w.lo, w.hi);
          if (n_parts <= 1 || owner_of(h, n_parts) == part) {
            ++acc_valid;
            const unsigned idx = (unsigned)(h >> (64 - p));
            const u64 rest = h << p;
            const unsigned rank = rest ? (unsigned)__clzll(rest) + 1u : 64u - p + 1u;
            atomicMax(&s_reg[idx], rank);
            if (mg.lo && (((q + j) & ((1u << kMgSampleShift) - 1)) == 0)) {  // sampled window
              const unsigned slot = atomicAdd(s_nit, 1u);
              it_lo[slot] = w.lo;
              it_hi[slot] = w.hi;
              it_b[slot] = (unsigned)(h >> (64 - kMgBucketBits));
            }
          }
        }
        if (j + 1 < kHllWpt) rw.roll();
      }
    }
    if (!mg.lo) continue;  // block-uniform
    __syncthreads();
    const unsigned n_items = *s_nit;
    __syncthreads();
    if (threadIdx.x == 0) *s_nit = 0;  // every thread has read the count
    // warp w: the items of buckets w and w + kHllWarps, in list order
    for (unsigned c = 0; c < n_items; c += 32) {
      const unsigned i = c + lane;
      unsigned own = __ballot_sync(0xffffffffu, i < n_items && (it_b[i] % kHllWarps) == warp);
      while (own) {
        const unsigned x = c + __ffs(own) - 1;
        own &= own - 1;
        const unsigned b = it_b[x];
        const u64 klo = it_lo[x], khi = it_hi[x];
        const unsigned s = b * kMgCounters + lane;
        const unsigned cc = mg_c[s];
        const bool match = cc && mg_lo[s] == klo && mg_hi[s] == khi;
        if (__ballot_sync(0xffffffffu, match)) {
          if (match) mg_c[s] = cc + 1;
        } else {
          const unsigned fm = __ballot_sync(0xffffffffu, cc == 0);
          if (fm) {
            if (lane == (unsigned)__ffs(fm) - 1) {
              mg_lo[s] = klo;
              mg_hi[s] = khi;
              mg_c[s] = 1;
            }
          } else {
            mg_c[s] = cc - 1;  // no free counter: every counter of the summary loses one
          }
        }
        if (lane == 0) mg_n[b] += 1;
        __syncwarp();
      }
    }
    __syncthreads();  // the item list is refilled by the next tile
  }
  __syncthreads();
  for (unsigned i = threadIdx.x; i < m; i += blockDim.x)
    if (s_reg[i]) atomicMax(&regs[i], s_reg[i]);
  if (mg.lo) {  // this CTA's summaries
    const u64 o = (u64)blockIdx.x * kMgBuckets * kMgCounters;
    for (unsigned i = threadIdx.x; i < kMgBuckets * kMgCounters; i += blockDim.x) {
      const unsigned c = mg_c[i];
      mg.count[o + i] = c;
      mg.lo[o + i] = c ? mg_lo[i] : 0ull;
      mg.hi[o + i] = c ? mg_hi[i] : 0ull;
    }
    if (threadIdx.x < kMgBuckets) mg.items[(u64)blockIdx.x * kMgBuckets + threadIdx.x] = mg_n[threadIdx.x];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc_valid += __shfl_down_sync(0xffffffffu, acc_valid, o);
  if ((threadIdx.x & 31) == 0 && acc_valid) atomicAdd(&st->valid_windows, (u64)acc_valid);
}

unsigned hll_grid(unsigned p, int num_sms) {
  int per_sm = 0;
  if (allow_dynamic_smem((const void*)hll_kernel, hll_smem(p)) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hll_kernel, kHllThreads, hll_smem(p)) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (unsigned)num_sms * (unsigned)(per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_hll(const PartWindows& w, unsigned k, unsigned canonical, unsigned n_parts, unsigned part,
                       unsigned p, unsigned* regs, DevStatus* st, const MgOut& mg, unsigned grid,
                       cudaStream_t stream) {
  const size_t smem = hll_smem(p);
  cudaError_t e = allow_dynamic_smem((const void*)hll_kernel, smem);
  if (e != cudaSuccess) return e;
  // every CTA runs (and writes its summaries) even when there are fewer tiles than CTAs
  hll_kernel<<<grid, kHllThreads, smem, stream>>>(w, k, canonical, n_parts, part, p, regs, st, mg);
  return cudaGetLastError();
}

}  // namespace kma
