// Partitioned mode of the counting passes: the paper's owner-computes scheme (Section 5.1:
// a deterministic k-mer -> owner map, every owner counting in a local table behind its own
// Bloom filter) applied on one GPU, with L2-sized partitions as the owners.
//
//   part_scatter_kernel  each window becomes a record {canonical key, extension info byte},
//                        appended to its partition's bucket (streaming writes); buckets
//                        have a fixed capacity and spill into a shared overflow area
//   part_pass_kernel     buckets processed in order: Bloom test-and-set in the partition's
//                        sub-filter, insert/count in its sub-table, or (recount) the first
//                        sightings added to k-mers that reached the table
//
// The random atomics of one partition touch only its sub-filter and sub-table, sized to stay
// resident in L2, instead of the whole multi-GB filter and table in HBM.
#include "kma_device.cuh"

namespace kma {

__device__ __forceinline__ unsigned char info_of(const Window& w) {
  return (unsigned char)(w.lb | ((unsigned)w.lu << 2) | (w.rb << 3) | ((unsigned)w.ru << 5));
}

__device__ __forceinline__ void window_of(unsigned char inf, Window& w) {
  w.lb = inf & 3u;
  w.lu = (inf >> 2) & 1u;
  w.rb = (inf >> 3) & 3u;
  w.ru = (inf >> 5) & 1u;
}

// Window at q of the batch, canonical key hashed, owner filter applied.
__device__ __forceinline__ bool part_window(const PartGeom& G, const PartWindows& W, u64 q,
                                            Window& w, u64& h) {
  if (!load_window(W.codes, W.rcodes, W.inv, W.hq, G.k, G.canonical, q, w)) return false;
  h = key_hash(w.lo, w.hi);
  if (G.n_parts > 1 && owner_of(h, G.n_parts) != G.part) return false;
  return true;
}

constexpr int kPartThreads = 256;

// ------------------------------------------------------------------ scatter
//
// One tile = kPartThreads * kScatterWpt consecutive window starts.
//  1. extract the windows, stage key + info in shared memory, rank each window inside its
//     partition for this tile (shared-memory atomics);
//  2. exclusive scan of the per-partition counts (the tile's records sorted by partition) and
//     one global reservation per partition present (bucket part, overflow part);
//  3. permute the staged records into partition order and write them out: consecutive
//     threads write consecutive records of the same bucket, so the stores coalesce.

constexpr int kScatterWpt = 16;
constexpr int kScatterTile = kPartThreads * kScatterWpt;  // 4096 (< 2^13: ranks and slots fit)

__host__ __device__ constexpr size_t scatter_smem(unsigned P, int kw) {
  return (size_t)kScatterTile * (kw * 8) +   // staged keys
         (size_t)kScatterTile +              // staged info
         (size_t)kScatterTile * 4 +          // sorted order: slot | partition << 16
         (size_t)P * (4 + 4 + 4 + 8 + 8) +   // cnt, off, n1, gbase, obase
         256;                                // warp sums, tile total, alignment
}

template <int KW>
__global__ void __launch_bounds__(kPartThreads) part_scatter_kernel(const __grid_constant__ PartGeom G,
                                                                    const __grid_constant__ PartWindows W,
                                                                    const __grid_constant__ PartRecords R) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const unsigned P = G.P;
  u64* s_keys = reinterpret_cast<u64*>(s_raw);                                   // [tile * KW]
  u64* s_gbase = s_keys + (size_t)kScatterTile * KW;                             // [P]
  u64* s_obase = s_gbase + P;                                                    // [P]
  unsigned* s_order = reinterpret_cast<unsigned*>(s_obase + P);                  // [tile]
  unsigned* s_cnt = s_order + kScatterTile;                                      // [P]
  unsigned* s_off = s_cnt + P;                                                   // [P]
  unsigned* s_n1 = s_off + P;                                                    // [P]
  unsigned* s_wsum = s_n1 + P;                                                   // [8 + 1]
  unsigned char* s_info = reinterpret_cast<unsigned char*>(s_wsum + 16);         // [tile]
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const u64 n_tiles = (W.q1 - W.q0 + kScatterTile - 1) / kScatterTile;
  const u64 pol = policy_evict_first();
  u64 acc_valid = 0;
  for (unsigned p = threadIdx.x; p < P; p += blockDim.x) s_cnt[p] = 0;
  __syncthreads();
  for (u64 t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    // 1: windows -> staged records, rank inside the partition
    unsigned pr[kScatterWpt];  // partition << 13 | rank, or ~0u
#pragma unroll
    for (int j = 0; j < kScatterWpt; ++j) {
      const unsigned slot = j * kPartThreads + threadIdx.x;
      const u64 q = W.q0 + t * kScatterTile + slot;
      pr[j] = 0xFFFFFFFFu;
      Window w;
      u64 h = 0;
      const bool ok = (q - lane) < W.q1 && q < W.q1 && part_window(G, W, q, w, h);
      acc_valid += __popc(__ballot_sync(0xffffffffu, ok));
      if (ok) {
        const unsigned p = part_of(h, P);
        pr[j] = (p << 13) | atomicAdd(&s_cnt[p], 1u);
        s_keys[(size_t)slot * KW] = w.lo;
        if (KW == 2) s_keys[(size_t)slot * KW + 1] = w.hi;
        s_info[slot] = info_of(w);
      }
    }
    __syncthreads();
    // 2a: exclusive scan of the counts (each thread a contiguous chunk of partitions)
    const unsigned per = (P + kPartThreads - 1) / kPartThreads;
    const unsigned p0 = threadIdx.x * per, p1 = min(P, p0 + per);
    unsigned local = 0;
    for (unsigned p = p0; p < p1; ++p) local += s_cnt[p];
    unsigned incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += v;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned run = 0;
      for (int x = 0; x < kPartThreads / 32; ++x) {
        const unsigned v = s_wsum[x];
        s_wsum[x] = run;
        run += v;
      }
      s_wsum[8] = run;  // records in this tile
    }
    __syncthreads();
    unsigned run = s_wsum[warp] + incl - local;
    for (unsigned p = p0; p < p1; ++p) {
      s_off[p] = run;
      run += s_cnt[p];
    }
    // 2b: reserve each partition's run: bucket first, the rest in the overflow area
    for (unsigned p = threadIdx.x; p < P; p += blockDim.x) {
      const unsigned c = s_cnt[p];
      if (c) {
        const u64 b = atomicAdd(&R.fill[p], (u64)c);
        const u64 room = b < R.cap ? R.cap - b : 0;
        const unsigned n1 = (unsigned)(room < c ? room : c);
        s_gbase[p] = (u64)p * R.cap + (b < R.cap ? b : 0);
        s_n1[p] = n1;
        s_obase[p] = n1 < c ? atomicAdd(&R.fill[P], (u64)(c - n1)) : 0;
      }
    }
    __syncthreads();
    // 3a: sorted order (partition-major) of the staged records
#pragma unroll
    for (int j = 0; j < kScatterWpt; ++j) {
      if (pr[j] == 0xFFFFFFFFu) continue;
      const unsigned p = pr[j] >> 13, r = pr[j] & 8191u;
      s_order[s_off[p] + r] = (j * kPartThreads + threadIdx.x) | (p << 16);
    }
    for (unsigned p = threadIdx.x; p < P; p += blockDim.x) s_cnt[p] = 0;  // for the next tile
    __syncthreads();
    // 3b: write out in sorted order (coalesced runs per bucket)
    const unsigned total = s_wsum[8];
    for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
      const unsigned e = s_order[i];
      const unsigned slot = e & 0xFFFFu, p = e >> 16;
      const unsigned r = i - s_off[p];
      u64 gi;
      if (r < s_n1[p]) {
        gi = s_gbase[p] + r;
      } else {
        const u64 o = s_obase[p] + (r - s_n1[p]);
        if (o >= R.ocap) {  // overflow area full: reported, never dropped silently
          atomicOr(&G.status->flags, kFlagFull);
          continue;
        }
        gi = (u64)P * R.cap + o;
      }
      if (KW == 1) {
        st_stream(reinterpret_cast<u64*>(R.keys) + gi, s_keys[slot], pol);
      } else {
        st_stream(reinterpret_cast<ulonglong2*>(R.keys) + gi,
                  make_ulonglong2(s_keys[(size_t)slot * 2], s_keys[(size_t)slot * 2 + 1]), pol);
      }
      st_stream(R.info + gi, s_info[slot], pol);
    }
    __syncthreads();  // staged records and per-partition runs are reused by the next tile
  }
  if (lane == 0 && acc_valid) atomicAdd(&G.status->valid_windows, acc_valid);
}

// ------------------------------------------------------------------ record pass
//
// Tiles walk the buckets in partition order (then the overflow area), so at any moment the
// CTAs work on one or two partitions whose sub-filter and sub-table sit in L2.


template <int KW, int kRecPerThread>
__global__ void __launch_bounds__(kPartThreads) part_pass_kernel(const __grid_constant__ PartGeom G,
                                                                 const __grid_constant__ PartRecords R,
                                                                 unsigned mode) {
  constexpr int kRecTile = kPartThreads * kRecPerThread;
  const unsigned lane = threadIdx.x & 31;
  const u64 tpb = (R.cap + kRecTile - 1) / kRecTile;          // tiles per bucket
  const u64 otiles = (R.ocap + kRecTile - 1) / kRecTile;
  const u64 n_tiles = (u64)G.P * tpb + otiles;
  u64 acc_ins = 0, acc_first = 0;
  const u64 pol = policy_evict_first();
  for (u64 t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    // record range of this tile
    u64 base, end;
    if (t < (u64)G.P * tpb) {
      const u64 b = t / tpb;
      const u64 f = R.fill[b] < R.cap ? R.fill[b] : R.cap;
      const u64 lo = (t - b * tpb) * kRecTile;
      if (lo >= f) continue;  // tile-uniform
      base = b * R.cap + lo;
      end = b * R.cap + f;
    } else {
      const u64 f = R.fill[G.P] < R.ocap ? R.fill[G.P] : R.ocap;
      const u64 lo = (t - (u64)G.P * tpb) * kRecTile;
      if (lo >= f) continue;
      base = (u64)G.P * R.cap + lo;
      end = (u64)G.P * R.cap + f;
    }
    Window w[kRecPerThread];
    u64 h[kRecPerThread], idx[kRecPerThread];
    unsigned p[kRecPerThread];
    unsigned char inf[kRecPerThread];
    bool act[kRecPerThread];
    // stage 1: records (coalesced, streamed)
#pragma unroll
    for (int j = 0; j < kRecPerThread; ++j) {
      const u64 i = base + (u64)j * blockDim.x + threadIdx.x;
      act[j] = i < end;
      h[j] = 0;
      p[j] = 0;
      inf[j] = 0;
      if (act[j]) {
        inf[j] = (unsigned char)ld_stream(R.info + i, pol);
        if (mode == kModeRecount && !(inf[j] & kInfoFirst)) act[j] = false;  // keys not needed
      }
      if (act[j]) {
        if (KW == 1) {
          w[j].lo = ld_stream(reinterpret_cast<const u64*>(R.keys) + i, pol);
          w[j].hi = 0;
        } else {
          const ulonglong2 kk = ld_stream(reinterpret_cast<const ulonglong2*>(R.keys) + i, pol);
          w[j].lo = kk.x;
          w[j].hi = kk.y;
        }
        window_of(inf[j], w[j]);
        h[j] = key_hash(w[j].lo, w[j].hi);
        p[j] = part_of(h[j], G.P);
      }
    }
    // stage 2: Bloom test-and-set in the partition's sub-filter
    if (mode == kModeBloom) {
      u64 old[kRecPerThread], msk[kRecPerThread];
#pragma unroll
      for (int j = 0; j < kRecPerThread; ++j) {
        old[j] = msk[j] = 0;
        if (act[j]) {
          msk[j] = bloom_mask(h[j], G.bloom_h);
          old[j] = atomicOr(G.bloom + (u64)p[j] * G.Wp + bloom_index(h[j], G.Wp), msk[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kRecPerThread; ++j) {
        const bool first = act[j] && (old[j] & msk[j]) != msk[j];
        if (first) st_stream(R.info + base + (u64)j * blockDim.x + threadIdx.x, inf[j] | kInfoFirst, pol);
        acc_first += __popc(__ballot_sync(0xffffffffu, first));
        act[j] = act[j] && !first;
      }
    }
    // stage 3: first probe in the partition's sub-table
    ulonglong2 kv[kRecPerThread];
#pragma unroll
    for (int j = 0; j < kRecPerThread; ++j) {
      kv[j] = make_ulonglong2(0, 0);
      idx[j] = 0;
      if (act[j]) {
        idx[j] = table_index(h[j], G.Sp);
        kv[j] = __ldcg(reinterpret_cast<const ulonglong2*>(G.table + (u64)p[j] * G.Sp + idx[j]));
      }
    }
    // stage 4: resolve and count
#pragma unroll
    for (int j = 0; j < kRecPerThread; ++j) {
      Slot* s = nullptr;
      bool inserted = false;
      if (act[j]) {
        Slot* sub = G.table + (u64)p[j] * G.Sp;
        if (mode == kModeRecount) {
          bool full;
          s = resolve_find(sub, G.Sp, idx[j], kv[j], w[j].lo, w[j].hi, full);
          if (full) atomicOr(&G.status->flags, kFlagFull);
        } else {
          s = resolve_insert(sub, G.Sp, idx[j], kv[j], w[j].lo, w[j].hi, inserted);
          if (!s) atomicOr(&G.status->flags, kFlagFull);
        }
      }
      acc_ins += __popc(__ballot_sync(0xffffffffu, inserted));
      if (s) add_occurrence(s, w[j], 1u, G.status);
    }
  }
  if (lane == 0) {
    if (acc_ins) atomicAdd(&G.status->table_keys, acc_ins);
    if (acc_first) atomicAdd(&G.status->first_sightings, acc_first);
  }
}

// ------------------------------------------------------------------ launchers

static int grid_for(const void* fn, int threads, size_t smem, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return num_sms * (per_sm > 0 ? per_sm : 1);
}

cudaError_t launch_part_scatter(const PartGeom& g, const PartWindows& w, const PartRecords& r,
                                cudaStream_t stream, int num_sms) {
  if (w.q1 <= w.q0) return cudaSuccess;
  const int kw = g.k > 32 ? 2 : 1;
  const size_t smem = scatter_smem(g.P, kw);
  const void* fn = kw == 2 ? (const void*)part_scatter_kernel<2> : (const void*)part_scatter_kernel<1>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const u64 tiles = (w.q1 - w.q0 + kScatterTile - 1) / kScatterTile;
  u64 grid = grid_for(fn, kPartThreads, smem, num_sms);
  if (grid > tiles) grid = tiles;
  if (kw == 2) part_scatter_kernel<2><<<(unsigned)grid, kPartThreads, smem, stream>>>(g, w, r);
  else part_scatter_kernel<1><<<(unsigned)grid, kPartThreads, smem, stream>>>(g, w, r);
  return cudaGetLastError();
}

template <int KW, int RPT>
static cudaError_t launch_pass_rt(const PartGeom& g, const PartRecords& r, unsigned mode, cudaStream_t stream,
                                  int num_sms) {
  constexpr int tile = kPartThreads * RPT;
  const u64 tiles = (u64)g.P * ((r.cap + tile - 1) / tile) + (r.ocap + tile - 1) / tile;
  if (tiles == 0) return cudaSuccess;
  u64 grid = grid_for((const void*)part_pass_kernel<KW, RPT>, kPartThreads, 0, num_sms);
  if (grid > tiles) grid = tiles;
  part_pass_kernel<KW, RPT><<<(unsigned)grid, kPartThreads, 0, stream>>>(g, r, mode);
  return cudaGetLastError();
}

cudaError_t launch_part_pass(const PartGeom& g, const PartRecords& r, unsigned mode, cudaStream_t stream,
                             int num_sms) {
  if (g.rpt >= 4)
    return g.k > 32 ? launch_pass_rt<2, 4>(g, r, mode, stream, num_sms)
                    : launch_pass_rt<1, 4>(g, r, mode, stream, num_sms);
  return g.k > 32 ? launch_pass_rt<2, 2>(g, r, mode, stream, num_sms)
                  : launch_pass_rt<1, 2>(g, r, mode, stream, num_sms);
}

}  // namespace kma
