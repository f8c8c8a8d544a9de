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
#include <mutex>
#include <utility>
#include <vector>

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

constexpr int kPartThreads = 256;

// ------------------------------------------------------------------ scatter
//
// One tile = kScatterThreads * kScatterWpt consecutive window starts; thread t takes the
// kScatterWpt consecutive starts t * kScatterWpt + j.
//  1. extract the windows (one set of word loads per thread, then the forward k-mer and its
//     reverse complement are rolled one base at a time), stage key + info in shared memory,
//     rank each window inside its partition for this tile (shared-memory atomics);
//  2. thread t owns a contiguous chunk of partitions: it reserves each present partition's
//     run in the bucket (one global atomic, bucket first, the rest in the overflow area) and,
//     while those atomics are in flight, takes part in the exclusive scan of the counts that
//     sorts the tile's records by partition;
//  3. permute the staged records into partition order and write them out: consecutive
//     threads write consecutive records of the same bucket, so the stores coalesce.
// A CTA of 512 threads with its 4096-window tile leaves room for two CTAs per SM (with up to
// about a thousand partitions), so one CTA's block barriers and reservation round trips
// overlap the other's extraction and stores.

constexpr int kScatterThreads = 1024;
constexpr int kScatterWpt = 8;
constexpr int kScatterTile = kScatterThreads * kScatterWpt;  // 4096: ranks and slots < 2^12
constexpr int kScatterMaxChunk = 4;                          // partitions per thread (4096 / 512)

__host__ __device__ constexpr size_t scatter_smem(unsigned P, int kw) {
  return (size_t)kScatterTile * (kw * 8) +   // staged keys
         (size_t)kScatterTile * 4 +          // sorted order: slot | partition << 12
         (size_t)P * 20 +                    // cnt, off, gbase, n1, obase (32-bit each)
         (size_t)32 * 4 +                    // warp sums
         (size_t)kScatterTile;               // staged info
}

static_assert(scatter_smem(kMaxPartitions, 1) <= 227 * 1024 && scatter_smem(kMaxPartitionsWide, 2) <= 227 * 1024,
              "the scatter's shared memory must fit one CTA for every allowed partition count");
static_assert(kMaxPartitions <= kScatterThreads * kScatterMaxChunk,
              "partition numbers must fit the sorted order's 12 bits and the threads' chunks");

template <int KW>
__global__ void __launch_bounds__(kScatterThreads, 1) part_scatter_kernel(const __grid_constant__ PartGeom G,
                                                                          const __grid_constant__ PartWindows W,
                                                                          const __grid_constant__ PartRecords R) {
  constexpr int kWarps = kScatterThreads / 32;
  extern __shared__ __align__(16) unsigned char s_raw[];
  const unsigned P = G.P;
  u64* s_keys = reinterpret_cast<u64*>(s_raw);                              // [tile * KW]
  unsigned* s_order = reinterpret_cast<unsigned*>(s_keys + kScatterTile * KW);  // [tile]
  unsigned* s_cnt = s_order + kScatterTile;                                 // [P] records in this tile
  unsigned* s_off = s_cnt + P;                                              // [P] first sorted position
  unsigned* s_gbase = s_off + P;                                            // [P] run start in the bucket
  unsigned* s_n1 = s_gbase + P;                                             // [P] records of the run in the bucket
  unsigned* s_obase = s_n1 + P;                                             // [P] rest: overflow area position
  unsigned* s_wsum = s_obase + P;                                           // [32]
  unsigned char* s_info = reinterpret_cast<unsigned char*>(s_wsum + 32);    // [tile]
  const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned n_tiles = (unsigned)((W.q1 - W.q0 + kScatterTile - 1) / kScatterTile);
  const u64 pol = policy_evict_first();
  const unsigned per = (P + kScatterThreads - 1) / kScatterThreads;  // partitions per thread (<= 8)
  const unsigned p0 = min(P, tid * per), p1 = min(P, p0 + per);
  const u64 cap = R.cap, ocap = R.ocap;
  unsigned acc_valid = 0;
  for (unsigned p = tid; p < P; p += kScatterThreads) s_cnt[p] = 0;
  __syncthreads();
  for (unsigned t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    // 1: windows -> staged records, rank inside the partition
    unsigned pr[kScatterWpt];  // partition << 13 | rank, or ~0u
#pragma unroll
    for (int j = 0; j < kScatterWpt; ++j) pr[j] = 0xFFFFFFFFu;
    const u64 q = W.q0 + (u64)t * kScatterTile + (u64)tid * kScatterWpt;
    if (q < W.q1) {  // q1 - q0 is a multiple of 64: all kScatterWpt starts are inside
      RollingWindows rw;
      rw.init(W, G.k, q);
#pragma unroll
      for (int j = 0; j < kScatterWpt; ++j) {
        Window w;
        if (rw.get(j, G.canonical, w)) {
          const u64 h = key_hash(w.lo, w.hi);
          if (G.n_parts <= 1 || owner_of(h, G.n_parts) == G.part) {
            ++acc_valid;
            const unsigned slot = j * kScatterThreads + tid;
            const unsigned p = part_of(h, P);
            pr[j] = (p << 13) | atomicAdd(&s_cnt[p], 1u);
            if (KW == 1) s_keys[slot] = w.lo;
            else reinterpret_cast<ulonglong2*>(s_keys)[slot] = make_ulonglong2(w.lo, w.hi);
            s_info[slot] = info_of(w);
          }
        }
        if (j + 1 < kScatterWpt) rw.roll();
      }
    }
    __syncthreads();
    // 2: reservations of this thread's partitions (in flight during the scan), then the
    // exclusive scan of the counts
    unsigned long long res[kScatterMaxChunk];
    unsigned local = 0;
#pragma unroll
    for (unsigned x = 0; x < kScatterMaxChunk; ++x) {
      const unsigned p = p0 + x;
      res[x] = 0;
      if (p < p1) {
        const unsigned c = s_cnt[p];
        local += c;
        if (c) res[x] = atomicAdd(&R.fill[p], (u64)c);
      }
    }
    unsigned incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += v;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    // prefix of the warp totals (every warp scans the 16 sums itself)
    unsigned ws = s_wsum[lane], wincl = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, wincl, o);
      if (lane >= (unsigned)o) wincl += v;
    }
    const unsigned total = __shfl_sync(0xffffffffu, wincl, kWarps - 1);  // records in this tile
    unsigned run = __shfl_sync(0xffffffffu, wincl - ws, warp) + incl - local;
#pragma unroll
    for (unsigned x = 0; x < kScatterMaxChunk; ++x) {
      const unsigned p = p0 + x;
      if (p < p1) {
        const unsigned c = s_cnt[p];
        s_off[p] = run;
        run += c;
        if (c) {
          const u64 b = res[x];
          const u64 room = b < cap ? cap - b : 0;
          const unsigned n1 = (unsigned)(room < c ? room : c);
          s_gbase[p] = (unsigned)(b < cap ? b : 0);
          s_n1[p] = n1;
          s_obase[p] = n1 < c ? (unsigned)min(atomicAdd(&R.fill[P], (u64)(c - n1)), ocap) : 0u;
        }
        s_cnt[p] = 0;  // for the next tile
      }
    }
    __syncthreads();
    // 3a: sorted order (partition-major) of the staged records
#pragma unroll
    for (int j = 0; j < kScatterWpt; ++j) {
      if (pr[j] == 0xFFFFFFFFu) continue;
      const unsigned p = pr[j] >> 13, r = pr[j] & 8191u;
      s_order[s_off[p] + r] = (p << 13) | (j * kScatterThreads + tid);
    }
    __syncthreads();
    // 3b: write out in sorted order (coalesced runs per bucket)
    for (unsigned i = tid; i < total; i += kScatterThreads) {
      const unsigned e = s_order[i];
      const unsigned slot = e & 8191u, p = e >> 13;
      const unsigned r = i - s_off[p], n1 = s_n1[p];
      u64 gi;
      if (r < n1) {
        gi = (u64)p * cap + s_gbase[p] + r;
      } else {
        const u64 o = (u64)s_obase[p] + (r - n1);
        if (o >= ocap) {  // overflow area full: reported, never dropped silently
          atomicOr(&G.status->flags, kFlagFull);
          continue;
        }
        gi = (u64)P * cap + o;
      }
      if (KW == 1) {
        st_stream(reinterpret_cast<u64*>(R.keys) + gi, s_keys[slot], pol);
      } else {
        st_stream(reinterpret_cast<ulonglong2*>(R.keys) + gi, reinterpret_cast<const ulonglong2*>(s_keys)[slot], pol);
      }
      st_stream(R.info + gi, s_info[slot], pol);
    }
    __syncthreads();  // staged records and per-partition runs are reused by the next tile
  }
  // valid windows: reduce inside the warp first
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc_valid += __shfl_down_sync(0xffffffffu, acc_valid, o);
  if (lane == 0 && acc_valid) atomicAdd(&G.status->valid_windows, (u64)acc_valid);
}

// ------------------------------------------------------------------ record pass
//
// Tiles walk the buckets in partition order (then the overflow area), so at any moment the
// CTAs work on one or two partitions whose sub-filter and sub-table sit in L2. Every warp
// works on its own tiles of 32 * RPT records, staged in shared memory with 1-D bulk copies
// and double-buffered: while the lanes resolve the atomics of one tile, the warp's next tile
// is on its way. Warps never wait for each other (no block barriers), so a warp whose
// probes take long does not hold up the others.

template <int KW, int RPT>
struct WarpStage {
  static constexpr int kTile = 32 * RPT;  // a multiple of 16
  u64 keys[2][kTile * KW];
  unsigned char info[2][kTile];
  unsigned char dup[64];                  // equal keys among a round of 32 records: a lane per hash slot
  unsigned acc[32][10];                   // per group leader: occurrences by left / right outcome
  unsigned walk[8];                       // lane 0's tile walk: t, c_end, c_next, cb, cf, kept
                                          // here: as registers they took five in every lane
                                          // and the Bloom pass spilled
  unsigned long long bar[2];
};
static_assert(sizeof(WarpStage<1, 2>) % 16 == 0 && sizeof(WarpStage<2, 2>) % 16 == 0 &&
                  sizeof(WarpStage<1, 4>) % 16 == 0 && sizeof(WarpStage<2, 4>) % 16 == 0,
              "every warp's staging buffers must start on a 16-byte boundary");

// Records of launch tile t: the first one (base) and their number, 0 if the tile is empty.
// The launch numbers its tiles from 0: first the nb tiles of the buckets of partitions
// [p_begin, p_end), tpb per bucket, then the tiles of the overflow area (if the launch covers
// it). Tile numbers, bucket numbers and record counts within a bucket fit 32 bits (the host
// checks each record batch). cb / cf: the bucket whose record count was loaded last.
// tinv: 0, or tile_inverse(tpb), with which the bucket number is a multiply-high instead of a
// division.
template <int TILE>
__device__ __forceinline__ unsigned rec_tile(const PartGeom& G, const PartRecords& R, unsigned tpb, unsigned nb,
                                             unsigned t, u64& base, unsigned& cb, unsigned& cf, u64 tinv) {
  unsigned f, lo;
  u64 b0;
  if (t < nb) {
    const unsigned q = tinv ? (tpb == 1 ? t : (unsigned)__umul64hi((u64)t, tinv)) : t / tpb;
    const unsigned b = R.p_begin + q;
    if (b != cb) {
      const u64 x = R.fill[b];
      cb = b;
      cf = (unsigned)(x < R.cap ? x : R.cap);
    }
    f = cf;
    lo = (t - q * tpb) * TILE;
    b0 = (u64)b * R.cap;
  } else {
    const u64 x = R.fill[G.P];
    f = (unsigned)(x < R.ocap ? x : R.ocap);
    lo = (t - nb) * TILE;
    b0 = (u64)G.P * R.cap;
  }
  if (lo >= f) return 0;
  base = b0 + lo;
  return f - lo < (unsigned)TILE ? f - lo : (unsigned)TILE;
}

// Tiles are handed out in launch order from a global queue, kQueueChunk consecutive tiles at a
// time, so every warp works at the front of the partition sequence: the warps never spread
// over more partitions than the front touches, and those partitions' sub-filters and
// sub-tables stay in L2. (Tiles assigned to warps in a fixed pattern let fast and slow warps
// drift apart over the partitions, and their structures evicted one another from L2.)
// Lane 0 holds the warp's current chunk (tiles up to c_end) and the next chunk, grabbed one
// ahead so that its queue round trip is hidden.
constexpr unsigned kQueueChunk = 8;

// floor(t / d) = high word of t * (floor((2^64 - 1) / d) + 1) for every t < 2^32 and 2 <= d <
// 2^32 (division by an invariant integer through a rounded-up reciprocal, Granlund and
// Montgomery, PLDI 1994): the product's error t * e / 2^64, e <= 1, stays below 1 / d.
__device__ __forceinline__ u64 tile_inverse(unsigned d) { return d > 1 ? ~0ull / d + 1 : 0ull; }

// Lane 0: the next non-empty tile from t on (its first record in base, t moved past it),
// moving through the warp's chunks; returns its record count, 0 when no tile is left.
template <int TILE>
__device__ __forceinline__ unsigned rec_next(const PartGeom& G, const PartRecords& R, unsigned tpb, unsigned nb,
                                             unsigned n_tiles, unsigned& t, unsigned& c_end, unsigned& c_next,
                                             u64& base, unsigned& cb, unsigned& cf, u64 tinv = 0) {
  while (true) {
    if (t >= c_end) {  // chunk done: take the one grabbed ahead, grab the following one
      t = c_next * kQueueChunk;
      c_end = t + kQueueChunk;
      c_next = atomicAdd(R.queue, 1u);
    }
    if (t >= n_tiles) return 0;
    const unsigned n = rec_tile<TILE>(G, R, tpb, nb, t, base, cb, cf, tinv);
    ++t;
    if (n) return n;
  }
}

// Lane 0: stage the n records from `base` into buffer `buf` (sizes rounded up to 16 records,
// which stays inside the bucket because cap and ocap are multiples of 16).
template <int KW, int RPT>
__device__ __forceinline__ void rec_issue(WarpStage<KW, RPT>& S, const PartRecords& R, int buf, u64 base, unsigned n,
                                          u64 pol) {
  const unsigned n16 = (n + 15u) & ~15u;
  const unsigned kb = n16 * 8u * KW;
  const unsigned bar = smem_u32(&S.bar[buf]);
  fence_proxy_async_smem();
  mbar_expect_tx(bar, kb + n16);
  tma_load_1d_hint(smem_u32(S.keys[buf]), reinterpret_cast<const u64*>(R.keys) + base * KW, kb, bar, pol);
  tma_load_1d_hint(smem_u32(S.info[buf]), R.info + base, n16, bar, pol);
}

// Lane 0: the same staging copy into explicit buffers (keys, info) completing on `bar`.
template <int KW>
__device__ __forceinline__ void rec_issue_raw(u64* keys, unsigned char* info, unsigned bar, const PartRecords& R,
                                              u64 base, unsigned n, u64 pol) {
  const unsigned n16 = (n + 15u) & ~15u;
  const unsigned kb = n16 * 8u * KW;
  fence_proxy_async_smem();
  mbar_expect_tx(bar, kb + n16);
  tma_load_1d_hint(smem_u32(keys), reinterpret_cast<const u64*>(R.keys) + base * KW, kb, bar, pol);
  tma_load_1d_hint(smem_u32(info), R.info + base, n16, bar, pol);
}

__device__ __forceinline__ u64 shfl0(u64 v) { return __shfl_sync(0xffffffffu, v, 0); }

template <int KW, int RPT, unsigned MODE, bool GROUP>
__global__ void __launch_bounds__(kPartThreads, RPT == 2 ? 4 : 2) part_pass_kernel(const __grid_constant__ PartGeom G,
                                                                                  const __grid_constant__ PartRecords R) {
  static_assert(MODE == kModeBloom || MODE == kModeCount, "the recount has its own kernel");
  constexpr int kTile = WarpStage<KW, RPT>::kTile;
  constexpr int kWarps = kPartThreads / 32;
  __shared__ __align__(128) WarpStage<KW, RPT> stage[kWarps];
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpStage<KW, RPT>& S = stage[warp];
  const unsigned tpb = (unsigned)((R.cap + kTile - 1) / kTile);  // tiles per bucket
  const unsigned ofill = (unsigned)(R.fill[G.P] < R.ocap ? R.fill[G.P] : R.ocap);
  const unsigned nb = (R.p_end - R.p_begin) * tpb;  // bucket tiles of this launch
  const unsigned n_tiles = nb + (R.overflow ? (ofill + kTile - 1) / kTile : 0u);
  const u64 pol = policy_evict_first();
  unsigned acc_ins = 0, acc_first = 0;  // per warp: below 2^32
  unsigned phases = 0;  // bit b: parity to wait for on buffer b (same in every lane)

  // lane 0's walk over the queue's chunks
  unsigned& t = S.walk[0];
  unsigned& c_end = S.walk[1];
  unsigned& c_next = S.walk[2];
  unsigned& cb = S.walk[3];
  unsigned& cf = S.walk[4];
  u64 base = 0;
  unsigned n = 0;
  if (lane == 0) {
    t = 0;
    cb = ~0u;
    cf = 0;
    c_end = 0;
    mbar_init(smem_u32(&S.bar[0]), 1);
    mbar_init(smem_u32(&S.bar[1]), 1);
    c_next = atomicAdd(R.queue, 1u);
    n = rec_next<kTile>(G, R, tpb, nb, n_tiles, t, c_end, c_next, base, cb, cf);
    if (n) rec_issue(S, R, 0, base, n, pol);
  }
  __syncwarp();  // barriers initialised before any lane polls them
  n = __shfl_sync(0xffffffffu, n, 0);
  base = shfl0(base);
  int buf = 0;
  while (n) {
    // stage the warp's next non-empty tile into the other buffer, then wait for this one
    u64 nbase = 0;
    unsigned nn = 0;
    if (lane == 0) {
      nn = rec_next<kTile>(G, R, tpb, nb, n_tiles, t, c_end, c_next, nbase, cb, cf);
      if (nn) rec_issue(S, R, buf ^ 1, nbase, nn, pol);
    }
    nn = __shfl_sync(0xffffffffu, nn, 0);
    nbase = shfl0(nbase);
    const unsigned bar = smem_u32(&S.bar[buf]);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, (phases >> buf) & 1u, G.wait_limit));
    if (!ok) {  // give up: report, let the copies in flight land (bounded), stop the warp
      if (lane == 0) {
        atomicOr(&G.status->flags, kFlagTimeout);
        mbar_drain(bar, (phases >> buf) & 1u, G.wait_limit);
        if (nn) mbar_drain(smem_u32(&S.bar[buf ^ 1]), (phases >> (buf ^ 1)) & 1u, G.wait_limit);
      }
      return;
    }
    phases ^= 1u << buf;
    const u64* sk = S.keys[buf];
    const unsigned char* si = S.info[buf];

    Window w[RPT];
    u64 h[RPT];
    unsigned p[RPT], rec[RPT];
    bool act[RPT];
    // stage 1: records from shared memory
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      const unsigned k = j * 32 + lane;
      act[j] = k < n;
      rec[j] = k;
      h[j] = 0;
      p[j] = 0;
      if (act[j]) {
        const unsigned i = rec[j];
        if (KW == 1) {
          w[j].lo = sk[i];
          w[j].hi = 0;
        } else {
          const ulonglong2 kk = reinterpret_cast<const ulonglong2*>(sk)[i];
          w[j].lo = kk.x;
          w[j].hi = kk.y;
        }
        window_of(si[i], w[j]);
        h[j] = key_hash(w[j].lo, w[j].hi);
        p[j] = part_of(h[j], G.P);
      }
    }
    // Equal keys in a round of 32 records (frequent k-mers: satellites, low-complexity
    // sequence) act as one group: only its leader does the Bloom test-and-set and the table
    // probe, and the group's counter updates are summed in shared memory and applied once
    // (the paper accumulates frequent k-mers locally before a global reduction, Section 5.1;
    // here the locality is the warp). Each lane writes its lane number at a slot chosen by its
    // hash; a lane whose slot holds another lane with the same key joins that lane's group.
    // Only with GROUP (the heavy_hitters parameter): elsewhere every lane is its own group.
    bool dup[RPT];
    unsigned ldr[RPT];
    bool anydup = false;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      dup[j] = false;
      ldr[j] = lane;
    }
    if (GROUP) {
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        const unsigned slot = (unsigned)h[j] & 63u;
        if (act[j]) S.dup[slot] = (unsigned char)lane;
        __syncwarp();
        const unsigned wl = act[j] ? S.dup[slot] : lane;
        const u64 wlo = __shfl_sync(0xffffffffu, w[j].lo, wl), whi = __shfl_sync(0xffffffffu, w[j].hi, wl);
        dup[j] = act[j] && wl != lane && wlo == w[j].lo && whi == w[j].hi;
        ldr[j] = dup[j] ? wl : lane;
        anydup |= __any_sync(0xffffffffu, dup[j]);
        __syncwarp();  // the slots are rewritten by the next round
      }
    }
    // stage 2: Bloom test-and-set in the partition's sub-filter; first sightings flagged
    if (MODE == kModeBloom) {
      u64 old[RPT], msk[RPT];
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        old[j] = msk[j] = 0;
        if (act[j]) {
          msk[j] = bloom_mask(h[j], G.bloom_h);
          if (!dup[j]) old[j] = atomicOr(G.bloom + (u64)p[j] * G.Wp + bloom_index(h[j], G.Wp), msk[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        // a group's members come after its leader: they have been seen
        const bool first = act[j] && !dup[j] && (old[j] & msk[j]) != msk[j];
        if (first) st_stream(R.info + base + rec[j], (unsigned)si[rec[j]] | kInfoFirst, pol);
        acc_first += __popc(__ballot_sync(0xffffffffu, first));
        act[j] = act[j] && !first;
        // a group whose leader was the first sighting: its members resolve on their own
        if (GROUP && __shfl_sync(0xffffffffu, first, ldr[j])) {
          dup[j] = false;
          ldr[j] = lane;
        }
      }
    }
    // stage 3: first probe in the partition's sub-table (group leaders only)
    ulonglong2 kv[RPT];
    u64 idx[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      kv[j] = make_ulonglong2(0, 0);
      idx[j] = 0;
      if (act[j] && !dup[j]) {
        idx[j] = table_index(h[j], G.Sp);
        kv[j] = __ldcg(reinterpret_cast<const ulonglong2*>(G.table + (u64)p[j] * G.Sp + idx[j]));
      }
    }
    // stage 4: resolve and count
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
      Slot* s = nullptr;
      bool inserted = false;
      if (act[j] && !dup[j]) {
        Slot* sub = G.table + (u64)p[j] * G.Sp;
        s = resolve_insert(sub, G.Sp, idx[j], kv[j], w[j].lo, w[j].hi, inserted);
        if (!s) atomicOr(&G.status->flags, kFlagFull);
      }
      acc_ins += __popc(__ballot_sync(0xffffffffu, inserted));
      if (GROUP && anydup) {
        // sum each group's outcomes in its leader's block, then the leader applies them
        unsigned* blk = S.acc[lane];
#pragma unroll
        for (int c = 0; c < 10; ++c) blk[c] = 0;
        __syncwarp();
        if (act[j]) {
          atomicAdd(&S.acc[ldr[j]][w[j].lu ? w[j].lb : 4u], 1u);
          atomicAdd(&S.acc[ldr[j]][5u + (w[j].ru ? w[j].rb : 4u)], 1u);
        }
        __syncwarp();
        if (s) {
#pragma unroll
          for (int c = 0; c < 10; ++c) {
            const unsigned v = blk[c];
            if (!v) continue;
            unsigned* ctr = c < 4 ? &s->ext[c] : c == 4 ? &s->none[0] : c < 9 ? &s->ext[c - 1] : &s->none[1];
            if (G.no_overflow) red_add(ctr, v);
            else if (atomicAdd(ctr, v) > 0xFFFFFFFFu - v) atomicOr(&G.status->flags, kFlagOverflow);
          }
        }
        __syncwarp();  // the blocks are cleared by the next round
      } else if (s) {
        if (G.no_overflow) add_occurrence_red(s, w[j]);
        else add_occurrence(s, w[j], 1u, G.status);
      }
    }
    __syncwarp();  // buffer `buf` (and the list) are free for the next copy
    n = nn;
    base = nbase;
    buf ^= 1;
  }
  if (lane == 0) {
    if (acc_ins) atomicAdd(&G.status->table_keys, (u64)acc_ins);
    if (acc_first) atomicAdd(&G.status->first_sightings, (u64)acc_first);
  }
}

// ------------------------------------------------------------------ recount
//
// The first sightings marked by the Bloom pass (about two in five records, most of them k-mers
// seen once) are added to the k-mers that reached the table. Every warp stages its tiles like
// the other record passes, copies each tile's marked records into a ring in shared memory
// (the staging buffer is then free for the next copy), and resolves the ring in full rounds of
// 32 records, one per lane: key filter, then (for the few that pass it) the table probe and the
// count. Resolving tile by tile instead would leave most lanes idle in every round.

constexpr int kRing = 128;  // entries; a tile adds at most 64 to fewer than 32 left over

template <int KW>
struct RecountStage {
  static constexpr int kTile = 64;
  u64 keys[2][kTile * KW];
  u64 rkeys[kRing * KW];
  unsigned char info[2][kTile];
  unsigned char rinfo[kRing];
  unsigned walk[8];  // lane 0's tile walk: t, c_end, c_next, cb, cf (not in every lane's registers)
  unsigned long long bar[2];
};
static_assert(sizeof(RecountStage<1>) % 16 == 0 && sizeof(RecountStage<2>) % 16 == 0,
              "every warp's staging buffers must start on a 16-byte boundary");

// One round: lane l resolves ring entry (head + l), if act.
template <int KW>
__device__ __forceinline__ void recount_round(const PartGeom& G, const RecountStage<KW>& S, unsigned e, bool act) {
  if (!act) return;
  Window w;
  if (KW == 1) {
    w.lo = S.rkeys[e];
    w.hi = 0;
  } else {
    const ulonglong2 kk = reinterpret_cast<const ulonglong2*>(S.rkeys)[e];
    w.lo = kk.x;
    w.hi = kk.y;
  }
  const u64 h = key_hash(w.lo, w.hi);
  const unsigned p = part_of(h, G.P);
  // most first sightings are of k-mers seen once, which never reached the table: the key
  // filter (every inserted key set its bits) rules them out without a probe
  if (G.Wk) {
    const u64 m = keyfilter_mask(h, G.bloom_h);
    if ((__ldcg(G.keyfilter + (u64)p * G.Wk + keyfilter_index(h, G.Wk)) & m) != m) return;
  }
  window_of(S.rinfo[e], w);  // extension outcomes: only for the sightings that may count
  Slot* sub = G.table + (u64)p * G.Sp;
  const u64 idx = table_index(h, G.Sp);
  const ulonglong2 kv = __ldcg(reinterpret_cast<const ulonglong2*>(sub + idx));
  bool full;
  Slot* s = resolve_find(sub, G.Sp, idx, kv, w.lo, w.hi, full);
  if (full) atomicOr(&G.status->flags, kFlagFull);
  if (s) {
    if (G.no_overflow) add_occurrence_red(s, w);
    else add_occurrence(s, w, 1u, G.status);
  }
}

template <int KW>
__global__ void __launch_bounds__(kPartThreads, 6) part_recount_kernel(const __grid_constant__ PartGeom G,
                                                                    const __grid_constant__ PartRecords R) {
  constexpr int kTile = RecountStage<KW>::kTile;
  constexpr int kWarps = kPartThreads / 32;
  __shared__ __align__(128) RecountStage<KW> stage[kWarps];
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RecountStage<KW>& S = stage[warp];
  const unsigned tpb = (unsigned)((R.cap + kTile - 1) / kTile);
  const unsigned ofill = (unsigned)(R.fill[G.P] < R.ocap ? R.fill[G.P] : R.ocap);
  const unsigned nb = (R.p_end - R.p_begin) * tpb;
  const unsigned n_tiles = nb + (R.overflow ? (ofill + kTile - 1) / kTile : 0u);
  const u64 pol = policy_evict_first();
  unsigned phases = 0;
  unsigned head = 0, tail = 0;  // ring: entries [head, tail) are waiting (same in every lane)
  const u64 tinv = tile_inverse(tpb);  // lane 0's tile walk: bucket numbers without a division

  unsigned& t = S.walk[0];
  unsigned& c_end = S.walk[1];
  unsigned& c_next = S.walk[2];
  unsigned& cb = S.walk[3];
  unsigned& cf = S.walk[4];
  u64 base = 0;
  unsigned n = 0;
  if (lane == 0) {
    t = 0;
    cb = ~0u;
    cf = 0;
    c_end = 0;
    mbar_init(smem_u32(&S.bar[0]), 1);
    mbar_init(smem_u32(&S.bar[1]), 1);
    c_next = atomicAdd(R.queue, 1u);
    n = rec_next<kTile>(G, R, tpb, nb, n_tiles, t, c_end, c_next, base, cb, cf, tinv);
    if (n) rec_issue_raw<KW>(S.keys[0], S.info[0], smem_u32(&S.bar[0]), R, base, n, pol);
  }
  __syncwarp();
  n = __shfl_sync(0xffffffffu, n, 0);
  base = shfl0(base);
  int buf = 0;
  while (n) {
    u64 nbase = 0;
    unsigned nn = 0;
    if (lane == 0) {
      nn = rec_next<kTile>(G, R, tpb, nb, n_tiles, t, c_end, c_next, nbase, cb, cf, tinv);
      if (nn) rec_issue_raw<KW>(S.keys[buf ^ 1], S.info[buf ^ 1], smem_u32(&S.bar[buf ^ 1]), R, nbase, nn, pol);
    }
    nn = __shfl_sync(0xffffffffu, nn, 0);
    nbase = shfl0(nbase);
    const unsigned bar = smem_u32(&S.bar[buf]);
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, (phases >> buf) & 1u, G.wait_limit));
    if (!ok) {  // give up: report, let the copies in flight land (bounded), stop the warp
      if (lane == 0) {
        atomicOr(&G.status->flags, kFlagTimeout);
        mbar_drain(bar, (phases >> buf) & 1u, G.wait_limit);
        if (nn) mbar_drain(smem_u32(&S.bar[buf ^ 1]), (phases >> (buf ^ 1)) & 1u, G.wait_limit);
      }
      return;
    }
    phases ^= 1u << buf;
    // the tile's marked records into the ring
#pragma unroll
    for (int j = 0; j < kTile / 32; ++j) {
      const unsigned i = j * 32 + lane;
      const bool f = i < n && (S.info[buf][i] & kInfoFirst);
      const unsigned m = __ballot_sync(0xffffffffu, f);
      if (f) {
        const unsigned e = (tail + __popc(m & ((1u << lane) - 1u))) & (kRing - 1);
        if (KW == 1) S.rkeys[e] = S.keys[buf][i];
        else reinterpret_cast<ulonglong2*>(S.rkeys)[e] = reinterpret_cast<const ulonglong2*>(S.keys[buf])[i];
        S.rinfo[e] = S.info[buf][i];
      }
      tail += __popc(m);
    }
    __syncwarp();  // ring entries visible to every lane; buffer `buf` free for the next copy
    while (tail - head >= 32) {
      recount_round<KW>(G, S, (head + lane) & (kRing - 1), true);
      head += 32;
    }
    __syncwarp();  // ring slots are rewritten by the next tile
    n = nn;
    base = nbase;
    buf ^= 1;
  }
  recount_round<KW>(G, S, (head + lane) & (kRing - 1), lane < tail - head);
}

// ------------------------------------------------------------------ key filter
//
// After the Bloom pass: every key in the table sets its bits in its partition's key filter.
// One CTA chunk = kKeyChunk consecutive slots of one partition (slot keys read once, in order).

constexpr int kKeyThreads = 256;
constexpr int kKeyChunk = kKeyThreads * 8;

__global__ void __launch_bounds__(kKeyThreads) keyfilter_build_kernel(const __grid_constant__ PartGeom G) {
  const u64 chunks_per_part = (G.Sp + kKeyChunk - 1) / kKeyChunk;
  const u64 n_chunks = chunks_per_part * G.P;
  for (u64 c = blockIdx.x; c < n_chunks; c += gridDim.x) {
    const u64 p = c / chunks_per_part;
    const u64 s0 = (c - p * chunks_per_part) * kKeyChunk;
    const Slot* sub = G.table + p * G.Sp;
    u64* kf = G.keyfilter + p * G.Wk;
    // all of the thread's slot keys are loaded before the first atomic: the loads of a chunk
    // are in flight together instead of one round trip each
    constexpr int kPer = kKeyChunk / kKeyThreads;
    ulonglong2 kv[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const u64 i = s0 + (u64)j * kKeyThreads + threadIdx.x;
      kv[j] = i < G.Sp ? __ldcs(reinterpret_cast<const ulonglong2*>(sub + i)) : make_ulonglong2(kEmpty, kEmpty);
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (kv[j].x == kEmpty && kv[j].y == kEmpty) continue;
      const u64 h = key_hash(kv[j].x, kv[j].y);
      atomicOr(kf + keyfilter_index(h, G.Wk), keyfilter_mask(h, G.bloom_h));
    }
  }
}

// ------------------------------------------------------------------ launchers

cudaError_t allow_dynamic_smem(const void* fn, size_t need) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> done;  // (kernel, device) -> limit
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  int limit = -1;
  for (const auto& d : done)
    if (d.first.first == fn && d.first.second == dev) limit = d.second;
  if (limit < 0) {
    int optin = 0;
    cudaFuncAttributes fa;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess)
      return e;
    limit = optin - (int)fa.sharedSizeBytes;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess) return e;
    done.push_back({{fn, dev}, limit});
  }
  return need <= (size_t)limit ? cudaSuccess : cudaErrorInvalidValue;
}

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
  cudaError_t e = allow_dynamic_smem(fn, smem);
  if (e != cudaSuccess) return e;
  const u64 tiles = (w.q1 - w.q0 + kScatterTile - 1) / kScatterTile;
  u64 grid = grid_for(fn, kScatterThreads, smem, num_sms);
  if (grid > tiles) grid = tiles;
  if (kw == 2) part_scatter_kernel<2><<<(unsigned)grid, kScatterThreads, smem, stream>>>(g, w, r);
  else part_scatter_kernel<1><<<(unsigned)grid, kScatterThreads, smem, stream>>>(g, w, r);
  return cudaGetLastError();
}

template <int KW, int RPT, unsigned MODE, bool GROUP>
static cudaError_t launch_pass_rt(const PartGeom& g, const PartRecords& r, cudaStream_t stream, int num_sms) {
  constexpr int tile = 32 * RPT;
  if (r.p_begin > r.p_end || r.p_end > g.P) return cudaErrorInvalidValue;
  const u64 tiles = (u64)(r.p_end - r.p_begin) * ((r.cap + tile - 1) / tile) +
                    (r.overflow ? (r.ocap + tile - 1) / tile : 0);
  if (tiles == 0) return cudaSuccess;
  if ((r.cap | r.ocap) & 15 || (reinterpret_cast<uintptr_t>(r.keys) | reinterpret_cast<uintptr_t>(r.info)) & 15)
    return cudaErrorInvalidValue;  // staging needs 16-record buckets on 16-byte boundaries
  const void* fn = (const void*)part_pass_kernel<KW, RPT, MODE, GROUP>;
  u64 grid = grid_for(fn, kPartThreads, 0, num_sms);
  if (grid > tiles) grid = tiles;
  cudaError_t e = cudaMemsetAsync(r.queue, 0, sizeof(unsigned), stream);  // the launch's tile queue
  if (e != cudaSuccess) return e;
  part_pass_kernel<KW, RPT, MODE, GROUP><<<(unsigned)grid, kPartThreads, 0, stream>>>(g, r);
  return cudaGetLastError();
}

template <int KW>
static cudaError_t launch_recount(const PartGeom& g, const PartRecords& r, cudaStream_t stream, int num_sms) {
  constexpr int tile = RecountStage<KW>::kTile;
  if (r.p_begin > r.p_end || r.p_end > g.P) return cudaErrorInvalidValue;
  const u64 tiles = (u64)(r.p_end - r.p_begin) * ((r.cap + tile - 1) / tile) +
                    (r.overflow ? (r.ocap + tile - 1) / tile : 0);
  if (tiles == 0) return cudaSuccess;
  if ((r.cap | r.ocap) & 15 || (reinterpret_cast<uintptr_t>(r.keys) | reinterpret_cast<uintptr_t>(r.info)) & 15)
    return cudaErrorInvalidValue;  // staging needs 16-record buckets on 16-byte boundaries
  const void* fn = (const void*)part_recount_kernel<KW>;
  u64 grid = grid_for(fn, kPartThreads, 0, num_sms);
  if (grid > tiles) grid = tiles;
  cudaError_t e = cudaMemsetAsync(r.queue, 0, sizeof(unsigned), stream);  // the launch's tile queue
  if (e != cudaSuccess) return e;
  part_recount_kernel<KW><<<(unsigned)grid, kPartThreads, 0, stream>>>(g, r);
  return cudaGetLastError();
}

template <int KW, int RPT>
static cudaError_t launch_pass_mode(const PartGeom& g, const PartRecords& r, unsigned mode, cudaStream_t stream,
                                    int num_sms) {
  // equal-key grouping (heavy hitters) is built for the 2-records-per-lane passes that count
  const bool group = g.group && RPT == 2;
  if (mode == kModeBloom)
    return group ? launch_pass_rt<KW, RPT, kModeBloom, true>(g, r, stream, num_sms)
                 : launch_pass_rt<KW, RPT, kModeBloom, false>(g, r, stream, num_sms);
  if (mode == kModeCount)
    return group ? launch_pass_rt<KW, RPT, kModeCount, true>(g, r, stream, num_sms)
                 : launch_pass_rt<KW, RPT, kModeCount, false>(g, r, stream, num_sms);
  return launch_recount<KW>(g, r, stream, num_sms);
}

cudaError_t launch_keyfilter_build(const PartGeom& g, cudaStream_t stream, int num_sms) {
  if (!g.Wk || !g.keyfilter) return cudaSuccess;
  const u64 chunks = g.P * ((g.Sp + kKeyChunk - 1) / kKeyChunk);
  u64 grid = grid_for((const void*)keyfilter_build_kernel, kKeyThreads, 0, num_sms);
  if (grid > chunks) grid = chunks;
  keyfilter_build_kernel<<<(unsigned)grid, kKeyThreads, 0, stream>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_part_pass(const PartGeom& g, const PartRecords& r, unsigned mode, cudaStream_t stream,
                             int num_sms) {
  if (g.rpt >= 4)
    return g.k > 32 ? launch_pass_mode<2, 4>(g, r, mode, stream, num_sms)
                    : launch_pass_mode<1, 4>(g, r, mode, stream, num_sms);
  return g.k > 32 ? launch_pass_mode<2, 2>(g, r, mode, stream, num_sms)
                  : launch_pass_mode<1, 2>(g, r, mode, stream, num_sms);
}

}  // namespace kma
