// CUDA kernels of the k-mer analysis stage (HipMer, arXiv 1705.11147, Sections 2 and 5.1),
// written for sm_103a. All of the work is integer hashing, bit manipulation and atomics on
// HBM-resident structures: no tensor cores.
//
//   pack_kernel       reads (ASCII + Phred) -> 2-bit codes, invalid bits, high-quality bits
//   pass_kernel       one thread per window start: extraction of the forward and reverse
//                     complement 2-bit words (one 128-bit value covers k <= 63), canonical
//                     key, then per mode
//                       Bloom:   test-and-set of the k-mer's bits in one 64-bit Bloom word
//                                (atomicOr). Already set -> insert-if-absent + count.
//                                Not set -> this window is the k-mer's first sighting: mark it.
//                       Count:   no Bloom filter: insert-if-absent + count every window.
//                       Recount: marked windows add their count/extensions if their k-mer
//                                made it into the table (it was seen at least twice).
//   classify_kernel   depth filter, side codes, compaction into output arrays
//   query_kernel      read-only lookups, answers re-oriented to the query
//
// Exactness with a Bloom filter (Section 5.1 keeps k-mers the filter reports as seen):
// all bits of a k-mer live in one word and are set by one atomicOr, so across all
// occurrences of a k-mer at most one observes "not all set" (exactly one unless a false
// positive). That occurrence is marked and counted in the recount pass if, and only if, the
// k-mer reached the table through another occurrence. Every occurrence of every k-mer with
// two or more occurrences is therefore counted exactly once; singletons are either absent
// or (false positives) present with count 1, which any min_depth >= 2 removes.
#include "kma_internal.cuh"

namespace kma {

typedef unsigned long long u64;
typedef unsigned __int128 u128;

// ------------------------------------------------------------------ hashing

// 64-bit finaliser of MurmurHash3 (Appleby).
__device__ __forceinline__ u64 fmix64(u64 x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__device__ __forceinline__ u64 key_hash(u64 lo, u64 hi) {
  return fmix64(lo ^ fmix64(hi + 0x9e3779b97f4a7c15ull));
}

__device__ __forceinline__ u64 table_index(u64 h, u64 slots) { return __umul64hi(fmix64(h ^ 0x2545f4914f6cdd1dull), slots); }
__device__ __forceinline__ u64 bloom_index(u64 h, u64 words) { return __umul64hi(h, words); }
__device__ __forceinline__ unsigned owner_of(u64 h, unsigned n_parts) {
  return (unsigned)__umul64hi(fmix64(h ^ 0x9fb21c651e98df25ull), n_parts);
}

__device__ __forceinline__ u64 bloom_mask(u64 h, unsigned nbits) {
  u64 g = fmix64(h + 0x632be59bd9b4e019ull);
  u64 m = 0;
  for (unsigned i = 0; i < nbits; ++i) m |= 1ull << ((g >> (6 * i)) & 63);
  return m;
}

// ------------------------------------------------------------------ 2-bit words

// Reverse the order of the 32 two-bit groups of x.
__device__ __forceinline__ u64 rev2(u64 x) {
  x = __brevll(x);
  return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

// Reverse complement of a k-mer held in the low 2k bits of (hi:lo).
__device__ __forceinline__ void revcomp(u64 lo, u64 hi, unsigned k, u64& rlo, u64& rhi) {
  u128 r = ((u128)rev2(lo) << 64) | (u128)rev2(hi);
  r = ~r;
  r >>= (128 - 2 * k);
  rlo = (u64)r;
  rhi = (u64)(r >> 64);
}

__device__ __forceinline__ unsigned code_at(const u64* codes, u64 p) {
  return (unsigned)(codes[p >> 5] >> (62 - 2 * (p & 31))) & 3u;
}

__device__ __forceinline__ unsigned bit_at(const u64* bits, u64 p) {
  return (unsigned)(bits[p >> 6] >> (63 - (p & 63))) & 1u;
}

struct Window {
  u64 lo, hi;        // canonical key
  unsigned lb, rb;   // extension bases in the key's orientation
  bool lu, ru;       // usable (exists, A/C/G/T, Phred >= threshold)
};

// Window starting at arena position q: returns false if any of its k positions is invalid.
__device__ __forceinline__ bool load_window(const PassDesc& D, u64 q, Window& w) {
  const unsigned k = D.k;
  const u64 v = q >> 6;
  const unsigned t = (unsigned)(q & 63);
  u64 x = D.inv[v] << t;
  if (t) x |= D.inv[v + 1] >> (64 - t);
  if (x >> (64 - k)) return false;

  const u64 wi = q >> 5;
  const unsigned s = 2 * (unsigned)(q & 31);
  const u64 a = D.codes[wi], b = D.codes[wi + 1], c = D.codes[wi + 2];
  u128 top = ((u128)a << 64) | (u128)b;
  if (s) top = (top << s) | (u128)(c >> (64 - s));
  const u128 fw = top >> (128 - 2 * k);
  const u64 flo = (u64)fw, fhi = (u64)(fw >> 64);

  // Extension bases: position q-1 (before) and q+k (after).
  const bool bu = q > 0 && bit_at(D.hq, q - 1);
  const bool au = bit_at(D.hq, q + k) != 0;
  const unsigned bb = q > 0 ? code_at(D.codes, q - 1) : 0u;
  const unsigned ab = (unsigned)(top >> (126 - 2 * k)) & 3u;  // the base right after the window

  u64 rlo, rhi;
  revcomp(flo, fhi, k, rlo, rhi);
  const bool forward = !D.canonical || (fhi < rhi) || (fhi == rhi && flo <= rlo);
  if (forward) {
    w.lo = flo; w.hi = fhi;
    w.lb = bb; w.lu = bu;
    w.rb = ab; w.ru = au;
  } else {
    w.lo = rlo; w.hi = rhi;
    w.lb = 3u - ab; w.lu = au;
    w.rb = 3u - bb; w.ru = bu;
  }
  return true;
}

// ------------------------------------------------------------------ table

__device__ __forceinline__ void cas128(Slot* s, u64 cmp_lo, u64 cmp_hi, u64 new_lo, u64 new_hi,
                                       u64& old_lo, u64& old_hi) {
  asm volatile(
      "{\n\t"
      ".reg .b128 d, c, n;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 n, {%4, %5};\n\t"
      "atom.global.cas.b128 d, [%6], c, n;\n\t"
      "mov.b128 {%0, %1}, d;\n\t"
      "}"
      : "=l"(old_lo), "=l"(old_hi)
      : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(s)
      : "memory");
}

// Insert-if-absent. Keys are written once (empty -> key) by a 16-byte CAS and never change
// again. A plain 16-byte load may observe a half-written slot; any value with a word still
// equal to the empty pattern is therefore resolved by the CAS itself, which is atomic.
// Returns the slot or nullptr (probe limit reached: the table is full).
__device__ __forceinline__ Slot* find_or_insert(Slot* table, u64 slots, u64 lo, u64 hi, u64 h,
                                                bool& inserted) {
  u64 idx = table_index(h, slots);
  const u64 limit = slots < kMaxProbe ? slots : kMaxProbe;
  inserted = false;
  for (u64 n = 0; n < limit; ++n) {
    Slot* s = table + idx;
    const ulonglong2 kv = __ldcg(reinterpret_cast<const ulonglong2*>(s));
    if (kv.x == lo && kv.y == hi) return s;
    if (kv.y == kEmpty || kv.x == kEmpty) {
      u64 olo, ohi;
      cas128(s, kEmpty, kEmpty, lo, hi, olo, ohi);
      if (olo == kEmpty && ohi == kEmpty) { inserted = true; return s; }
      if (olo == lo && ohi == hi) return s;
    }
    idx = (idx + 1 == slots) ? 0 : idx + 1;
  }
  return nullptr;
}

// Lookup in a table no thread is modifying. nullptr if absent; sets `full` if the probe
// limit was reached without finding an empty slot.
__device__ __forceinline__ const Slot* find(const Slot* table, u64 slots, u64 lo, u64 hi, u64 h,
                                            bool& full) {
  u64 idx = table_index(h, slots);
  const u64 limit = slots < kMaxProbe ? slots : kMaxProbe;
  full = false;
  for (u64 n = 0; n < limit; ++n) {
    const Slot* s = table + idx;
    const ulonglong2 kv = __ldcg(reinterpret_cast<const ulonglong2*>(s));
    if (kv.x == lo && kv.y == hi) return s;
    if (kv.y == kEmpty) return nullptr;
    idx = (idx + 1 == slots) ? 0 : idx + 1;
  }
  full = true;
  return nullptr;
}

__device__ __forceinline__ void add_occurrence(Slot* s, const Window& w, unsigned inc,
                                               DevStatus* st) {
  const unsigned old = atomicAdd(&s->count, inc);
  if (old > 0xFFFFFFFFu - inc) atomicOr(&st->flags, kFlagOverflow);
  if (w.lu) atomicAdd(&s->ext[w.lb], 1u);
  if (w.ru) atomicAdd(&s->ext[4 + w.rb], 1u);
}

// Warp-aggregated variant: lanes in `act` holding the same slot merge their count into one
// atomic, and lanes adding to the same extension counter merge theirs.
__device__ __forceinline__ void add_occurrence_agg(unsigned act, Slot* s, const Window& w,
                                                   DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(act, reinterpret_cast<u64>(s));
  if (lane == __ffs(peers) - 1) {
    const unsigned inc = __popc(peers);
    const unsigned old = atomicAdd(&s->count, inc);
    if (old > 0xFFFFFFFFu - inc) atomicOr(&st->flags, kFlagOverflow);
  }
  const unsigned lact = __ballot_sync(act, w.lu);
  if (w.lu) {
    unsigned* a = &s->ext[w.lb];
    const unsigned m = __match_any_sync(lact, reinterpret_cast<u64>(a));
    if (lane == __ffs(m) - 1) atomicAdd(a, (unsigned)__popc(m));
  }
  const unsigned ract = __ballot_sync(act, w.ru);
  if (w.ru) {
    unsigned* a = &s->ext[4 + w.rb];
    const unsigned m = __match_any_sync(ract, reinterpret_cast<u64>(a));
    if (lane == __ffs(m) - 1) atomicAdd(a, (unsigned)__popc(m));
  }
}

// ------------------------------------------------------------------ pass kernel

__device__ __forceinline__ int find_pass_sample(const PassBatch& B, u64 t) {
  int lo = 0, hi = (int)B.n;  // largest s with tile_begin <= t
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.d[mid].tile_begin <= t) lo = mid; else hi = mid;
  }
  return lo;
}

template <bool AGG>
__global__ void __launch_bounds__(1024) pass_kernel(const __grid_constant__ PassBatch B, int wpt) {
  const unsigned lane = threadIdx.x & 31;
  const u64 tile = (u64)blockDim.x * (u64)wpt;
  // Per-warp running totals, flushed when the warp moves to another sample.
  int cur = -1;
  u64 acc_valid = 0, acc_ins = 0, acc_first = 0;

  for (u64 t = blockIdx.x; t < B.total_tiles; t += gridDim.x) {
    const int si = find_pass_sample(B, t);
    const PassDesc& D = B.d[si];
    if (si != cur) {
      if (cur >= 0 && lane == 0) {
        if (acc_valid) atomicAdd(&B.d[cur].status->valid_windows, acc_valid);
        if (acc_ins) atomicAdd(&B.d[cur].status->table_keys, acc_ins);
        if (acc_first) atomicAdd(&B.d[cur].status->first_sightings, acc_first);
      }
      cur = si;
      acc_valid = acc_ins = acc_first = 0;
    }
    const u64 base = D.q0 + (t - D.tile_begin) * tile;
    for (int j = 0; j < wpt; ++j) {
      const u64 q = base + (u64)j * blockDim.x + threadIdx.x;
      if (q - lane >= D.q1) break;  // whole warp past the end (q1 is a multiple of 64)
      Window w;
      if (D.mode == kModeRecount) {
        const unsigned mw = D.marks[q >> 5];
        if (!((mw >> lane) & 1u)) continue;
        if (!load_window(D, q, w)) continue;  // cannot happen: marks are set on valid windows
        const u64 h = key_hash(w.lo, w.hi);
        bool full;
        Slot* s = const_cast<Slot*>(find(D.table, D.slots, w.lo, w.hi, h, full));
        if (full) atomicOr(&D.status->flags, kFlagFull);
        if (s) add_occurrence(s, w, 1u, D.status);
        continue;
      }
      bool valid = q < D.q1 && load_window(D, q, w);
      u64 h = 0;
      if (valid) {
        h = key_hash(w.lo, w.hi);
        if (D.n_parts > 1 && owner_of(h, D.n_parts) != D.part) valid = false;  // not ours
      }
      bool count_it = valid;
      if (D.mode == kModeBloom) {
        bool first = false;
        if (valid) {
          const u64 m = bloom_mask(h, D.bloom_h);
          const u64 old = atomicOr(D.bloom + bloom_index(h, D.bloom_words), m);
          first = (old & m) != m;
        }
        const unsigned mark = __ballot_sync(0xffffffffu, first);
        if (lane == 0) D.marks[q >> 5] = mark;
        acc_first += __popc(mark);
        count_it = valid && !first;
      }
      const unsigned nv = __popc(__ballot_sync(0xffffffffu, valid));
      acc_valid += nv;
      Slot* s = nullptr;
      bool inserted = false;
      if (count_it) {
        s = find_or_insert(D.table, D.slots, w.lo, w.hi, h, inserted);
        if (!s) atomicOr(&D.status->flags, kFlagFull);
      }
      acc_ins += __popc(__ballot_sync(0xffffffffu, inserted));
      if (AGG) {
        const unsigned act = __ballot_sync(0xffffffffu, s != nullptr);
        if (s) add_occurrence_agg(act, s, w, D.status);
      } else {
        if (s) add_occurrence(s, w, 1u, D.status);
      }
    }
  }
  if (cur >= 0 && lane == 0) {
    if (acc_valid) atomicAdd(&B.d[cur].status->valid_windows, acc_valid);
    if (acc_ins) atomicAdd(&B.d[cur].status->table_keys, acc_ins);
    if (acc_first) atomicAdd(&B.d[cur].status->first_sightings, acc_first);
  }
}

// ------------------------------------------------------------------ pack kernel

__device__ __forceinline__ int find_pack_sample(const PackBatch& B, u64 w) {
  int lo = 0, hi = (int)B.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.d[mid].word_begin <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// One thread per 64 arena positions: writes two code words, one invalid word, one hq word.
__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ PackBatch B) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 w = (u64)blockIdx.x * blockDim.x + threadIdx.x; w < B.total_words; w += stride) {
    const int si = find_pack_sample(B, w);
    const PackDesc& D = B.d[si];
    const u64 lw = w - D.word_begin;
    const u64 p0 = lw * 64;  // batch-relative position
    const u64* off = D.offsets;
    const u64 o0 = off[0];
    if (lw == 0 && off[D.n_reads] - o0 != D.n_bases) atomicOr(&D.status->flags, kFlagBadOffsets);
    // Read r starts at ps_r = offsets[r] - o0 + r; find the last read starting at or before p0.
    u64 r = 0;
    if (D.n_reads > 0) {
      u64 lo = 0, hi = D.n_reads;
      while (hi - lo > 1) {
        const u64 mid = (lo + hi) >> 1;
        if (off[mid] - o0 + mid <= p0) lo = mid; else hi = mid;
      }
      r = lo;
    }
    u64 rs = D.n_reads ? off[r] - o0 + r : 0;        // start of read r
    u64 re = D.n_reads ? off[r + 1] - o0 + r : 0;    // its separator position
    if (D.n_reads && off[r + 1] < off[r]) atomicOr(&D.status->flags, kFlagBadOffsets);
    u64 c0 = 0, c1 = 0, inv = 0, hq = 0;
    for (int i = 0; i < 64; ++i) {
      const u64 p = p0 + i;
      while (r < D.n_reads && p > re) {  // move to the read containing p
        ++r;
        if (r < D.n_reads) {
          rs = off[r] - o0 + r;
          re = off[r + 1] - o0 + r;
          if (off[r + 1] < off[r]) atomicOr(&D.status->flags, kFlagBadOffsets);
        }
      }
      unsigned code = 0, valid = 0, good = 0;
      // batch-relative base index; only bases inside [0, n_bases) are ever read
      const u64 bidx = off[r] - o0 + (p - rs);
      if (r < D.n_reads && p < re && p >= rs && bidx < D.n_bases) {
        const u64 b = o0 + bidx - (u64)D.delta;
        const unsigned ch = D.seq[b] & 0xDFu;
        valid = (ch == 'A') | (ch == 'C') | (ch == 'G') | (ch == 'T');
        code = ch == 'C' ? 1u : ch == 'G' ? 2u : ch == 'T' ? 3u : 0u;
        good = valid && (unsigned)D.qual[b] >= D.qual_min;
      }
      if (i < 32) c0 |= (u64)code << (62 - 2 * i);
      else c1 |= (u64)code << (62 - 2 * (i - 32));
      inv |= (u64)(!valid) << (63 - i);
      hq |= (u64)good << (63 - i);
    }
    const u64 gw = (D.q0 >> 6) + lw;
    D.codes[2 * gw] = c0;
    D.codes[2 * gw + 1] = c1;
    D.inv[gw] = inv;
    D.hq[gw] = hq;
  }
}

// ------------------------------------------------------------------ classify + compact

__device__ __forceinline__ unsigned side_code(const unsigned* e, unsigned min_ext) {
  unsigned n = 0, b = 0;
#pragma unroll
  for (unsigned j = 0; j < 4; ++j)
    if (e[j] >= min_ext) { ++n; b = j; }
  return n == 0 ? 4u : (n >= 2 ? 5u : b);
}

__device__ __forceinline__ int find_class_sample(const ClassBatch& B, u64 blk) {
  int lo = 0, hi = (int)B.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.d[mid].block_begin <= blk) lo = mid; else hi = mid;
  }
  return lo;
}

constexpr int kClassThreads = 256;
constexpr int kClassItems = 4;  // slots per thread per block tile

__global__ void __launch_bounds__(kClassThreads) classify_kernel(const __grid_constant__ ClassBatch B) {
  __shared__ unsigned warp_tot[kClassThreads / 32];
  __shared__ u64 blk_base;
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int cur = -1;
  u64 acc_uu = 0;
  for (u64 blk = blockIdx.x; blk < B.total_blocks; blk += gridDim.x) {
    const int si = find_class_sample(B, blk);
    const ClassDesc& D = B.d[si];
    if (si != cur) {
      if (cur >= 0 && acc_uu) atomicAdd(&B.d[cur].status->n_uu, acc_uu);
      cur = si;
      acc_uu = 0;
    }
    const u64 first = (blk - D.block_begin) * (u64)(kClassThreads * kClassItems);
    bool keep[kClassItems];
    unsigned nk = 0;
#pragma unroll
    for (int it = 0; it < kClassItems; ++it) {
      const u64 i = first + (u64)it * kClassThreads + threadIdx.x;
      keep[it] = false;
      if (i < D.slots) {
        const Slot* s = D.table + i;
        if (__ldcg(&s->hi) != kEmpty && __ldcg(&s->count) >= D.min_depth) keep[it] = true;
      }
      nk += keep[it];
    }
    // block-wide exclusive scan of nk
    unsigned incl = nk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned wbase = 0, btot = 0;
    for (int x = 0; x < kClassThreads / 32; ++x) {
      if ((unsigned)x < warp) wbase += warp_tot[x];
      btot += warp_tot[x];
    }
    if (threadIdx.x == 0) blk_base = btot ? atomicAdd(&D.status->n_out, (u64)btot) : 0;
    __syncthreads();
    u64 pos = blk_base + wbase + (incl - nk);
#pragma unroll
    for (int it = 0; it < kClassItems; ++it) {
      if (!keep[it]) continue;
      const u64 i = first + (u64)it * kClassThreads + threadIdx.x;
      const Slot* s = D.table + i;
      const ulonglong2 kv = __ldcg(reinterpret_cast<const ulonglong2*>(s));
      const unsigned c = __ldcg(&s->count);
      const uint4 e0 = __ldcg(reinterpret_cast<const uint4*>(&s->ext[0]));
      const uint4 e1 = __ldcg(reinterpret_cast<const uint4*>(&s->ext[4]));
      const unsigned el[4] = {e0.x, e0.y, e0.z, e0.w};
      const unsigned er[4] = {e1.x, e1.y, e1.z, e1.w};
      const unsigned lc = side_code(el, D.min_ext), rc = side_code(er, D.min_ext);
      acc_uu += (lc < 4 && rc < 4);
      if (pos < D.out_cap) {
        reinterpret_cast<ulonglong2*>(D.out_keys)[pos] = kv;
        D.out_counts[pos] = c;
        reinterpret_cast<uint4*>(D.out_ext)[2 * pos] = e0;
        reinterpret_cast<uint4*>(D.out_ext)[2 * pos + 1] = e1;
        reinterpret_cast<uchar2*>(D.out_codes)[pos] = make_uchar2((unsigned char)lc, (unsigned char)rc);
      } else {
        atomicOr(&D.status->flags, kFlagFull);
      }
      ++pos;
    }
    __syncthreads();  // warp_tot / blk_base reuse
  }
  // n_uu: reduce inside the warp first
  if (cur >= 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_uu += __shfl_down_sync(0xffffffffu, acc_uu, o);
    if (lane == 0 && acc_uu) atomicAdd(&B.d[cur].status->n_uu, acc_uu);
  }
}

// ------------------------------------------------------------------ query

__global__ void __launch_bounds__(256) query_kernel(const Slot* table, u64 slots, unsigned k,
                                                    unsigned canonical, unsigned min_depth,
                                                    unsigned min_ext, const u64* keys, u64 n,
                                                    unsigned* counts, unsigned* ext,
                                                    unsigned char* codes, DevStatus* st) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u64 qlo = keys[2 * i], qhi = keys[2 * i + 1];
    // bits at or above 2k must be clear
    const bool in_range = (2 * k >= 64) ? (2 * k == 128 || (qhi >> (2 * k - 64)) == 0)
                                        : (qhi == 0 && (qlo >> (2 * k)) == 0);
    unsigned e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned c = 0;
    if (in_range) {
      u64 rlo, rhi;
      revcomp(qlo, qhi, k, rlo, rhi);
      const bool forward = !canonical || (qhi < rhi) || (qhi == rhi && qlo <= rlo);
      const u64 lo = forward ? qlo : rlo, hi = forward ? qhi : rhi;
      bool full;
      const Slot* s = find(table, slots, lo, hi, key_hash(lo, hi), full);
      if (full) atomicOr(&st->flags, kFlagFull);
      if (s && s->count >= min_depth) {
        c = s->count;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (forward) {
            e[b] = s->ext[b];
            e[4 + b] = s->ext[4 + b];
          } else {
            e[3 - b] = s->ext[4 + b];   // query's left = complement of key's right
            e[4 + 3 - b] = s->ext[b];   // query's right = complement of key's left
          }
        }
      }
    }
    counts[i] = c;
#pragma unroll
    for (int j = 0; j < 8; ++j) ext[8 * i + j] = e[j];
    codes[2 * i] = (unsigned char)(c ? side_code(e, min_ext) : 4u);
    codes[2 * i + 1] = (unsigned char)(c ? side_code(e + 4, min_ext) : 4u);
  }
}

// ------------------------------------------------------------------ table init

__global__ void __launch_bounds__(256) table_init_kernel(Slot* table, u64 slots) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const ulonglong2 empty = make_ulonglong2(kEmpty, kEmpty);
  const ulonglong2 zero = make_ulonglong2(0, 0);
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += stride) {
    ulonglong2* s = reinterpret_cast<ulonglong2*>(table + i);
    __stcg(s + 0, empty);
    __stcg(s + 1, zero);
    __stcg(s + 2, zero);
    __stcg(s + 3, zero);
  }
}

// ------------------------------------------------------------------ launchers

int pass_max_ctas_per_sm(int block_threads, int wpt, bool agg) {
  (void)wpt;
  int n = 0;
  cudaError_t e = agg ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pass_kernel<true>, block_threads, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pass_kernel<false>, block_threads, 0);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_pass(const PassBatch& b, const LaunchShape& shape, bool agg, cudaStream_t stream) {
  if (b.total_tiles == 0) return cudaSuccess;
  u64 grid = (u64)shape.grid;
  if (grid > b.total_tiles) grid = b.total_tiles;
  if (agg) pass_kernel<true><<<(unsigned)grid, shape.block_threads, 0, stream>>>(b, shape.windows_per_thread);
  else pass_kernel<false><<<(unsigned)grid, shape.block_threads, 0, stream>>>(b, shape.windows_per_thread);
  return cudaGetLastError();
}

cudaError_t launch_pack(const PackBatch& b, cudaStream_t stream, int num_sms) {
  if (b.total_words == 0) return cudaSuccess;
  u64 blocks = (b.total_words + 255) / 256;
  const u64 cap = (u64)num_sms * 8;
  if (blocks > cap) blocks = cap;
  pack_kernel<<<(unsigned)blocks, 256, 0, stream>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_classify(const ClassBatch& b, cudaStream_t stream, int num_sms) {
  if (b.total_blocks == 0) return cudaSuccess;
  u64 grid = b.total_blocks;
  const u64 cap = (u64)num_sms * 8;
  if (grid > cap) grid = cap;
  classify_kernel<<<(unsigned)grid, kClassThreads, 0, stream>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_table_init(Slot* table, u64 slots, cudaStream_t stream) {
  if (slots == 0) return cudaSuccess;
  u64 blocks = (slots + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  table_init_kernel<<<(unsigned)blocks, 256, 0, stream>>>(table, slots);
  return cudaGetLastError();
}

cudaError_t launch_query(const Slot* table, u64 slots, unsigned k, unsigned canonical,
                         unsigned min_depth, unsigned min_ext, const u64* keys, u64 n,
                         unsigned* counts, unsigned* ext, unsigned char* codes, DevStatus* st,
                         cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  u64 blocks = (n + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  query_kernel<<<(unsigned)blocks, 256, 0, stream>>>(table, slots, k, canonical, min_depth, min_ext,
                                                     keys, n, counts, ext, codes, st);
  return cudaGetLastError();
}

}  // namespace kma
