// Device helpers shared by the library's kernels (not part of the C ABI): hashing, 2-bit
// k-mer words, window extraction from the packed-read arena, and the hash-table operations.
#pragma once
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

// 64-bit hash of a 128-bit key: the high word is spread by an odd multiplier (plus a
// constant), folded into the low word, and the result mixed by one finaliser.
__device__ __forceinline__ u64 key_hash(u64 lo, u64 hi) {
  return fmix64(lo ^ (hi * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull));
}

// Everything derived from the 64-bit key hash h uses cheap 32-bit slices of h and of two
// more products, instead of further 64-bit mixes:
//   on-chip partition   high 32 bits of h                  (part_of)
//   Bloom word          low 32 bits of h                   (bloom_index; < 2^32 words)
//   table slot          high 32 bits of h * phi            (table_index; < 2^32 slots per part)
//   Bloom bit positions 6-bit fields from the top of (h ^ h >> 32) * c   (bloom_mask)
// The bit positions must not depend on the low bits of h alone: those also pick the word, and
// keys sharing a word would then share most of their bits (a much higher false-positive rate).
__device__ __forceinline__ u64 scramble(u64 h) { return h * 0x9e3779b97f4a7c15ull; }
__device__ __forceinline__ u64 table_index(u64 h, u64 slots) {
  return __umulhi((unsigned)(scramble(h) >> 32), (unsigned)slots);
}
__device__ __forceinline__ u64 bloom_index(u64 h, u64 words) {
  return __umulhi((unsigned)h, (unsigned)words);
}
// Owner GPU of a k-mer (multi-GPU owner-computes), independent of the bits above.
__device__ __forceinline__ unsigned owner_of(u64 h, unsigned n_parts) {
  return __umulhi((unsigned)(fmix64(h ^ 0x9fb21c651e98df25ull) >> 32), n_parts);
}

// On-chip partition (partitioned mode) of a k-mer with hash h, 0 .. P-1.
__device__ __forceinline__ unsigned part_of(u64 h, unsigned P) {
  return __umulhi((unsigned)(h >> 32), P);
}

// Mask with bit x set for each 6-bit field x taken from the top of g (field i at bits
// 58 - 6i .. 63 - 6i, i < nbits <= kMaxHashBits), built in 32-bit halves. The loop is unrolled
// so that every field is extracted with constant shifts.
constexpr unsigned kMaxHashBits = 10;
__device__ __forceinline__ u64 mask_from_fields(u64 g, unsigned nbits) {
  const unsigned gh = (unsigned)(g >> 32), gl = (unsigned)g;
  unsigned lo = 0, hi = 0;
#pragma unroll
  for (int i = 0; i < (int)kMaxHashBits; ++i) {
    if (i < (int)nbits) {
      const int off = 58 - 6 * i;
      const unsigned x = off >= 32 ? (gh >> (off - 32)) & 63u
                                   : (off + 6 <= 32 ? (gl >> off) & 63u : __funnelshift_r(gl, gh, off) & 63u);
      const unsigned bit = 1u << (x & 31u);
      if (x & 32u) hi |= bit; else lo |= bit;
    }
  }
  return ((u64)hi << 32) | lo;
}

__device__ __forceinline__ u64 bloom_mask(u64 h, unsigned nbits) {
  return mask_from_fields((h ^ (h >> 32)) * 0xd6e8feb86659fd93ull, nbits);
}

// Key filter (partitioned recount): one 64-bit word per key, chosen by the low half of
// h * phi (the table slot uses its high half), bits from the top of (h ^ h >> 32) * c' with a
// multiplier of its own.
__device__ __forceinline__ u64 keyfilter_index(u64 h, u64 words) {
  return __umulhi((unsigned)scramble(h), (unsigned)words);
}
__device__ __forceinline__ u64 keyfilter_mask(u64 h, unsigned nbits) {
  return mask_from_fields((h ^ (h >> 32)) * 0x94d049bb133111ebull, nbits);
}

// L2 cache policy for data read or written once (record streams): evict first, so the
// partition's Bloom sub-filter and sub-table stay resident.
__device__ __forceinline__ u64 policy_evict_first() {
  u64 pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ ulonglong2 ld_stream(const ulonglong2* p, u64 pol) {
  ulonglong2 v;
  asm volatile("ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
               : "=l"(v.x), "=l"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ u64 ld_stream(const u64* p, u64 pol) {
  u64 v;
  asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ unsigned ld_stream(const unsigned char* p, u64 pol) {
  unsigned v;
  asm volatile("ld.global.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_stream(ulonglong2* p, ulonglong2 v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::"l"(p), "l"(v.x), "l"(v.y), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_stream(u64* p, u64 v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_stream(unsigned char* p, unsigned v, u64 pol) {
  asm volatile("st.global.L2::cache_hint.u8 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}


// ------------------------------------------------------------------ bulk copies (TMA)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 1-D TMA bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16),
// completion signalled on the mbarrier as transaction bytes.
__device__ __forceinline__ void tma_load_1d(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// The same copy with an L2 cache policy (evict-first for streams read once).
__device__ __forceinline__ void tma_load_1d_hint(unsigned dst, const void* src, unsigned bytes, unsigned bar,
                                                 u64 pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(pol) : "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before later bulk
// copies into it (a buffer read by the CTA, then refilled by a copy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Test for the phase; while it is incomplete the thread may be suspended, and it resumes when
// the phase completes or after at most kWaitHintNs nanoseconds. A waiting warp therefore
// sleeps instead of spinning (no issue slots spent on polling).
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned phase) {
  unsigned done;
  asm volatile("{\n\t.reg .pred p;\n\t"
               "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(done) : "r"(bar), "r"(phase), "n"(kWaitHintNs) : "memory");
  return done != 0;
}

// Bounded wait for the mbarrier phase: returns false (and the caller raises a status flag)
// if the copies have not completed after `limit` polls (at most limit * kWaitHintNs ns).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned phase, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// After a wait that gave up: before the CTA may exit, the bulk copies already issued into its
// shared memory must land. Waits up to 8 times the first limit (still bounded; copies that
// have not landed by then are reported by the flag the caller already raised).
__device__ __forceinline__ bool mbar_drain(unsigned bar, unsigned phase, unsigned limit) {
  for (unsigned r = 0; r < 8; ++r)
    if (mbar_wait_bounded(bar, phase, limit)) return true;
  return false;
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

// (a:b) << s, top 64 bits, for 0 <= s < 64.
__device__ __forceinline__ u64 fshl(u64 a, u64 b, unsigned s) { return s ? (a << s) | (b >> (64 - s)) : a; }
// (b:a) >> s, low 64 bits, for 0 <= s < 64.
__device__ __forceinline__ u64 fshr(u64 a, u64 b, unsigned s) { return s ? (a >> s) | (b << (64 - s)) : a; }

// Window starting at arena position q: returns false if any of its k positions is invalid.
// The forward k-mer is read MSB-first from `codes`, its reverse complement LSB-first from
// `rcodes` (both one funnel shift per 64-bit word), the canonical key is the smaller.
__device__ __forceinline__ bool load_window(const u64* codes, const u64* rcodes, const u64* inv,
                                            const u64* hq, unsigned k, unsigned canonical, u64 q,
                                            Window& w) {
  const u64 v = q >> 6;
  const unsigned t = (unsigned)(q & 63);
  if (fshl(inv[v], inv[v + 1], t) >> (64 - k)) return false;

  const u64 wi = q >> 5;
  const unsigned s = 2 * (unsigned)(q & 31);
  const u64 a = codes[wi], b = codes[wi + 1];
  const u64 top = fshl(a, b, s);  // first 32 bases of the window, MSB-first
  u64 flo, fhi, rlo, rhi;
  const u64 r0 = rcodes[wi], r1 = rcodes[wi + 1];
  const u64 bot = fshr(r0, r1, s);  // reverse complement, low 64 bits
  if (k > 32) {
    const u64 c = codes[wi + 2];
    const u64 mid = fshl(b, c, s);
    const unsigned sh = 128 - 2 * k;  // 2 .. 62
    flo = (mid >> sh) | (top << (64 - sh));
    fhi = top >> sh;
    const u64 r2 = rcodes[wi + 2];
    rlo = bot;
    rhi = fshr(r1, r2, s) & ((1ull << (2 * k - 64)) - 1);
  } else {
    flo = top >> (64 - 2 * k);
    fhi = 0;
    rlo = k == 32 ? bot : bot & ((1ull << (2 * k)) - 1);
    rhi = 0;
  }

  // Extension bases: position q-1 (before) and q+k (after).
  const bool bu = q > 0 && bit_at(hq, q - 1);
  const bool au = bit_at(hq, q + k) != 0;
  const unsigned bb = q > 0 ? code_at(codes, q - 1) : 0u;
  const unsigned ab = code_at(codes, q + k);

  const bool forward = !canonical || (fhi < rhi) || (fhi == rhi && flo <= rlo);
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

__device__ __forceinline__ bool load_window(const PassDesc& D, u64 q, Window& w) {
  return load_window(D.codes, D.rcodes, D.inv, D.hq, D.k, D.canonical, q, w);
}

// Consecutive windows starting at q (a multiple of 8), one at a time: the state
// holds the forward k-mer F and its reverse complement R of the current window, the next
// bases to enter (MSB first), and the invalid / high-quality bits around the windows.
struct RollingWindows {
  u64 fhi, flo, rhi, rlo;  // F and R as 2k-bit numbers (first base most / least significant)
  u64 nxt;                 // bases q + k, q + k + 1, ... (MSB first)
  u64 iv0, iv1;            // invalid bits from q (MSB first), 128 of them
  u64 hl, hr;              // hq bits from q - 1 (left extensions) and from q + k (right)
  unsigned left;           // base at q - 1 (left extension of window q)
  unsigned k;

  __device__ __forceinline__ void init(const PartWindows& W, unsigned kk, u64 q) {
    k = kk;
    const u64 v = q >> 6;
    const unsigned t = (unsigned)(q & 63);
    const u64 i0 = W.inv[v], i1 = W.inv[v + 1], i2 = W.inv[v + 2];
    iv0 = fshl(i0, i1, t);
    iv1 = fshl(i1, i2, t);
    const u64 h0 = W.hq[v];
    if (q > 0) {
      const u64 vl = (q - 1) >> 6;
      hl = fshl(W.hq[vl], W.hq[vl + 1], (unsigned)((q - 1) & 63));
      left = code_at(W.codes, q - 1);
    } else {
      hl = h0 >> 1;  // no position before the arena: unusable
      left = 0;
    }
    const u64 qr = q + k, vr = qr >> 6;
    hr = fshl(W.hq[vr], W.hq[vr + 1], (unsigned)(qr & 63));
    const u64 wr = qr >> 5;
    nxt = fshl(W.codes[wr], W.codes[wr + 1], 2 * (unsigned)(qr & 31));
    // window q itself, as in load_window
    const u64 wi = q >> 5;
    const unsigned sh2 = 2 * (unsigned)(q & 31);
    const u64 a = W.codes[wi], b = W.codes[wi + 1];
    const u64 top = fshl(a, b, sh2);
    const u64 r0 = W.rcodes[wi], r1 = W.rcodes[wi + 1];
    const u64 bot = fshr(r0, r1, sh2);
    if (k > 32) {
      const u64 mid = fshl(b, W.codes[wi + 2], sh2);
      const unsigned sh = 128 - 2 * k;
      flo = (mid >> sh) | (top << (64 - sh));
      fhi = top >> sh;
      rlo = bot;
      rhi = fshr(r1, W.rcodes[wi + 2], sh2) & ((1ull << (2 * k - 64)) - 1);
    } else {
      flo = top >> (64 - 2 * k);
      fhi = 0;
      rlo = k == 32 ? bot : bot & ((1ull << (2 * k)) - 1);
      rhi = 0;
    }
  }

  // Window j of the run (the state holds window j): valid flag and the canonical window.
  __device__ __forceinline__ bool get(unsigned j, unsigned canonical, Window& w) const {
    const u64 bad = (j ? (iv0 << j) | (iv1 >> (64 - j)) : iv0) >> (64 - k);
    if (bad) return false;
    const unsigned ab = (unsigned)(nxt >> 62);              // base q + j + k
    const bool au = (hr >> (63 - j)) & 1u;
    const bool bu = (hl >> (63 - j)) & 1u;                 // base q + j - 1
    const bool forward = !canonical || (fhi < rhi) || (fhi == rhi && flo <= rlo);
    if (forward) {
      w.lo = flo; w.hi = fhi;
      w.lb = left; w.lu = bu;
      w.rb = ab; w.ru = au;
    } else {
      w.lo = rlo; w.hi = rhi;
      w.lb = 3u - ab; w.lu = au;
      w.rb = 3u - left; w.ru = bu;
    }
    return true;
  }

  // Move to the next window: the base at q + j + k enters, the first base leaves.
  __device__ __forceinline__ void roll() {
    const unsigned b = (unsigned)(nxt >> 62);
    nxt <<= 2;
    if (k > 32) {
      left = (unsigned)(fhi >> (2 * k - 66)) & 3u;
      fhi = ((fhi << 2) | (flo >> 62)) & ((1ull << (2 * k - 64)) - 1);
      flo = (flo << 2) | b;
      rlo = (rlo >> 2) | (rhi << 62);
      rhi = (rhi >> 2) | ((u64)(3u - b) << (2 * k - 66));
    } else {
      left = (unsigned)(flo >> (2 * k - 2)) & 3u;
      flo = ((flo << 2) | b) & (k == 32 ? ~0ull : ((1ull << (2 * k)) - 1));
      rlo = (rlo >> 2) | ((u64)(3u - b) << (2 * k - 2));
    }
  }
};

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

// Counter of the occurrence's left / right outcome.
__device__ __forceinline__ unsigned* left_counter(Slot* s, const Window& w) {
  return w.lu ? &s->ext[w.lb] : &s->none[0];
}
__device__ __forceinline__ unsigned* right_counter(Slot* s, const Window& w) {
  return w.ru ? &s->ext[4 + w.rb] : &s->none[1];
}

// One occurrence (inc of them) of the slot's key, with wrap detection: every counter is at
// most the key's count, so a wrap of either updated counter is the only way one can be lost
// (a total count above 2^32 is caught when the counters are summed).
__device__ __forceinline__ void add_occurrence(Slot* s, const Window& w, unsigned inc,
                                               DevStatus* st) {
  const unsigned a = atomicAdd(left_counter(s, w), inc);
  const unsigned b = atomicAdd(right_counter(s, w), inc);
  if (a > 0xFFFFFFFFu - inc || b > 0xFFFFFFFFu - inc) atomicOr(&st->flags, kFlagOverflow);
}

// Count update when no counter can reach 2^32 (the host bounds the occurrences a key can
// have before the next reset): reductions without a returned value, nothing to wait for.
__device__ __forceinline__ void red_add(unsigned* a, unsigned v) {
  asm volatile("red.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void add_occurrence_red(Slot* s, const Window& w) {
  red_add(left_counter(s, w), 1u);
  red_add(right_counter(s, w), 1u);
}

// Warp-aggregated variant: lanes in `act` adding to the same counter merge their updates.
__device__ __forceinline__ void add_occurrence_agg(unsigned act, Slot* s, const Window& w,
                                                   DevStatus* st) {
  const int lane = threadIdx.x & 31;
  unsigned* l = left_counter(s, w);
  unsigned* r = right_counter(s, w);
  const unsigned ml = __match_any_sync(act, reinterpret_cast<u64>(l));
  const unsigned mr = __match_any_sync(act, reinterpret_cast<u64>(r));
  bool wrap = false;
  if (lane == __ffs(ml) - 1) {
    const unsigned inc = __popc(ml);
    wrap |= atomicAdd(l, inc) > 0xFFFFFFFFu - inc;
  }
  if (lane == __ffs(mr) - 1) {
    const unsigned inc = __popc(mr);
    wrap |= atomicAdd(r, inc) > 0xFFFFFFFFu - inc;
  }
  if (wrap) atomicOr(&st->flags, kFlagOverflow);
}

// Count of a slot (sum of its left outcomes), flagged if it does not fit 32 bits.
__device__ __forceinline__ unsigned slot_count(unsigned none_l, uint4 el, DevStatus* st) {
  const u64 c = (u64)none_l + el.x + el.y + el.z + el.w;
  if (c > 0xFFFFFFFFull) {
    atomicOr(&st->flags, kFlagOverflow);
    return 0xFFFFFFFFu;
  }
  return (unsigned)c;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Insert-if-absent continuing from a first probe whose slot (index idx) is already loaded.
__device__ __forceinline__ Slot* resolve_insert(Slot* table, u64 slots, u64 idx, ulonglong2 kv,
                                                u64 lo, u64 hi, bool& inserted) {
  const u64 limit = slots < kMaxProbe ? slots : kMaxProbe;
  inserted = false;
  for (u64 n = 0; n < limit; ++n) {
    Slot* s = table + idx;
    if (n) kv = __ldcg(reinterpret_cast<const ulonglong2*>(s));
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

// Lookup (table not being modified) continuing from a loaded first probe.
__device__ __forceinline__ Slot* resolve_find(Slot* table, u64 slots, u64 idx, ulonglong2 kv,
                                              u64 lo, u64 hi, bool& full) {
  const u64 limit = slots < kMaxProbe ? slots : kMaxProbe;
  full = false;
  for (u64 n = 0; n < limit; ++n) {
    Slot* s = table + idx;
    if (n) kv = __ldcg(reinterpret_cast<const ulonglong2*>(s));
    if (kv.x == lo && kv.y == hi) return s;
    if (kv.y == kEmpty) return nullptr;
    idx = (idx + 1 == slots) ? 0 : idx + 1;
  }
  full = true;
  return nullptr;
}

__device__ __forceinline__ unsigned side_code(const unsigned* e, unsigned min_ext) {
  unsigned n = 0, b = 0;
#pragma unroll
  for (unsigned j = 0; j < 4; ++j)
    if (e[j] >= min_ext) { ++n; b = j; }
  return n == 0 ? 4u : (n >= 2 ? 5u : b);
}

}  // namespace kma
