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
#include "kma_device.cuh"

namespace kma {

// ------------------------------------------------------------------ pass kernel

__device__ __forceinline__ int find_pass_sample(const PassBatch& B, u64 t) {
  int lo = 0, hi = (int)B.n;  // largest s with tile_begin <= t
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.d[mid].tile_begin <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// One tile = blockDim.x * WPT consecutive window starts; thread t takes starts
// base + j * blockDim.x + t (j < WPT), so a warp always covers 32 consecutive, 32-aligned
// starts (one marks word). The WPT windows of a thread go through the memory stages
// together: all Bloom atomics (with an L2 prefetch of each window's first table slot) are in
// flight at once, then all first probes, then the updates.
template <int WPT, bool AGG>
__global__ void __launch_bounds__(256, WPT <= 2 ? 4 : 1) pass_kernel(const __grid_constant__ PassBatch B) {
  const unsigned lane = threadIdx.x & 31;
  const u64 tile = (u64)blockDim.x * WPT;
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
    const u64 base = D.q0 + (t - D.tile_begin) * tile + threadIdx.x;
    const unsigned mode = D.mode;
    Window w[WPT];
    u64 h[WPT];
    bool in[WPT], act[WPT];

    // stage 1: extract the windows (packed reads are read coalesced through L1)
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      const u64 q = base + (u64)j * blockDim.x;
      in[j] = (q - lane) < D.q1;  // warp-uniform: q1 is a multiple of 64
      act[j] = false;
      h[j] = 0;
      if (in[j]) {
        bool ok = (mode != kModeRecount) || ((D.marks[q >> 5] >> lane) & 1u);
        ok = ok && load_window(D, q, w[j]);
        if (ok) {
          h[j] = key_hash(w[j].lo, w[j].hi);
          if (D.n_parts > 1 && owner_of(h[j], D.n_parts) != D.part) ok = false;  // not ours
        }
        act[j] = ok;
      }
    }

    // stage 2: Bloom test-and-set of every window, first sightings marked
    if (mode == kModeBloom) {
      u64 old[WPT], msk[WPT];
#pragma unroll
      for (int j = 0; j < WPT; ++j) {
        old[j] = 0;
        msk[j] = 0;
        if (act[j]) {
          msk[j] = bloom_mask(h[j], D.bloom_h);
          if (B.prefetch) prefetch_l2(D.table + table_index(h[j], D.slots));
          old[j] = atomicOr(D.bloom + bloom_index(h[j], D.bloom_words), msk[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < WPT; ++j) {
        if (!in[j]) continue;
        const bool first = act[j] && (old[j] & msk[j]) != msk[j];
        const unsigned mark = __ballot_sync(0xffffffffu, first);
        if (lane == 0) D.marks[(base + (u64)j * blockDim.x) >> 5] = mark;
        acc_first += __popc(mark);
        acc_valid += __popc(__ballot_sync(0xffffffffu, act[j]));
        act[j] = act[j] && !first;
      }
    } else if (mode == kModeCount) {
#pragma unroll
      for (int j = 0; j < WPT; ++j)
        if (in[j]) acc_valid += __popc(__ballot_sync(0xffffffffu, act[j]));
    }

    // stage 3: first probe of every window that counts
    ulonglong2 kv[WPT];
    u64 idx[WPT];
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      kv[j] = make_ulonglong2(0, 0);
      idx[j] = 0;
      if (act[j]) {
        idx[j] = table_index(h[j], D.slots);
        kv[j] = __ldcg(reinterpret_cast<const ulonglong2*>(D.table + idx[j]));
      }
    }

    // stage 4: finish the probe (insert-if-absent, or find in the recount) and count
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      Slot* s = nullptr;
      bool inserted = false;
      if (act[j]) {
        if (mode == kModeRecount) {
          bool full;
          s = resolve_find(D.table, D.slots, idx[j], kv[j], w[j].lo, w[j].hi, full);
          if (full) atomicOr(&D.status->flags, kFlagFull);
        } else {
          s = resolve_insert(D.table, D.slots, idx[j], kv[j], w[j].lo, w[j].hi, inserted);
          if (!s) atomicOr(&D.status->flags, kFlagFull);
        }
      }
      if (!in[j]) continue;
      acc_ins += __popc(__ballot_sync(0xffffffffu, inserted));
      if (AGG) {
        const unsigned a = __ballot_sync(0xffffffffu, s != nullptr);
        if (s) add_occurrence_agg(a, s, w[j], D.status);
      } else if (s) {
        if (D.no_overflow) add_occurrence_red(s, w[j]);
        else add_occurrence(s, w[j], 1u, D.status);
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

__device__ __forceinline__ int find_pack_sample(const PackBatch& B, u64 c) {
  int lo = 0, hi = (int)B.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (B.d[mid].chunk_begin <= c) lo = mid; else hi = mid;
  }
  return lo;
}

// Last read r with start ps_r = offsets[r] - o0 + r <= p, found by a warp: the answer lies in [lo, hi) and offsets[lo] - o0 + lo <= p;
// each round the 32 lanes test 32 evenly spaced reads, so ~log32(hi - lo) dependent loads
// instead of log2. Called by all lanes of a warp with the same arguments; all return it.
// With non-decreasing offsets the lanes that qualify are a prefix of the warp; `bad` is set
// when they are not (decreasing offsets), and the caller reports it.
__device__ __forceinline__ u64 read_at_warp(const u64* off, u64 o0, u64 lo, u64 hi, u64 p, bool& bad) {
  const unsigned lane = threadIdx.x & 31;
  while (hi - lo > 1) {
    const u64 step = (hi - lo + 31) / 32;
    const u64 idx = lo + lane * step;
    const bool le = idx < hi && off[idx] - o0 + idx <= p;  // a prefix of the lanes (starts increase)
    const unsigned m = __ballot_sync(0xffffffffu, le);
    bad |= (m & (m + 1u)) != 0u;
    const u64 nlo = m ? lo + (u64)(31 - __clz(m)) * step : lo;
    hi = nlo + step < hi ? nlo + step : hi;
    lo = nlo;
  }
  return lo;
}

// Same answer as read_at_warp, trying first the 32 reads around `guess` in one round of
// loads: with reads of similar length a proportional guess lands within a few reads, which
// saves the ~log32(hi - lo) dependent rounds of a search over all the batch's reads.
__device__ __forceinline__ u64 read_at_warp_near(const u64* off, u64 o0, u64 lo, u64 hi, u64 p, u64 guess,
                                                 bool& bad) {
  if (hi - lo > 32) {
    const unsigned lane = threadIdx.x & 31;
    u64 g0 = guess > lo + 16 ? guess - 16 : lo;
    if (g0 > hi - 32) g0 = hi - 32;
    const u64 idx = g0 + lane;  // inside [lo, hi)
    const unsigned m = __ballot_sync(0xffffffffu, off[idx] - o0 + idx <= p);  // a prefix of the lanes
    bad |= (m & (m + 1u)) != 0u;
    // the last read starting at or before p is inside the window: its first read qualifies and
    // a later one does not (or the window ends at hi)
    if ((m & 1u) && (m != 0xffffffffu || g0 + 32 == hi)) return g0 + (u64)(31 - __clz(m));
  }
  return read_at_warp(off, o0, lo, hi, p, bad);
}

// Batch-relative index of the first base at or after arena position p (clamped to n_bases),
// given the read r containing p.
__device__ __forceinline__ u64 base_at_or_after(const PackDesc& D, u64 o0, u64 r, u64 p) {
  const u64* off = D.offsets;
  const u64 rs = off[r] - o0 + r;
  const u64 len = off[r + 1] - off[r];
  const u64 b = (p - rs < len) ? off[r] - o0 + (p - rs) : off[r + 1] - o0;
  return b < D.n_bases ? b : D.n_bases;
}

// Four bytes starting at byte offset a of a shared-memory buffer (read as two aligned words;
// the buffer has slack past its last staged byte).
__device__ __forceinline__ unsigned load4(const unsigned* w, unsigned a) {
  const u64 v = ((u64)w[(a >> 2) + 1] << 32) | w[a >> 2];
  return (unsigned)(v >> ((a & 3u) * 8u));
}

// First position of read rr + 1 relative to the chunk start P0 (saturated: past the last read
// or beyond 32 bits).
__device__ __forceinline__ unsigned pack_next_start(const u64* off, u64 o0, u64 P0, u64 nr, u64 rr) {
  if (rr >= nr) return 0xFFFFFFFFu;
  const u64 sn = off[rr + 1] - o0 + rr + 1 - P0;
  return sn < 0xFFFFFFFFull ? (unsigned)sn : 0xFFFFFFFFu;
}

// Four positions that are all bases of one read: s = their sequence bytes, q = their quality
// bytes (first position in the low byte). Byte-parallel arithmetic gives per byte the 2-bit
// code (A0 C1 G2 T3 from bits 1..3 of the character, either case), whether the character is
// A/C/G/T at all (it must equal the upper-case letter its code names), and code/valid/quality
// flags; multiplications by sparse constants then gather the four results into
//   f8: the four codes, first position in the top bits (forward words are MSB-first),
//   r8: the four complemented codes, first position in the low bits (reverse words),
//   i4: invalid flags and h4: high-quality flags, first position in bit 3.
// An invalid position has code 0 and complemented code 3. gmask = 0 when no byte can reach
// the quality threshold (threshold above 255).
__device__ __forceinline__ void pack_group4(unsigned s, unsigned q, unsigned qmin4, unsigned gmask, unsigned& f8,
                                            unsigned& r8, unsigned& i4, unsigned& h4) {
  const unsigned H = 0x80808080u, L1 = 0x01010101u;
  unsigned code = ((s >> 1) ^ (s >> 2)) & 0x03030303u;
  const unsigned b0 = code & L1, b1 = (code >> 1) & L1;
  const unsigned letter = 0x41414141u + 2u * b0 + 6u * b1 + 11u * (b0 & b1);  // A C G T
  const unsigned d = (s & 0xDFDFDFDFu) ^ letter;
  const unsigned nz = (((d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | d) & H;  // bit 7: byte of d non-zero
  const unsigned valid = (~nz & H) >> 7;
  code &= valid * 3u;
  // per byte q >= qmin (unsigned): the low 7 bits compared by a borrow-free subtraction
  const unsigned sq = (q | H) - (qmin4 & ~H);
  const unsigned ge = ((q & ~qmin4) | (~(q ^ qmin4) & sq)) & H;
  const unsigned good = (ge >> 7) & valid & gmask;
  f8 = (code * 0x40100401u) >> 24;                   // byte k's code to bits 6 - 2k
  r8 = ((~code & 0x03030303u) * 0x01041040u) >> 24;  // byte k's complement to bits 2k
  i4 = (((valid ^ L1) * 0x08040201u) >> 24) & 0xFu;  // byte k's flag to bit 3 - k
  h4 = ((good * 0x08040201u) >> 24) & 0xFu;
}

constexpr int kPackThreads = 256;                     // 8 warps, one 64-position word per thread
constexpr int kPackChunk = kPackThreads * 64;         // positions per CTA chunk
constexpr int kPackBuf = kPackChunk + 32;             // staged bytes (+ alignment slack)

// One CTA chunk = 256 words of 64 arena positions of one sample. The bases (and qualities)
// the chunk covers are one contiguous byte range of the input; thread 0 locates it and
// stages it into shared memory with two 1-D TMA bulk copies. Thread t then builds word t of
// the chunk (its code, complemented-code, invalid and high-quality words) four positions at
// a time: four positions inside one read take the byte-parallel path (pack_group4), a group
// that holds a read's separator or starts a new read is done position by position. The
// words of consecutive threads are consecutive, so the stores coalesce.
__global__ void __launch_bounds__(kPackThreads, 4) pack_kernel(const __grid_constant__ PackBatch B) {
  __shared__ __align__(16) unsigned char s_seq[kPackBuf];
  __shared__ __align__(16) unsigned char s_qual[kPackBuf];
  __shared__ __align__(8) unsigned long long s_bar;
  __shared__ u64 s_b0, s_b1, s_r0, s_r1;
  __shared__ unsigned s_lead, s_ok;
  const unsigned bar = smem_u32(&s_bar);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  unsigned phase = 0;

  for (u64 c = blockIdx.x; c < B.total_chunks; c += gridDim.x) {
    const int si = find_pack_sample(B, c);
    const PackDesc& D = B.d[si];
    const u64* off = D.offsets;
    const u64 o0 = off[0];
    const u64 words = D.n_pos / 64;
    const u64 w0 = (c - D.chunk_begin) * kPackThreads;
    const u64 w1 = (w0 + kPackThreads < words) ? w0 + kPackThreads : words;
    // warp 0 finds the read at the chunk's first position, warp 1 the one at its end
    const unsigned warp = threadIdx.x >> 5;
    if (warp < 2) {
      const u64 p = (warp == 0 ? w0 : w1) * 64;
      u64 r = 0, b = 0;
      if (D.n_reads) {
        const u64 guess = (u64)((double)p * (double)D.n_reads / (double)(D.n_bases + D.n_reads));
        bool bad = false;
        r = read_at_warp_near(off, o0, 0, D.n_reads, p, guess, bad);
        if (bad && (threadIdx.x & 31) == 0) atomicOr(&D.status->flags, kFlagBadOffsets);
        b = base_at_or_after(D, o0, r, p);
      }
      if ((threadIdx.x & 31) == 0) {
        if (warp == 0) {
          s_b0 = b;
          s_r0 = r;
        } else {
          s_b1 = b;
          s_r1 = r;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (w0 == 0 && off[D.n_reads] - o0 != D.n_bases) atomicOr(&D.status->flags, kFlagBadOffsets);
      const u64 b0 = s_b0;
      u64 b1 = s_b1;
      unsigned ok = 1;
      if (b1 < b0 || b1 - b0 > (u64)kPackChunk || s_r1 < s_r0) {  // only with inconsistent offsets
        atomicOr(&D.status->flags, kFlagBadOffsets);
        b1 = b0;
        ok = 0;
      }
      const u64 a = reinterpret_cast<u64>(D.seq) + o0 + b0 - (u64)D.delta;
      const u64 aq = reinterpret_cast<u64>(D.qual) + o0 + b0 - (u64)D.delta;
      const unsigned lead = (unsigned)(a & 15);
      // the quality array must share the alignment phase to reuse `lead`; otherwise
      // stage it from its own aligned base (lead differs) -- handled by two leads below
      const unsigned leadq = (unsigned)(aq & 15);
      const unsigned n = (unsigned)(b1 - b0);
      s_b1 = b1;
      s_lead = lead | (leadq << 8);
      s_ok = ok;
      if (n) {
        const unsigned bytes = (lead + n + 15u) & ~15u;
        const unsigned bytesq = (leadq + n + 15u) & ~15u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, bytes + bytesq);
        if (!B.skip_copy) {
          tma_load_1d(smem_u32(s_seq), reinterpret_cast<const void*>(a - lead), bytes, bar);
          tma_load_1d(smem_u32(s_qual), reinterpret_cast<const void*>(aq - leadq), bytesq, bar);
        }
      }
    }
    // thread 0 waits for the two copies (bounded); the block barrier then publishes the
    // staged bytes to every thread
    if (threadIdx.x == 0 && s_b1 > s_b0) {
      if (mbar_wait_bounded(bar, phase, B.wait_limit)) {
        phase ^= 1u;
      } else {
        atomicOr(&D.status->flags, kFlagTimeout);
        if (!B.skip_copy) mbar_drain(bar, phase, B.wait_limit);  // copies may still land
        s_ok = 2;
      }
    }
    __syncthreads();
    if (s_ok == 2) return;  // uniform: the chunk's input never arrived
    // the chunk's reads must not decrease (device offsets are not checked on the host)
    for (u64 r = s_r0 + threadIdx.x; r < s_r1 && r < D.n_reads; r += kPackThreads)
      if (off[r + 1] < off[r]) atomicOr(&D.status->flags, kFlagBadOffsets);
    const unsigned nb = (unsigned)(s_b1 - s_b0);  // staged bases
    const unsigned lead = s_lead & 0xFF, leadq = s_lead >> 8;
    const u64 ww0 = w0 + warp * 32;                  // first word of this warp
    const u64 gw = (D.q0 >> 6) + w0 + threadIdx.x;  // the word this thread stores
    if (ww0 < w1 && s_ok) {
      // Positions are handled relative to the chunk start P0 (32-bit). A base of read r at
      // position p has batch base index p - r; the chunk's staged bytes start at the base of
      // the chunk's first position, so its byte offset is (p - P0) - (r - r0).
      const u64 nr = D.n_reads, P0 = w0 * 64, r0 = s_r0;
      bool bad = false;
      const u64 rw = nr ? read_at_warp(off, o0, s_r0, s_r1 + 1, ww0 * 64, bad) : 0;
      if (bad && (threadIdx.x & 31) == 0) atomicOr(&D.status->flags, kFlagBadOffsets);
      if (w0 + threadIdx.x < w1) {
        // the read holding this word's first position (binary search from the warp's read)
        const u64 pos = (w0 + threadIdx.x) * 64;
        u64 lo = rw, hi = nr ? s_r1 + 1 : rw;
        while (hi - lo > 1) {
          const u64 mid = (lo + hi) >> 1;
          if (off[mid] - o0 + mid <= pos) lo = mid; else hi = mid;
        }
        unsigned rd = (unsigned)(lo - r0);  // read index relative to the chunk's first read
        unsigned snext = pack_next_start(off, o0, P0, nr, lo);
        const unsigned nrd = (unsigned)(nr - r0);
        const unsigned* sw = reinterpret_cast<const unsigned*>(s_seq);
        const unsigned* qw = reinterpret_cast<const unsigned*>(s_qual);
        const unsigned qmin4 = (D.qual_min & 0xFFu) * 0x01010101u;
        const unsigned gmask = D.qual_min <= 0xFFu ? 0xFFFFFFFFu : 0u;
        const unsigned pw = (unsigned)(pos - P0);
        u64 c[2], rc[2], inv = 0, hq = 0;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          u64 cc = 0, qq = 0;
#pragma unroll 2
          for (int g = 0; g < 8; ++g) {
            const unsigned pg = pw + 32u * half + 4u * g;
            while (rd < nrd && pg >= snext) snext = pack_next_start(off, o0, P0, nr, r0 + ++rd);
            // all four positions past the last read: invalid
            unsigned f8 = 0, r8 = 0xFFu, i4 = 0xFu, h4 = 0;
            if (rd < nrd) {
              // A group holds at most one read separator (position snext - 1) unless a read is
              // shorter than three bases. With the separator at s, the positions after it are
              // the next read's bases, one byte earlier in the staged bytes: one byte permute
              // of the group's four bytes, then position s (and, after the last read, the
              // positions behind it) marked invalid. Every lane takes this path, so a warp
              // does not diverge at read boundaries.
              const unsigned bi = pg - rd;  // staged byte of position pg
              const unsigned s = snext - 1u - pg;  // separator index in the group, >= 4: none
              bool simple = bi + 4u <= nb;
              unsigned rdn = rd, snn = snext;
              if (s < 4u) {
                rdn = rd + 1u;
                snn = rdn < nrd ? pack_next_start(off, o0, P0, nr, r0 + rdn) : 0xFFFFFFFFu;
                simple = bi + 3u <= nb && (rdn >= nrd || snn - 1u >= pg + 4u);
              }
              if (simple) {
                const unsigned ss = s < 4u ? s : 4u;
                const unsigned sel = 0x3210u - (0x1110u & (0xFFF0u << (4u * ss)));
                pack_group4(__byte_perm(load4(sw, lead + bi), 0u, sel), __byte_perm(load4(qw, leadq + bi), 0u, sel),
                            qmin4, gmask, f8, r8, i4, h4);
                if (s < 4u) {
                  unsigned fm = 3u << (6u - 2u * s), rm = 3u << (2u * s), im = 1u << (3u - s);
                  if (rdn >= nrd) {  // no read after the separator
                    fm |= (1u << (6u - 2u * s)) - 1u;
                    rm |= (0xFFu << (2u * s + 2u)) & 0xFFu;
                    im |= (1u << (3u - s)) - 1u;
                  }
                  f8 &= ~fm;
                  r8 |= rm;
                  i4 |= im;
                  h4 &= ~im;
                  rd = rdn;
                  snext = snn;
                }
              } else {  // reads shorter than three bases, or inconsistent offsets
                f8 = 0, r8 = 0, i4 = 0, h4 = 0;
                for (unsigned i = 0; i < 4; ++i) {
                  const unsigned p = pg + i;
                  while (rd < nrd && p >= snext) snext = pack_next_start(off, o0, P0, nr, r0 + ++rd);
                  unsigned code = 0, valid = 0, good = 0;
                  const unsigned b = p - rd;
                  if (rd < nrd && p + 1u != snext && b < nb) {
                    const unsigned ch = s_seq[lead + b];
                    const unsigned u = (ch & 0xDFu) - 0x40u;  // A C G T (either case) -> bits 1 3 7 20
                    valid = u < 32u ? (0x10008Au >> u) & 1u : 0u;
                    code = valid ? ((ch >> 1) ^ (ch >> 2)) & 3u : 0u;  // A0 C1 G2 T3
                    good = valid && (unsigned)s_qual[leadq + b] >= D.qual_min;
                  }
                  f8 |= code << (6u - 2u * i);
                  r8 |= (~code & 3u) << (2u * i);
                  i4 |= (valid ^ 1u) << (3u - i);
                  h4 |= good << (3u - i);
                }
              }
            }
            cc = (cc << 8) | f8;                // first position ends in the top bits
            qq = (qq >> 8) | ((u64)r8 << 56);   // first position ends in the low bits
            inv = (inv << 4) | i4;
            hq = (hq << 4) | h4;
          }
          c[half] = cc;
          rc[half] = qq;
        }
        reinterpret_cast<ulonglong2*>(D.codes)[gw] = make_ulonglong2(c[0], c[1]);
        reinterpret_cast<ulonglong2*>(D.rcodes)[gw] = make_ulonglong2(rc[0], rc[1]);
        D.inv[gw] = inv;
        D.hq[gw] = hq;
      }
    } else if (w0 + threadIdx.x < w1) {
      reinterpret_cast<ulonglong2*>(D.codes)[gw] = make_ulonglong2(0, 0);
      reinterpret_cast<ulonglong2*>(D.rcodes)[gw] = make_ulonglong2(~0ull, ~0ull);
      D.inv[gw] = ~0ull;
      D.hq[gw] = 0;
    }
    __syncthreads();  // shared buffers are reused by the next chunk
  }
}

// ------------------------------------------------------------------ classify + compact

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
        if (__ldcg(&s->hi) != kEmpty) {  // count = left outcomes (none + A C G T)
          const uint4 el = __ldcg(reinterpret_cast<const uint4*>(&s->ext[0]));
          const u64 c = (u64)__ldcg(&s->none[0]) + el.x + el.y + el.z + el.w;
          keep[it] = c >= D.min_depth;
        }
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
      const uint4 e0 = __ldcg(reinterpret_cast<const uint4*>(&s->ext[0]));
      const uint4 e1 = __ldcg(reinterpret_cast<const uint4*>(&s->ext[4]));
      const unsigned c = slot_count(__ldcg(&s->none[0]), e0, D.status);
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

// slots = slots per partition, parts = on-chip partitions (1: one table).
__global__ void __launch_bounds__(256) query_kernel(const Slot* table, u64 slots, unsigned parts,
                                                    unsigned k,
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
      const u64 h = key_hash(lo, hi);
      const Slot* sub = parts > 1 ? table + (u64)part_of(h, parts) * slots : table;
      const Slot* s = find(sub, slots, lo, hi, h, full);
      if (full) atomicOr(&st->flags, kFlagFull);
      const unsigned sc = s ? slot_count(s->none[0], *reinterpret_cast<const uint4*>(&s->ext[0]), st) : 0u;
      if (s && sc >= min_depth) {
        c = sc;
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

// Consecutive threads write consecutive 16-byte pieces of the table (every warp store covers
// 512 contiguous bytes): the key piece of a slot gets the empty pattern, the rest zero.
__global__ void __launch_bounds__(256) table_init_kernel(Slot* table, u64 slots) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 pieces = slots * (sizeof(Slot) / 16);
  ulonglong2* t = reinterpret_cast<ulonglong2*>(table);
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < pieces; i += stride) {
    const u64 v = (i & 3) == 0 ? kEmpty : 0ull;
    __stcs(t + i, make_ulonglong2(v, v));
  }
}

// ------------------------------------------------------------------ launchers

template <int WPT, bool AGG>
static cudaError_t launch_pass_t(const PassBatch& b, int grid, int threads, cudaStream_t stream) {
  pass_kernel<WPT, AGG><<<(unsigned)grid, threads, 0, stream>>>(b);
  return cudaGetLastError();
}

template <int WPT, bool AGG>
static int occupancy_t(int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pass_kernel<WPT, AGG>, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int pass_max_ctas_per_sm(int block_threads, int wpt, bool agg) {
  switch (wpt) {
    case 1: return agg ? occupancy_t<1, true>(block_threads) : occupancy_t<1, false>(block_threads);
    case 2: return agg ? occupancy_t<2, true>(block_threads) : occupancy_t<2, false>(block_threads);
    case 4: return agg ? occupancy_t<4, true>(block_threads) : occupancy_t<4, false>(block_threads);
    default: return agg ? occupancy_t<8, true>(block_threads) : occupancy_t<8, false>(block_threads);
  }
}

cudaError_t launch_pass(const PassBatch& b, const LaunchShape& shape, bool agg, cudaStream_t stream) {
  if (b.total_tiles == 0) return cudaSuccess;
  u64 grid = (u64)shape.grid;
  if (grid > b.total_tiles) grid = b.total_tiles;
  const int g = (int)grid, th = shape.block_threads;
  switch (shape.windows_per_thread) {
    case 1: return agg ? launch_pass_t<1, true>(b, g, th, stream) : launch_pass_t<1, false>(b, g, th, stream);
    case 2: return agg ? launch_pass_t<2, true>(b, g, th, stream) : launch_pass_t<2, false>(b, g, th, stream);
    case 4: return agg ? launch_pass_t<4, true>(b, g, th, stream) : launch_pass_t<4, false>(b, g, th, stream);
    default: return agg ? launch_pass_t<8, true>(b, g, th, stream) : launch_pass_t<8, false>(b, g, th, stream);
  }
}

cudaError_t launch_pack(const PackBatch& b, cudaStream_t stream, int num_sms) {
  if (b.total_chunks == 0) return cudaSuccess;
  u64 blocks = b.total_chunks;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pack_kernel, kPackThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 4;
  }
  const u64 cap = (u64)num_sms * (per_sm > 0 ? per_sm : 1);
  if (blocks > cap) blocks = cap;
  pack_kernel<<<(unsigned)blocks, kPackThreads, 0, stream>>>(b);
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

cudaError_t launch_query(const Slot* table, u64 slots, unsigned parts, unsigned k, unsigned canonical,
                         unsigned min_depth, unsigned min_ext, const u64* keys, u64 n,
                         unsigned* counts, unsigned* ext, unsigned char* codes, DevStatus* st,
                         cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  u64 blocks = (n + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  query_kernel<<<(unsigned)blocks, 256, 0, stream>>>(table, slots, parts, k, canonical, min_depth, min_ext,
                                                     keys, n, counts, ext, codes, st);
  return cudaGetLastError();
}

}  // namespace kma
