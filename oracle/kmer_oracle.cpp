// Plain CPU oracle for the k-mer analysis stage of HipMer (arXiv 1705.11147, Sections 2 and 5.1).
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product library may include, link or call this
// file; only the tests, the package's smoke check and the benchmark's CPU-baseline leg use it.
// It shares no code with the CUDA path: it works on character strings, uses std::unordered_map
// and has no Bloom filter (the Bloom filter may never change the result, Section 5.1).
//
// What it computes, step by step in the paper's terms:
//  1. Chopping (Section 2, item 1; Fig. "combined"(b)): every read of length L yields the
//     L-k+1 overlapping substrings of length k ("windows"). A window is kept only if all of
//     its k characters are A, C, G or T after case folding (the paper does not say how N or
//     other symbols are treated; reading: they invalidate every window that covers them).
//  2. Canonical form (not stated in the paper; reverse complements are named in Section 7):
//     the key of a window w is the lexicographically smaller of w and its reverse complement,
//     with A < C < G < T. With canonical = 0 the key is w itself (the paper's k = 3 figures).
//  3. Counting (Section 5.1): count[key] += 1 for every window.
//  4. Extensions (Section 5.1: two arrays of four counters per k-mer, one per end): the base
//     before the window and the base after it are each counted if they exist, are ACGT and
//     have Phred quality >= qual_threshold. When the key is the reverse complement of w, the
//     sides swap and the bases are complemented.
//  5. Error filter (Section 2 item 1, Section 5.1): keep keys with count >= min_depth
//     (the paper keeps k-mers seen more than epsilon times: min_depth = epsilon + 1).
//  6. High-quality extensions (Section 5.1, threshold t_hq): on each side the set
//     H = {b : ext[b] >= min_ext_count}. The side code is b if |H| = 1, X (no neighbour,
//     Section 4.1) if |H| = 0 and F (fork, excluded from contigs, Section 2) if |H| >= 2.
//     Unique-extension (UU, Section 5.2) k-mers have A/C/G/T on both sides.
//  7. Owner-computes partitioning (Section 5.1: a fixed k-mer -> owner map): with n_parts > 1
//     only keys with fnv1a(key string) mod n_parts == part are kept (or, with a set of parts,
//     keys whose part is in the set); the union over all parts equals the whole result. The
//     FNV-1a hash here is the oracle's own.
//
// Output: records sorted by key; key = 2-bit codes A0 C1 G2 T3, first base most
// significant, as a 128-bit number split into (lo, hi) 64-bit words.

#include <algorithm>
#include <array>
#include <cstdint>
#include <cmath>
#include <cstring>
#include <memory>
#include <memory_resource>
#include <sys/mman.h>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

struct Params {
  uint32_t k;
  uint32_t min_depth;
  uint32_t min_ext_count;
  uint32_t qual_threshold;
  uint32_t qual_offset;
  uint32_t canonical;
};

struct Rec {
  uint32_t count = 0;
  uint32_t ext[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // left A C G T, right A C G T
};

using Key = std::array<uint64_t, 2>;  // (lo, hi)

struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = k[0] * 0x9E3779B97F4A7C15ull ^ (k[1] + 0x632BE59BD9B4E019ull + (k[0] >> 17));
    return (size_t)(h ^ (h >> 29));
  }
};

// Each thread's map draws its nodes from its own monotonic arena (large chunks), so counting
// threads do not contend on the system allocator.
using Map = std::pmr::unordered_map<Key, Rec, KeyHash>;

// Upstream of the arenas: 2 MiB-aligned blocks marked for transparent huge pages, so that
// touching fresh node memory costs few page faults.
class HugeBlocks : public std::pmr::memory_resource {
  void* do_allocate(size_t bytes, size_t) override {
    const size_t a = size_t(2) << 20;
    void* p = std::aligned_alloc(a, (bytes + a - 1) / a * a);
    if (!p) throw std::bad_alloc();
    madvise(p, (bytes + a - 1) / a * a, MADV_HUGEPAGE);
    return p;
  }
  void do_deallocate(void* p, size_t, size_t) override { std::free(p); }
  bool do_is_equal(const std::pmr::memory_resource& o) const noexcept override { return this == &o; }
};

HugeBlocks g_huge_blocks;

struct ArenaMap {
  std::unique_ptr<std::pmr::monotonic_buffer_resource> arena;
  std::unique_ptr<Map> map;
  ArenaMap()
      : arena(new std::pmr::monotonic_buffer_resource(size_t(64) << 20, &g_huge_blocks)),
        map(new Map(arena.get())) {}
};

char fold(uint8_t c) { return (c >= 'a' && c <= 'z') ? (char)(c - 'a' + 'A') : (char)c; }

bool is_acgt(char c) { return c == 'A' || c == 'C' || c == 'G' || c == 'T'; }

int code_of(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    default: return 3;  // 'T'
  }
}

char complement(char c) {
  switch (c) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    default: return 'A';  // 'T'
  }
}

std::string reverse_complement(const std::string& w) {
  std::string r(w.rbegin(), w.rend());
  for (char& c : r) c = complement(c);
  return r;
}

Key pack(const std::string& key) {
  unsigned __int128 v = 0;
  for (char c : key) v = (v << 2) | (unsigned __int128)code_of(c);
  return Key{(uint64_t)v, (uint64_t)(v >> 64)};
}

std::string unpack(const Key& key, uint32_t k) {
  unsigned __int128 v = ((unsigned __int128)key[1] << 64) | key[0];
  std::string s(k, 'A');
  for (uint32_t i = 0; i < k; ++i) s[k - 1 - i] = "ACGT"[(int)(v & 3)], v >>= 2;
  return s;
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (char c : s) h = (h ^ (uint8_t)c) * 0x100000001b3ull;
  return h;
}

bool usable(const std::string& s, const uint8_t* q, int64_t j, const Params& p) {
  if (j < 0 || j >= (int64_t)s.size()) return false;
  if (!is_acgt(s[(size_t)j])) return false;
  return (int)q[j] - (int)p.qual_offset >= (int)p.qual_threshold;
}

Key pack_chars(const char* key, int64_t k) {
  unsigned __int128 v = 0;
  for (int64_t j = 0; j < k; ++j) v = (v << 2) | (unsigned __int128)code_of(key[j]);
  return Key{(uint64_t)v, (uint64_t)(v >> 64)};
}

uint64_t fnv1a_chars(const char* s, int64_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (int64_t j = 0; j < n; ++j) h = (h ^ (uint8_t)s[j]) * 0x100000001b3ull;
  return h;
}

// Steps 1-4 over reads [r0, r1) into map m; returns the number of valid windows seen
// (before partition filtering). Windows and their reverse complements are built in
// fixed-size character buffers (k <= 63), so no step allocates per window.
// keep[i] != 0: keys of owner partition i (of n_parts) are counted.
uint64_t count_reads(const uint8_t* seq, const uint8_t* qual, const uint64_t* offsets,
                     uint64_t r0, uint64_t r1, const Params& p, const uint8_t* keep,
                     uint32_t n_parts, Map& m) {
  uint64_t valid_windows = 0;
  const int64_t k = p.k;
  std::string s;
  std::vector<int64_t> bad;  // bad[j] = number of non-ACGT characters in s[0, j)
  char rc[64];
  for (uint64_t r = r0; r < r1; ++r) {
    const int64_t L = (int64_t)(offsets[r + 1] - offsets[r]);
    const uint8_t* q = qual + offsets[r];
    s.assign((size_t)L, ' ');
    bad.assign((size_t)L + 1, 0);
    for (int64_t j = 0; j < L; ++j) {
      s[(size_t)j] = fold(seq[offsets[r] + j]);
      bad[(size_t)j + 1] = bad[(size_t)j] + (is_acgt(s[(size_t)j]) ? 0 : 1);
    }
    for (int64_t i = 0; i + k <= L; ++i) {
      if (bad[(size_t)(i + k)] != bad[(size_t)i]) continue;  // window has a non-ACGT character
      ++valid_windows;
      const char* w = s.data() + i;
      for (int64_t j = 0; j < k; ++j) rc[j] = complement(w[k - 1 - j]);
      const bool forward = !p.canonical || std::memcmp(w, rc, (size_t)k) <= 0;
      const char* key = forward ? w : rc;
      if (n_parts > 1 && !keep[fnv1a_chars(key, k) % n_parts]) continue;
      Rec& rec = m[pack_chars(key, k)];
      rec.count += 1;
      const bool left_ok = usable(s, q, i - 1, p);
      const bool right_ok = usable(s, q, i + k, p);
      if (forward) {
        if (left_ok) rec.ext[0 + code_of(s[(size_t)(i - 1)])] += 1;
        if (right_ok) rec.ext[4 + code_of(s[(size_t)(i + k)])] += 1;
      } else {
        // Reverse-complement orientation: the base after w precedes the key (complemented),
        // the base before w follows it (complemented).
        if (right_ok) rec.ext[0 + code_of(complement(s[(size_t)(i + k)]))] += 1;
        if (left_ok) rec.ext[4 + code_of(complement(s[(size_t)(i - 1)]))] += 1;
      }
    }
  }
  return valid_windows;
}

uint8_t side_code(const uint32_t* e, uint32_t min_ext) {
  int n = 0, b = 0;
  for (int j = 0; j < 4; ++j)
    if (e[j] >= min_ext) ++n, b = j;
  if (n == 0) return 4;  // X
  if (n >= 2) return 5;  // F
  return (uint8_t)b;
}

struct Result {
  Params p;
  uint64_t valid_windows = 0;
  std::vector<Key> keys;
  std::vector<Rec> recs;
  // all counted keys (before the min_depth filter), split by KeyHash % parts.size()
  std::vector<ArenaMap> parts;
  const Rec* find(const Key& k) const {
    const Map& m = *parts[KeyHash()(k) % parts.size()].map;
    auto it = m.find(k);
    return it == m.end() ? nullptr : &it->second;
  }
};

bool key_less(const Key& a, const Key& b) { return a[1] != b[1] ? a[1] < b[1] : a[0] < b[0]; }

}  // namespace

extern "C" {

typedef struct {
  uint32_t k, min_depth, min_ext_count, qual_threshold, qual_offset, canonical;
} oracle_params;

// keep[0 .. n_parts): which owner partitions to count (NULL or n_parts <= 1: all keys).
void* oracle_run_parts(const uint8_t* seq, const uint8_t* qual, const uint64_t* offsets,
                       uint64_t n_reads, const oracle_params* op, const uint8_t* keep_in,
                       uint32_t n_parts, int n_threads) {
  Params p{op->k, op->min_depth, op->min_ext_count, op->qual_threshold, op->qual_offset,
           op->canonical};
  if (n_parts == 0 || !keep_in) n_parts = 1;
  const std::vector<uint8_t> keep(keep_in && n_parts > 1 ? keep_in : nullptr,
                                  keep_in && n_parts > 1 ? keep_in + n_parts : nullptr);
  if (n_threads < 1) n_threads = 1;
  const size_t T = (size_t)n_threads;
  // 1. each thread counts the windows of its share of the reads (steps 1-4)
  std::vector<ArenaMap> maps(T);
  std::vector<uint64_t> windows(T, 0);
  {
    std::vector<std::thread> th;
    for (size_t t = 0; t < T; ++t) {
      const uint64_t r0 = n_reads * t / T, r1 = n_reads * (t + 1) / T;
      th.emplace_back([&, t, r0, r1] {
        windows[t] = count_reads(seq, qual, offsets, r0, r1, p, keep.data(), n_parts, *maps[t].map);
      });
    }
    for (auto& x : th) x.join();
  }
  // 2. merge: thread u sums every key with KeyHash % T == u over all thread maps
  Result* res = new Result();
  res->p = p;
  for (size_t t = 0; t < T; ++t) res->valid_windows += windows[t];
  res->parts.resize(T);
  std::vector<std::vector<std::pair<Key, Rec>>> kept(T);
  {
    std::vector<std::thread> th;
    for (size_t u = 0; u < T; ++u) {
      th.emplace_back([&, u] {
        Map& dst = *res->parts[u].map;
        for (size_t t = 0; t < T; ++t)
          for (const auto& kv : *maps[t].map) {
            if (KeyHash()(kv.first) % T != u) continue;
            Rec& r = dst[kv.first];
            r.count += kv.second.count;
            for (int j = 0; j < 8; ++j) r.ext[j] += kv.second.ext[j];
          }
        // 3. depth filter (step 5)
        for (const auto& kv : dst)
          if (kv.second.count >= p.min_depth) kept[u].push_back(kv);
      });
    }
    for (auto& x : th) x.join();
  }
  std::vector<ArenaMap>().swap(maps);
  std::vector<std::pair<Key, Rec>> all;
  for (auto& v : kept) {
    all.insert(all.end(), v.begin(), v.end());
    std::vector<std::pair<Key, Rec>>().swap(v);
  }
  std::sort(all.begin(), all.end(), [](const std::pair<Key, Rec>& a, const std::pair<Key, Rec>& b) {
    return key_less(a.first, b.first);
  });
  res->keys.reserve(all.size());
  res->recs.reserve(all.size());
  for (auto& kv : all) res->keys.push_back(kv.first), res->recs.push_back(kv.second);
  return res;
}

// One owner partition `part` of n_parts (n_parts <= 1: every key).
void* oracle_run(const uint8_t* seq, const uint8_t* qual, const uint64_t* offsets,
                 uint64_t n_reads, const oracle_params* op, uint32_t part, uint32_t n_parts,
                 int n_threads) {
  if (n_parts <= 1) return oracle_run_parts(seq, qual, offsets, n_reads, op, nullptr, 1, n_threads);
  std::vector<uint8_t> keep(n_parts, 0);
  if (part < n_parts) keep[part] = 1;
  return oracle_run_parts(seq, qual, offsets, n_reads, op, keep.data(), n_parts, n_threads);
}

uint64_t oracle_size(void* h) { return ((Result*)h)->keys.size(); }

uint64_t oracle_valid_windows(void* h) { return ((Result*)h)->valid_windows; }

void oracle_fetch(void* h, uint64_t* keys, uint32_t* counts, uint32_t* ext, uint8_t* codes) {
  Result* r = (Result*)h;
  for (size_t i = 0; i < r->keys.size(); ++i) {
    keys[2 * i] = r->keys[i][0];
    keys[2 * i + 1] = r->keys[i][1];
    counts[i] = r->recs[i].count;
    std::memcpy(ext + 8 * i, r->recs[i].ext, sizeof(uint32_t) * 8);
    codes[2 * i] = side_code(r->recs[i].ext, r->p.min_ext_count);
    codes[2 * i + 1] = side_code(r->recs[i].ext + 4, r->p.min_ext_count);
  }
}

// Lookup (the read-only phase, Section 4.2 use case GRO). A query k-mer may be given in
// either orientation; the answer is expressed in the query's own orientation. Keys below
// min_depth (or absent) answer count 0, zero extensions and codes X/X.
void oracle_query(void* h, const uint64_t* qkeys, uint64_t n, uint32_t* counts, uint32_t* ext,
                  uint8_t* codes) {
  Result* r = (Result*)h;
  const Params& p = r->p;
  for (uint64_t i = 0; i < n; ++i) {
    std::string w = unpack(Key{qkeys[2 * i], qkeys[2 * i + 1]}, p.k);
    std::string rc = reverse_complement(w);
    const bool forward = !p.canonical || w <= rc;
    const Rec* rec = r->find(pack(forward ? w : rc));
    uint32_t e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t c = 0;
    if (rec && rec->count >= p.min_depth) {
      c = rec->count;
      for (int b = 0; b < 4; ++b) {
        if (forward) {
          e[b] = rec->ext[b];
          e[4 + b] = rec->ext[4 + b];
        } else {
          // the query's left neighbours are the complements of the key's right neighbours
          e[code_of(complement("ACGT"[b]))] = rec->ext[4 + b];
          e[4 + code_of(complement("ACGT"[b]))] = rec->ext[b];
        }
      }
    }
    counts[i] = c;
    std::memcpy(ext + 8 * i, e, sizeof(e));
    codes[2 * i] = c ? side_code(e, p.min_ext_count) : 4;
    codes[2 * i + 1] = c ? side_code(e + 4, p.min_ext_count) : 4;
  }
}

void oracle_free(void* h) { delete (Result*)h; }

// The oracle's owner map (step 7): partition id of each packed key.
void oracle_partition_of(const uint64_t* keys, uint64_t n, uint32_t k, uint32_t n_parts,
                         uint32_t* out) {
  for (uint64_t i = 0; i < n; ++i)
    out[i] = (uint32_t)(fnv1a(unpack(Key{keys[2 * i], keys[2 * i + 1]}, k)) % n_parts);
}

// 2-bit packing of k-mer strings (ACGT only, length k each, concatenated), as the oracle
// packs keys; lets tests state inputs and expected keys as text.
void oracle_pack_strings(const char* s, uint64_t n, uint32_t k, uint64_t* keys) {
  for (uint64_t i = 0; i < n; ++i) {
    Key key = pack(std::string(s + i * k, k));
    keys[2 * i] = key[0];
    keys[2 * i + 1] = key[1];
  }
}

void oracle_unpack_keys(const uint64_t* keys, uint64_t n, uint32_t k, char* out) {
  for (uint64_t i = 0; i < n; ++i) {
    std::string s = unpack(Key{keys[2 * i], keys[2 * i + 1]}, k);
    std::memcpy(out + i * k, s.data(), k);
  }
}

// ---- Contig generation (Section 5.2), walked one k-mer at a time ------------------------
// Vertices: the k-mers of a k-mer analysis result without a fork on either side (Section 2
// excludes the vertices with non-unique neighbours; a side code X means no neighbour there,
// as in the two-letter codes of Section 4.1). The right neighbour of a k-mer x (in the
// orientation of its key) is y = x[1..k) + R, R its right extension; the left neighbour is
// L + x[0..k-1). The neighbour is looked up by its key (with canonical keys: the smaller of y
// and its reverse complement). Reading taken here (Section 5.2 extends a subcontig while the
// lookup succeeds): the step is taken only if the neighbour is a vertex whose own extension
// on the facing side points back to x (mutual), and never from a k-mer to itself. Components
// are then simple paths or cycles; a contig is a path's k-mers merged (length = k-mers + k - 1).
// A cycle is cut at its smallest key, on that k-mer's left side, and becomes a path.

struct ContigResult {
  std::string bases;
  std::vector<uint64_t> offsets{0};
  uint64_t cycles = 0;
};

std::string canonical_of(const std::string& w, int canonical) {
  if (!canonical) return w;
  std::string rc = reverse_complement(w);
  return rc < w ? rc : w;
}

// ---- HyperLogLog sketch (Section 5.1's cardinality pass), from its definition ----------
// The sketch of a set of distinct keys with m = 2^p registers: each key (lo, hi) is hashed to
// 64 bits by the sketch's hash h = fmix64(lo XOR (hi * 0x9e3779b97f4a7c15 + 0x632be59bd9b4e019)),
// fmix64 being the MurmurHash3 64-bit finaliser (Appleby); register j = the top p bits of h;
// the register holds the largest rank over its keys, rank = 1 + number of leading zeros of
// the other 64 - p bits (64 - p + 1 if they are all zero). Written here on its own; the hash
// is part of the sketch's definition, so both sides must agree on it bit for bit.

uint64_t sketch_fmix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

void oracle_hll_registers(const uint64_t* keys, uint64_t n, uint32_t p, uint8_t* regs) {
  const uint64_t m = 1ull << p;
  for (uint64_t j = 0; j < m; ++j) regs[j] = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t lo = keys[2 * i], hi = keys[2 * i + 1];
    const uint64_t h = sketch_fmix64(lo ^ (hi * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull));
    const uint64_t j = h >> (64 - p);
    // leading zeros of the remaining 64 - p bits, counted one bit at a time
    uint32_t rank = 1;
    for (uint32_t b = 0; b < 64 - p; ++b) {
      if ((h >> (63 - p - b)) & 1) break;
      ++rank;
    }
    if (rank > regs[j]) regs[j] = (uint8_t)rank;
  }
}

// Flajolet, Fusy, Gandouet, Meunier (2007): E = alpha_m m^2 / sum_j 2^(-M[j]); if E <= 5m/2
// and V > 0 registers are zero, E = m ln(m / V) (linear counting). With 64-bit hashes the
// large-range correction of the 32-bit original is not needed.
// Heavy hitters (Section 5.1: frequent k-mers found in the cardinality pass).
//
// The sampled stream: the canonical keys of the valid windows that start at every
// `sample`-th position of the reads laid out back to back with one separator after each read
// (read r's base j at offsets[r] - offsets[0] + r + j), in read order.
struct KeyStream {
  std::vector<uint64_t> keys;  // (lo, hi) pairs
};

void* oracle_sampled_stream(const uint8_t* seq, const uint8_t* qual, const uint64_t* offsets, uint64_t n_reads,
                            const oracle_params* op, uint32_t sample) {
  (void)qual;
  KeyStream* out = new KeyStream();
  const int64_t k = op->k;
  std::string s;
  char rc[64];
  for (uint64_t r = 0; r < n_reads; ++r) {
    const int64_t L = (int64_t)(offsets[r + 1] - offsets[r]);
    const uint64_t start = offsets[r] - offsets[0] + r;  // position of the read's first base
    s.assign((size_t)L, ' ');
    for (int64_t j = 0; j < L; ++j) s[(size_t)j] = fold(seq[offsets[r] + j]);
    for (int64_t i = 0; i + k <= L; ++i) {
      if ((start + (uint64_t)i) % sample != 0) continue;
      bool ok = true;
      for (int64_t j = 0; j < k; ++j) ok = ok && is_acgt(s[(size_t)(i + j)]);
      if (!ok) continue;
      const char* w = s.data() + i;
      for (int64_t j = 0; j < k; ++j) rc[j] = complement(w[k - 1 - j]);
      const bool forward = !op->canonical || std::memcmp(w, rc, (size_t)k) <= 0;
      const Key key = pack_chars(forward ? w : rc, k);
      out->keys.push_back(key[0]);
      out->keys.push_back(key[1]);
    }
  }
  return out;
}

uint64_t oracle_stream_size(void* h) { return ((KeyStream*)h)->keys.size() / 2; }

void oracle_stream_fetch(void* h, uint64_t* keys) {
  const KeyStream* st = (KeyStream*)h;
  std::memcpy(keys, st->keys.data(), st->keys.size() * sizeof(uint64_t));
}

void oracle_stream_free(void* h) { delete (KeyStream*)h; }

// Sub-stream of a key: the top `bits` bits of the sketch hash (the same hash as the
// HyperLogLog registers).
void oracle_stream_bucket(const uint64_t* keys, uint64_t n, uint32_t bits, uint32_t* out) {
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t lo = keys[2 * i], hi = keys[2 * i + 1];
    const uint64_t h = sketch_fmix64(lo ^ (hi * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull));
    out[i] = (uint32_t)(h >> (64 - bits));
  }
}

// Misra and Gries (1982), "Finding repeated elements", taken item by item over a stream of
// keys with m counters: a key that holds a counter increments it; otherwise, if a counter is
// free (zero), the key takes it with count 1; otherwise every counter is decremented (those
// reaching zero are freed) and the item is dropped. Returns the number of keys left with a
// positive count; keys/counts receive them (up to m rows), in counter order.
uint64_t oracle_misra_gries(const uint64_t* stream, uint64_t n, uint32_t m, uint64_t* keys, uint64_t* counts) {
  std::vector<Key> held(m);
  std::vector<uint64_t> c(m, 0);
  for (uint64_t i = 0; i < n; ++i) {
    const Key x{stream[2 * i], stream[2 * i + 1]};
    int64_t at = -1, free_at = -1;
    for (uint32_t j = 0; j < m; ++j) {
      if (c[j] > 0 && held[j] == x) at = j;
      if (c[j] == 0 && free_at < 0) free_at = j;
    }
    if (at >= 0) {
      ++c[(size_t)at];
    } else if (free_at >= 0) {
      held[(size_t)free_at] = x;
      c[(size_t)free_at] = 1;
    } else {
      for (uint32_t j = 0; j < m; ++j) --c[j];
    }
  }
  uint64_t out = 0;
  for (uint32_t j = 0; j < m; ++j)
    if (c[j] > 0) {
      keys[2 * out] = held[j][0];
      keys[2 * out + 1] = held[j][1];
      counts[out] = c[j];
      ++out;
    }
  return out;
}

double oracle_hll_estimate(const uint8_t* regs, uint32_t p) {
  const uint64_t m = 1ull << p;
  const double md = (double)m;
  double alpha;
  if (m == 16) alpha = 0.673;
  else if (m == 32) alpha = 0.697;
  else if (m == 64) alpha = 0.709;
  else alpha = 0.7213 / (1.0 + 1.079 / md);
  double sum = 0.0;
  uint64_t zeros = 0;
  for (uint64_t j = 0; j < m; ++j) {
    sum += std::pow(2.0, -(double)regs[j]);
    if (regs[j] == 0) ++zeros;
  }
  const double e = alpha * md * md / sum;
  if (e <= 2.5 * md && zeros > 0) return md * std::log(md / (double)zeros);
  return e;
}

void* oracle_contigs(const uint64_t* keys, const uint8_t* codes, uint64_t n, uint32_t k, int canonical) {
  auto* res = new ContigResult();
  std::vector<std::string> str;
  std::vector<int> lc, rc;
  std::unordered_map<std::string, int64_t> index;
  for (uint64_t i = 0; i < n; ++i) {
    if (codes[2 * i] == 5 || codes[2 * i + 1] == 5) continue;  // a fork on either side
    index[unpack(Key{keys[2 * i], keys[2 * i + 1]}, k)] = (int64_t)str.size();
    str.push_back(unpack(Key{keys[2 * i], keys[2 * i + 1]}, k));
    lc.push_back(codes[2 * i]);
    rc.push_back(codes[2 * i + 1]);
  }
  const int64_t m = (int64_t)str.size();
  // adj[u][side] = (v, side of v it enters), side 0 = left, 1 = right; v = -1: none
  std::vector<std::array<std::pair<int64_t, int>, 2>> adj(m);
  for (int64_t u = 0; u < m; ++u) {
    const std::string& x = str[u];
    for (int side = 0; side < 2; ++side) {
      adj[u][side] = {-1, 0};
      if ((side ? rc[u] : lc[u]) == 4) continue;  // X: no neighbour on this side
      const std::string y = side ? x.substr(1) + "ACGT"[rc[u]] : std::string(1, "ACGT"[lc[u]]) + x.substr(0, k - 1);
      const std::string key = canonical_of(y, canonical);
      auto it = index.find(key);
      if (it == index.end() || it->second == u) continue;
      const int64_t v = it->second;
      const bool same = key == y;  // v read in the orientation of its key
      int enter;
      bool mutual;
      if (side == 1) {  // leaving x to the right: x[0] must be v's extension on the facing side
        enter = same ? 0 : 1;
        mutual = same ? lc[v] == code_of(x[0]) : rc[v] == code_of(complement(x[0]));
      } else {          // leaving x to the left: x[k-1] must be v's extension on the facing side
        enter = same ? 1 : 0;
        mutual = same ? rc[v] == code_of(x[k - 1]) : lc[v] == code_of(complement(x[k - 1]));
      }
      if (mutual) adj[u][side] = {v, enter};
    }
  }
  std::vector<char> seen(m, 0);
  for (int64_t u0 = 0; u0 < m; ++u0) {
    if (seen[u0]) continue;
    // the component of u0
    std::vector<int64_t> comp{u0};
    seen[u0] = 1;
    for (size_t i = 0; i < comp.size(); ++i)
      for (int side = 0; side < 2; ++side) {
        const int64_t v = adj[comp[i]][side].first;
        if (v >= 0 && !seen[v]) seen[v] = 1, comp.push_back(v);
      }
    // an end of the path: one with a free left side if there is one (forward keys: the start)
    int64_t end = -1;
    for (int64_t v : comp)
      if (adj[v][0].first < 0) { end = v; break; }
    if (end < 0)
      for (int64_t v : comp)
        if (adj[v][1].first < 0) { end = v; break; }
    if (end < 0) {  // a cycle: cut it at the smallest key, on that k-mer's left side
      int64_t mn = comp[0];
      for (int64_t v : comp)
        if (str[v] < str[mn]) mn = v;
      const auto [w, t] = adj[mn][0];
      adj[w][t] = {-1, 0};
      adj[mn][0] = {-1, 0};
      end = mn;
      ++res->cycles;
    }
    // walk from the end: forward if its left side is free, else in reverse
    bool fwd = adj[end][0].first < 0;
    std::string contig = fwd ? str[end] : reverse_complement(str[end]);
    int64_t cur = end;
    int exit = fwd ? 1 : 0;
    while (true) {
      const auto [v, t] = adj[cur][exit];
      if (v < 0) break;
      if (t == 0) {  // entered v on its left: v read forward
        contig.push_back(str[v][k - 1]);
        exit = 1;
      } else {
        contig.push_back(complement(str[v][0]));
        exit = 0;
      }
      cur = v;
    }
    res->bases += contig;
    res->offsets.push_back(res->bases.size());
  }
  return res;
}

uint64_t oracle_contigs_n(void* h) { return ((ContigResult*)h)->offsets.size() - 1; }
uint64_t oracle_contigs_bases(void* h) { return ((ContigResult*)h)->bases.size(); }
uint64_t oracle_contigs_cycles(void* h) { return ((ContigResult*)h)->cycles; }
void oracle_contigs_fetch(void* h, char* bases, uint64_t* offsets) {
  auto* r = (ContigResult*)h;
  std::memcpy(bases, r->bases.data(), r->bases.size());
  std::memcpy(offsets, r->offsets.data(), r->offsets.size() * 8);
}
void oracle_contigs_free(void* h) { delete (ContigResult*)h; }

}  // extern "C"
