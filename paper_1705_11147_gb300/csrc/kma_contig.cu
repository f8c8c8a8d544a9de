// Contig generation (HipMer, arXiv 1705.11147, Section 5.2; Section 2 defines contigs as the
// connected components of the de Bruijn graph of k-mers once the fork vertices are removed).
//
// Vertices: the finalized k-mers with no fork on either side (side codes A/C/G/T or X). The
// neighbour of a vertex x on its right is y = x[1..k) + R (R = its right code), on its left
// L + x[0..k-1); it is looked up by its key (canonical keys: the smaller of y and its reverse
// complement) and becomes an edge only if it is another vertex whose code on the facing side
// points back to x (mutual). Every vertex then has at most one edge per side: components are
// simple paths or cycles.
//
// GPU-native traversal instead of the paper's per-processor walks with conflict resolution:
// the edges define a successor function on the 2m directed states (vertex, direction of
// travel), and pointer jumping (Wyllie's list ranking, ceil(log2 2m) + 1 rounds) gives every
// state its distance to the end of its chain and that end. A path appears as two opposite
// chains; every vertex picks the chain whose head has the smaller key (with forward keys:
// always the forward chain), which fixes its contig, its position and its orientation.
// Cycles (chains that never end) are cut at their smallest key, on that vertex's left side,
// found by a second pointer-jumping pass that carries the minimum, and then ranked again.
// Contig offsets come from two exclusive scans; each vertex writes its own base.
#include <utility>
#include <vector>

#include "kma_device.cuh"

namespace kma {

constexpr unsigned kNil = 0xFFFFFFFFu;
constexpr int kCgThreads = 256;

static unsigned blocks_for(u64 n) { return (unsigned)((n + kCgThreads - 1) / kCgThreads); }

// ------------------------------------------------------------------ vertices and their map

// flag[i] = 1 if record i is a vertex (no fork on either side); flag[n] = 0 (scan total slot)
__global__ void cg_flag_kernel(const unsigned char* codes, u64 n, u64* flag) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = codes[2 * i] != 5 && codes[2 * i + 1] != 5;
  else if (i == n) flag[i] = 0;
}

__global__ void cg_compact_kernel(const unsigned char* codes, u64 n, const u64* pos, unsigned* vrec) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && codes[2 * i] != 5 && codes[2 * i + 1] != 5) vrec[pos[i]] = (unsigned)i;
}

__device__ __forceinline__ u64 cg_slot(u64 lo, u64 hi, unsigned log2s) {
  return (key_hash(lo, hi) * 0x9e3779b97f4a7c15ull) >> (64 - log2s);
}

__global__ void cg_map_init_kernel(ulonglong2* mkey, unsigned* midx, u64 S) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < S) {
    mkey[i] = make_ulonglong2(kEmpty, kEmpty);
    midx[i] = kNil;
  }
}

// Insert vertex u's key (keys are distinct; the table has at least twice as many slots).
__global__ void cg_map_insert_kernel(const u64* keys, const unsigned* vrec, u64 m, ulonglong2* mkey, unsigned* midx,
                                     unsigned log2s, unsigned* flags) {
  const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= m) return;
  const u64 r = vrec[u], lo = keys[2 * r], hi = keys[2 * r + 1];
  const u64 S = 1ull << log2s;
  u64 s = cg_slot(lo, hi, log2s);
  for (u64 n = 0; n < S; ++n) {
    u64 olo, ohi;
    cas128(reinterpret_cast<Slot*>(reinterpret_cast<ulonglong2*>(mkey) + s), kEmpty, kEmpty, lo, hi, olo, ohi);
    if (olo == kEmpty && ohi == kEmpty) {
      midx[s] = (unsigned)u;
      return;
    }
    s = (s + 1) & (S - 1);
  }
  atomicOr(flags, kFlagFull);
}

__device__ __forceinline__ unsigned cg_find(const ulonglong2* mkey, const unsigned* midx, unsigned log2s, u64 lo,
                                            u64 hi) {
  const u64 S = 1ull << log2s;
  u64 s = cg_slot(lo, hi, log2s);
  for (u64 n = 0; n < S; ++n) {
    const ulonglong2 kv = mkey[s];
    if (kv.x == lo && kv.y == hi) return midx[s];
    if (kv.x == kEmpty && kv.y == kEmpty) return kNil;
    s = (s + 1) & (S - 1);
  }
  return kNil;
}

// ------------------------------------------------------------------ edges

// nbr[2u + side] = (v << 1) | side of v entered, or kNil (side 0 = left, 1 = right).
__global__ void cg_edge_kernel(const u64* keys, const unsigned char* codes, const unsigned* vrec, u64 m, unsigned k,
                               unsigned canonical, const ulonglong2* mkey, const unsigned* midx, unsigned log2s,
                               unsigned* nbr) {
  const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * m) return;
  const u64 u = t >> 1;
  const unsigned side = (unsigned)(t & 1);
  const u64 r = vrec[u];
  const u64 lo = keys[2 * r], hi = keys[2 * r + 1];
  const unsigned code = codes[2 * r + side];
  nbr[t] = kNil;
  if (code >= 4) return;  // X: no neighbour on this side
  const u128 x = ((u128)hi << 64) | lo;
  const u128 mask = k == 64 ? ~(u128)0 : (((u128)1 << (2 * k)) - 1);
  const unsigned first = (unsigned)(x >> (2 * (k - 1))) & 3u, last = (unsigned)x & 3u;
  const u128 y = side ? (((x << 2) | code) & mask) : (((u128)code << (2 * (k - 1))) | (x >> 2));
  u64 ylo = (u64)y, yhi = (u64)(y >> 64), clo = ylo, chi = yhi;
  bool same = true;
  if (canonical) {
    u64 rlo, rhi;
    revcomp(ylo, yhi, k, rlo, rhi);
    if (rhi < yhi || (rhi == yhi && rlo < ylo)) {
      clo = rlo;
      chi = rhi;
      same = false;
    }
  }
  const unsigned v = cg_find(mkey, midx, log2s, clo, chi);
  if (v == kNil || v == u) return;
  const u64 vr = vrec[v];
  const unsigned vl = codes[2 * vr], vrc = codes[2 * vr + 1];
  unsigned enter;
  bool mutual;
  if (side) {  // leaving x to the right: x's first base must be v's extension on the facing side
    enter = same ? 0u : 1u;
    mutual = same ? vl == first : vrc == 3u - first;
  } else {     // leaving x to the left: x's last base must be v's extension on the facing side
    enter = same ? 1u : 0u;
    mutual = same ? vrc == last : vl == 3u - last;
  }
  if (mutual) nbr[t] = (v << 1) | enter;
}

// ------------------------------------------------------------------ list ranking

// State s = 2u + d: vertex u travelled forward (d = 0, leaving through its right side) or
// backward (d = 1, leaving through its left). Its successor follows the edge on that side and
// leaves the next vertex through the side opposite to the one it entered.
__global__ void cg_succ_kernel(const unsigned* nbr, u64 m, unsigned* nxt, unsigned* dist, unsigned* endst) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 2 * m) return;
  // edge (v << 1) | side of v entered: entering v on its left means leaving it on its right,
  // i.e. state 2v + 0, on its right state 2v + 1 -- the same number
  const unsigned n = nbr[(s & ~1ull) | (1u - (unsigned)(s & 1))];
  nxt[s] = n;
  dist[s] = n == kNil ? 0u : 1u;
  endst[s] = (unsigned)s;
}

// One pointer-jumping round from (nxt, dist, endst) into the *2 arrays; *live is set when a
// state still has a successor (every writer stores the same value).
__global__ void cg_jump_kernel(const unsigned* nxt, const unsigned* dist, const unsigned* endst, u64 n_states,
                               unsigned* nxt2, unsigned* dist2, unsigned* endst2, unsigned long long* live) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_states) return;
  const unsigned n = nxt[s];
  if (n == kNil) {
    nxt2[s] = kNil;
    dist2[s] = dist[s];
    endst2[s] = endst[s];
    return;
  }
  const unsigned nn = nxt[n];
  nxt2[s] = nn;
  dist2[s] = dist[s] + dist[n];
  endst2[s] = endst[n];
  if (nn != kNil) *live = 1ull;
}

__device__ __forceinline__ bool key_lt(const u64* keys, const unsigned* vrec, unsigned a, unsigned b) {
  const u64 ra = vrec[a], rb = vrec[b];
  const u64 ahi = keys[2 * ra + 1], bhi = keys[2 * rb + 1];
  return ahi != bhi ? ahi < bhi : keys[2 * ra] < keys[2 * rb];
}

// Cycle minimum: states still live after ranking lie on cycles; carry the vertex with the
// smallest key along the cycle by pointer jumping (mn = vertex index, nxt a fresh successor).
__global__ void cg_min_init_kernel(const unsigned* live_nxt, const unsigned* succ, u64 n_states, unsigned* mn,
                                   unsigned* nxt) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_states) return;
  const bool on_cycle = live_nxt[s] != kNil;
  mn[s] = on_cycle ? (unsigned)(s >> 1) : kNil;
  nxt[s] = on_cycle ? succ[s] : kNil;
}

__global__ void cg_min_jump_kernel(const u64* keys, const unsigned* vrec, const unsigned* mn, const unsigned* nxt,
                                   u64 n_states, unsigned* mn2, unsigned* nxt2) {
  const u64 s = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_states) return;
  const unsigned n = nxt[s];
  if (n == kNil) {
    mn2[s] = mn[s];
    nxt2[s] = kNil;
    return;
  }
  const unsigned a = mn[s], b = mn[n];
  mn2[s] = key_lt(keys, vrec, b, a) ? b : a;
  nxt2[s] = nxt[n];
}

// Cut every cycle at its smallest vertex, on that vertex's left side (both ends of the edge).
__global__ void cg_cut_kernel(const unsigned* mn, u64 m, unsigned* nbr, unsigned long long* cycles) {
  const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= m || mn[2 * u] != (unsigned)u) return;
  const unsigned e = nbr[2 * u];
  if (e != kNil) nbr[((u64)(e >> 1) << 1) | (e & 1u)] = kNil;
  nbr[2 * u] = kNil;
  atomicAdd(cycles, 1ull);
}

// ------------------------------------------------------------------ contigs

// Per vertex: the chosen chain (head with the smaller key; forward keys: the forward chain),
// position in it, and the contig length in bases (heads only) for the offset scan.
__global__ void cg_place_kernel(const u64* keys, const unsigned* vrec, const unsigned* dist, const unsigned* endst,
                                u64 m, unsigned k, unsigned canonical, unsigned* head, unsigned* pos,
                                unsigned char* dir, u64* head_flag, u64* head_len) {
  const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (u > m) return;
  if (u == m) {  // scan total slots
    head_flag[m] = 0;
    head_len[m] = 0;
    return;
  }
  const unsigned endF = endst[2 * u] >> 1, endB = endst[2 * u + 1] >> 1;
  const unsigned distF = dist[2 * u], distB = dist[2 * u + 1];
  // chain (u, 0) starts at endB, chain (u, 1) at endF
  const bool fwd = !canonical || endB == endF || key_lt(keys, vrec, endB, endF);
  head[u] = fwd ? endB : endF;
  pos[u] = fwd ? distB : distF;
  dir[u] = fwd ? 0 : 1;
  const bool is_head = (fwd ? distB : distF) == 0;
  head_flag[u] = is_head;
  head_len[u] = is_head ? (u64)distF + distB + k : 0;  // k-mers + k - 1
}

__global__ void cg_offsets_kernel(const u64* head_flag_scan, const u64* head_len_scan, const unsigned* pos, u64 m,
                                  u64* offsets) {
  const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < m && pos[u] == 0) offsets[head_flag_scan[u]] = head_len_scan[u];
  if (u == m) offsets[head_flag_scan[m]] = head_len_scan[m];
}

__global__ void cg_bases_kernel(const u64* keys, const unsigned* vrec, const unsigned* head, const unsigned* pos,
                                const unsigned char* dir, const u64* head_len_scan, u64 m, unsigned k, char* seq) {
  const u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= m) return;
  const u64 r = vrec[u];
  u64 lo = keys[2 * r], hi = keys[2 * r + 1];
  if (dir[u]) {
    u64 rlo, rhi;
    revcomp(lo, hi, k, rlo, rhi);
    lo = rlo;
    hi = rhi;
  }
  const u128 x = ((u128)hi << 64) | lo;
  const u64 base = head_len_scan[head[u]];
  if (pos[u] == 0) {
    for (unsigned i = 0; i < k; ++i) seq[base + i] = "ACGT"[(unsigned)(x >> (2 * (k - 1 - i))) & 3u];
  } else {
    seq[base + pos[u] + k - 1] = "ACGT"[(unsigned)x & 3u];
  }
}

// ------------------------------------------------------------------ driver

// The whole pass on `stream`; temporaries from `pool`. On success *seq_out / *offsets_out are
// pool allocations the caller owns.
int contig_pass(const u64* keys, const unsigned char* codes, u64 n, unsigned k, unsigned canonical,
                cudaMemPool_t pool, cudaStream_t st, char** seq_out, u64** offsets_out, u64* n_contigs,
                u64* n_bases, u64* n_vertices, u64* n_cycles, unsigned* dev_flags, cudaError_t* err) {
  std::vector<void*> temps;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, u64 bytes) -> bool {
    if (e != cudaSuccess) return false;
    e = cudaMallocFromPoolAsync(p, bytes ? bytes : 8, pool, st);
    if (e == cudaSuccess) temps.push_back(*p);
    return e == cudaSuccess;
  };
  auto fail = [&](int code) {
    for (void* p : temps) cudaFreeAsync(p, st);
    *err = e;
    return code;
  };
#define CG_TRY(x)                                                       \
  do {                                                                  \
    e = (x);                                                            \
    if (e != cudaSuccess) return fail(-7);                              \
  } while (0)
  *seq_out = nullptr;
  *offsets_out = nullptr;
  *n_contigs = *n_bases = *n_vertices = *n_cycles = 0;
  // vertices
  u64 *flag = nullptr, *scan_tmp = nullptr;
  if (!alloc((void**)&flag, (n + 1) * 8) || !alloc((void**)&scan_tmp, scan_scratch_items(n + 1) * 8))
    return fail(-2);
  cg_flag_kernel<<<blocks_for(n + 1), kCgThreads, 0, st>>>(codes, n, flag);
  CG_TRY(cudaGetLastError());
  CG_TRY(scan_exclusive(flag, n + 1, scan_tmp, st));
  u64 m = 0;
  CG_TRY(cudaMemcpyAsync(&m, flag + n, 8, cudaMemcpyDeviceToHost, st));
  CG_TRY(cudaStreamSynchronize(st));
  *n_vertices = m;
  if (m >= (1ull << 31)) return fail(-8);  // 2m directed states must fit 32-bit indices
  unsigned* vrec = nullptr;
  if (!alloc((void**)&vrec, m * 4)) return fail(-2);
  cg_compact_kernel<<<blocks_for(n), kCgThreads, 0, st>>>(codes, n, flag, vrec);
  CG_TRY(cudaGetLastError());
  // vertex map
  unsigned log2s = 6;
  while ((1ull << log2s) < 2 * m) ++log2s;
  const u64 S = 1ull << log2s;
  ulonglong2* mkey = nullptr;
  unsigned* midx = nullptr;
  if (!alloc((void**)&mkey, S * 16) || !alloc((void**)&midx, S * 4)) return fail(-2);
  cg_map_init_kernel<<<blocks_for(S), kCgThreads, 0, st>>>(mkey, midx, S);
  CG_TRY(cudaGetLastError());
  if (m) cg_map_insert_kernel<<<blocks_for(m), kCgThreads, 0, st>>>(keys, vrec, m, mkey, midx, log2s, dev_flags);
  CG_TRY(cudaGetLastError());
  // edges
  const u64 ns = 2 * m;
  unsigned *nbr = nullptr, *nxt = nullptr, *dist = nullptr, *endst = nullptr, *nxt2 = nullptr, *dist2 = nullptr,
           *endst2 = nullptr;
  unsigned long long* cnt = nullptr;  // [0] live states, [1] cycles
  if (!alloc((void**)&nbr, ns * 4) || !alloc((void**)&nxt, ns * 4) || !alloc((void**)&dist, ns * 4) ||
      !alloc((void**)&endst, ns * 4) || !alloc((void**)&nxt2, ns * 4) || !alloc((void**)&dist2, ns * 4) ||
      !alloc((void**)&endst2, ns * 4) || !alloc((void**)&cnt, 16))
    return fail(-2);
  CG_TRY(cudaMemsetAsync(cnt, 0, 16, st));
  if (ns) cg_edge_kernel<<<blocks_for(ns), kCgThreads, 0, st>>>(keys, codes, vrec, m, k, canonical, mkey, midx,
                                                              log2s, nbr);
  CG_TRY(cudaGetLastError());
  // list ranking (twice if there are cycles: rank, cut the cycles, rank again)
  unsigned rounds = 1;
  while ((1ull << rounds) < ns + 1) ++rounds;
  ++rounds;
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (ns) cg_succ_kernel<<<blocks_for(ns), kCgThreads, 0, st>>>(nbr, m, nxt, dist, endst);
    CG_TRY(cudaGetLastError());
    unsigned long long live = 0;
    for (unsigned it = 0; it < rounds && ns; ++it) {
      CG_TRY(cudaMemsetAsync(cnt, 0, 8, st));
      cg_jump_kernel<<<blocks_for(ns), kCgThreads, 0, st>>>(nxt, dist, endst, ns, nxt2, dist2, endst2, cnt);
      CG_TRY(cudaGetLastError());
      std::swap(nxt, nxt2);
      std::swap(dist, dist2);
      std::swap(endst, endst2);
      CG_TRY(cudaMemcpyAsync(&live, cnt, 8, cudaMemcpyDeviceToHost, st));
      CG_TRY(cudaStreamSynchronize(st));
      if (live == 0) break;
    }
    if (live == 0) break;
    if (attempt == 1) return fail(-1);  // cycles left after cutting: cannot happen
    // states still live lie on cycles: find each cycle's smallest vertex and cut there
    unsigned *mnA = nullptr, *mnB = nullptr, *nxA = nullptr, *nxB = nullptr;
    if (!alloc((void**)&mnA, ns * 4) || !alloc((void**)&mnB, ns * 4) || !alloc((void**)&nxA, ns * 4) ||
        !alloc((void**)&nxB, ns * 4))
      return fail(-2);
    cg_succ_kernel<<<blocks_for(ns), kCgThreads, 0, st>>>(nbr, m, nxB, dist2, endst2);  // fresh successors
    CG_TRY(cudaGetLastError());
    cg_min_init_kernel<<<blocks_for(ns), kCgThreads, 0, st>>>(nxt, nxB, ns, mnA, nxA);
    CG_TRY(cudaGetLastError());
    unsigned* mn = mnA;
    for (unsigned it = 0; it < rounds; ++it) {
      cg_min_jump_kernel<<<blocks_for(ns), kCgThreads, 0, st>>>(keys, vrec, mnA, nxA, ns, mnB, nxB);
      CG_TRY(cudaGetLastError());
      std::swap(mnA, mnB);
      std::swap(nxA, nxB);
      mn = mnA;
    }
    cg_cut_kernel<<<blocks_for(m), kCgThreads, 0, st>>>(mn, m, nbr, cnt + 1);
    CG_TRY(cudaGetLastError());
  }
  // placement, offsets, bases
  unsigned *head = nxt2, *pos = dist2;
  unsigned char* dir = nullptr;
  u64 *hflag = nullptr, *hlen = nullptr;
  if (!alloc((void**)&dir, m) || !alloc((void**)&hflag, (m + 1) * 8) || !alloc((void**)&hlen, (m + 1) * 8))
    return fail(-2);
  cg_place_kernel<<<blocks_for(m + 1), kCgThreads, 0, st>>>(keys, vrec, dist, endst, m, k, canonical, head, pos, dir,
                                                           hflag, hlen);
  CG_TRY(cudaGetLastError());
  CG_TRY(scan_exclusive(hflag, m + 1, scan_tmp, st));
  CG_TRY(scan_exclusive(hlen, m + 1, scan_tmp, st));
  u64 back[3] = {0, 0, 0};
  CG_TRY(cudaMemcpyAsync(&back[0], hflag + m, 8, cudaMemcpyDeviceToHost, st));
  CG_TRY(cudaMemcpyAsync(&back[1], hlen + m, 8, cudaMemcpyDeviceToHost, st));
  CG_TRY(cudaMemcpyAsync(&back[2], cnt + 1, 8, cudaMemcpyDeviceToHost, st));
  CG_TRY(cudaStreamSynchronize(st));
  const u64 nc = back[0], nb = back[1];
  char* seq = nullptr;
  u64* offsets = nullptr;
  e = cudaMallocFromPoolAsync((void**)&seq, nb ? nb : 8, pool, st);
  if (e != cudaSuccess) return fail(-2);
  e = cudaMallocFromPoolAsync((void**)&offsets, (nc + 1) * 8, pool, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(seq, st);
    return fail(-2);
  }
  cg_offsets_kernel<<<blocks_for(m + 1), kCgThreads, 0, st>>>(hflag, hlen, pos, m, offsets);
  e = cudaGetLastError();
  if (e == cudaSuccess && m)
    cg_bases_kernel<<<blocks_for(m), kCgThreads, 0, st>>>(keys, vrec, head, pos, dir, hlen, m, k, seq);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (void* p : temps) cudaFreeAsync(p, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(seq, st);
    cudaFreeAsync(offsets, st);
    *err = e;
    return -7;
  }
  *seq_out = seq;
  *offsets_out = offsets;
  *n_contigs = nc;
  *n_bases = nb;
  *n_cycles = back[2];
  return 0;
#undef CG_TRY
}

}  // namespace kma
