/*
 * Seeded synthetic read sets shaped like the paper's workloads (Section 6: Illumina-style
 * short reads of 100-250 bp sampled from both strands of a genome at coverage d).
 *
 * This file is the one input generator that both the CPU oracle and the CUDA path are
 * fed from. It contains no k-mer arithmetic: it only draws a genome, plants repeats,
 * samples reads with substitution errors, N bases and Phred qualities.
 *
 * Every random value is a pure function of (seed, stream, counter) through the
 * splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), so reads can be generated in any order and on any number
 * of threads with identical output, on x86-64 and aarch64 alike. Probabilities are
 * compared as 64-bit integers against thresholds computed once on the host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

static inline uint64_t sm_mix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* One 64-bit draw for counter `ctr` of stream `stream` under `seed`. */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return sm_mix(sm_mix(seed ^ (stream * 0xD1B54A32D192ED03ull)) + ctr);
}

/* Unbiased-enough bounded draw: high 64 bits of a 64x64 product (Lemire). */
static inline uint64_t bounded(uint64_t r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)r * n) >> 64);
}

enum { ST_GENOME = 1, ST_REPEAT = 2, ST_READ = 3, ST_BASE = 4, ST_META = 5 };

/* Genome of G bases, codes 0..3 (A,C,G,T), i.i.d. uniform. */
void synth_genome(uint64_t seed, uint64_t G, uint8_t* out) {
  for (uint64_t w = 0; w * 32 < G; ++w) {
    uint64_t r = draw(seed, ST_GENOME, w);
    uint64_t n = G - w * 32 < 32 ? G - w * 32 : 32;
    for (uint64_t j = 0; j < n; ++j) out[w * 32 + j] = (uint8_t)((r >> (2 * j)) & 3);
  }
}

/*
 * Plant repeats: copy j takes a source segment of length U[min_len, max_len] at a random
 * position and pastes it at another random position, each pasted base substituted with
 * probability `div_thresh / 2^64` by one of the other three bases. Copies are added in
 * order j = 0, 1, ... until `n_copies` copies (if non-zero) or until the pasted bases reach
 * `target_bases`. Returns the number of bases pasted.
 */
uint64_t synth_plant_repeats(uint64_t seed, uint8_t* g, uint64_t G, uint64_t n_copies,
                             uint64_t target_bases, uint32_t min_len, uint32_t max_len,
                             uint64_t div_thresh) {
  uint64_t pasted = 0;
  uint8_t* buf = (uint8_t*)malloc(max_len ? max_len : 1);
  if (!buf || max_len < min_len || (uint64_t)max_len >= G) { free(buf); return 0; }
  for (uint64_t j = 0;; ++j) {
    if (n_copies ? j >= n_copies : pasted >= target_bases) break;
    uint64_t len = min_len + bounded(draw(seed, ST_REPEAT, 4 * j), (uint64_t)(max_len - min_len) + 1);
    uint64_t src = bounded(draw(seed, ST_REPEAT, 4 * j + 1), G - len + 1);
    uint64_t dst = bounded(draw(seed, ST_REPEAT, 4 * j + 2), G - len + 1);
    uint64_t sub_key = draw(seed, ST_REPEAT, 4 * j + 3);
    memcpy(buf, g + src, len);
    for (uint64_t i = 0; i < len; ++i) {
      uint64_t u = draw(sub_key, ST_BASE, 2 * i);
      if (u < div_thresh) buf[i] = (uint8_t)((buf[i] + 1 + bounded(draw(sub_key, ST_BASE, 2 * i + 1), 3)) & 3);
    }
    memcpy(g + dst, buf, len);
    pasted += len;
  }
  free(buf);
  return pasted;
}

typedef struct {
  uint64_t seed;
  const uint8_t* g;
  uint64_t G;
  const uint32_t* lens;   /* per-read length, or NULL for fixed L */
  uint32_t L;
  const uint64_t* offsets;
  uint64_t r0, r1;
  uint64_t err_thresh, n_thresh;
  uint8_t* seq;
  uint8_t* qual;
} read_job;

static void* read_worker(void* arg) {
  static const char ACGT[4] = {'A', 'C', 'G', 'T'};
  read_job* jb = (read_job*)arg;
  for (uint64_t r = jb->r0; r < jb->r1; ++r) {
    uint64_t L = jb->lens ? jb->lens[r] : jb->L;
    uint64_t o = jb->offsets[r];
    uint64_t rr = draw(jb->seed, ST_READ, r);
    uint64_t start = bounded(rr, jb->G - L + 1);
    int minus = (int)(draw(jb->seed, ST_READ, r ^ 0x8000000000000000ull) >> 63);
    uint64_t key = draw(jb->seed, ST_READ, r ^ 0x4000000000000000ull);
    for (uint64_t j = 0; j < L; ++j) {
      int b = minus ? 3 - jb->g[start + L - 1 - j] : jb->g[start + j];
      uint64_t u = draw(key, ST_BASE, 4 * j);
      uint64_t v = draw(key, ST_BASE, 4 * j + 1);
      uint64_t w = draw(key, ST_BASE, 4 * j + 2);
      uint8_t q;
      if (jb->n_thresh && w < jb->n_thresh) {
        jb->seq[o + j] = 'N';
        jb->qual[o + j] = (uint8_t)(33 + 2);
        continue;
      }
      if (u < jb->err_thresh) {
        b = (b + 1 + (int)bounded(v, 3)) & 3;
        q = (uint8_t)(2 + bounded(draw(key, ST_BASE, 4 * j + 3), 14));   /* U{2..15} */
      } else {
        q = (uint8_t)(25 + bounded(draw(key, ST_BASE, 4 * j + 3), 16));  /* U{25..40} */
      }
      jb->seq[o + j] = (uint8_t)ACGT[b];
      jb->qual[o + j] = (uint8_t)(33 + q);
    }
  }
  return NULL;
}

/*
 * Sample n_reads reads into seq/qual (ASCII, Phred+33) at `offsets` (n_reads+1 entries,
 * filled here from the lengths). Read r: start U[0, G-L], strand Bernoulli(1/2) (minus =
 * reverse complement of the genome segment), per base substitution with probability
 * err_thresh/2^64 (to one of the other three bases, Phred U{2..15}); correct bases get
 * Phred U{25..40}; with probability n_thresh/2^64 a base is 'N' with Phred 2.
 */
void synth_reads(uint64_t seed, const uint8_t* g, uint64_t G, uint64_t n_reads, uint32_t L,
                 const uint32_t* lens, uint64_t err_thresh, uint64_t n_thresh,
                 uint8_t* seq, uint8_t* qual, uint64_t* offsets, int n_threads) {
  offsets[0] = 0;
  for (uint64_t r = 0; r < n_reads; ++r) offsets[r + 1] = offsets[r] + (lens ? lens[r] : L);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  read_job jobs[256];
  for (int t = 0; t < n_threads; ++t) {
    read_job* jb = &jobs[t];
    jb->seed = seed; jb->g = g; jb->G = G; jb->lens = lens; jb->L = L; jb->offsets = offsets;
    jb->r0 = n_reads * (uint64_t)t / (uint64_t)n_threads;
    jb->r1 = n_reads * (uint64_t)(t + 1) / (uint64_t)n_threads;
    jb->err_thresh = err_thresh; jb->n_thresh = n_thresh; jb->seq = seq; jb->qual = qual;
    if (pthread_create(&th[t], NULL, read_worker, jb) != 0) { read_worker(jb); th[t] = 0; }
  }
  for (int t = 0; t < n_threads; ++t) if (th[t]) pthread_join(th[t], NULL);
}

/* Raw counter-based draws, exposed so the Python side derives per-sample / per-job
 * parameters (sizes, coverages, arrival gaps) from the same generator. */
void synth_draws(uint64_t seed, uint64_t stream, uint64_t ctr0, uint64_t n, uint64_t* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = draw(seed, ST_META + stream, ctr0 + i);
}
