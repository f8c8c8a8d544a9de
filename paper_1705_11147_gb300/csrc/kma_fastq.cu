// FASTQ text -> reads (the input side of the k-mer analysis stage, Section 2 item 1: the
// stage reads sequencing reads with per-base qualities). A FASTQ record is four lines:
// "@name", the bases, "+" (optionally followed by the name again) and the qualities, one
// character per base. Quality lines may begin with '@' or '+', so records are found by line
// number (line 4r starts record r), never by scanning for markers.
//
// Device steps (all on the caller's stream):
//   1. newlines per 16 KiB chunk of text            fastq_count_kernel
//   2. exclusive scan of the chunk counts           scan kernels (device-wide, u64)
//   3. newline positions, in order                  fastq_lines_kernel
//   4. per record: check the '@' and '+' lines, base and quality line lengths equal
//                                                   fastq_record_kernel
//   5. exclusive scan of the base counts -> offsets scan kernels
//   6. bases and qualities copied out, one warp per record
//                                                   fastq_copy_kernel
// A line may end in "\r\n"; the '\r' is not part of it. A final line without '\n' counts.
#include "kma_device.cuh"

namespace kma {

constexpr int kFqThreads = 1024;
constexpr int kFqBytesPerThread = 16;
constexpr u64 kFqChunk = (u64)kFqThreads * kFqBytesPerThread;  // 16 KiB of text per CTA

// ------------------------------------------------------------------ device-wide scan (u64)

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr u64 kScanBlock = (u64)kScanThreads * kScanItems;

// Exclusive scan of one block's kScanBlock items in place; the block's total to sums[blk].
__global__ void __launch_bounds__(kScanThreads) scan_block_kernel(u64* data, u64 n, u64* sums) {
  __shared__ u64 warp_tot[kScanThreads / 32];
  const u64 base = (u64)blockIdx.x * kScanBlock + (u64)threadIdx.x * kScanItems;
  u64 v[kScanItems];
  u64 local = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? data[base + j] : 0;
    local += v[j];
  }
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const u64 w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
    u64 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (unsigned)o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
    if (lane == kScanThreads / 32 - 1 && sums) sums[blockIdx.x] = wi;
  }
  __syncthreads();
  u64 run = warp_tot[warp] + incl - local;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) data[base + j] = run;
    run += v[j];
  }
}

__global__ void scan_add_kernel(u64* data, u64 n, const u64* block_offsets) {
  const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) data[i] += block_offsets[i / kScanBlock];
}

// Exclusive scan of data[0, n) in place; `tmp` holds scan_scratch_items(n) u64.
u64 scan_scratch_items(u64 n) {
  u64 total = 0;
  while (n > kScanBlock) {
    n = (n + kScanBlock - 1) / kScanBlock;
    total += n;
  }
  return total + 1;
}

cudaError_t scan_exclusive(u64* data, u64 n, u64* tmp, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const u64 blocks = (n + kScanBlock - 1) / kScanBlock;
  if (blocks == 1) {
    scan_block_kernel<<<1, kScanThreads, 0, stream>>>(data, n, nullptr);
    return cudaGetLastError();
  }
  u64* sums = tmp;
  scan_block_kernel<<<(unsigned)blocks, kScanThreads, 0, stream>>>(data, n, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = scan_exclusive(sums, blocks, tmp + blocks, stream)) != cudaSuccess) return e;
  scan_add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(data, n, sums);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ FASTQ kernels

// Newlines in each 16 KiB chunk (plus one for a final line that does not end in '\n').
__global__ void __launch_bounds__(kFqThreads) fastq_count_kernel(const unsigned char* text, u64 n,
                                                                 u64* chunk_counts) {
  __shared__ unsigned warp_cnt[kFqThreads / 32];
  const u64 c = blockIdx.x;
  const u64 b0 = c * kFqChunk + (u64)threadIdx.x * kFqBytesPerThread;
  unsigned cnt = 0;
#pragma unroll
  for (int j = 0; j < kFqBytesPerThread; ++j) {
    const u64 i = b0 + j;
    if (i < n) cnt += (text[i] == '\n') | (i == n - 1 && text[i] != '\n');
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    u64 t = 0;
    for (int w = 0; w < kFqThreads / 32; ++w) t += warp_cnt[w];
    chunk_counts[c] = t;
  }
}

// Line ends (position of each '\n', or n for an unterminated last line), in text order.
__global__ void __launch_bounds__(kFqThreads) fastq_lines_kernel(const unsigned char* text, u64 n,
                                                                 const u64* chunk_offsets, u64* line_end) {
  __shared__ unsigned warp_off[kFqThreads / 32];
  const u64 c = blockIdx.x;
  const u64 b0 = c * kFqChunk + (u64)threadIdx.x * kFqBytesPerThread;
  unsigned cnt = 0;
#pragma unroll
  for (int j = 0; j < kFqBytesPerThread; ++j) {
    const u64 i = b0 + j;
    if (i < n) cnt += (text[i] == '\n') | (i == n - 1 && text[i] != '\n');
  }
  const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += t;
  }
  if (lane == 31) warp_off[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int w = 0; w < kFqThreads / 32; ++w) {
      const unsigned t = warp_off[w];
      warp_off[w] = run;
      run += t;
    }
  }
  __syncthreads();
  u64 out = chunk_offsets[c] + warp_off[warp] + incl - cnt;
#pragma unroll
  for (int j = 0; j < kFqBytesPerThread; ++j) {
    const u64 i = b0 + j;
    if (i < n && text[i] == '\n') line_end[out++] = i;
    else if (i == n - 1 && i < n) line_end[out++] = n;  // unterminated last line
  }
}

// Line l occupies [start, end) with the '\r' of a "\r\n" ending removed.
__device__ __forceinline__ void line_span(const unsigned char* text, const u64* line_end, u64 l, u64& s, u64& e) {
  s = l ? line_end[l - 1] + 1 : 0;
  e = line_end[l];
  if (e > s && text[e - 1] == '\r') --e;
}

// Record r: '@' line, bases, '+' line, qualities; bases per record to seq_len[r]. The first
// malformed record's index goes to *bad (atomicMin).
__global__ void fastq_record_kernel(const unsigned char* text, const u64* line_end, u64 n_reads, u64* seq_len,
                                    unsigned long long* bad) {
  const u64 r = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_reads) return;
  u64 s0, e0, s1, e1, s2, e2, s3, e3;
  line_span(text, line_end, 4 * r, s0, e0);
  line_span(text, line_end, 4 * r + 1, s1, e1);
  line_span(text, line_end, 4 * r + 2, s2, e2);
  line_span(text, line_end, 4 * r + 3, s3, e3);
  const bool ok = e0 > s0 && text[s0] == '@' && e2 > s2 && text[s2] == '+' && e1 - s1 == e3 - s3;
  seq_len[r] = ok ? e1 - s1 : 0;
  if (!ok) atomicMin(bad, (unsigned long long)r);
}

// One warp per record: bases and qualities to their place in the output.
__global__ void fastq_copy_kernel(const unsigned char* text, const u64* line_end, u64 n_reads, const u64* offsets,
                                  unsigned char* seq, unsigned char* qual) {
  const u64 r = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31;
  if (r >= n_reads) return;
  u64 s1, e1, s3, e3;
  line_span(text, line_end, 4 * r + 1, s1, e1);
  line_span(text, line_end, 4 * r + 3, s3, e3);
  const u64 o = offsets[r], len = e1 - s1;
  for (u64 i = lane; i < len; i += 32) {
    seq[o + i] = text[s1 + i];
    qual[o + i] = text[s3 + i];
  }
}

// ------------------------------------------------------------------ launchers

u64 fastq_chunks(u64 n_bytes) { return (n_bytes + kFqChunk - 1) / kFqChunk; }

cudaError_t launch_fastq_count(const unsigned char* text, u64 n, u64* chunk_counts, cudaStream_t stream) {
  const u64 chunks = fastq_chunks(n);
  if (!chunks) return cudaSuccess;
  fastq_count_kernel<<<(unsigned)chunks, kFqThreads, 0, stream>>>(text, n, chunk_counts);
  return cudaGetLastError();
}

cudaError_t launch_fastq_lines(const unsigned char* text, u64 n, const u64* chunk_offsets, u64* line_end,
                               cudaStream_t stream) {
  const u64 chunks = fastq_chunks(n);
  if (!chunks) return cudaSuccess;
  fastq_lines_kernel<<<(unsigned)chunks, kFqThreads, 0, stream>>>(text, n, chunk_offsets, line_end);
  return cudaGetLastError();
}

cudaError_t launch_fastq_records(const unsigned char* text, const u64* line_end, u64 n_reads, u64* seq_len,
                                 unsigned long long* bad, cudaStream_t stream) {
  if (!n_reads) return cudaSuccess;
  fastq_record_kernel<<<(unsigned)((n_reads + 255) / 256), 256, 0, stream>>>(text, line_end, n_reads, seq_len, bad);
  return cudaGetLastError();
}

cudaError_t launch_fastq_copy(const unsigned char* text, const u64* line_end, u64 n_reads, const u64* offsets,
                              unsigned char* seq, unsigned char* qual, cudaStream_t stream) {
  if (!n_reads) return cudaSuccess;
  const u64 threads = n_reads * 32;
  fastq_copy_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(text, line_end, n_reads, offsets, seq,
                                                                          qual);
  return cudaGetLastError();
}

}  // namespace kma
