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
#include "kma_device.cuh"

namespace kma {

constexpr int kHllThreads = 512;
constexpr int kHllWpt = 8;
constexpr int kHllTile = kHllThreads * kHllWpt;

__global__ void __launch_bounds__(kHllThreads) hll_kernel(const __grid_constant__ PartWindows W, unsigned k,
                                                          unsigned canonical, unsigned n_parts, unsigned part,
                                                          unsigned p, unsigned* regs, DevStatus* st) {
  extern __shared__ unsigned s_reg[];  // [2^p]
  const unsigned m = 1u << p;
  for (unsigned i = threadIdx.x; i < m; i += blockDim.x) s_reg[i] = 0;
  __syncthreads();
  const u64 n_tiles = (W.q1 - W.q0 + kHllTile - 1) / kHllTile;
  unsigned acc_valid = 0;
  for (u64 t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const u64 q = W.q0 + t * kHllTile + (u64)threadIdx.x * kHllWpt;
    if (q >= W.q1) continue;  // q1 - q0 is a multiple of 64: all kHllWpt starts are inside
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
        }
      }
      if (j + 1 < kHllWpt) rw.roll();
    }
  }
  __syncthreads();
  for (unsigned i = threadIdx.x; i < m; i += blockDim.x)
    if (s_reg[i]) atomicMax(&regs[i], s_reg[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc_valid += __shfl_down_sync(0xffffffffu, acc_valid, o);
  if ((threadIdx.x & 31) == 0 && acc_valid) atomicAdd(&st->valid_windows, (u64)acc_valid);
}

cudaError_t launch_hll(const PartWindows& w, unsigned k, unsigned canonical, unsigned n_parts, unsigned part,
                       unsigned p, unsigned* regs, DevStatus* st, cudaStream_t stream, int num_sms) {
  if (w.q1 <= w.q0) return cudaSuccess;
  const size_t smem = (size_t)4 << p;
  cudaError_t e = cudaFuncSetAttribute(hll_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hll_kernel, kHllThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  const u64 tiles = (w.q1 - w.q0 + kHllTile - 1) / kHllTile;
  u64 grid = (u64)num_sms * (per_sm > 0 ? per_sm : 1);
  if (grid > tiles) grid = tiles;
  hll_kernel<<<(unsigned)grid, kHllThreads, smem, stream>>>(w, k, canonical, n_parts, part, p, regs, st);
  return cudaGetLastError();
}

}  // namespace kma
