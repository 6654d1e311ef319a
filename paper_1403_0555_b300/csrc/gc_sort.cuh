// Stable least-significant-digit radix sort of 64-bit keys with 32- or 64-bit
// values: it orders the copy pool by (F, first start) for the fetch and the
// paper's F-quantised minima (Section III sorts its quantised minima on the
// GPU too, by a bitonic sort; a stable radix sort gives the same order in
// fewer passes over the data and keeps equal keys in input order).
//
// One pass per 8-bit digit that varies among the keys (the OR and AND of all
// keys, read back once, say which do), three kernels per pass:
//   radix_hist_kernel    -- per tile of 2048 keys, the 256-bin digit histogram,
//                           stored digit-major: hist[digit * tiles + tile];
//   radix_scan_kernel    -- one CTA: exclusive prefix sum over that array, so
//                           entry (digit, tile) is where the tile's first key
//                           with that digit goes;
//   radix_scatter_kernel -- per tile, in eight rounds of 256 keys (key order
//                           = round-major, thread order within a round): each
//                           key's rank among the earlier keys of its digit
//                           (warp peers by __match_any_sync, earlier warps by
//                           a per-digit prefix over the warps in shared
//                           memory, earlier rounds by a running base), so the
//                           pass is stable.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gc {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr unsigned kSortTile = kSortThreads * kSortRounds;   // keys per tile
constexpr int kSortBins = 256;

__host__ __device__ inline unsigned sort_tiles(unsigned n) { return (n + kSortTile - 1) / kSortTile; }

// or_and[0] |= every key, or_and[1] &= every key (caller sets 0 / ~0 first)
__global__ void __launch_bounds__(256) key_bits_kernel(const unsigned long long* keys, unsigned n,
                                                       unsigned long long* or_and) {
  unsigned long long o = 0ull, a = ~0ull;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long k = keys[i];
    o |= k;
    a &= k;
  }
  for (int s = 16; s > 0; s >>= 1) {
    o |= __shfl_xor_sync(0xffffffffu, o, s);
    a &= __shfl_xor_sync(0xffffffffu, a, s);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicOr(or_and, o);
    atomicAnd(or_and + 1, a);
  }
}

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const unsigned long long* keys, unsigned n,
                                                                 int shift, unsigned* hist, unsigned tiles) {
  __shared__ unsigned h[kSortBins];
  h[threadIdx.x] = 0u;
  __syncthreads();
  const unsigned base = blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const unsigned i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// exclusive prefix sum of m entries in place, one CTA of 1024 threads: each
// thread sums a contiguous chunk, the chunk sums are scanned in shared memory,
// then each thread rewrites its chunk
__global__ void __launch_bounds__(1024) radix_scan_kernel(unsigned* a, unsigned m) {
  __shared__ unsigned part[1024];
  const unsigned t = threadIdx.x;
  const unsigned chunk = (m + 1023u) / 1024u;
  const unsigned lo = t * chunk, hi = lo + chunk < m ? lo + chunk : m;
  unsigned s = 0u;
  for (unsigned i = lo; i < hi; ++i) s += a[i];
  part[t] = s;
  __syncthreads();
  for (unsigned off = 1; off < 1024u; off <<= 1) {   // Hillis-Steele inclusive scan
    const unsigned v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned run = part[t] - s;                        // exclusive prefix of this chunk
  for (unsigned i = lo; i < hi; ++i) {
    const unsigned v = a[i];
    a[i] = run;
    run += v;
  }
}

template <typename VT>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const unsigned long long* kin, const VT* vin,
                                                                    unsigned long long* kout, VT* vout, unsigned n,
                                                                    int shift, const unsigned* offs,
                                                                    unsigned tiles) {
  constexpr int W = kSortThreads / 32;
  __shared__ unsigned base[kSortBins];
  __shared__ unsigned wcnt[W][kSortBins];
  const unsigned t = threadIdx.x, warp = t >> 5, lane = t & 31u;
  base[t] = offs[(size_t)t * tiles + blockIdx.x];
  const unsigned tile0 = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
#pragma unroll
    for (int w = 0; w < W; ++w) wcnt[w][t] = 0u;
    __syncthreads();
    const unsigned i = tile0 + r * kSortThreads + t;
    const bool valid = i < n;
    unsigned long long k = 0ull;
    VT v{};
    unsigned dg = kSortBins;                        // out-of-range keys form their own group
    if (valid) {
      k = kin[i];
      v = vin[i];
      dg = (unsigned)(k >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, dg);
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[warp][dg] = __popc(peers);
    __syncthreads();
    // per digit (thread t owns digit t): where each warp's keys of the digit start
    unsigned run = base[t];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const unsigned c = wcnt[w][t];
      wcnt[w][t] = run;
      run += c;
    }
    base[t] = run;
    __syncthreads();
    if (valid) {
      const unsigned pos = wcnt[warp][dg] + rank;
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
  }
}

}  // namespace gc
