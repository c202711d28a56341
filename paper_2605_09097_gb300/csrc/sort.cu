// Stable least-significant-digit radix sort of (uint64 key, uint32 value)
// pairs, 8 bits per pass.  Used to keep particles in Morton order of their
// base grid node (equal codes keep their incoming order).
//
// Per pass: (1) every block counts the digits of its tile; (2) one block
// scans the counts in (digit, block) order; (3) every block scatters its
// tile in order, ranking equal digits inside a 256-element chunk by warp
// and lane, so the pass is stable.
#include <cuda_runtime.h>

#include "osmpm_internal.h"

namespace osmpm {

namespace {

constexpr int kRsThreads = 256;
constexpr int kRsTile = 4096;  // elements per block per pass
constexpr int kRsWarps = kRsThreads / 32;

__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, unsigned* hist, int nb) {
  __shared__ unsigned cnt[256];
  cnt[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t start = (int64_t)blockIdx.x * kRsTile;
  int64_t end = start + kRsTile;
  if (end > n) end = n;
  for (int64_t i = start + threadIdx.x; i < end; i += kRsThreads)
    atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of `total` counters by one block of 1024 threads.
__global__ void k_rs_scan(unsigned* hist, int64_t total) {
  __shared__ unsigned sh[1024];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  for (int64_t base = 0; base < total; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const unsigned v = i < total ? hist[i] : 0u;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const unsigned t = threadIdx.x >= (unsigned)off ? sh[threadIdx.x - off] : 0u;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < total) hist[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
}

__global__ void k_rs_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                             uint32_t* vout, int64_t n, int shift, const unsigned* hist, int nb) {
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[kRsWarps][256];
  __shared__ unsigned tot[256];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  run[t] = hist[(int64_t)t * nb + blockIdx.x];
  for (int w = 0; w < kRsWarps; ++w) wcnt[w][t] = 0u;
  __syncthreads();
  const int64_t start = (int64_t)blockIdx.x * kRsTile;
  int64_t end = start + kRsTile;
  if (end > n) end = n;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int64_t c0 = start; c0 < end; c0 += kRsThreads) {
    const int64_t i = c0 + t;
    const bool valid = i < end;
    uint64_t key = 0;
    uint32_t val = 0;
    unsigned digit = 256u;  // invalid lanes form their own group
    if (valid) {
      key = kin[i];
      val = vin[i];
      digit = (unsigned)(key >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, digit);
    const unsigned rank = __popc(peers & lt_mask);
    if (valid && rank == 0u) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    {
      unsigned acc = 0u;
      for (int w = 0; w < kRsWarps; ++w) {
        const unsigned c = wcnt[w][t];
        wcnt[w][t] = acc;
        acc += c;
      }
      tot[t] = acc;
    }
    __syncthreads();
    if (valid) {
      const unsigned pos = run[digit] + wcnt[warp][digit] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    run[t] += tot[t];
    for (int w = 0; w < kRsWarps; ++w) wcnt[w][t] = 0u;
    __syncthreads();
  }
}

}  // namespace

int64_t radix_tiles(int64_t n) { return n <= 0 ? 1 : (n + kRsTile - 1) / kRsTile; }

void radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                      int64_t n, int bits, unsigned* hist, cudaStream_t s) {
  if (n <= 1) return;
  const int nb = (int)radix_tiles(n);
  uint64_t *ka = keys, *kb = keys_alt;
  uint32_t *va = vals, *vb = vals_alt;
  int passes = (bits + 7) / 8;
  if (passes < 1) passes = 1;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    g_launch_count += 3;
    k_rs_hist<<<nb, kRsThreads, 0, s>>>(ka, n, shift, hist, nb);
    k_rs_scan<<<1, 1024, 0, s>>>(hist, (int64_t)256 * nb);
    k_rs_scatter<<<nb, kRsThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist, nb);
    uint64_t* tk = ka;
    ka = kb;
    kb = tk;
    uint32_t* tv = va;
    va = vb;
    vb = tv;
  }
  if (ka != keys) {
    cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
  }
}

}  // namespace osmpm
