// Device-wide exclusive scan of uint32 values and a stable LSD radix sort of
// (uint32 key, uint32 value) pairs, 8 bits per pass.
//
// Sort pass, for a tile of 2048 keys per block:
//   1. histogram: per-tile digit counts, stored digit-major (digit * tiles + tile)
//   2. exclusive scan of the digit-major counts: global base of (digit, tile)
//   3. scatter: the stable rank of every key inside its tile comes from warp
//      __match_any_sync groups, combined across warps and rounds in shared
//      memory; keys are first ordered by digit in shared memory and then written
//      out so that runs of equal digits land on consecutive addresses.
// The element count may live on the device (it is produced by an earlier
// kernel); grids are sized for the capacity and blocks past the count return
// early, so a whole build can be captured in a CUDA graph.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanTile = kScanThreads * kScanPerThread;  // 2048

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / kWarp;
constexpr int kSortPerThread = 8;
constexpr int kSortTile = kSortThreads * kSortPerThread;  // 2048
constexpr int kBins = 256;

// Exclusive scan across a block of kScanThreads threads; returns the prefix
// of this thread and writes the block total to *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[kScanThreads / kWarp];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < kScanThreads / kWarp ? warp_sums[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFullMask, si, o);
      if (lane >= o) si += t;
    }
    if (lane < kScanThreads / kWarp) warp_sums[lane] = si - s;
    if (lane == kScanThreads / kWarp - 1) *total = si;
  }
  __syncthreads();
  uint32_t r = warp_sums[warp] + incl - v;
  __syncthreads();
  return r;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n,
                                   uint32_t* __restrict__ partial) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < kScanPerThread; ++r) {
    int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  __shared__ uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// One block scans all partials (exclusive, in place) and stores the total.
__global__ void scan_partials_kernel(uint32_t* __restrict__ partial, int64_t nb,
                                     uint32_t* __restrict__ total_out) {
  __shared__ uint32_t total;
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    uint32_t v = i < nb ? partial[i] : 0u;
    uint32_t ex = block_exclusive_scan(v, &total);
    if (i < nb) partial[i] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

// in and out may be the same array (each thread reads its elements before
// writing them).
__global__ void scan_down_kernel(const uint32_t* in, int64_t n,
                                 const uint32_t* __restrict__ partial, uint32_t* out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPerThread;
  uint32_t v[kScanPerThread];
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < kScanPerThread; ++r) {
    int64_t i = base + r;
    v[r] = i < n ? in[i] : 0u;
    s += v[r];
  }
  __shared__ uint32_t total;
  uint32_t run = block_exclusive_scan(s, &total) + partial[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kScanPerThread; ++r) {
    int64_t i = base + r;
    if (i < n) out[i] = run;
    run += v[r];
  }
}

__device__ __forceinline__ uint32_t load_count(const uint32_t* d_n, int64_t n_max) {
  if (d_n == nullptr) return (uint32_t)n_max;
  uint32_t n = *d_n;
  return (int64_t)n > n_max ? (uint32_t)n_max : n;
}

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, const uint32_t* d_n,
                                  int64_t n_max, int shift, uint32_t* __restrict__ hist,
                                  int64_t n_tiles) {
  __shared__ uint32_t cnt[kBins];
  const uint32_t n = load_count(d_n, n_max);
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int d = threadIdx.x; d < kBins; d += kSortThreads) cnt[d] = 0;
  __syncthreads();
  if (base < (int64_t)n) {
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r) {
      int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
      bool ok = i < (int64_t)n;
      uint32_t d = ok ? (keys[i] >> shift) & (kBins - 1) : kBins;
      uint32_t peers = __match_any_sync(kFullMask, d);
      if (ok && (peers & lanemask_lt()) == 0) atomicAdd(&cnt[d], __popc(peers));
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kBins; d += kSortThreads)
    hist[(int64_t)d * n_tiles + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                     uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                     const uint32_t* d_n, int64_t n_max, int shift,
                     const uint32_t* __restrict__ hist, const uint32_t* __restrict__ offs,
                     int64_t n_tiles) {
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t warp_cnt[kSortWarps][kBins];   // (round << 16) | count
  __shared__ uint32_t warp_base[kSortWarps][kBins];
  __shared__ uint32_t tile_start[kBins];
  __shared__ uint32_t running[kBins];
  __shared__ uint32_t total;

  const uint32_t n = load_count(d_n, n_max);
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  if (base >= (int64_t)n) return;
  const int tile_n = (int)min((int64_t)kSortTile, (int64_t)n - base);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // digit starts inside this tile (kSortThreads == kBins: one digit per thread)
  {
    uint32_t c = hist[(int64_t)threadIdx.x * n_tiles + blockIdx.x];
    tile_start[threadIdx.x] = block_exclusive_scan(c, &total);
    running[threadIdx.x] = 0;
    for (int w = 0; w < kSortWarps; ++w) warp_cnt[w][threadIdx.x] = 0xffff0000u;
  }
  __syncthreads();

  for (int r = 0; r < kSortPerThread; ++r) {
    const int li = r * kSortThreads + threadIdx.x;
    const bool ok = li < tile_n;
    uint32_t key = ok ? keys_in[base + li] : 0u;
    uint32_t val = ok ? vals_in[base + li] : 0u;
    uint32_t d = ok ? (key >> shift) & (kBins - 1) : kBins;
    uint32_t peers = __match_any_sync(kFullMask, d);
    uint32_t lt = peers & lanemask_lt();
    if (ok && lt == 0) warp_cnt[warp][d] = ((uint32_t)r << 16) | (uint32_t)__popc(peers);
    __syncthreads();
    {
      const int t = threadIdx.x;
      uint32_t run = running[t];
      for (int w = 0; w < kSortWarps; ++w) {
        uint32_t e = warp_cnt[w][t];
        uint32_t c = (e >> 16) == (uint32_t)r ? (e & 0xffffu) : 0u;
        warp_base[w][t] = run;
        run += c;
      }
      running[t] = run;
    }
    __syncthreads();
    if (ok) {
      uint32_t pos = tile_start[d] + warp_base[warp][d] + (uint32_t)__popc(lt);
      s_keys[pos] = key;
      s_vals[pos] = val;
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < tile_n; p += kSortThreads) {
    uint32_t key = s_keys[p];
    uint32_t d = (key >> shift) & (kBins - 1);
    uint32_t dst = offs[(int64_t)d * n_tiles + blockIdx.x] + ((uint32_t)p - tile_start[d]);
    keys_out[dst] = key;
    vals_out[dst] = s_vals[p];
  }
}

}  // namespace

int64_t scan_partials_count(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

size_t scan_workspace_bytes(int64_t n_max) {
  return align_up((size_t)(scan_partials_count(n_max) + 1) * sizeof(uint32_t));
}

cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n,
                               uint32_t* total_out, void* ws, cudaStream_t stream) {
  if (n <= 0) {
    if (total_out) return cudaMemsetAsync(total_out, 0, sizeof(uint32_t), stream);
    return cudaSuccess;
  }
  const int64_t nb = scan_partials_count(n);
  uint32_t* partial = static_cast<uint32_t*>(ws);
  scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, partial);
  scan_partials_kernel<<<1, kScanThreads, 0, stream>>>(partial, nb, total_out);
  scan_down_kernel<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, n, partial, out);
  note_launches(3);
  return cudaGetLastError();
}

int64_t radix_tiles(int64_t n_max) { return (n_max + kSortTile - 1) / kSortTile; }

size_t radix_sort_workspace_bytes(int64_t n_max) {
  const int64_t hist_n = radix_tiles(n_max) * kBins;
  return 2 * align_up((size_t)hist_n * sizeof(uint32_t)) + scan_workspace_bytes(hist_n);
}

int radix_sort_passes(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }

cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                             int64_t n_max, const uint32_t* d_n, int bits, void* ws,
                             cudaStream_t stream) {
  if (n_max <= 0) return cudaSuccess;
  const int64_t tiles = radix_tiles(n_max);
  const int64_t hist_n = tiles * kBins;
  char* p = static_cast<char*>(ws);
  uint32_t* hist = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)hist_n * sizeof(uint32_t));
  uint32_t* offs = reinterpret_cast<uint32_t*>(p);
  p += align_up((size_t)hist_n * sizeof(uint32_t));
  void* scan_ws = p;
  const int passes = radix_sort_passes(bits);
  uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * 8;
    radix_hist_kernel<<<(unsigned)tiles, kSortThreads, 0, stream>>>(ki, d_n, n_max, shift, hist,
                                                                     tiles);
    cudaError_t e = exclusive_scan_u32(hist, offs, hist_n, nullptr, scan_ws, stream);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<<<(unsigned)tiles, kSortThreads, 0, stream>>>(
        ki, vi, ko, vo, d_n, n_max, shift, hist, offs, tiles);
    note_launches(2);
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  return cudaGetLastError();
}

}  // namespace gpf
