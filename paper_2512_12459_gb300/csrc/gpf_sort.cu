// Device-wide exclusive scan of uint32 values and a stable LSD radix sort of
// (uint32 key, uint32 value) pairs, 8 bits per pass.
//
// Sort (single pass per digit, decoupled look-back; Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016, and
// Adinets and Merrill, "Onesweep", 2022):
//   0. one kernel counts the digits of every pass over all keys (the global
//      digit counts do not depend on the order the earlier passes leave);
//   1. per pass, one kernel: a block claims the next tile of 3072 keys from
//      an atomic counter (so every earlier tile is held by a block that is
//      already running); each warp ranks its own 384 keys, 32 at a time
//      (groups of equal digits from bit ballots, per-warp digit counters in
//      shared memory);
//      the block publishes its digit counts, orders its keys by digit in
//      shared memory, adds up the counts the earlier tiles published for each
//      digit, walking back until a tile whose inclusive prefix is known,
//      publishes its own inclusive prefix and writes its keys out in digit
//      order (runs of equal digits land on consecutive addresses).
//   Every wait in the walk is bounded: after kSpinLimit polls the block sets
//   the caller's stall flag, stops waiting and writes only in-bounds
//   addresses; the sorted output is then invalid and the flag says so.
//   Counts are below kMaxSortN = 2^30 (30-bit status values).
// The element count may live on the device (it is produced by an earlier
// kernel); grids are sized for the capacity and blocks past the count return
// early, so a whole build can be captured in a CUDA graph.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 8;
constexpr int kScanTile = kScanThreads * kScanPerThread;  // 2048

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / kWarp;
constexpr int kSortPerThread = 12;
constexpr int kSortTile = kSortThreads * kSortPerThread;  // 3072
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

// ---- single-pass (decoupled look-back) sort

constexpr int kMaxPasses = kSortMaxPasses;     // 32-bit keys
static_assert(kSortBins == kBins, "8-bit digits");
constexpr uint32_t kFlagAgg = 1u << 30;        // the tile's own count is published
constexpr uint32_t kFlagPre = 2u << 30;        // the inclusive prefix is published
constexpr uint32_t kValMask = kFlagAgg - 1u;
constexpr uint32_t kSpinLimit = 1u << 22;      // polls of one status word before giving up

__device__ __forceinline__ uint32_t ld_status(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_status(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Digit counts of every pass over all keys: ghist[pass * 256 + digit].
__global__ void onesweep_hist_kernel(const uint32_t* __restrict__ keys, const uint32_t* d_n,
                                     int64_t n_max, int passes, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t cnt[kMaxPasses * kBins];
  for (int i = threadIdx.x; i < kMaxPasses * kBins; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const uint32_t n = load_count(d_n, n_max);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // plain shared-memory atomics: cheaper here than grouping equal digits first
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n; i += stride) {
    const uint32_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&cnt[p * kBins + ((k >> (8 * p)) & (kBins - 1))], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kBins; i += blockDim.x)
    if (cnt[i]) atomicAdd(&ghist[i], cnt[i]);
}

__global__ void __launch_bounds__(kSortThreads)
onesweep_pass_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                     uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                     const uint32_t* d_n, int64_t n_max, int shift,
                     const uint32_t* __restrict__ ghist, uint32_t* status,
                     uint32_t* tile_counter, uint32_t tile_base, uint32_t spin_limit,
                     uint32_t* stalled) {
  constexpr int kWarpKeys = kSortPerThread * kWarp;   // each warp ranks its own 384 keys
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t wcnt[kSortWarps][kBins];   // digit counts of each warp, then its bases
  __shared__ uint32_t tile_start[kBins];
  __shared__ uint32_t out_base[kBins];
  __shared__ uint32_t total;
  __shared__ uint32_t s_tile;

  const int t = threadIdx.x;        // kSortThreads == kBins: thread t owns digit t
  const int lane = t & 31, warp = t >> 5;
  if (t == 0) s_tile = tile_base + atomicAdd(tile_counter, 1u);
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) wcnt[w][t] = 0;
  __syncthreads();
  const uint32_t n = load_count(d_n, n_max);
  const uint32_t tile = s_tile;
  const int64_t base = (int64_t)tile * kSortTile;
  if (base >= (int64_t)n) return;                    // the whole block
  const int tile_n = (int)min((int64_t)kSortTile, (int64_t)n - base);

  // 1. ranks inside the warp's 384 keys (taken 32 at a time in order):
  //    (rank << 9) | digit, digit kBins for the positions past the tile
  uint32_t rd[kSortPerThread];
#pragma unroll
  for (int it = 0; it < kSortPerThread; ++it) {
    const int li = warp * kWarpKeys + it * kWarp + lane;
    const bool ok = li < tile_n;
    const uint32_t d = ok ? (keys_in[base + li] >> shift) & (kBins - 1) : kBins;
    // the lanes with the same digit: nine ballots (validity, then each digit
    // bit), cheaper here than __match_any_sync
    uint32_t peers = __ballot_sync(kFullMask, ok);
    if (!ok) peers = ~peers;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint32_t m = __ballot_sync(kFullMask, (d >> b) & 1u);
      peers &= ((d >> b) & 1u) ? m : ~m;
    }
    uint32_t r0 = 0;
    if (ok) r0 = wcnt[warp][d];
    __syncwarp();
    if (ok && (peers & lanemask_lt()) == 0) wcnt[warp][d] = r0 + (uint32_t)__popc(peers);
    __syncwarp();
    rd[it] = ((r0 + (uint32_t)__popc(peers & lanemask_lt())) << 9) | d;
  }
  __syncthreads();
  // 2. digit t: the warps' bases and the tile's count; publish the count
  //    (tile 0: its inclusive prefix)
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t x = wcnt[w][t];
    wcnt[w][t] = c;
    c += x;
  }
  st_status(status + (int64_t)tile * kBins + t, (tile == 0 ? kFlagPre : kFlagAgg) | c);
  tile_start[t] = block_exclusive_scan(c, &total);
  const uint32_t digit_start = block_exclusive_scan(ghist[t], &total);
  // 3. keys in digit order in shared memory (reloaded: the tile is in L1/L2)
#pragma unroll
  for (int it = 0; it < kSortPerThread; ++it) {
    const uint32_t d = rd[it] & 511u;
    if (d < (uint32_t)kBins) {
      const int li = warp * kWarpKeys + it * kWarp + lane;
      const uint32_t pos = tile_start[d] + wcnt[warp][d] + (rd[it] >> 9);
      s_keys[pos] = keys_in[base + li];
      s_vals[pos] = vals_in[base + li];
    }
  }
  // 4. digit t in the earlier tiles: walk back to the nearest inclusive prefix
  uint32_t excl = 0;
  if (tile > 0) {
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (j >= 0) {
      const uint32_t sv = ld_status(status + j * kBins + t);
      const uint32_t flag = sv & ~kValMask;
      if (flag == 0u) {
        if (++spins >= spin_limit) {
          atomicExch(stalled, 1u);
          break;
        }
        __nanosleep(64);
        continue;
      }
      excl += sv & kValMask;
      if (flag == kFlagPre) break;
      --j;
    }
    st_status(status + (int64_t)tile * kBins + t, kFlagPre | ((excl + c) & kValMask));
  }
  out_base[t] = digit_start + excl - tile_start[t];
  __syncthreads();
  // 5. out in digit order: runs of one digit go to consecutive addresses
  for (int p = t; p < tile_n; p += kSortThreads) {
    const uint32_t k = s_keys[p];
    const uint32_t dst = out_base[(k >> shift) & (kBins - 1)] + (uint32_t)p;
    if (dst < n) {
      keys_out[dst] = k;
      vals_out[dst] = s_vals[p];
    }
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

// The digit counts and tile counters of every pass, then the per-pass tile
// status words.
size_t radix_sort_workspace_bytes(int64_t n_max) {
  const int64_t hist_n = radix_tiles(n_max) * kBins;
  return align_up(sizeof(uint32_t) * (kMaxPasses * kBins + kMaxPasses)) +
         align_up((size_t)kMaxPasses * hist_n * sizeof(uint32_t));
}

int radix_sort_passes(int bits) { return bits <= 0 ? 0 : (bits + 7) / 8; }

// Two tiles of keys and values in and out, the digit counts and tile
// counter of one pass, two tiles of status words.
size_t sort_wait_probe_bytes() {
  return sizeof(uint32_t) * (8 * (size_t)kSortTile + kBins + 1 + 2 * kBins);
}

cudaError_t launch_sort_wait_probe(void* buf, uint32_t spin_limit, uint32_t* stalled,
                                   cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(buf, 0, sort_wait_probe_bytes(), stream);
  if (e != cudaSuccess) return e;
  uint32_t* w = static_cast<uint32_t*>(buf);
  uint32_t* keys_in = w;
  uint32_t* vals_in = w + 2 * kSortTile;
  uint32_t* keys_out = w + 4 * kSortTile;
  uint32_t* vals_out = w + 6 * kSortTile;
  uint32_t* ghist = w + 8 * kSortTile;
  uint32_t* counter = ghist + kBins;
  uint32_t* status = counter + 1;
  // one block, claiming tile 1 (tile_base 1): tile 0 is never processed, so
  // its status words stay 0 and the walk back from tile 1 waits on them
  onesweep_pass_kernel<<<1, kSortThreads, 0, stream>>>(
      keys_in, vals_in, keys_out, vals_out, nullptr, 2 * kSortTile, 0, ghist, status, counter,
      1u, spin_limit, stalled);
  note_launches(1);
  return cudaGetLastError();
}

uint32_t* radix_sort_counts(void* ws) { return static_cast<uint32_t*>(ws); }

cudaError_t radix_sort_clear_counts(void* ws, cudaStream_t stream) {
  return cudaMemsetAsync(ws, 0, sizeof(uint32_t) * (kMaxPasses * kBins + kMaxPasses), stream);
}

cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                             int64_t n_max, const uint32_t* d_n, int bits, void* ws,
                             uint32_t* stalled, cudaStream_t stream, bool counted) {
  if (n_max <= 0) return cudaSuccess;
  if (n_max >= kMaxSortN) return cudaErrorInvalidValue;
  const int64_t tiles = radix_tiles(n_max);
  const int passes = radix_sort_passes(bits);
  if (passes == 0) return cudaSuccess;
  char* p = static_cast<char*>(ws);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(p);        // [kMaxPasses][kBins]
  uint32_t* counters = ghist + kMaxPasses * kBins;          // [kMaxPasses]
  p += align_up(sizeof(uint32_t) * (kMaxPasses * kBins + kMaxPasses));
  uint32_t* status = reinterpret_cast<uint32_t*>(p);        // [passes][tiles][kBins]
  cudaError_t e;
  if (!counted && (e = radix_sort_clear_counts(ws, stream)) != cudaSuccess) return e;
  e = cudaMemsetAsync(status, 0, sizeof(uint32_t) * (size_t)passes * tiles * kBins, stream);
  if (e != cudaSuccess) return e;
  if (!counted) {
    const unsigned hblocks = (unsigned)std::min<int64_t>(tiles, 1024);
    onesweep_hist_kernel<<<hblocks, kSortThreads, 0, stream>>>(k0, d_n, n_max, passes, ghist);
    note_launches(1);
  }
  uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int pass = 0; pass < passes; ++pass) {
    onesweep_pass_kernel<<<(unsigned)tiles, kSortThreads, 0, stream>>>(
        ki, vi, ko, vo, d_n, n_max, pass * 8, ghist + pass * kBins,
        status + (size_t)pass * tiles * kBins, counters + pass, 0u, kSpinLimit, stalled);
    uint32_t* tmp;
    tmp = ki; ki = ko; ko = tmp;
    tmp = vi; vi = vo; vo = tmp;
  }
  note_launches(passes);
  return cudaGetLastError();
}

}  // namespace gpf
