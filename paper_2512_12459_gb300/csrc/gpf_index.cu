// gpf_build_index on a multi-level hashed grid.
//
// Level L has cubic cells of edge c0 * 2^L. Each Gaussian lives on the finest
// level on which its k-sigma bounds span at most S cells per axis, and is
// listed in the (level, cell) bucket of every cell of that box that holds a
// hit point. Lists of all levels share one array of 2^hash_bits buckets,
// radix-sorted by bucket (stable, so a list's order is deterministic).
// Hit points are sorted by their cell on the query level K (dense linear
// keys), which orders the forward's tiles and gives the backward the hit
// points of any query-level cell. Gaussians are also sorted by the
// query-level cell of their mean, the order the backward walks them in.
//
// Kernels, in stream order:
//   query_keys (hit point keys and per-cell counts, occupancy bits of every level)
//   preprocess (records, level boxes, entry counts, order keys, level mask)
//   sort hit points, per-cell starts (scan of the counts)
//   sort Gaussians into the backward's order
//   scan of entry counts -> emit (bucket, Gaussian) entries -> sort -> bucket ranges
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kThreads = 256;
constexpr int kBlockWarps = kThreads / kWarp;

// The sum over a block of kThreads threads of up to four per-thread counts,
// each in [0, 2^32); thread 0 gets the sums. The header counters take one
// atomic per block: atomics to one address are serialised, so per-warp
// updates from 10^6 threads cost tens of microseconds.
__device__ __forceinline__ void block_counts(uint32_t (&v)[4], uint32_t (*s)[4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = __reduce_add_sync(kFullMask, v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t t = 0;
      for (int w = 0; w < kBlockWarps; ++w) t += s[w][k];
      v[k] = t;
    }
  }
}
// Boxes with more cells than this on their level are refused (overflow flag).
constexpr int64_t kMaxBoxCells = int64_t(1) << 16;
constexpr uint32_t kNoBox = 0xffffffffu;
// gmask of a box of more than 31 cells: emit tests every cell's occupancy bit.
constexpr uint32_t kMaskAll = 0xffffffffu;

__device__ __forceinline__ bool occupied(const uint32_t* occ, uint32_t b) {
  return (occ[b >> 5] >> (b & 31u)) & 1u;
}

// GPF_BF16 / GPF_BF16_MEAN32 field -> float32 [(10 + C), n] rows: mean, quat, logscale,
// spectrum (the decoding stated at gpf_field).
__global__ void decode_bf16_kernel(gpf_field f, float* __restrict__ dec) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = f.n;
  if (g >= n) return;
  const float* anc = f.anchor + 4 * (g / GPF_BF16_GROUP);
  const uint16_t* quat = static_cast<const uint16_t*>(f.quat);
  const uint16_t* lsc = static_cast<const uint16_t*>(f.logscale);
  const uint16_t* spec = static_cast<const uint16_t*>(f.spectrum);
  const float4 a = *reinterpret_cast<const float4*>(anc);
  if (f.storage == GPF_BF16) {
    const uint16_t* mean = static_cast<const uint16_t*>(f.mean);
    dec[g] = __fadd_rn(a.x, bf16_to_f32(mean[g]));
    dec[n + g] = __fadd_rn(a.y, bf16_to_f32(mean[n + g]));
    dec[2 * n + g] = __fadd_rn(a.z, bf16_to_f32(mean[2 * n + g]));
  } else {
    const float* mean = static_cast<const float*>(f.mean);
#pragma unroll
    for (int k = 0; k < 3; ++k) dec[k * n + g] = mean[k * n + g];
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) dec[(3 + k) * n + g] = bf16_to_f32(quat[k * n + g]);
#pragma unroll
  for (int k = 0; k < 3; ++k) dec[(7 + k) * n + g] = __fadd_rn(a.w, bf16_to_f32(lsc[k * n + g]));
  for (int c = 0; c < f.channels; ++c) dec[(10 + c) * n + g] = bf16_to_f32(spec[c * n + g]);
}

// gpf_field_quantize: one half-warp per group of 16 Gaussians, one lane per
// Gaussian; min / max over the group by xor shuffles within the half-warp.
__global__ void quantize_bf16_kernel(gpf_field src, gpf_field dst) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = src.n;
  const bool live = g < n;
  const float* mean = static_cast<const float*>(src.mean);
  const float* quat = static_cast<const float*>(src.quat);
  const float* lsc = static_cast<const float*>(src.logscale);
  const float* spec = static_cast<const float*>(src.spectrum);
  float mu[3], l[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    mu[k] = live ? mean[k * n + g] : 0.0f;
    l[k] = live ? lsc[k * n + g] : 0.0f;
  }
  float lo[4], hi[4];
#pragma unroll
  for (int k = 0; k < 3; ++k) lo[k] = hi[k] = mu[k];
  lo[3] = fminf(l[0], fminf(l[1], l[2]));
  hi[3] = fmaxf(l[0], fmaxf(l[1], l[2]));
  if (!live) {
#pragma unroll
    for (int k = 0; k < 4; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
  }
#pragma unroll
  for (int o = GPF_BF16_GROUP / 2; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(kFullMask, lo[k], o, GPF_BF16_GROUP));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(kFullMask, hi[k], o, GPF_BF16_GROUP));
    }
  }
  float ref[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) ref[k] = __fmul_rn(__fadd_rn(lo[k], hi[k]), 0.5f);
  if (!live) return;
  if (g % GPF_BF16_GROUP == 0)
    *reinterpret_cast<float4*>(const_cast<float*>(dst.anchor) + 4 * (g / GPF_BF16_GROUP)) =
        make_float4(ref[0], ref[1], ref[2], ref[3]);
  const bool mean32 = dst.storage == GPF_BF16_MEAN32;
  uint16_t* dquat = static_cast<uint16_t*>(const_cast<void*>(dst.quat));
  uint16_t* dlsc = static_cast<uint16_t*>(const_cast<void*>(dst.logscale));
  uint16_t* dspec = static_cast<uint16_t*>(const_cast<void*>(dst.spectrum));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (mean32)
      static_cast<float*>(const_cast<void*>(dst.mean))[k * n + g] = mu[k];
    else
      static_cast<uint16_t*>(const_cast<void*>(dst.mean))[k * n + g] =
          f32_to_bf16(__fsub_rn(mu[k], ref[k]));
    dlsc[k * n + g] = f32_to_bf16(__fsub_rn(l[k], ref[3]));
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) dquat[k * n + g] = f32_to_bf16(quat[k * n + g]);
  for (int c = 0; c < src.channels; ++c) dspec[c * n + g] = f32_to_bf16(spec[c * n + g]);
}

// Per Gaussian: record, level box, the number of cells of that box holding a
// hit point (its list entries) and its key in the backward's order.
__global__ void __launch_bounds__(kThreads, 4)
preprocess_kernel(gpf_field f, Grid grid, float cutoff, int brute,
                                  float* __restrict__ rec, int rs, uint4* __restrict__ box,
                                  const uint32_t* __restrict__ occ,
                                  uint32_t* __restrict__ gcount, uint8_t* __restrict__ glive,
                                  uint32_t* __restrict__ gmask, uint2* __restrict__ qbox,
                                  uint32_t* __restrict__ okey, uint32_t* __restrict__ oval,
                                  DeviceHeader* header) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = f.n;
  uint32_t level_bit = 0;
  bool live = false, small = false, huge = false, bad = false;
  if (g < n) {
    const float* mean = static_cast<const float*>(f.mean);
    const float* spec = static_cast<const float*>(f.spectrum);
    const float mu[3] = {mean[g], mean[n + g], mean[2 * n + g]};
    const Frame fr = gaussian_frame(static_cast<const float*>(f.quat),
                                    static_cast<const float*>(f.logscale), n, g);
    // the record's first 16 floats in registers, stored as four float4 once
    // the level is known (rs is a multiple of 4, the record 16-byte aligned)
    float rv[16];
    const float smax = fmaxf(fr.s[0], fmaxf(fr.s[1], fr.s[2]));
    // non-finite parameters: an infinite log-scale shows in max s; the rest
    // in the record (checked where it is stored)
    uint32_t nf = ~__float_as_uint(smax) & 0x7f800000u ? 0u : 1u;
    rv[0] = mu[0]; rv[1] = mu[1]; rv[2] = mu[2];
    // bounding sphere of the k-sigma ellipsoid, widened by 1e-4 for rounding
    rv[3] = isinf(cutoff) ? INFINITY : cutoff * smax * 1.0001f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float inv = 1.0f / fr.s[j];
#pragma unroll
      for (int k = 0; k < 3; ++k) rv[4 + 3 * j + k] = fr.R[k][j] * inv;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) rv[13 + c] = c < f.channels ? spec[(int64_t)c * n + g] : 0.0f;
    // the order the backward walks Gaussians in: class (0 = bounds within
    // 2 x 2 x 2 query-level cells, 1 = larger, 2 = no hit point in reach);
    // the large ones largest first (log4 of their bounds' volume in query
    // cells), so that none of them starts last; then the cell of the mean on
    // a coarse level
    const int K = grid.qlevel, os = grid.oshift;
    const uint32_t mkey =
        ((coord0(mu[2], grid.oz, grid.inv_cell0, grid.max0z) >> os) * grid.ody +
         (coord0(mu[1], grid.oy, grid.inv_cell0, grid.max0y) >> os)) * grid.odx +
        (coord0(mu[0], grid.ox, grid.inv_cell0, grid.max0x) >> os);
    const int cls_shift = grid.obits - 2;
    const int size_shift = cls_shift - kOrderSizeBits;
    uint32_t cls = 1, size_rank = 0;
    oval[g] = (uint32_t)g;
    if (!brute) {
      uint32_t lo[3], hi[3];
      gaussian_cells0(grid, fr, mu, cutoff, lo, hi);
      qbox[g] = pack_qbox(lo, hi, grid.qlevel);    // the backward's cell range
      if ((hi[0] >> K) - (lo[0] >> K) <= 1 && (hi[1] >> K) - (lo[1] >> K) <= 1 &&
          (hi[2] >> K) - (lo[2] >> K) <= 1) {
        cls = 0;
      } else {
        const uint64_t vq = (uint64_t)((hi[0] >> K) - (lo[0] >> K) + 1) *
                            ((hi[1] >> K) - (lo[1] >> K) + 1) * ((hi[2] >> K) - (lo[2] >> K) + 1);
        const uint32_t lg = 63u - (uint32_t)__clzll((long long)vq);
        const uint32_t top = (1u << kOrderSizeBits) - 1u;
        size_rank = top - min(lg >> 1, top);
      }
      int L = 0;
      for (; L < grid.levels - 1; ++L) {
        const uint32_t sx = (hi[0] >> L) - (lo[0] >> L), sy = (hi[1] >> L) - (lo[1] >> L),
                       sz = (hi[2] >> L) - (lo[2] >> L);
        if (max(sx, max(sy, sz)) < (uint32_t)grid.max_span) break;
      }
      const uint32_t lx = lo[0] >> L, ly = lo[1] >> L, lz = lo[2] >> L;
      const uint32_t sx = (hi[0] >> L) - lx, sy = (hi[1] >> L) - ly, sz = (hi[2] >> L) - lz;
      const int64_t vol = (int64_t)(sx + 1) * (sy + 1) * (sz + 1);
      uint32_t cnt = 0;
      if (sx > 255 || sy > 255 || sz > 255 || vol > kMaxBoxCells) {
        box[g] = make_uint4(kNoBox, kNoBox, kNoBox, 0);
        atomicExch(&header->overflow, 1u);
      } else {
        box[g] = make_uint4(lx | ((uint32_t)L << 20), ly, lz, sx | (sy << 8) | (sz << 16));
        rv[3] = rec_radius_with_level(rv[3], (uint32_t)L);
        level_bit = 1u << L;
        // bit c of the mask: the c-th cell of the box (x fastest) holds a
        // hit point; emit walks the set bits only
        uint32_t mask = 0;
        if (sx <= 2 && sy <= 2 && sz <= 2) {
          // at most 3 x 3 x 3 cells: the nine occupancy reads of a z slice
          // are independent and go out together
          for (uint32_t dz = 0; dz <= sz; ++dz) {
#pragma unroll
            for (uint32_t j = 0; j < 9; ++j) {
              const uint32_t dy = j / 3, dx = j % 3;
              if (dy <= sy && dx <= sx &&
                  occupied(occ, bucket_of(grid, L, lx + dx, ly + dy, lz + dz))) {
                ++cnt;
                mask |= 1u << ((dz * (sy + 1) + dy) * (sx + 1) + dx);
              }
            }
          }
        } else {
          uint32_t c = 0;
          for (uint32_t iz = lz; iz <= lz + sz; ++iz)
            for (uint32_t iy = ly; iy <= ly + sy; ++iy)
              for (uint32_t ix = lx; ix <= lx + sx; ++ix, ++c)
                if (occupied(occ, bucket_of(grid, L, ix, iy, iz))) {
                  ++cnt;
                  if (c < 32) mask |= 1u << c;
                }
        }
        gmask[g] = vol <= 31 ? mask : kMaskAll;
      }
      live = cnt > 0;
      if (grid.blevel >= 0) ++cnt;      // the centre entry (kept for every Gaussian)
      gcount[g] = cnt;
      if (!live) cls = 2;
      small = live && cls == 0;
      huge = live && cls == 1 && size_rank <= 1;
    }
    okey[g] = mkey | (size_rank << size_shift) | (cls << cls_shift);
    glive[g] = (brute || live) ? 1 : 0;
    float4* r4 = reinterpret_cast<float4*>(rec + g * rs);
#pragma unroll
    for (int v = 0; v < 4; ++v)
      r4[v] = make_float4(rv[4 * v], rv[4 * v + 1], rv[4 * v + 2], rv[4 * v + 3]);
    // every parameter finite: a NaN or infinite mean, quaternion or
    // log-scale leaves a non-finite value in the record's mean or M = S^-1 R^T
    // (an infinite log-scale in max s), and a spectrum value is stored as is
#pragma unroll
    for (int v = 0; v < 16; ++v)
      if (v != 3) nf |= ~__float_as_uint(rv[v]) & 0x7f800000u ? 0u : 1u;
    for (int c = 16; c < rs; ++c) {
      const float sv = c - 13 < f.channels ? spec[(int64_t)(c - 13) * n + g] : 0.0f;
      nf |= ~__float_as_uint(sv) & 0x7f800000u ? 0u : 1u;
      rec[g * rs + c] = sv;
    }
    bad = nf != 0u;
  }
  __shared__ uint32_t s_cnt[kBlockWarps][4];
  __shared__ uint32_t s_mask;
  if (threadIdx.x == 0) s_mask = 0;
  __syncthreads();
  const uint32_t m = __reduce_or_sync(kFullMask, level_bit);
  if ((threadIdx.x & 31) == 0 && m) atomicOr(&s_mask, m);
  uint32_t v[4] = {live ? 1u : 0u, small ? 1u : 0u, huge ? 1u : 0u, bad ? 1u : 0u};
  block_counts(v, s_cnt);      // its __syncthreads also orders s_mask
  if (threadIdx.x == 0) {
    // the level bits: only when this block adds one (the mask fills up early)
    if (s_mask & ~*(volatile uint32_t*)&header->level_mask) atomicOr(&header->level_mask, s_mask);
    if (v[0]) atomicAdd(&header->n_live, v[0]);
    if (v[1]) atomicAdd(&header->n_small, v[1]);
    if (v[2]) atomicAdd(&header->n_huge, v[2]);
    if (v[3]) atomicExch(&header->nonfinite, 1u);
  }
}

__global__ void query_keys_kernel(Grid grid, const float* __restrict__ x,
                                  const float* __restrict__ nrm, const float* __restrict__ wo,
                                  const uint8_t* __restrict__ valid, int64_t m,
                                  uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                                  uint32_t* __restrict__ occ, int mark,
                                  uint32_t* __restrict__ qcount, DeviceHeader* header) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool active = false, bad = false;
  uint32_t k = grid.key_inactive;  // sort key
  uint32_t kc = 0u;                 // query-level cell key
  uint32_t c0[3] = {0u, 0u, 0u};   // level-0 cell of an active hit point
  if (i < m) {
    // hemisphere gate n . w_o > 0: the float32 sum when it is far enough
    // from zero for its sign to be exact (its error is below 3 u sum|a_i b_i|,
    // u = 2^-24), else the float64 sum (the three products of float32 values
    // are exact in float64, so its sign is exact)
    const float a0 = nrm[i], a1 = nrm[m + i], a2 = nrm[2 * m + i];
    const float b0 = wo[i], b1 = wo[m + i], b2 = wo[2 * m + i];
    const float d32 = fmaf(a0, b0, fmaf(a1, b1, a2 * b2));
    const float mag = fabsf(a0 * b0) + fabsf(a1 * b1) + fabsf(a2 * b2);
    bool facing;
    if (fabsf(d32) > 1e-6f * mag && mag > 1e-30f) {
      facing = d32 > 0.0f;
    } else {
      const double d = __dadd_rn(__dadd_rn(__dmul_rn((double)a0, (double)b0),
                                           __dmul_rn((double)a1, (double)b1)),
                                 __dmul_rn((double)a2, (double)b2));
      facing = d > 0.0;
    }
    active = facing && (valid == nullptr || valid[i] != 0);
    if (active) {
      bad = !(isfinite(x[i]) && isfinite(x[m + i]) && isfinite(x[2 * m + i]));
      const uint32_t cx = coord0(x[i], grid.ox, grid.inv_cell0, grid.max0x);
      const uint32_t cy = coord0(x[m + i], grid.oy, grid.inv_cell0, grid.max0y);
      const uint32_t cz = coord0(x[2 * m + i], grid.oz, grid.inv_cell0, grid.max0z);
      const int K = grid.qlevel;
      kc = qkey_of(grid, cx >> K, cy >> K, cz >> K);
      k = kc;
      if (grid.qsub > 0) {
        // then the Morton code of the sub-cell on level K - qsub (x in the
        // lowest bit of each triple), so that a run of 32 hit points covers
        // a compact part of its cell
        const int s = K - grid.qsub;
        uint32_t mort = 0u;
        for (int b = grid.qsub - 1; b >= 0; --b)
          mort = (mort << 3) | (((cz >> (s + b)) & 1u) << 2) | (((cy >> (s + b)) & 1u) << 1) |
                 ((cx >> (s + b)) & 1u);
        k = (kc << (3 * grid.qsub)) | mort;
      }
      c0[0] = cx; c0[1] = cy; c0[2] = cz;
    }
    key[i] = k;
    val[i] = (uint32_t)i;
  }
  if (mark) {
    // occupancy bits of every level: all levels' words are read at once,
    // then on each level the first lane of every run of lanes in the same
    // cell (all of a warp's on the coarse ones) sets its bit where it is not
    // set yet
    uint32_t bkt[kMaxLevels], word[kMaxLevels];
#pragma unroll
    for (int L = 0; L < kMaxLevels; ++L) {
      bkt[L] = active && L < grid.levels
                   ? bucket_of(grid, L, c0[0] >> L, c0[1] >> L, c0[2] >> L)
                   : 0xffffffffu;
      word[L] = bkt[L] != 0xffffffffu ? occ[bkt[L] >> 5] : 0xffffffffu;
    }
#pragma unroll
    for (int L = 0; L < kMaxLevels; ++L) {
      if (L >= grid.levels) break;
      const uint32_t b = bkt[L];
      // setting a bit twice is harmless: skipping a lane whose left
      // neighbour has the same cell removes nearly all repeats cheaply
      const uint32_t left = __shfl_up_sync(kFullMask, b, 1);
      const uint32_t bit = 1u << (b & 31u);
      if (b != 0xffffffffu && ((threadIdx.x & 31) == 0 || left != b) && !(word[L] & bit))
        atomicOr(&occ[b >> 5], bit);
    }
  }
  // per-cell counts: one atomic per distinct cell of the warp (neighbouring
  // pixels share query cells)
  const uint32_t peers = __match_any_sync(kFullMask, active ? kc : 0xffffffffu);
  if (active && (peers & lanemask_lt()) == 0) atomicAdd(&qcount[kc], (uint32_t)__popc(peers));
  __shared__ uint32_t s_cnt[kBlockWarps][4];
  uint32_t v[4] = {active ? 1u : 0u, bad ? 1u : 0u, 0u, 0u};
  block_counts(v, s_cnt);
  if (threadIdx.x == 0 && v[0]) atomicAdd(&header->n_active, v[0]);
  if (threadIdx.x == 0 && v[1]) atomicExch(&header->nonfinite, 1u);
}

// One (bucket, Gaussian) entry per occupied cell of every Gaussian's level
// box, in the box's cell order, at the Gaussian's offset (the exclusive scan
// of the counts). A Gaussian whose cells share a bucket appears there on
// consecutive entries; the pair loops take only the first.
__global__ void emit_kernel(Grid grid, int64_t n, int64_t p_max, const float* __restrict__ rec,
                            int rs, const uint4* __restrict__ box,
                            const uint32_t* __restrict__ occ, const uint32_t* __restrict__ gmask,
                            const uint32_t* __restrict__ goffset,
                            uint32_t* __restrict__ gkey, uint32_t* __restrict__ gval,
                            int passes, uint32_t* __restrict__ digit_counts,
                            uint32_t* __restrict__ cocc, uint32_t* __restrict__ focc,
                            DeviceHeader* header) {
  // the digit counts of the entry sort, added here as the keys are written
  __shared__ uint32_t cnt[kSortMaxPasses * kSortBins];
  for (int i = threadIdx.x; i < passes * kSortBins; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0 && (int64_t)header->n_pairs > p_max) atomicExch(&header->overflow, 1u);
  auto put = [&](int64_t pos, uint32_t bucket, uint32_t v) {
    if (pos >= p_max) return;
    gkey[pos] = bucket;
    gval[pos] = v;
    for (int p = 0; p < passes; ++p) atomicAdd(&cnt[p * kSortBins + ((bucket >> (8 * p)) & 255u)], 1u);
  };
  if (g < n) {
    const uint4 bw = box[g];
    int64_t pos = goffset[g];
    if (grid.blevel >= 0) {
      // the centre entry: the cell of the mean on the centre level
      const float* r = rec + g * rs;
      const int Lb = grid.blevel;
      const uint32_t cx = coord0(r[0], grid.ox, grid.inv_cell0, grid.max0x) >> Lb;
      const uint32_t cy = coord0(r[1], grid.oy, grid.inv_cell0, grid.max0y) >> Lb;
      const uint32_t cz = coord0(r[2], grid.oz, grid.inv_cell0, grid.max0z) >> Lb;
      const CellHash h = cell_hash(grid, Lb, cx, cy, cz, kCentreSalt);
      put(pos, h.bucket, (uint32_t)g | h.tag);
      const uint32_t bit = cocc_bit(grid, cx, cy, cz);
      atomicOr(cocc + (bit >> 5), 1u << (bit & 31u));
      if (grid.fwords) atomicOr(focc + focc_word(grid, cx, cy, cz), 1u << (cx & 31u));
      ++pos;
    }
    if (bw.x != kNoBox) {
      const LevelBox b = unpack_box(bw);
      uint32_t mask = gmask[g];
      if (mask != kMaskAll) {
        // the set bits only, in increasing cell order (x fastest): cell c of
        // the box is (c mod nx, (c / nx) mod ny, c / (nx ny)); c < 31, so the
        // quotients computed as floor((c + 0.5) / d) in float32 are exact
        const uint32_t nx = b.hx - b.lx + 1, nxy = nx * (b.hy - b.ly + 1);
        const float inx = 1.0f / (float)nx, inxy = 1.0f / (float)nxy;
        while (mask) {
          const uint32_t c = (uint32_t)__ffs(mask) - 1u;
          mask &= mask - 1u;
          const uint32_t dz = (uint32_t)(((float)c + 0.5f) * inxy);
          const uint32_t r = c - dz * nxy;
          const uint32_t dy = (uint32_t)(((float)r + 0.5f) * inx);
          const uint32_t dx = r - dy * nx;
          const CellHash h = cell_hash(grid, b.level, b.lx + dx, b.ly + dy, b.lz + dz);
          put(pos, h.bucket, (uint32_t)g | h.tag);
          ++pos;
        }
      } else {
        for (uint32_t iz = b.lz; iz <= b.hz; ++iz)
          for (uint32_t iy = b.ly; iy <= b.hy; ++iy)
            for (uint32_t ix = b.lx; ix <= b.hx; ++ix) {
              const CellHash h = cell_hash(grid, b.level, ix, iy, iz);
              if (!occupied(occ, h.bucket)) continue;
              put(pos, h.bucket, (uint32_t)g | h.tag);
              ++pos;
            }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kSortBins; i += blockDim.x)
    if (cnt[i]) atomicAdd(&digit_counts[i], cnt[i]);
}

// [start, end) of every non-empty bucket from the boundaries of the sorted
// keys (the other buckets keep the [0, 0) of the memset).
__global__ void bucket_range_kernel(const uint32_t* __restrict__ keys, const DeviceHeader* header,
                                    int64_t n_cap, uint2* __restrict__ range) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (header->stalled) return;
  int64_t n = header->n_pairs;
  if (n > n_cap) n = n_cap;
  if (i >= n) return;
  const uint32_t k = keys[i];
  if (i == 0 || keys[i - 1] != k) range[k].x = (uint32_t)i;
  if (i == n - 1 || keys[i + 1] != k) range[k].y = (uint32_t)(i + 1);
}

__global__ void index_flags_kernel(const DeviceHeader* header, uint32_t* flags) {
  *flags = index_flags(header);
}

inline unsigned blocks_for(int64_t n, int t = kThreads) {
  return (unsigned)((n + t - 1) / t);
}

}  // namespace

gpf_field float32_view(const IndexDims& d, const IndexBuffers& b, const gpf_field& f) {
  if (f.storage == GPF_F32) return f;
  // rows of the field's own length n, packed at the start of the buffer
  const int64_t n = f.n;
  gpf_field v = f;
  v.storage = GPF_F32;
  v.mean = b.dec;
  v.quat = b.dec + 3 * n;
  v.logscale = b.dec + 7 * n;
  v.spectrum = b.dec + 10 * n;
  v.anchor = nullptr;
  return v;
}

cudaError_t launch_build(const IndexDims& d, const IndexBuffers& b, const gpf_field& f_in,
                         const gpf_queries& q, cudaStream_t stream) {
  const Grid& grid = d.grid;
  cudaError_t e = cudaMemsetAsync(b.header, 0, sizeof(DeviceHeader), stream);
  if (e != cudaSuccess) return e;
  // 0. 16-bit storage: decode every parameter to float32 once
  if (f_in.storage != GPF_F32 && f_in.n > 0) {
    decode_bf16_kernel<<<blocks_for(f_in.n), kThreads, 0, stream>>>(f_in, b.dec);
    note_launches(1);
  }
  const gpf_field f = float32_view(d, b, f_in);
  if (!d.brute) {
    e = cudaMemsetAsync(b.occ, 0, sizeof(uint32_t) * ((grid.n_buckets + 31) / 32), stream);
    if (e != cudaSuccess) return e;
  }
  // hit points per query-level cell, counted by the key pass
  e = cudaMemsetAsync(b.qstart, 0, sizeof(uint32_t) * ((size_t)grid.n_keys + 2), stream);
  if (e != cudaSuccess) return e;
  // 1. hit point keys and occupancy bits of every level
  if (q.m > 0) {
    query_keys_kernel<<<blocks_for(q.m), kThreads, 0, stream>>>(
        grid, q.x, q.normal, q.wo, q.valid, q.m, b.qkey[0], b.qval[0], b.occ, d.brute ? 0 : 1,
        b.qstart, b.header);
    note_launches(1);
  }
  // 2. Gaussian records, level boxes, entry counts, order keys, level mask
  if (f.n > 0) {
    preprocess_kernel<<<blocks_for(f.n), kThreads, 0, stream>>>(
        f, grid, d.cutoff, d.brute ? 1 : 0, b.rec, rec_stride(d.channels), b.box, b.occ,
        b.gcount, b.glive, b.gmask, b.qbox, b.okey[0], b.oval[0], b.header);
    note_launches(1);
  }
  // 3. hit points sorted by query-level cell (inactive ones last), cell starts
  e = radix_sort_pairs(b.qkey[0], b.qval[0], b.qkey[1], b.qval[1], q.m, nullptr, grid.key_bits,
                       b.qsort_ws, &b.header->stalled, stream);
  if (e != cudaSuccess) return e;
  e = exclusive_scan_u32(b.qstart, b.qstart, (int64_t)grid.n_keys + 2, nullptr, b.scan_ws,
                         stream);
  if (e != cudaSuccess) return e;
  // 4. Gaussians in the backward's order
  e = radix_sort_pairs(b.okey[0], b.oval[0], b.okey[1], b.oval[1], f.n, nullptr, grid.obits,
                       b.osort_ws, &b.header->stalled, stream);
  if (e != cudaSuccess) return e;
  if (d.brute || f.n == 0) return cudaGetLastError();
  // 5. (bucket, Gaussian) entries: scan, emit, sort, bucket starts
  e = exclusive_scan_u32(b.gcount, b.goffset, f.n, &b.header->n_pairs, b.scan_ws, stream);
  if (e != cudaSuccess) return e;
  e = radix_sort_clear_counts(b.gsort_ws, stream);
  if (e != cudaSuccess) return e;
  if (grid.blevel >= 0) {
    e = cudaMemsetAsync(
        b.cocc, 0, sizeof(uint32_t) * (((size_t)grid.cdx * grid.cdy * grid.cdz + 31) / 32), stream);
    if (e != cudaSuccess) return e;
    if (grid.fwords && (e = cudaMemsetAsync(b.focc, 0, sizeof(uint32_t) * focc_words(grid),
                                            stream)) != cudaSuccess)
      return e;
  }
  emit_kernel<<<blocks_for(f.n), kThreads, 0, stream>>>(
      grid, f.n, d.p_max, b.rec, rec_stride(d.channels), b.box, b.occ, b.gmask, b.goffset,
      b.gkey[0], b.gval[0], radix_sort_passes(grid.hash_bits), radix_sort_counts(b.gsort_ws),
      b.cocc, b.focc, b.header);
  note_launches(1);
  e = radix_sort_pairs(b.gkey[0], b.gval[0], b.gkey[1], b.gval[1], d.p_max, &b.header->n_pairs,
                       grid.hash_bits, b.gsort_ws, &b.header->stalled, stream, true);
  if (e != cudaSuccess) return e;
  // bucket ranges from the boundaries of the sorted keys
  e = cudaMemsetAsync(b.brange, 0, sizeof(uint2) * (size_t)grid.n_buckets, stream);
  if (e != cudaSuccess) return e;
  if (d.p_max > 0) {
    bucket_range_kernel<<<blocks_for(d.p_max), kThreads, 0, stream>>>(
        b.gkey[b.gsorted], b.header, d.p_max, b.brange);
    note_launches(1);
  }
  if (d.split_items > 0 && q.m > 0) {
    e = launch_tile_split(d, b, q, stream);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_index_flags(const DeviceHeader* header, uint32_t* flags, cudaStream_t stream) {
  index_flags_kernel<<<1, 1, 0, stream>>>(header, flags);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_quantize(const gpf_field& src, const gpf_field& dst, cudaStream_t stream) {
  if (src.n == 0) return cudaSuccess;
  // whole groups per block: kThreads is a multiple of GPF_BF16_GROUP
  quantize_bf16_kernel<<<blocks_for(src.n), kThreads, 0, stream>>>(src, dst);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gpf
