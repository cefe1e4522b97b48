// gpf_radiance_fwd: radiance at hit points (Sec. 4.2, aggregation equation;
// the soft falloff and soft normalisation of the query listing of Algorithm S3).
//
// One warp per tile of 32 consecutive hit points in cell-sorted order. For
// every grid level that holds Gaussians, the lanes find their cell on that
// level and group equal cells (__match_any_sync):
//   * few distinct cells (the Gaussians of this level are large next to the
//     tile): warp-cooperative mode. The lanes walk the lists of those cells
//     together, 32 entries at a time; each lane vets one candidate (it belongs
//     to this level and cell, it was not already taken from an earlier cell of
//     the tile, and neither its bounding sphere nor a lower bound of its
//     Mahalanobis distance rules out the tile's box of hit points). Survivors
//     are staged in shared memory and every lane evaluates all of them.
//   * many distinct cells (the Gaussians are small next to the spacing of the
//     hit points): pooled mode. The lanes' own cell lists are concatenated and
//     taken 32 (hit point, entry) items at a time, one per lane; a segmented
//     sum over the lanes returns each hit point's share to its lane.
// Every lane applies the exact predicate Q <= k^2, so the result equals the
// brute-force sum over {i : Q_i <= k^2}. With no cell lists (k = +INF or
// brute force) the candidates are all Gaussians, in index order.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdint.h>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kFwdWarps = 4;
constexpr int kFwdThreads = kFwdWarps * kWarp;
// A tile whose hit points fall in at most Grid::coop cells of a level walks
// that level cooperatively; kUnionMax bounds that threshold.
constexpr int kUnionMax = GPF_MAX_COOP_CELLS;

struct FwdArgs {
  Grid grid;
  const uint32_t* qkey;    // sorted query-level keys of hit points
  const uint32_t* qval;    // sorted hit point ids
  const DeviceHeader* header;
  const float* x;          // [3,M]
  const float* albedo;     // [C,M] or null
  int64_t m;
  const float* rec;
  const uint4* box;
  const uint2* brange;     // [n_buckets] [start, end) of each bucket's list
  const uint32_t* gval;    // sorted entries (Gaussian ids)
  int64_t n;               // Gaussians (brute force)
  int mode;
  float r, r2, inv_rr;     // falloff radius, its square, 1/max(r, 1e-6)
  float eps;
  float kde_scale;         // disk kernel: 1 / (pi r^2)
  float cut, cut2;         // k, k^2
  float tscale;            // sqrt(3 log2 e) / max(r, 1e-6): the falloff root in base 2
  float* out;              // [C,M]
  float* z;                // [M] or null
  unsigned long long* counts;  // count mode: [candidates, included]
  unsigned long long* next_tile;  // work counter, zero at launch
  const uint32_t* tparts;  // split forward: parts of each tile (null: no splitting)
  const uint4* xunit;      // split forward: (tile, part, parts, valid) of each split unit
  float* xsum;             // split forward: [unit][C + 1][32] partial sums
};

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(kFullMask, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFullMask, v, o));
  return v;
}

// Pair kernels: the Gaussian weight alone, with the soft falloff psi, or the
// disk of the photon density estimate.
constexpr int kKernGauss = 0, kKernFalloff = 1, kKernDisk = 2;
constexpr float kNegHalfLog2e = -0.72134752044448170368f;   // -log2(e) / 2

// |d| from d2 = |d|^2 > 0: one reciprocal square root and one Newton step
// on the square root (residual d2 - s^2 by a fused multiply-add), which
// leaves about 1 ulp of relative error, as a correctly rounded square root
// would within an ulp, without its special-case branch.
__device__ __forceinline__ float dist_of(float d2) {
  const float y = rsqrtf(d2);
  const float s = d2 * y;
  return fmaf(0.5f * y, fmaf(-s, s, d2), s);
}

// w = exp(-Q/2) psi(|d|) of an included pair as 2^-(Q log2(e)/2 + t'^2), with
// t' = sqrt(3 log2 e) (|d| - r)/r beyond the falloff radius r (zero within).
template <int KERN>
__device__ __forceinline__ float pair_exp2(float Q, float dx, float dy, float dz,
                                           const FwdArgs& a) {
  float e = Q * kNegHalfLog2e;
  if (KERN == kKernFalloff) {
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (d2 > a.r2) {
      const float t = (dist_of(d2) - a.r) * a.tscale;   // as staged_weight: same w bit for bit
      e = fmaf(-t, t, e);
    }
  }
  return ex2_approx(e);
}

// Weight of one pair: w = exp(-Q/2) psi(|d|) when Q <= k^2 (hit = true); for
// the disk kernel w = 1 when |d| <= r (Eq. kde; 1/(pi r^2) is applied once
// per hit point). In count mode only evaluated and included pairs are counted.
template <int KERN, bool COUNT>
__device__ __forceinline__ float pair_weight(const float* __restrict__ r, float px, float py,
                                             float pz, const FwdArgs& a, bool& hit,
                                             uint32_t& n_eval, uint32_t& n_inc) {
  const float dx = px - r[0], dy = py - r[1], dz = pz - r[2];
  if (KERN == kKernDisk) {
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    hit = d2 <= a.r2;
    if (COUNT) {
      ++n_eval;
      n_inc += hit ? 1u : 0u;
      hit = false;
    }
    return hit ? 1.0f : 0.0f;
  }
  const float u0 = fmaf(r[4], dx, fmaf(r[5], dy, r[6] * dz));
  const float u1 = fmaf(r[7], dx, fmaf(r[8], dy, r[9] * dz));
  const float u2 = fmaf(r[10], dx, fmaf(r[11], dy, r[12] * dz));
  const float Q = fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
  if (COUNT) {
    ++n_eval;
    n_inc += Q <= a.cut2 ? 1u : 0u;
    hit = false;
    return 0.0f;
  }
  hit = Q <= a.cut2;
  if (!hit) return 0.0f;
  return pair_exp2<KERN>(Q, dx, dy, dz, a);
}

// Accumulate one Gaussian record r into this lane's sums (or count it).
template <int C, int KERN, bool COUNT>
__device__ __forceinline__ void eval_pair(const float* __restrict__ r, float px, float py, float pz,
                                          const FwdArgs& a, float (&L)[C], float& Z,
                                          uint32_t& n_eval, uint32_t& n_inc) {
  bool hit;
  const float w = pair_weight<KERN, COUNT>(r, px, py, pz, a, hit, n_eval, n_inc);
  if (hit) {
#pragma unroll
    for (int c = 0; c < C; ++c) L[c] = fmaf(w, r[13 + c], L[c]);
    Z += w;
  }
}

// Weight of a staged record r at (px, py, pz) without branches: 0 unless
// Q <= k^2, else pair_exp2's weight, bit for bit.
template <int KERN>
__device__ __forceinline__ float staged_weight(const float* __restrict__ r, float px, float py,
                                               float pz, const FwdArgs& a) {
  const float dx = px - r[0], dy = py - r[1], dz = pz - r[2];
  const float u0 = fmaf(r[4], dx, fmaf(r[5], dy, r[6] * dz));
  const float u1 = fmaf(r[7], dx, fmaf(r[8], dy, r[9] * dz));
  const float u2 = fmaf(r[10], dx, fmaf(r[11], dy, r[12] * dz));
  const float Q = fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
  float e = Q * kNegHalfLog2e;
  if (KERN == kKernFalloff) {
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float t = (dist_of(d2) - a.r) * a.tscale;   // not used when d2 <= r^2
    e = d2 > a.r2 ? fmaf(-t, t, e) : e;
  }
  return ex2_approx(Q <= a.cut2 ? e : -INFINITY);             // 2^-inf = +0
}

// Every staged record of the cooperative mode at this lane's hit point, four
// at a time as straight-line code. A group may reach past nk (never past the
// 32 staged slots): those slots hold zeros or earlier finite records, and
// their weight is forced to 0, so the sums are those of the first nk in order.
template <int C, int KERN, bool COUNT>
__device__ __forceinline__ void eval_staged(const float* __restrict__ recs, int nk, float px,
                                            float py, float pz, const FwdArgs& a, float (&L)[C],
                                            float& Z, uint32_t& n_eval, uint32_t& n_inc) {
  constexpr int RS = rec_stride(C);
  if (COUNT || KERN == kKernDisk) {
    for (int s = 0; s < nk; ++s) eval_pair<C, KERN, COUNT>(recs + s * RS, px, py, pz, a, L, Z,
                                                           n_eval, n_inc);
    return;
  }
  constexpr int kGroup = 4;
  for (int s = 0; s < nk; s += kGroup) {
    float w[kGroup];
#pragma unroll
    for (int j = 0; j < kGroup; ++j) {
      const float wj = staged_weight<KERN>(recs + (s + j) * RS, px, py, pz, a);
      w[j] = s + j < nk ? wj : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kGroup; ++j) {
      const float* r = recs + (s + j) * RS;
#pragma unroll
      for (int c = 0; c < C; ++c) L[c] = fmaf(w[j], r[13 + c], L[c]);
      Z += w[j];
    }
  }
}

// Hands the per-lane partial sums pc of the lanes with f set to their owner
// key (owner lane) in acc[c][key]. The flushing lanes of one key are
// contiguous, so a segmented inclusive sum over the lanes leaves each key's
// total in its last lane, which adds it to acc. Lanes that flush restart
// from zero.
template <int C>
__device__ __forceinline__ void pooled_flush(float (*acc)[kWarp], int lane, int key_in, bool f,
                                             float (&pc)[C + 1]) {
  const int key = f ? key_in : 2 * kWarp + lane;
  float t[C + 1];
#pragma unroll
  for (int c = 0; c <= C; ++c) t[c] = f ? pc[c] : 0.0f;
#pragma unroll
  for (int d = 1; d < kWarp; d <<= 1) {
    const int kd = __shfl_up_sync(kFullMask, key, d);
    float u[C + 1];
#pragma unroll
    for (int c = 0; c <= C; ++c) u[c] = __shfl_up_sync(kFullMask, t[c], d);
    if (lane >= d && kd == key) {
#pragma unroll
      for (int c = 0; c <= C; ++c) t[c] += u[c];
    }
  }
  const int kn = __shfl_down_sync(kFullMask, key, 1);
  if (f && (lane == kWarp - 1 || kn != key)) {
#pragma unroll
    for (int c = 0; c <= C; ++c) acc[c][key] += t[c];
  }
  if (f) {
#pragma unroll
    for (int c = 0; c <= C; ++c) pc[c] = 0.0f;
  }
  __syncwarp();
}

template <int RS>
__device__ __forceinline__ void load_rec(const float* __restrict__ rec, uint32_t g, float (&r)[RS]) {
  const float4* src = reinterpret_cast<const float4*>(rec + (int64_t)g * RS);
#pragma unroll
  for (int v = 0; v < RS / 4; ++v) {
    const float4 t = __ldg(src + v);
    r[4 * v] = t.x; r[4 * v + 1] = t.y; r[4 * v + 2] = t.z; r[4 * v + 3] = t.w;
  }
}

// COUNT: count the evaluated and included pairs instead of summing radiance.
// SPLIT: the index splits heavy tiles into parts (a separate instantiation,
// so that an index without splitting runs the plain tile loop).
template <int C, bool BRUTE, int KERN, bool COUNT, bool SPLIT>
__global__ void __launch_bounds__(kFwdThreads, C <= 4 ? 6 : 5)
fwd_kernel(FwdArgs a) {
  constexpr int RS = rec_stride(C);
  __shared__ __align__(16) float s_rec[kFwdWarps][kWarp * RS];
  __shared__ unsigned long long s_cell[kFwdWarps][kUnionMax];
  __shared__ int s_leader[kFwdWarps][kUnionMax];
  __shared__ uint2 s_range[kFwdWarps][kMaxLevels][kWarp];
  __shared__ float s_acc[kFwdWarps][C + 1][kWarp];  // pooled-mode sums per hit point
  // the warp's work unit: its tile's part and number of parts (kept here, not
  // in registers, which the pair loops need)
  __shared__ uint32_t s_part[kFwdWarps], s_parts[kFwdWarps];

  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (index_unusable(a.header)) return;
  // the staged slots start finite: eval_staged reads whole groups of four
  for (int i = lane; i < kWarp * RS; i += kWarp) s_rec[wib][i] = 0.0f;
  const int64_t n_act = a.header->n_active;
  const int64_t n_tiles = (a.m + kWarp - 1) / kWarp;
  // split tiles (heavy ones, when the index asks for it) come first as
  // n_x units, one per part; then every tile as one unit (a split tile's is
  // skipped)
  const int64_t n_x = SPLIT ? (int64_t)a.header->n_xunits : 0;
  uint32_t n_eval = 0, n_inc = 0;
  // persistent: every warp takes the next unit until none is left, so a
  // warp that drew a light tile goes on with another one
  for (;;) {
  __syncwarp();
  unsigned long long unit_u = 0;
  if (lane == 0) unit_u = atomicAdd(a.next_tile, 1ull);
  const int64_t unit = (int64_t)__shfl_sync(kFullMask, unit_u, 0);
  if (unit >= n_x + n_tiles) break;
  int64_t tile;
  uint32_t part = 0, parts = 1;
  if (SPLIT && unit < n_x) {
    const uint4 xu = a.xunit[unit];
    if (!xu.w) continue;                      // a slot left over at the capacity edge
    tile = xu.x;
    part = xu.y;
    parts = xu.z;
  } else {
    tile = unit - n_x;
    if (SPLIT && n_x && a.tparts[tile] > 1) continue;  // done by its parts
  }
  const bool split = SPLIT && parts > 1;
  if (SPLIT && lane == 0) {
    s_part[wib] = part;
    s_parts[wib] = parts;
  }
  if (SPLIT) __syncwarp();
  const int64_t base = tile * kWarp;
  const int64_t k = base + lane;
  const bool in_range = k < a.m;
  const bool active = k < n_act;
  const uint32_t q = in_range ? a.qval[k] : 0u;
  if (!COUNT && !split && in_range && !active) {
#pragma unroll
    for (int c = 0; c < C; ++c) a.out[(int64_t)c * a.m + q] = 0.0f;
    if (a.z) a.z[q] = 0.0f;
  }
  if (base >= n_act) continue;  // warp-uniform (never a split tile)
  uint32_t gchunk = 0;  // chunks of this tile's lists seen so far, all levels and modes

  float px = 0.f, py = 0.f, pz = 0.f;
  if (active) {
    px = a.x[q];
    py = a.x[a.m + q];
    pz = a.x[2 * a.m + q];
  }
  float L[C];
#pragma unroll
  for (int c = 0; c < C; ++c) L[c] = 0.0f;
  float Z = 0.0f;
  float* my_rec = s_rec[wib];
#pragma unroll
  for (int c = 0; c <= C; ++c) s_acc[wib][c][lane] = 0.0f;
  __syncwarp();

  if (BRUTE) {
    for (int64_t g0 = 0; g0 < a.n; g0 += kWarp) {
      const int64_t g = g0 + lane;
      const int cnt = (int)min((int64_t)kWarp, a.n - g0);
      if (g < a.n) {
        const float4* src = reinterpret_cast<const float4*>(a.rec + g * RS);
        float4* dst = reinterpret_cast<float4*>(my_rec + lane * RS);
#pragma unroll
        for (int v = 0; v < RS / 4; ++v) dst[v] = src[v];
      }
      __syncwarp();
      if (active)
        for (int s = 0; s < cnt; ++s)
          eval_pair<C, KERN, COUNT>(my_rec + s * RS, px, py, pz, a, L, Z, n_eval, n_inc);
      __syncwarp();
    }
  } else {
    const Grid& G = a.grid;
    const uint32_t c0x = coord0(px, G.ox, G.inv_cell0, G.max0x);
    const uint32_t c0y = coord0(py, G.oy, G.inv_cell0, G.max0y);
    const uint32_t c0z = coord0(pz, G.oz, G.inv_cell0, G.max0z);
    // tile box of the active hit points
    const float bx0 = warp_min(active ? px : INFINITY), bx1 = warp_max(active ? px : -INFINITY);
    const float by0 = warp_min(active ? py : INFINITY), by1 = warp_max(active ? py : -INFINITY);
    const float bz0 = warp_min(active ? pz : INFINITY), bz1 = warp_max(active ? pz : -INFINITY);
    const float cx = 0.5f * (bx0 + bx1), cy = 0.5f * (by0 + by1), cz = 0.5f * (bz0 + bz1);
    const float hx = 0.5f * (bx1 - bx0), hy = 0.5f * (by1 - by0), hz = 0.5f * (bz1 - bz0);
    const float cut_keep = a.cut * 1.0001f;
    const uint32_t lmask = a.header->level_mask;
    // the lane's bucket range on every used level, all looked up at once
#pragma unroll
    for (int lev = 0; lev < kMaxLevels; ++lev) {
      if (lev < G.levels && ((lmask >> lev) & 1u)) {
        uint2 rg = make_uint2(0u, 0u);
        if (active) rg = __ldg(a.brange + cell_hash(G, lev, c0x >> lev, c0y >> lev, c0z >> lev).bucket);
        s_range[wib][lev][lane] = rg;
      }
    }
    __syncwarp();

    for (int lev = 0; lev < G.levels; ++lev) {
      if (!((lmask >> lev) & 1u)) continue;
      const uint32_t lx = c0x >> lev, ly = c0y >> lev, lz = c0z >> lev;
      const unsigned long long packed =
          active ? ((unsigned long long)lx | ((unsigned long long)ly << 20) |
                    ((unsigned long long)lz << 40))
                 : ~0ull;
      const uint32_t peers = __match_any_sync(kFullMask, packed);
      const bool leader = active && (peers & lanemask_lt()) == 0;
      const uint32_t uniq = __ballot_sync(kFullMask, leader);
      const int nu = __popc(uniq);
      if (nu <= G.coop) {
        // ---- warp-cooperative mode over the tile's distinct cells
        if (leader) {
          const int slot = __popc(uniq & lanemask_lt());
          s_cell[wib][slot] = packed;
          s_leader[wib][slot] = lane;
        }
        __syncwarp();
        for (int j = 0; j < nu; ++j) {
          const unsigned long long cj = s_cell[wib][j];
          const uint32_t ux = (uint32_t)(cj & kCoordMax), uy = (uint32_t)((cj >> 20) & kCoordMax),
                         uz = (uint32_t)((cj >> 40) & kCoordMax);
          const uint32_t tag = cell_hash(G, lev, ux, uy, uz).tag;
          const uint2 rg = s_range[wib][lev][s_leader[wib][j]];
          // chunks of 32 entries; a split tile's part takes every parts-th
          // chunk of the tile's lists. The entry words of the next chunk are
          // fetched while the current one is being vetted.
          const uint32_t parts_ = SPLIT ? s_parts[wib] : 1u;
          uint32_t c_first = 0;
          if (SPLIT && parts_ > 1) {     // warp-uniform: only for split tiles
            c_first = (s_part[wib] + parts_ - gchunk % parts_) % parts_;
            gchunk += (rg.y - rg.x + kWarp - 1) / kWarp;
          }
          const uint32_t step = parts_ * kWarp;
          uint32_t e_first = rg.x + c_first * kWarp;
          uint32_t v = e_first + lane < rg.y ? __ldg(a.gval + e_first + lane) : 0u;
          uint32_t carry = 0xffffffffu;
          for (uint32_t e0 = e_first; e0 < rg.y; e0 += step) {
            const uint32_t e = e0 + lane;
            const uint32_t vn = e + step < rg.y ? __ldg(a.gval + e + step) : 0u;
            // a Gaussian listed twice in a bucket sits on consecutive entries
            uint32_t vprev = __shfl_up_sync(kFullMask, v, 1);
            if (lane == 0)
              vprev = parts_ == 1 ? carry : e0 > rg.x ? __ldg(a.gval + e0 - 1) : 0xffffffffu;
            carry = __shfl_sync(kFullMask, v, kWarp - 1);
            bool keep = e < rg.y && (v & ~G.id_mask) == tag && v != vprev;
            const uint32_t g = v & G.id_mask;
            float rr[RS];
            if (keep) {
              const uint4 bw = __ldg(a.box + g);
              load_rec<RS>(a.rec, g, rr);
              const LevelBox b = unpack_box(bw);
              // it must live on this level and cover this cell, and must not
              // have been taken from an earlier cell of this tile
              keep = b.level == lev && box_holds(b, ux, uy, uz);
              for (int jj = 0; jj < j && keep; ++jj) {
                const unsigned long long ci = s_cell[wib][jj];
                keep = !box_holds(b, (uint32_t)(ci & kCoordMax), (uint32_t)((ci >> 20) & kCoordMax),
                                  (uint32_t)((ci >> 40) & kCoordMax));
              }
              if (keep) {
                // sphere test: distance from mu to the tile box vs k * max s
                const float ex = fmaxf(fmaxf(bx0 - rr[0], rr[0] - bx1), 0.0f);
                const float ey = fmaxf(fmaxf(by0 - rr[1], rr[1] - by1), 0.0f);
                const float ez = fmaxf(fmaxf(bz0 - rr[2], rr[2] - bz1), 0.0f);
                keep = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= rr[3] * rr[3];
              }
              if (keep)
                keep = mahalanobis_lower_bound(rr + 4, rr[0], rr[1], rr[2], cx, cy, cz, hx, hy, hz) <=
                       cut_keep;
            }
            const uint32_t kb = __ballot_sync(kFullMask, keep);
            if (keep) {
              float4* dst = reinterpret_cast<float4*>(my_rec + __popc(kb & lanemask_lt()) * RS);
#pragma unroll
              for (int q4 = 0; q4 < RS / 4; ++q4)
                dst[q4] = make_float4(rr[4 * q4], rr[4 * q4 + 1], rr[4 * q4 + 2], rr[4 * q4 + 3]);
            }
            __syncwarp();
            const int nk = __popc(kb);
            if (active) eval_staged<C, KERN, COUNT>(my_rec, nk, px, py, pz, a, L, Z, n_eval, n_inc);
            __syncwarp();
            v = vn;
          }
        }
      } else {
        // ---- pooled mode: the lanes' lists are laid end to end and the warp
        // takes them 32 (hit point, entry) items at a time, one item per lane.
        // A lane sums what it evaluates for one owner at a time and hands the
        // sum over (pooled_flush) when the owner of its item slot changes, so
        // no lane waits for the longest list and every sum has a fixed order.
        // The cell-box test is not needed here: an entry that reached this
        // bucket from another cell on the same level has a box that misses
        // this hit point, so Q > k^2 rejects it; the level test and the
        // duplicate test keep any Gaussian from being counted twice.
        const uint32_t tag = cell_hash(G, lev, lx, ly, lz).tag;
        const uint2 rg = s_range[wib][lev][lane];  // (0, 0) for inactive lanes
        const uint32_t len = rg.y - rg.x;
        uint32_t incl = len;  // inclusive prefix sum of the list lengths
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
          const uint32_t t = __shfl_up_sync(kFullMask, incl, o);
          if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(kFullMask, incl, kWarp - 1);
        int cur = -1;  // owner of this lane's item slot in the previous chunk
        float pc[C + 1];
#pragma unroll
        for (int c = 0; c <= C; ++c) pc[c] = 0.0f;
        uint32_t o_first = 0, o_start = 0, o_tag = 0;
        float qx = 0.0f, qy = 0.0f, qz = 0.0f;
        uint32_t carry = 0xffffffffu;
        // owner of item i: the first lane whose inclusive end exceeds i
        // (kWarp: none); the entry word of the next chunk is fetched while
        // the current chunk is evaluated
        auto owner_of = [&](uint32_t i) {
          int o = 0;
#pragma unroll
          for (int st = 16; st > 0; st >>= 1) {
            const uint32_t pe = __shfl_sync(kFullMask, incl, o + st - 1);
            if (pe <= i) o += st;
          }
          return i < total ? o : kWarp;
        };
        auto entry_of = [&](uint32_t i, int o) {
          const int src = o & (kWarp - 1);
          const uint32_t first = __shfl_sync(kFullMask, incl - len, src);
          const uint32_t start = __shfl_sync(kFullMask, rg.x, src);
          return i < total ? __ldg(a.gval + start + (i - first)) : 0u;
        };
        // a split tile's part takes every parts-th chunk of 32 items
        const uint32_t parts_ = SPLIT ? s_parts[wib] : 1u;
        uint32_t c_first = 0;
        if (SPLIT && parts_ > 1) {
          c_first = (s_part[wib] + parts_ - gchunk % parts_) % parts_;
          gchunk += (total + kWarp - 1) / kWarp;
        }
        const uint32_t step = parts_ * kWarp;
        const uint32_t b_first = c_first * kWarp;
        int own_n = owner_of(b_first + lane);
        uint32_t v_n = entry_of(b_first + lane, own_n);
        for (uint32_t b = b_first; b < total; b += step) {
          const uint32_t i = b + lane;
          const bool live = i < total;
          const int own = own_n;
          const uint32_t v = v_n;
          own_n = owner_of(i + step);
          v_n = entry_of(i + step, own_n);
          const bool chg = own != cur;
          if (__any_sync(kFullMask, chg)) {
            pooled_flush<C>(s_acc[wib], lane, cur, chg && cur >= 0 && cur < kWarp, pc);
            const int src = own & (kWarp - 1);
            o_first = __shfl_sync(kFullMask, incl - len, src);
            o_start = __shfl_sync(kFullMask, rg.x, src);
            o_tag = __shfl_sync(kFullMask, tag, src);
            qx = __shfl_sync(kFullMask, px, src);
            qy = __shfl_sync(kFullMask, py, src);
            qz = __shfl_sync(kFullMask, pz, src);
            cur = own;
          }
          const uint32_t kk = i - o_first;  // position in the owner's list
          // the owner's previous entry is the previous item
          uint32_t vprev = __shfl_up_sync(kFullMask, v, 1);
          if (lane == 0)
            vprev = parts_ == 1 ? carry
                                : live && kk > 0 ? __ldg(a.gval + o_start + kk - 1) : 0xffffffffu;
          carry = __shfl_sync(kFullMask, v, kWarp - 1);
          if (live && (v & ~G.id_mask) == o_tag && !(kk > 0 && v == vprev)) {
            float rr[RS];
            load_rec<RS>(a.rec, v & G.id_mask, rr);
            if (rec_level(rr[3]) == (uint32_t)lev) {
              bool hit;
              const float w = pair_weight<KERN, COUNT>(rr, qx, qy, qz, a, hit, n_eval, n_inc);
              if (hit) {
#pragma unroll
                for (int c = 0; c < C; ++c) pc[c] = fmaf(w, rr[13 + c], pc[c]);
                pc[C] += w;
              }
            }
          }
        }
        pooled_flush<C>(s_acc[wib], lane, cur, cur >= 0 && cur < kWarp, pc);
      }
    }
  }

  if (!COUNT) {
    // the pooled-mode sums of this lane's hit point
    __syncwarp();
#pragma unroll
    for (int c = 0; c < C; ++c) L[c] += s_acc[wib][c][lane];
    Z += s_acc[wib][C][lane];
    if (SPLIT && s_parts[wib] > 1) {
      // this part's sums; fwd_split_combine_kernel adds the parts in order
      float* xs = a.xsum + (size_t)unit * (C + 1) * kWarp;
#pragma unroll
      for (int c = 0; c < C; ++c) xs[c * kWarp + lane] = L[c];
      xs[C * kWarp + lane] = Z;
    } else if (active) {
      float scale = 1.0f;
      if (a.mode == GPF_NORMALIZED) scale = 1.0f / fmaxf(Z, a.eps);
      else if (a.mode == GPF_DISK_KDE) scale = a.kde_scale;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float rho = a.albedo ? a.albedo[(int64_t)c * a.m + q] : 1.0f;
        a.out[(int64_t)c * a.m + q] = rho * (L[c] * scale);
      }
      if (a.z) a.z[q] = Z;
    }
  }
  }  // tile loop

  if (COUNT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_eval += __shfl_xor_sync(kFullMask, n_eval, o);
      n_inc += __shfl_xor_sync(kFullMask, n_inc, o);
    }
    if (lane == 0) {
      atomicAdd(&a.counts[0], (unsigned long long)n_eval);
      atomicAdd(&a.counts[1], (unsigned long long)n_inc);
    }
  }
}

// The split tiles' outputs: one warp per split unit of part 0, adding the
// tile's parts in part order, then the epilogue of fwd_kernel.
template <int C>
__global__ void fwd_split_combine_kernel(FwdArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (index_unusable(a.header) || u >= (int64_t)a.header->n_xunits) return;
  const uint4 xu = a.xunit[u];
  if (!xu.w || xu.y != 0u) return;
  const int64_t k = (int64_t)xu.x * kWarp + lane;
  float L[C], Z = 0.0f;
#pragma unroll
  for (int c = 0; c < C; ++c) L[c] = 0.0f;
  for (uint32_t p = 0; p < xu.z; ++p) {
    const float* xs = a.xsum + (size_t)(u + p) * (C + 1) * kWarp;
#pragma unroll
    for (int c = 0; c < C; ++c) L[c] += xs[c * kWarp + lane];
    Z += xs[C * kWarp + lane];
  }
  if (k >= a.m) return;
  const uint32_t q = a.qval[k];
  const bool active = k < (int64_t)a.header->n_active;
  float scale = 1.0f;
  if (a.mode == GPF_NORMALIZED) scale = 1.0f / fmaxf(Z, a.eps);
  else if (a.mode == GPF_DISK_KDE) scale = a.kde_scale;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const float rho = a.albedo ? a.albedo[(int64_t)c * a.m + q] : 1.0f;
    a.out[(int64_t)c * a.m + q] = active ? rho * (L[c] * scale) : 0.0f;
  }
  if (a.z) a.z[q] = active ? Z : 0.0f;
}

// Estimated work of every tile of 32 hit points, from a sample of eight of its
// points (every fourth: neighbouring points of the cell order see similar
// lists), on every used level: where the sample falls in at most
// Grid::coop cells, the distinct cells' lists, counted 8 times for the
// staged evaluation of their survivors by the whole warp; else the points'
// own lists, counted 4 times for the points not sampled. Then the tile's
// number of parts. Four tiles per warp, eight lanes each.
__global__ void tile_cost_kernel(Grid grid, const DeviceHeader* header, const float* __restrict__ x,
                                 const uint32_t* __restrict__ qval, int64_t m,
                                 const uint2* __restrict__ brange, int split_items,
                                 uint32_t* __restrict__ tparts, uint32_t* __restrict__ xparts) {
  const int lane = threadIdx.x & 31;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tile = gt >> 3;
  const int64_t n_tiles = (m + kWarp - 1) / kWarp;
  const int64_t n_act = header->n_active;
  const int64_t k = tile * kWarp + (lane & 7) * 4;
  const bool active = tile < n_tiles && k < n_act && !index_unusable(header);
  const uint32_t group = 0xffu << (lane & ~7);      // the 8 lanes of this tile
  uint32_t c0x = 0, c0y = 0, c0z = 0;
  uint2 rg[kMaxLevels];
  const uint32_t lmask = header->level_mask;
  if (active) {
    const uint32_t q = qval[k];
    c0x = coord0(x[q], grid.ox, grid.inv_cell0, grid.max0x);
    c0y = coord0(x[m + q], grid.oy, grid.inv_cell0, grid.max0y);
    c0z = coord0(x[2 * m + q], grid.oz, grid.inv_cell0, grid.max0z);
  }
#pragma unroll
  for (int lev = 0; lev < kMaxLevels; ++lev) {
    rg[lev] = make_uint2(0u, 0u);
    if (active && lev < grid.levels && ((lmask >> lev) & 1u))
      rg[lev] = __ldg(brange + cell_hash(grid, lev, c0x >> lev, c0y >> lev, c0z >> lev).bucket);
  }
  uint32_t cost = 0;
#pragma unroll
  for (int lev = 0; lev < kMaxLevels; ++lev) {
    if (lev >= grid.levels || !((lmask >> lev) & 1u)) continue;
    const unsigned long long packed =
        active ? ((unsigned long long)(c0x >> lev) | ((unsigned long long)(c0y >> lev) << 20) |
                  ((unsigned long long)(c0z >> lev) << 40))
               : ~0ull;
    const uint32_t peers = __match_any_sync(kFullMask, packed) & group;
    const bool leader = active && (peers & lanemask_lt()) == 0;
    const int nu = __popc(__ballot_sync(kFullMask, leader) & group);
    const uint32_t len = rg[lev].y - rg[lev].x;
    // (eight samples see at most 8 cells: all 8 distinct reads as more than 8)
    cost += nu <= min(grid.coop, 7) ? (leader ? 8u * len : 0u) : 4u * len;
  }
  // the eight lanes of a tile are consecutive: sum them
  cost += __shfl_xor_sync(kFullMask, cost, 1);
  cost += __shfl_xor_sync(kFullMask, cost, 2);
  cost += __shfl_xor_sync(kFullMask, cost, 4);
  if ((lane & 7) == 0 && tile < n_tiles) {
    uint32_t parts = 1;
    if (cost > (uint32_t)split_items)
      parts = min((cost + (uint32_t)split_items - 1) / (uint32_t)split_items,
                  (uint32_t)GPF_MAX_TILE_PARTS);
    tparts[tile] = parts;
    xparts[tile] = parts > 1 ? parts : 0u;
  }
}

// The split units: tile t's parts at xoff[t] .. xoff[t] + parts - 1 (the
// exclusive scan of the parts of split tiles); a tile whose units would not
// all fit under GPF_MAX_SPLIT_UNITS runs unsplit, and its slots below the
// limit are marked empty.
__global__ void tile_units_kernel(int64_t n_tiles, uint32_t* __restrict__ tparts,
                                  const uint32_t* __restrict__ xoff, uint4* __restrict__ xunit,
                                  uint32_t* n_units) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *n_units = min(xoff[n_tiles], (uint32_t)GPF_MAX_SPLIT_UNITS);
  if (t >= n_tiles) return;
  const uint32_t parts = tparts[t];
  if (parts <= 1) return;
  const uint32_t o = xoff[t];
  const bool fits = (uint64_t)o + parts <= (uint64_t)GPF_MAX_SPLIT_UNITS;
  if (!fits) tparts[t] = 1;
  for (uint32_t p = 0; p < parts && o + p < (uint32_t)GPF_MAX_SPLIT_UNITS; ++p)
    xunit[o + p] = make_uint4((uint32_t)t, p, parts, fits ? 1u : 0u);
}

}  // namespace

cudaError_t launch_split_units(int64_t n_tiles, uint32_t* tparts, uint32_t* xoff, uint4* xunit,
                               uint32_t* n_units, void* scan_ws, cudaStream_t stream) {
  cudaError_t e = exclusive_scan_u32(xoff, xoff, n_tiles + 1, nullptr, scan_ws, stream);
  if (e != cudaSuccess) return e;
  tile_units_kernel<<<(unsigned)((n_tiles + 256) / 256), 256, 0, stream>>>(n_tiles, tparts, xoff,
                                                                           xunit, n_units);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tile_split(const IndexDims& d, const IndexBuffers& b, const gpf_queries& q,
                              cudaStream_t stream) {
  const int64_t n_tiles = (q.m + kWarp - 1) / kWarp;
  tile_cost_kernel<<<(unsigned)((n_tiles * 8 + 255) / 256), 256, 0, stream>>>(
      d.grid, b.header, q.x, b.qval[b.qsorted], q.m, b.brange, d.split_items, b.tparts, b.xoff);
  note_launches(1);
  return launch_split_units(n_tiles, b.tparts, b.xoff, b.xunit, &b.header->n_xunits, b.scan_ws,
                            stream);
}

cudaError_t launch_forward(const IndexDims& d, const IndexBuffers& b, const gpf_queries& q,
                           const gpf_query_params& p, int64_t n, float* out, float* z,
                           unsigned long long* counts, const KernelEvents& ev,
                           cudaStream_t stream) {
  if (counts) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
  }
  if (q.m == 0) return cudaSuccess;
  FwdArgs a;
  a.grid = d.grid;
  a.qkey = b.qkey[b.qsorted];
  a.qval = b.qval[b.qsorted];
  a.header = b.header;
  a.x = q.x;
  a.albedo = q.albedo;
  a.m = q.m;
  a.rec = b.rec;
  a.box = b.box;
  a.brange = b.brange;
  a.gval = b.gval[b.gsorted];
  a.n = n;
  a.mode = p.mode;
  const bool psi = isfinite(p.r_max);
  a.r = psi ? p.r_max : 0.0f;
  a.r2 = psi ? p.r_max * p.r_max : 0.0f;
  a.inv_rr = psi ? 1.0f / fmaxf(p.r_max, 1e-6f) : 0.0f;
  a.eps = p.eps;
  a.kde_scale = psi ? (float)(1.0 / (M_PI * (double)p.r_max * (double)p.r_max)) : 0.0f;
  a.cut = d.cutoff;
  a.cut2 = isinf(d.cutoff) ? INFINITY : d.cutoff * d.cutoff;
  a.tscale = (float)((double)a.inv_rr * std::sqrt(3.0 * M_LOG2E));
  a.out = out;
  a.z = z;
  a.counts = counts;
  a.next_tile = &b.header->next_tile;
  const bool split = d.split_items > 0 && !d.brute;
  a.tparts = split ? b.tparts : nullptr;
  a.xunit = split ? b.xunit : nullptr;
  a.xsum = split ? b.xsum : nullptr;
  {
    const cudaError_t e = cudaMemsetAsync(a.next_tile, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
  }
  const int64_t tiles = (q.m + kWarp - 1) / kWarp + (split ? GPF_MAX_SPLIT_UNITS : 0);
  const int64_t want = (tiles + kFwdWarps - 1) / kFwdWarps;
#define GPF_FWD_LAUNCH2(CC, BR, PS, CN, SP)                                                \
  do {                                                                                    \
    const unsigned blocks = (unsigned)persistent_blocks(                                  \
        reinterpret_cast<const void*>(&fwd_kernel<CC, BR, PS, CN, SP>), kFwdThreads, want); \
    fwd_kernel<CC, BR, PS, CN, SP><<<blocks, kFwdThreads, 0, stream>>>(a);                \
  } while (0)
#define GPF_FWD_LAUNCH(CC, BR, PS, CN)                \
  do {                                                \
    if (!BR && split) GPF_FWD_LAUNCH2(CC, false, PS, CN, true); \
    else GPF_FWD_LAUNCH2(CC, BR, PS, CN, false);      \
  } while (0)
#define GPF_FWD_MODES(CC, BR)                                          \
  do {                                                                 \
    if (counts) GPF_FWD_LAUNCH(CC, BR, kKernGauss, true);              \
    else if (kern == kKernDisk) GPF_FWD_LAUNCH(CC, BR, kKernDisk, false); \
    else if (kern == kKernFalloff) GPF_FWD_LAUNCH(CC, BR, kKernFalloff, false); \
    else GPF_FWD_LAUNCH(CC, BR, kKernGauss, false);                    \
  } while (0)
#define GPF_FWD_CASE(CC)                                                              \
  case CC:                                                                            \
    if (d.brute) GPF_FWD_MODES(CC, true);                                             \
    else GPF_FWD_MODES(CC, false);                                                    \
    note_launches(1);                                                                 \
    if (split && !counts) {                                                           \
      fwd_split_combine_kernel<CC><<<GPF_MAX_SPLIT_UNITS / 4, 128, 0, stream>>>(a);   \
      note_launches(1);                                                               \
    }                                                                                 \
    break;
  const int kern = p.mode == GPF_DISK_KDE ? kKernDisk : psi ? kKernFalloff : kKernGauss;
  if (ev.start) {
    const cudaError_t e = cudaEventRecord(ev.start, stream);
    if (e != cudaSuccess) return e;
  }
  switch (d.channels) {
    GPF_FWD_CASE(1)
    GPF_FWD_CASE(2)
    GPF_FWD_CASE(3)
    GPF_FWD_CASE(4)
    GPF_FWD_CASE(5)
    GPF_FWD_CASE(6)
    GPF_FWD_CASE(7)
    GPF_FWD_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef GPF_FWD_CASE
#undef GPF_FWD_MODES
#undef GPF_FWD_LAUNCH
#undef GPF_FWD_LAUNCH2
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return ev.stop ? cudaEventRecord(ev.stop, stream) : cudaSuccess;
}

}  // namespace gpf
