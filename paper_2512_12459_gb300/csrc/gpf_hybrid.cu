// gpf_radiance_fwd with the paper's hybrid neighbourhood (GPF_NB_BALL_KNN;
// Sec. 4.2, Neighborhood Search; the query listing of Algorithm S3): the
// Gaussians whose mean lies within ball_r of the hit point, or, where fewer
// than k_min do, the k_min nearest means. The weights are the field's,
// exp(-Q/2) psi(|d|), without truncation; the output is summed or softly
// normalised as in the k-sigma forward.
//
// The means are listed once each under their cell on the centre level (cells
// of edge >= the index's ball_radius), hashed like the box lists under a
// separate key space, and marked in two occupancy bitmaps of those cells (a
// coarse one of 4 x 4 x 4 cells or more, and one bit per centre cell). One
// warp per tile of 32 cell-sorted hit points, taking tiles from the work
// counter:
//   * ball: the warp fetches the lists of the centre cells that the tile's
//     box, grown by ball_r, overlaps (32 cells at a time, empty cells
//     skipped) and spreads their entries over the lanes; each lane vets one
//     (its tag, its centre cell, its mean's distance to the tile's box);
//     survivors are staged in shared memory and every lane tests and sums
//     them for its own hit point (a tile whose grown box meets more than
//     kMaxTileCells cells walks the 3 x 3 x 3 cells around each hit point
//     lane by lane instead). Tiles whose boxes list many entries are split
//     into parts over those entries, and a finish pass adds the parts;
//   * kNN: the hit points whose ball holds fewer than k_min Gaussians take
//     the k_min nearest means instead, searched by the whole warp for one
//     group of such points at a time (those within one cell of each other):
//     rings of cells around the group's cells, slice by slice (slices and
//     cells with no mean skipped by the bitmaps), each slice's cells spread
//     over the lanes and their listed means 32 at a time, every point
//     keeping its own sorted list in shared memory; a cell beyond every
//     point's k-th distance is skipped, and a point is settled once its
//     k-th distance is within the searched box.
// The same selection serves the backward (Sec. 4.2, Differentiable
// Accumulation, with N(x) held fixed): a counting pass writes each hit
// point's number of selected Gaussians, their exclusive scan gives each
// point its offset, an emitting pass writes the (Gaussian, hit point) pairs
// there in the order the selection visits them, and a stable sort by
// Gaussian leaves every Gaussian's hit points in increasing order: the
// pairs, and so the backward's sums, do not depend on thread timing. A
// forward asked to (write_counts) leaves the counts and the kNN lists
// behind, so that the backward that follows needs neither the counting pass
// nor the kNN search.
#include <cuda_runtime.h>
#include <math.h>
#include <limits.h>
#include <stdint.h>

#include <algorithm>

#include "gpf_internal.h"

namespace gpf {

namespace {

constexpr int kHybWarps = 4;
constexpr int kHybThreads = kHybWarps * kWarp;
constexpr int kMaxTileCells = 512;   // larger grown boxes: per-lane 27-cell walks
constexpr int kMaxRing = 64;         // kNN rings searched at most (then: what was found)
// What a pass of the selection produces: the forward's sums, each hit
// point's number of selected pairs, or the pairs themselves.
constexpr int kHybSums = 0, kHybCount = 1, kHybEmit = 2;
// The phases of a split forward (sums): whole tiles only; the parts of the
// split tiles and the whole unsplit tiles; the split tiles' finish (their
// parts added in part order, then the kNN and the output as for a whole tile).
constexpr int kHybWhole = 0, kHybSplitParts = 1, kHybSplitFinish = 2;
// listed centre-cell entries of a tile's grown box above which the tile is
// split, and the entries each part takes (up to GPF_MAX_TILE_PARTS parts)
constexpr uint32_t kHybSplitEntries = 512;

struct HybArgs {
  Grid grid;
  const uint32_t* qval;
  const DeviceHeader* header;
  const float* x;
  const float* albedo;
  int64_t m;
  const float* rec;
  const uint2* brange;
  const uint32_t* gval;
  const uint32_t* cocc;    // centre occupancy bits (Grid::cshift cells)
  const uint32_t* focc;    // and per centre cell (Grid::fwords > 0)
  int mode;
  float r, r2, inv_rr;     // falloff radius psi
  float eps;
  float ball_r, ball_r2;
  int k_min;
  int64_t n;               // Gaussians (0: no lists to read; every sum is 0)
  float* out;
  float* z;
  unsigned long long* next_tile;
  uint32_t* nbcnt;         // count pass: pairs per point; emit pass: their offsets
  uint32_t* knn_ids;       // [M][GPF_MAX_KMIN] kNN ids of the points that fall back:
                           // written by the forward, read by an emit pass (knn_stored)
  bool knn_stored;
  uint32_t* nbkey;         // emit pass: Gaussian ids of the pairs
  uint32_t* nbval;         // emit pass: hit point positions of the pairs
  int64_t nb_max;          // capacity of nbkey / nbval
  int phase;               // kHybWhole, kHybSplitParts or kHybSplitFinish
  const uint32_t* hparts;  // split forward: parts of each tile
  const uint32_t* hitems;  // listed entries of each tile's box
  const uint4* hunit;      // (tile, part, parts, valid) of each unit
  float* hsum;             // [unit][C + 2][32] partial L, Z, count
};

// Does some mean lie in centre cell (cx, cy, cz)? The fine occupancy bits
// when the index has them, else every cell may hold one.
__device__ __forceinline__ bool centre_cell_occupied(const HybArgs& a, uint32_t cx, uint32_t cy,
                                                     uint32_t cz) {
  if (!a.grid.fwords) return true;
  return (__ldg(a.focc + focc_word(a.grid, cx, cy, cz)) >> (cx & 31u)) & 1u;
}

// Pair j of hit point position k (emit pass): written when it fits.
__device__ __forceinline__ void emit_pair(const HybArgs& a, uint32_t pos, uint32_t g, int64_t k) {
  if ((int64_t)pos < a.nb_max) {
    a.nbkey[pos] = g;
    a.nbval[pos] = (uint32_t)k;
  }
}

template <int RS>
__device__ __forceinline__ void hyb_load_rec(const float* __restrict__ rec, uint32_t g,
                                             float (&r)[RS]) {
  const float4* src = reinterpret_cast<const float4*>(rec + (int64_t)g * RS);
#pragma unroll
  for (int v = 0; v < RS / 4; ++v) {
    const float4 t = __ldg(src + v);
    r[4 * v] = t.x; r[4 * v + 1] = t.y; r[4 * v + 2] = t.z; r[4 * v + 3] = t.w;
  }
}

// Squared distance from the hit point to a record's mean.
__device__ __forceinline__ float mean_d2(const float* r, float px, float py, float pz) {
  const float dx = px - r[0], dy = py - r[1], dz = pz - r[2];
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// The field's weight exp(-Q/2) psi(|d|), no truncation.
template <bool PSI>
__device__ __forceinline__ float hyb_weight(const float* r, float px, float py, float pz,
                                            const HybArgs& a) {
  const float dx = px - r[0], dy = py - r[1], dz = pz - r[2];
  const float u0 = fmaf(r[4], dx, fmaf(r[5], dy, r[6] * dz));
  const float u1 = fmaf(r[7], dx, fmaf(r[8], dy, r[9] * dz));
  const float u2 = fmaf(r[10], dx, fmaf(r[11], dy, r[12] * dz));
  float e = -0.5f * fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
  if (PSI) {
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    if (d2 > a.r2) {
      const float t = (sqrtf(d2) - a.r) * a.inv_rr;
      e = fmaf(-3.0f * t, t, e);
    }
  }
  return ex2_approx(e * kLog2e);
}

// Is a Gaussian listed in centre cell (cx, cy, cz), rather than in another
// cell of the same bucket with an equal tag? Its mean decides.
__device__ __forceinline__ bool in_centre_cell(const Grid& G, const float* r, uint32_t cx,
                                               uint32_t cy, uint32_t cz) {
  const int Lb = G.blevel;
  return (coord0(r[0], G.ox, G.inv_cell0, G.max0x) >> Lb) == cx &&
         (coord0(r[1], G.oy, G.inv_cell0, G.max0y) >> Lb) == cy &&
         (coord0(r[2], G.oz, G.inv_cell0, G.max0z) >> Lb) == cz;
}

// Lane-by-lane ball sum over the 3 x 3 x 3 centre cells around the lane's own
// (or its count, or its pairs from offset pos for hit point position k).
template <int C, bool PSI, int MODE>
__device__ void lane_ball(const HybArgs& a, float px, float py, float pz, float (&L)[C],
                          float& Z, int& cnt, uint32_t pos, int64_t k) {
  constexpr int RS = rec_stride(C);
  const Grid& G = a.grid;
  const int Lb = G.blevel;
  const int hx = (int)(coord0(px, G.ox, G.inv_cell0, G.max0x) >> Lb);
  const int hy = (int)(coord0(py, G.oy, G.inv_cell0, G.max0y) >> Lb);
  const int hz = (int)(coord0(pz, G.oz, G.inv_cell0, G.max0z) >> Lb);
  const int mx = (int)(G.max0x >> Lb), my = (int)(G.max0y >> Lb), mz = (int)(G.max0z >> Lb);
  for (int cz = max(hz - 1, 0); cz <= min(hz + 1, mz); ++cz)
    for (int cy = max(hy - 1, 0); cy <= min(hy + 1, my); ++cy)
      for (int cx = max(hx - 1, 0); cx <= min(hx + 1, mx); ++cx) {
        const CellHash h = cell_hash(G, Lb, cx, cy, cz, kCentreSalt);
        const uint2 rg = __ldg(a.brange + h.bucket);
        for (uint32_t e = rg.x; e < rg.y; ++e) {
          const uint32_t v = __ldg(a.gval + e);
          if ((v & ~G.id_mask) != h.tag) continue;
          float rr[RS];
          hyb_load_rec<RS>(a.rec, v & G.id_mask, rr);
          if (!in_centre_cell(G, rr, cx, cy, cz)) continue;
          if (mean_d2(rr, px, py, pz) > a.ball_r2) continue;
          if (MODE == kHybSums) {
            const float w = hyb_weight<PSI>(rr, px, py, pz, a);
#pragma unroll
            for (int c = 0; c < C; ++c) L[c] = fmaf(w, rr[13 + c], L[c]);
            Z += w;
          } else if (MODE == kHybEmit) {
            emit_pair(a, pos + (uint32_t)cnt, v & G.id_mask, k);
          }
          ++cnt;
        }
      }
}

// Floats as unsigned keys of the same order (and back), for warp min / max.
__device__ __forceinline__ uint32_t ord_f(float v) {
  const uint32_t u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Cell j of the border of the rectangle [x0, x1] x [y0, y1] (both sides at
// least 3 cells): along y0, up x1, back along y1, down x0.
__device__ __forceinline__ void slice_border_cell(int j, int x0, int y0, int x1, int y1, int& x,
                                                  int& y) {
  const int wx = x1 - x0 + 1, wy = y1 - y0 + 1;
  if (j < wx - 1) { x = x0 + j; y = y0; return; }
  j -= wx - 1;
  if (j < wy - 1) { x = x1; y = y0 + j; return; }
  j -= wy - 1;
  if (j < wx - 1) { x = x1 - j; y = y1; return; }
  j -= wx - 1;
  x = x0;
  y = y1 - j;
}

// Distance along one axis from [lo, hi] (points) to the cell spanning finest
// cells [c_lo, c_hi) from the origin o, grown by half a finest cell.
__device__ __forceinline__ float cell_gap(float o, float cell0, int c_lo, int c_hi, float lo,
                                          float hi) {
  const float a = o + ((float)c_lo - 0.5f) * cell0;
  const float b = o + ((float)c_hi + 0.5f) * cell0;
  return fmaxf(fmaxf(a - hi, lo - b), 0.0f);
}

// A warp's kNN lists in shared memory: entry i of lane l at d[i][l], g[i][l].
struct KnnList {
  float (*d)[kWarp];
  uint32_t (*g)[kWarp];
};

// The k_min nearest means of the tile's points that need them (need: the
// ball held fewer), searched by the whole warp together, one centre cell of
// needing points at a time: the points of a cell have the same rings of
// cells around them, which are now read once for all of them instead of
// once per point. Ring 0 is the cell itself, ring R the cells at Chebyshev
// distance R from it; the lanes share a ring's rows (a row of cells along
// x; away from the ring's outer faces only its two end cells belong to the
// ring), each lane walking its rows' entries, and every round the warp
// stages one mean per lane in shared memory, where each needing lane of the
// cell offers all of them to its own sorted list of the nearest (squared
// distance, then index). A point is settled once it holds k_min means and
// the k-th is no farther than the searched box's nearest face with cells
// beyond it (every other mean lies beyond that face); a cell is done when
// all its points are settled, or after kMaxRing rings. Then each needing
// lane sums its nearest (or writes their pairs from offset pos); returns
// how many it found.
template <int C, bool PSI, int MODE>
__device__ int warp_knn(const HybArgs& a, bool need, float px, float py, float pz,
                        float (&L)[C], float& Z, uint32_t pos, int64_t k_pos,
                        float4* s_cand, KnnList s_list) {
  constexpr int RS = rec_stride(C);
  const Grid& G = a.grid;
  const int Lb = G.blevel;
  const int k = a.k_min;
  const int lane = threadIdx.x & 31;
  uint32_t todo = __ballot_sync(kFullMask, need);
  if (todo == 0u) return 0;
  float* kd = s_list.d[0] + lane;     // this lane's sorted list: entry i at [i * kWarp]
  uint32_t* kg = s_list.g[0] + lane;
  float thr_d = INFINITY;
  uint32_t thr_g = 0xffffffffu;
  int found = 0;
  // the point in units of the finest cell (the cell index before flooring),
  // and its centre cell
  const float tx = __fmul_rn(__fsub_rn(px, G.ox), G.inv_cell0);
  const float ty = __fmul_rn(__fsub_rn(py, G.oy), G.inv_cell0);
  const float tz = __fmul_rn(__fsub_rn(pz, G.oz), G.inv_cell0);
  const int hx = (int)(coord0(px, G.ox, G.inv_cell0, G.max0x) >> Lb);
  const int hy = (int)(coord0(py, G.oy, G.inv_cell0, G.max0y) >> Lb);
  const int hz = (int)(coord0(pz, G.oz, G.inv_cell0, G.max0z) >> Lb);
  const int mx = (int)(G.max0x >> Lb), my = (int)(G.max0y >> Lb), mz = (int)(G.max0z >> Lb);
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int gx = __shfl_sync(kFullMask, hx, leader);
    const int gy = __shfl_sync(kFullMask, hy, leader);
    const int gz = __shfl_sync(kFullMask, hz, leader);
    const bool mine = ((todo >> lane) & 1u) && abs(hx - gx) <= 1 && abs(hy - gy) <= 1 &&
                      abs(hz - gz) <= 1;
    todo &= ~__ballot_sync(kFullMask, mine);
    // the box of their cells (at most 3 x 3 x 3)
    const int qx0 = __reduce_min_sync(kFullMask, mine ? hx : INT_MAX);
    const int qy0 = __reduce_min_sync(kFullMask, mine ? hy : INT_MAX);
    const int qz0 = __reduce_min_sync(kFullMask, mine ? hz : INT_MAX);
    const int qx1 = __reduce_max_sync(kFullMask, mine ? hx : INT_MIN);
    const int qy1 = __reduce_max_sync(kFullMask, mine ? hy : INT_MIN);
    const int qz1 = __reduce_max_sync(kFullMask, mine ? hz : INT_MIN);
    // the box of the cell's needing points
    const float bx0 = unord_f(__reduce_min_sync(kFullMask, mine ? ord_f(px) : 0xffffffffu));
    const float by0 = unord_f(__reduce_min_sync(kFullMask, mine ? ord_f(py) : 0xffffffffu));
    const float bz0 = unord_f(__reduce_min_sync(kFullMask, mine ? ord_f(pz) : 0xffffffffu));
    const float bx1 = unord_f(__reduce_max_sync(kFullMask, mine ? ord_f(px) : 0u));
    const float by1 = unord_f(__reduce_max_sync(kFullMask, mine ? ord_f(py) : 0u));
    const float bz1 = unord_f(__reduce_max_sync(kFullMask, mine ? ord_f(pz) : 0u));
    const int rmax = max(max(max(qx0, mx - qx1), max(qy0, my - qy1)), max(qz0, mz - qz1));
    for (int R = 0; R <= min(rmax, kMaxRing); ++R) {
      const int x0 = qx0 - R, x1 = qx1 + R, y0 = qy0 - R, y1 = qy1 + R, z0 = qz0 - R, z1 = qz1 + R;
      // the ring slice by slice along z: the grown box's rectangle on its
      // two z faces (every slice for R = 0), the rectangle's border between
      const int wx = x1 - x0 + 1, wy = y1 - y0 + 1;
      const int per = 2 * (wx + wy) - 4;
      const float rwx = 1.0f / (float)wx;
      // the occupancy cells under the rectangle (clipped to the grid)
      const int cs = G.cshift - Lb;
      const int ux0 = max(x0, 0) >> cs, uy0 = max(y0, 0) >> cs;
      const int unx = (min(x1, mx) >> cs) - ux0 + 1, nu = unx * ((min(y1, my) >> cs) - uy0 + 1);
      const float runx = 1.0f / (float)unx;
      // the fine bits' words under the rectangle: rows fy0.., words fw0..
      const int fx0 = max(x0, 0), fx1 = min(x1, mx), fy0 = max(y0, 0);
      const int fw0 = fx0 >> 5, fnw = (fx1 >> 5) - fw0 + 1;
      const int fn = G.fwords ? fnw * (min(y1, my) - fy0 + 1) : 0;
      const float rfnw = 1.0f / (float)fnw;
      for (int sz = max(z0, 0); sz <= min(z1, mz); ++sz) {
        // a slice with no mean under its rectangle is skipped whole: first by
        // the coarse bits (a few words in cache), then by the fine ones
        uint32_t any = 0u;
        for (int u = lane; u < nu; u += kWarp) {
          const int uy = (int)(((float)u + 0.5f) * runx);   // u / unx, exact at these sizes
          const uint32_t bit = ((uint32_t)(sz >> cs) * G.cdy + (uint32_t)(uy0 + uy)) * G.cdx +
                               (uint32_t)(ux0 + u - uy * unx);
          any |= (__ldg(a.cocc + (bit >> 5)) >> (bit & 31u)) & 1u;
        }
        if (!__any_sync(kFullMask, any != 0u)) continue;
        if (G.fwords) {
          any = 0u;
          for (int u = lane; u < fn; u += kWarp) {
            const int r = (int)(((float)u + 0.5f) * rfnw);  // u / fnw, exact at these sizes
            const int w = fw0 + u - r * fnw;
            // the bits of word w inside [fx0, fx1]
            const int b0 = max(fx0 - 32 * w, 0), b1 = min(fx1 - 32 * w, 31);
            const uint32_t m = (b1 == 31 ? 0xffffffffu : (2u << b1) - 1u) & ~((1u << b0) - 1u);
            any |= __ldg(a.focc + ((uint32_t)sz * G.fdy + (uint32_t)(fy0 + r)) * G.fwords +
                         (uint32_t)w) & m;
          }
          if (!__any_sync(kFullMask, any != 0u)) continue;
        }
        const bool face = R == 0 || sz == z0 || sz == z1;
        const int n_slice = face ? wx * wy : per;
        for (int c0 = 0; c0 < n_slice; c0 += kWarp) {
          // one cell of the slice per lane: its entries, unless the cell lies
          // beyond every needing point's k-th distance (box grown by half a
          // finest cell for the rounding of the cell coordinates)
          const uint32_t tmax = __reduce_max_sync(
              kFullMask, mine ? __float_as_uint(found == k ? thr_d : INFINITY) : 0u);
          int cx = 0, cy = 0;
          const int cz = sz;
          uint32_t cnt = 0, eb = 0, tag = 0;
          const int j = c0 + lane;
          if (j < n_slice) {
            if (face) {
              const int q = (int)(((float)j + 0.5f) * rwx);   // j / wx, exact at these sizes
              cy = y0 + q;
              cx = x0 + j - q * wx;
            } else {
              slice_border_cell(j, x0, y0, x1, y1, cx, cy);
            }
            if (cx >= 0 && cx <= mx && cy >= 0 && cy <= my) {
              const float dx = cell_gap(G.ox, G.cell0, cx << Lb, (cx + 1) << Lb, bx0, bx1);
              const float dy = cell_gap(G.oy, G.cell0, cy << Lb, (cy + 1) << Lb, by0, by1);
              const float dz = cell_gap(G.oz, G.cell0, cz << Lb, (cz + 1) << Lb, bz0, bz1);
              const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * 0.99999f;
              bool occupied;
              if (G.fwords) {
                occupied = (__ldg(a.focc + focc_word(G, (uint32_t)cx, (uint32_t)cy, (uint32_t)cz)) >>
                            (cx & 31)) & 1u;
              } else {
                const uint32_t bit = cocc_bit(G, (uint32_t)cx, (uint32_t)cy, (uint32_t)cz);
                occupied = (__ldg(a.cocc + (bit >> 5)) >> (bit & 31u)) & 1u;
              }
              if (!(d2 > __uint_as_float(tmax)) && occupied) {
                const CellHash h =
                    cell_hash(G, Lb, (uint32_t)cx, (uint32_t)cy, (uint32_t)cz, kCentreSalt);
                const uint2 rg = __ldg(a.brange + h.bucket);
                eb = rg.x;
                cnt = rg.y - rg.x;
                tag = h.tag;
              }
            }
          }
          uint32_t incl = cnt;
#pragma unroll
          for (int o = 1; o < kWarp; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFullMask, incl, o);
            if (lane >= o) incl += t;
          }
          const uint32_t total = __shfl_sync(kFullMask, incl, kWarp - 1);
          // the cells' entries, 32 at a time: entry f of the chunk belongs to
          // the first lane whose inclusive count exceeds f
          for (uint32_t f0 = 0; f0 < total; f0 += kWarp) {
            const uint32_t f = f0 + lane;
            int o = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1)
              if (__shfl_sync(kFullMask, incl, o + st - 1) <= f) o += st;
            const uint32_t e = __shfl_sync(kFullMask, eb, o) + f -
                               (__shfl_sync(kFullMask, incl, o) - __shfl_sync(kFullMask, cnt, o));
            const uint32_t otag = __shfl_sync(kFullMask, tag, o);
            const int ox = __shfl_sync(kFullMask, cx, o);
            const int oy = __shfl_sync(kFullMask, cy, o);
            const int oz = __shfl_sync(kFullMask, cz, o);
            bool have = false;
            float4 cand = make_float4(0.f, 0.f, 0.f, 0.f);
            if (f < total) {
              const uint32_t v = __ldg(a.gval + e);
              if ((v & ~G.id_mask) == otag) {
                const uint32_t g = v & G.id_mask;
                const float4 t = __ldg(reinterpret_cast<const float4*>(a.rec + (int64_t)g * RS));
                const float mu[3] = {t.x, t.y, t.z};
                if (in_centre_cell(G, mu, (uint32_t)ox, (uint32_t)oy, (uint32_t)oz)) {
                  cand = make_float4(t.x, t.y, t.z, __uint_as_float(g));
                  have = true;
                }
              }
            }
            const uint32_t hm = __ballot_sync(kFullMask, have);
            if (hm == 0u) continue;
            if (have) s_cand[__popc(hm & lanemask_lt())] = cand;
            __syncwarp();
            if (mine) {
              const int nc = __popc(hm);
              for (int s = 0; s < nc; ++s) {
                const float4 c4 = s_cand[s];
                const uint32_t g = __float_as_uint(c4.w);
                const float ddx = px - c4.x, ddy = py - c4.y, ddz = pz - c4.z;
                const float d2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
                if (!(d2 < thr_d || (d2 == thr_d && g < thr_g))) continue;
                // insertion: the larger entries move up one slot (the k-th drops out)
                int j = found < k ? found : k - 1;
                for (; j > 0; --j) {
                  const float pd = kd[(j - 1) * kWarp];
                  const uint32_t pg = kg[(j - 1) * kWarp];
                  if (pd < d2 || (pd == d2 && pg < g)) break;
                  kd[j * kWarp] = pd;
                  kg[j * kWarp] = pg;
                }
                kd[j * kWarp] = d2;
                kg[j * kWarp] = g;
                if (found < k) ++found;
                if (found == k) {
                  thr_d = kd[(k - 1) * kWarp];
                  thr_g = kg[(k - 1) * kWarp];
                }
              }
            }
            __syncwarp();
          }
        }
      }
      // the point's distance to the box's faces that have cells beyond them,
      // in finest cells; half a cell less covers the rounding of the cell
      // coordinates (below 2^-3 cells each at 2^20 cells)
      bool settled = true;
      if (mine) {
        float gap = INFINITY;
        if (x0 > 0) gap = fminf(gap, tx - (float)(x0 << Lb));
        if (x1 < mx) gap = fminf(gap, (float)((x1 + 1) << Lb) - tx);
        if (y0 > 0) gap = fminf(gap, ty - (float)(y0 << Lb));
        if (y1 < my) gap = fminf(gap, (float)((y1 + 1) << Lb) - ty);
        if (z0 > 0) gap = fminf(gap, tz - (float)(z0 << Lb));
        if (z1 < mz) gap = fminf(gap, (float)((z1 + 1) << Lb) - tz);
        const float reach = fmaxf(gap - 0.5f, 0.0f) * G.cell0 * 0.999999f;
        settled = found == k && thr_d <= reach * reach;
      }
      if (__all_sync(kFullMask, settled)) break;
    }
  }
  if (!need) return 0;
  for (int i = 0; i < found; ++i) {
    if (MODE == kHybSums) {
      float rr[RS];
      hyb_load_rec<RS>(a.rec, kg[i * kWarp], rr);
      const float w = hyb_weight<PSI>(rr, px, py, pz, a);
#pragma unroll
      for (int c = 0; c < C; ++c) L[c] = fmaf(w, rr[13 + c], L[c]);
      Z += w;
      if (a.knn_ids) a.knn_ids[k_pos * GPF_MAX_KMIN + i] = kg[i * kWarp];
    } else if (MODE == kHybEmit) {
      emit_pair(a, pos + (uint32_t)i, kg[i * kWarp], k_pos);
    }
  }
  return found;
}

template <int C, bool PSI, int MODE>
__global__ void __launch_bounds__(kHybThreads, 4)
hybrid_fwd_kernel(HybArgs a) {
  constexpr int RS = rec_stride(C);
  __shared__ __align__(16) float s_rec[kHybWarps][kWarp * RS];
  __shared__ uint32_t s_gid[kHybWarps][kWarp];
  __shared__ float4 s_cand[kHybWarps][kWarp];     // the kNN search's staged means
  __shared__ float s_kd[kHybWarps][GPF_MAX_KMIN][kWarp];     // and sorted lists
  __shared__ uint32_t s_kg[kHybWarps][GPF_MAX_KMIN][kWarp];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (index_unusable(a.header)) return;
  if (MODE == kHybEmit && (int64_t)a.header->nb_pairs > a.nb_max) {
    // more pairs than room: flag it once; every later kernel leaves its outputs
    if (blockIdx.x == 0 && threadIdx.x == 0)
      atomicExch(const_cast<uint32_t*>(&a.header->overflow), 1u);
    return;
  }
  const Grid& G = a.grid;
  const int Lb = G.blevel;
  const int64_t n_act = a.header->n_active;
  const int64_t n_tiles = (a.m + kWarp - 1) / kWarp;
  float* my_rec = s_rec[wib];
  const int64_t n_units = a.phase != kHybWhole ? (int64_t)a.header->n_hunits : 0;
  for (;;) {
    __syncwarp();
    unsigned long long item_u = 0;
    if (lane == 0) item_u = atomicAdd(a.next_tile, 1ull);
    const int64_t item = (int64_t)__shfl_sync(kFullMask, item_u, 0);
    // the item: a whole tile, one part of a split tile (its partial sums
    // only), or a split tile's finish
    int64_t tile = item;
    uint32_t part = 0, parts = 1;
    if (a.phase == kHybSplitParts) {
      if (item < n_units) {
        const uint4 u = a.hunit[item];
        if (!u.w) continue;
        tile = u.x;
        part = u.y;
        parts = u.z;
      } else {
        tile = item - n_units;
        if (tile < n_tiles && a.hparts[tile] > 1) continue;
      }
    } else if (a.phase == kHybSplitFinish) {
      if (item >= n_units) break;
      const uint4 u = a.hunit[item];
      if (!u.w || u.y != 0) continue;
      tile = u.x;
      parts = u.z;
    }
    if (tile >= n_tiles) break;
    const bool partial = a.phase == kHybSplitParts && parts > 1;
    const bool finish = a.phase == kHybSplitFinish;
    const int64_t k = tile * kWarp + lane;
    const bool in_range = k < a.m;
    const bool active = k < n_act;
    const uint32_t q = in_range ? a.qval[k] : 0u;
    if (MODE == kHybSums && in_range && !active && !partial) {
#pragma unroll
      for (int c = 0; c < C; ++c) a.out[(int64_t)c * a.m + q] = 0.0f;
      if (a.z) a.z[q] = 0.0f;
    }
    // (the forward writes the counts too when asked to)
    const bool counts = MODE == kHybCount || (MODE == kHybSums && a.nbcnt != nullptr);
    if (counts && in_range && !active && !partial) a.nbcnt[k] = 0u;
    if (tile * kWarp >= n_act) continue;  // warp-uniform
    uint32_t pos = MODE == kHybEmit && active ? a.nbcnt[k] : 0u;
    if (MODE == kHybEmit && partial) {
      // after the ball pairs of the tile's earlier parts (their counts from
      // the counting pass)
      for (uint32_t p = 0; p < part; ++p)
        pos += (uint32_t)__float_as_int(a.hsum[(size_t)(item - part + p) * (C + 2) * kWarp +
                                               (C + 1) * kWarp + lane]);
    }
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
    int cnt = 0;
    // the tile's box, and the centre cells of the box grown by the ball radius
    float b0 = active ? px : INFINITY, b1 = active ? py : INFINITY, b2 = active ? pz : INFINITY;
    float b3 = active ? px : -INFINITY, b4 = active ? py : -INFINITY, b5 = active ? pz : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      b0 = fminf(b0, __shfl_xor_sync(kFullMask, b0, o));
      b1 = fminf(b1, __shfl_xor_sync(kFullMask, b1, o));
      b2 = fminf(b2, __shfl_xor_sync(kFullMask, b2, o));
      b3 = fmaxf(b3, __shfl_xor_sync(kFullMask, b3, o));
      b4 = fmaxf(b4, __shfl_xor_sync(kFullMask, b4, o));
      b5 = fmaxf(b5, __shfl_xor_sync(kFullMask, b5, o));
    }
    const uint32_t cx0 = coord0(b0 - a.ball_r, G.ox, G.inv_cell0, G.max0x) >> Lb;
    const uint32_t cy0 = coord0(b1 - a.ball_r, G.oy, G.inv_cell0, G.max0y) >> Lb;
    const uint32_t cz0 = coord0(b2 - a.ball_r, G.oz, G.inv_cell0, G.max0z) >> Lb;
    const uint32_t cx1 = coord0(b3 + a.ball_r, G.ox, G.inv_cell0, G.max0x) >> Lb;
    const uint32_t cy1 = coord0(b4 + a.ball_r, G.oy, G.inv_cell0, G.max0y) >> Lb;
    const uint32_t cz1 = coord0(b5 + a.ball_r, G.oz, G.inv_cell0, G.max0z) >> Lb;
    const int64_t n_cells = (int64_t)(cx1 - cx0 + 1) * (cy1 - cy0 + 1) * (cz1 - cz0 + 1);
    if (finish) {
      // the parts' sums, added in part order
      for (uint32_t p = 0; p < parts; ++p) {
        const float* src = a.hsum + (size_t)(item + p) * (C + 2) * kWarp + lane;
#pragma unroll
        for (int c = 0; c < C; ++c) L[c] += src[c * kWarp];
        Z += src[C * kWarp];
        cnt += __float_as_int(src[(C + 1) * kWarp]);
      }
    } else if (a.n == 0) {
      // no Gaussians: the build left no lists to read
    } else if (n_cells <= kMaxTileCells) {
      // the box's listed entries in cell order; a part takes its share of them
      uint32_t u_lo = 0, u_hi = 0xffffffffu;
      if (partial) {
        const uint64_t items = a.hitems[tile];
        u_lo = (uint32_t)(items * part / parts);
        u_hi = (uint32_t)(items * (part + 1) / parts);
      }
      // 32 cells at a time, one per lane, then their entries 32 at a time:
      // entry f of the chunk belongs to the first lane whose inclusive count
      // exceeds f
      const uint32_t nx = cx1 - cx0 + 1, ny = cy1 - cy0 + 1;
      uint32_t off = 0;     // entries of the chunks before this one
      for (uint32_t c0 = 0; c0 < (uint32_t)n_cells && off < u_hi; c0 += kWarp) {
        const uint32_t ci = c0 + lane;
        uint32_t ccx = 0, ccy = 0, ccz = 0, eb = 0, len = 0, tag = 0;
        if (ci < (uint32_t)n_cells) {
          ccx = cx0 + ci % nx;
          ccy = cy0 + (ci / nx) % ny;
          ccz = cz0 + ci / (nx * ny);
          // (a cell that holds no mean is not looked up: hyb_cost_kernel
          // skips the same cells)
          if (centre_cell_occupied(a, ccx, ccy, ccz)) {
            const CellHash h = cell_hash(G, Lb, ccx, ccy, ccz, kCentreSalt);
            const uint2 rg = __ldg(a.brange + h.bucket);
            eb = rg.x;
            len = rg.y - rg.x;
            tag = h.tag;
          }
        }
        uint32_t incl = len;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
          const uint32_t t = __shfl_up_sync(kFullMask, incl, o);
          if (lane >= o) incl += t;
        }
        const uint32_t total = __shfl_sync(kFullMask, incl, kWarp - 1);
        const uint32_t f_lo = u_lo > off ? min(u_lo - off, total) : 0u;
        const uint32_t f_hi = min(u_hi - off, total);
        off += total;
        for (uint32_t f0 = f_lo; f0 < f_hi; f0 += kWarp) {
          const uint32_t f = f0 + lane;
          int o = 0;
#pragma unroll
          for (int st = 16; st > 0; st >>= 1)
            if (__shfl_sync(kFullMask, incl, o + st - 1) <= f) o += st;
          const uint32_t e = __shfl_sync(kFullMask, eb, o) + f -
                             (__shfl_sync(kFullMask, incl, o) - __shfl_sync(kFullMask, len, o));
          const uint32_t otag = __shfl_sync(kFullMask, tag, o);
          const uint32_t ox = __shfl_sync(kFullMask, ccx, o);
          const uint32_t oy = __shfl_sync(kFullMask, ccy, o);
          const uint32_t oz = __shfl_sync(kFullMask, ccz, o);
          const uint32_t v = f < f_hi ? __ldg(a.gval + e) : 0u;
          bool keep = f < f_hi && (v & ~G.id_mask) == otag;
          float rr[RS];
          if (keep) {
            hyb_load_rec<RS>(a.rec, v & G.id_mask, rr);
            keep = in_centre_cell(G, rr, ox, oy, oz);
            if (keep) {
              // the mean's distance to the tile's box, against ball_r
              const float ex = fmaxf(fmaxf(b0 - rr[0], rr[0] - b3), 0.0f);
              const float ey = fmaxf(fmaxf(b1 - rr[1], rr[1] - b4), 0.0f);
              const float ez = fmaxf(fmaxf(b2 - rr[2], rr[2] - b5), 0.0f);
              keep = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= a.ball_r2;
            }
          }
          const uint32_t kb = __ballot_sync(kFullMask, keep);
          if (kb == 0u) continue;
          if (keep) {
            const int slot = __popc(kb & lanemask_lt());
            float4* dst = reinterpret_cast<float4*>(my_rec + slot * RS);
#pragma unroll
            for (int q4 = 0; q4 < RS / 4; ++q4)
              dst[q4] = make_float4(rr[4 * q4], rr[4 * q4 + 1], rr[4 * q4 + 2], rr[4 * q4 + 3]);
            s_gid[wib][slot] = v & G.id_mask;
          }
          __syncwarp();
          const int nk = __popc(kb);
          if (active)
            for (int s = 0; s < nk; ++s) {
              const float* r = my_rec + s * RS;
              if (mean_d2(r, px, py, pz) > a.ball_r2) continue;
              if (MODE == kHybSums) {
                const float w = hyb_weight<PSI>(r, px, py, pz, a);
#pragma unroll
                for (int c = 0; c < C; ++c) L[c] = fmaf(w, r[13 + c], L[c]);
                Z += w;
              } else if (MODE == kHybEmit) {
                emit_pair(a, pos + (uint32_t)cnt, s_gid[wib][s], k);
              }
              ++cnt;
            }
          __syncwarp();
        }
      }
    } else if (active) {
      lane_ball<C, PSI, MODE>(a, px, py, pz, L, Z, cnt, pos, k);
    }
    if (partial) {
      // the part's sums (its ball count in the counting pass); the emitting
      // pass has written its pairs and keeps the counts
      if (MODE == kHybEmit) continue;
      float* dst = a.hsum + (size_t)item * (C + 2) * kWarp + lane;
#pragma unroll
      for (int c = 0; c < C; ++c) dst[c * kWarp] = L[c];
      dst[C * kWarp] = Z;
      dst[(C + 1) * kWarp] = __int_as_float(cnt);
      continue;
    }
    // sparse neighbourhoods: the k_min nearest instead (in the emit pass they
    // take the slots the ball's pairs were written to: there are at least as
    // many of them, min(k_min, N) > cnt)
    const bool need = active && a.n > 0 && cnt < a.k_min;
    if (need) {
#pragma unroll
      for (int c = 0; c < C; ++c) L[c] = 0.0f;
      Z = 0.0f;
    }
    if (MODE == kHybEmit && a.knn_stored) {
      // the forward's search, in its order: as many ids as the point's pairs
      if (need) {
        const uint32_t end = k + 1 < a.m ? a.nbcnt[k + 1] : a.header->nb_pairs;
        const uint32_t nk = end - pos;
        for (uint32_t i = 0; i < nk; ++i)
          emit_pair(a, pos + i, a.knn_ids[k * GPF_MAX_KMIN + i], k);
        cnt = (int)nk;
      }
    } else if (a.n > 0) {
      const int nk = warp_knn<C, PSI, MODE>(a, need, px, py, pz, L, Z, pos, k, s_cand[wib],
                                              KnnList{s_kd[wib], s_kg[wib]});
      if (need) cnt = nk;
    }
    if (counts && active) a.nbcnt[k] = (uint32_t)cnt;
    if (MODE == kHybSums && active) {
      float scale = 1.0f;
      if (a.mode == GPF_NORMALIZED) scale = 1.0f / fmaxf(Z, a.eps);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float rho = a.albedo ? a.albedo[(int64_t)c * a.m + q] : 1.0f;
        a.out[(int64_t)c * a.m + q] = rho * (L[c] * scale);
      }
      if (a.z) a.z[q] = Z;
    }
  }
}

// The split forward's plan: each tile's listed centre-cell entries in its
// box grown by ball_r (the cells the ball sums walk, in the same order), and
// from them its parts (1: whole); one warp per tile.
template <int C>
__global__ void __launch_bounds__(kHybThreads)
hyb_cost_kernel(HybArgs a, uint32_t* __restrict__ hparts, uint32_t* __restrict__ hoff,
                uint32_t* __restrict__ hitems) {
  const int lane = threadIdx.x & 31;
  const int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_tiles = (a.m + kWarp - 1) / kWarp;
  if (tile >= n_tiles) return;
  const Grid& G = a.grid;
  const int Lb = G.blevel;
  const int64_t n_act = a.header->n_active;
  uint32_t items = 0;
  if (!index_unusable(a.header) && tile * kWarp < n_act && a.n > 0) {
    const int64_t k = tile * kWarp + lane;
    const bool active = k < n_act;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (active) {
      const uint32_t q = a.qval[k];
      px = a.x[q];
      py = a.x[a.m + q];
      pz = a.x[2 * a.m + q];
    }
    float b0 = active ? px : INFINITY, b1 = active ? py : INFINITY, b2 = active ? pz : INFINITY;
    float b3 = active ? px : -INFINITY, b4 = active ? py : -INFINITY, b5 = active ? pz : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      b0 = fminf(b0, __shfl_xor_sync(kFullMask, b0, o));
      b1 = fminf(b1, __shfl_xor_sync(kFullMask, b1, o));
      b2 = fminf(b2, __shfl_xor_sync(kFullMask, b2, o));
      b3 = fmaxf(b3, __shfl_xor_sync(kFullMask, b3, o));
      b4 = fmaxf(b4, __shfl_xor_sync(kFullMask, b4, o));
      b5 = fmaxf(b5, __shfl_xor_sync(kFullMask, b5, o));
    }
    const uint32_t cx0 = coord0(b0 - a.ball_r, G.ox, G.inv_cell0, G.max0x) >> Lb;
    const uint32_t cy0 = coord0(b1 - a.ball_r, G.oy, G.inv_cell0, G.max0y) >> Lb;
    const uint32_t cz0 = coord0(b2 - a.ball_r, G.oz, G.inv_cell0, G.max0z) >> Lb;
    const uint32_t cx1 = coord0(b3 + a.ball_r, G.ox, G.inv_cell0, G.max0x) >> Lb;
    const uint32_t cy1 = coord0(b4 + a.ball_r, G.oy, G.inv_cell0, G.max0y) >> Lb;
    const uint32_t cz1 = coord0(b5 + a.ball_r, G.oz, G.inv_cell0, G.max0z) >> Lb;
    const uint32_t nx = cx1 - cx0 + 1, ny = cy1 - cy0 + 1;
    const int64_t n_cells = (int64_t)nx * ny * (cz1 - cz0 + 1);
    if (n_cells <= kMaxTileCells) {
      for (uint32_t i = lane; i < (uint32_t)n_cells; i += kWarp) {
        const uint32_t cx = cx0 + i % nx, cy = cy0 + (i / nx) % ny, cz = cz0 + i / (nx * ny);
        if (!centre_cell_occupied(a, cx, cy, cz)) continue;
        const uint2 rg = __ldg(a.brange + cell_hash(G, Lb, cx, cy, cz, kCentreSalt).bucket);
        items += rg.y - rg.x;
      }
      items = __reduce_add_sync(kFullMask, items);
    }
  }
  if (lane == 0) {
    uint32_t parts = 1;
    if (items > kHybSplitEntries)
      parts = min((items + kHybSplitEntries - 1) / kHybSplitEntries, (uint32_t)GPF_MAX_TILE_PARTS);
    hparts[tile] = parts;
    hoff[tile] = parts > 1 ? parts : 0u;
    hitems[tile] = items;
  }
}

}  // namespace

namespace {

HybArgs hyb_args(const IndexDims& d, const IndexBuffers& b, const gpf_queries& q,
                 const gpf_query_params& p, int64_t n) {
  HybArgs a{};
  a.grid = d.grid;
  a.qval = b.qval[b.qsorted];
  a.header = b.header;
  a.x = q.x;
  a.albedo = q.albedo;
  a.m = q.m;
  a.rec = b.rec;
  a.brange = b.brange;
  a.gval = b.gval[b.gsorted];
  a.cocc = b.cocc;
  a.focc = b.focc;
  a.mode = p.mode;
  const bool psi = isfinite(p.r_max);
  a.r = psi ? p.r_max : 0.0f;
  a.r2 = psi ? p.r_max * p.r_max : 0.0f;
  a.inv_rr = psi ? 1.0f / fmaxf(p.r_max, 1e-6f) : 0.0f;
  a.eps = p.eps;
  a.ball_r = p.ball_r;
  a.ball_r2 = p.ball_r * p.ball_r;
  a.k_min = (int64_t)p.k_min < n ? p.k_min : (int)n;
  a.n = n;
  a.next_tile = &b.header->next_tile;
  return a;
}

// One pass of the selection kernel (persistent, tiles from the work counter).
template <int MODE>
cudaError_t hyb_pass(const HybArgs& a, int channels, bool psi, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(a.next_tile, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (a.m + kWarp - 1) / kWarp;
  const int64_t want = (tiles + kHybWarps - 1) / kHybWarps;
#define GPF_HYB_LAUNCH(CC, PS)                                                               \
  do {                                                                                       \
    const unsigned blocks = (unsigned)persistent_blocks(                                     \
        reinterpret_cast<const void*>(&hybrid_fwd_kernel<CC, PS, MODE>), kHybThreads, want); \
    hybrid_fwd_kernel<CC, PS, MODE><<<blocks, kHybThreads, 0, stream>>>(a);                  \
  } while (0)
#define GPF_HYB_CASE(CC)              \
  case CC:                            \
    if (psi) GPF_HYB_LAUNCH(CC, true); \
    else GPF_HYB_LAUNCH(CC, false);   \
    note_launches(1);                 \
    break;
  switch (channels) {
    GPF_HYB_CASE(1)
    GPF_HYB_CASE(2)
    GPF_HYB_CASE(3)
    GPF_HYB_CASE(4)
    GPF_HYB_CASE(5)
    GPF_HYB_CASE(6)
    GPF_HYB_CASE(7)
    GPF_HYB_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef GPF_HYB_CASE
#undef GPF_HYB_LAUNCH
  return cudaGetLastError();
}

// [start, end) of every Gaussian's run of the sorted pairs (the others keep
// the [0, 0) of the memset).
__global__ void nb_range_kernel(const uint32_t* __restrict__ keys, const DeviceHeader* header,
                                int64_t n_cap, uint2* __restrict__ range) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (index_unusable(header)) return;
  const int64_t n = header->nb_pairs;
  if (i >= n || i >= n_cap) return;
  const uint32_t k = keys[i];
  if (i == 0 || keys[i - 1] != k) range[k].x = (uint32_t)i;
  if (i == n - 1 || keys[i + 1] != k) range[k].y = (uint32_t)(i + 1);
}

// The split plan of a selection pass: each tile's listed ball entries and
// parts (hyb_cost_kernel), the unit list of the split tiles, and the
// buffers that the passes read it from.
cudaError_t hyb_split_plan(HybArgs& a, const IndexDims& d, const IndexBuffers& b,
                           const gpf_queries& q, cudaStream_t stream) {
  const int64_t n_tiles = (q.m + kWarp - 1) / kWarp;
  const unsigned blocks = (unsigned)((n_tiles + kHybWarps - 1) / kHybWarps);
  switch (d.channels) {
#define GPF_HYB_COST(CC)                                                                      \
  case CC:                                                                                    \
    hyb_cost_kernel<CC><<<blocks, kHybThreads, 0, stream>>>(a, b.hparts, b.hoff, b.hitems); \
    break;
    GPF_HYB_COST(1) GPF_HYB_COST(2) GPF_HYB_COST(3) GPF_HYB_COST(4)
    GPF_HYB_COST(5) GPF_HYB_COST(6) GPF_HYB_COST(7) GPF_HYB_COST(8)
#undef GPF_HYB_COST
    default:
      return cudaErrorInvalidValue;
  }
  note_launches(1);
  cudaError_t e = launch_split_units(n_tiles, b.hparts, b.hoff, b.hunit, &b.header->n_hunits,
                                     b.scan_ws, stream);
  if (e != cudaSuccess) return e;
  a.hparts = b.hparts;
  a.hitems = b.hitems;
  a.hunit = b.hunit;
  a.hsum = b.hsum;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_hybrid_forward(const IndexDims& d, const IndexBuffers& b,
                                  const gpf_queries& q, const gpf_query_params& p, int64_t n,
                                  float* out, float* z, bool write_counts,
                                  const KernelEvents& ev, cudaStream_t stream) {
  if (q.m == 0) return cudaSuccess;
  HybArgs a = hyb_args(d, b, q, p, n);
  a.out = out;
  a.z = z;
  if (write_counts) {
    a.nbcnt = b.nbcnt;
    a.knn_ids = b.nbknn;
  }
  cudaError_t e;
  if (ev.start && (e = cudaEventRecord(ev.start, stream)) != cudaSuccess) return e;
  const bool psi = isfinite(p.r_max);
  if (n > 0) {
    if ((e = hyb_split_plan(a, d, b, q, stream)) != cudaSuccess) return e;
    a.phase = kHybSplitParts;
    if ((e = hyb_pass<kHybSums>(a, d.channels, psi, stream)) != cudaSuccess) return e;
    a.phase = kHybSplitFinish;
  }
  if ((e = hyb_pass<kHybSums>(a, d.channels, psi, stream)) != cudaSuccess) return e;
  return ev.stop ? cudaEventRecord(ev.stop, stream) : cudaSuccess;
}

cudaError_t launch_hybrid_pairs(const IndexDims& d, const IndexBuffers& b, const gpf_queries& q,
                                const gpf_query_params& p, int64_t n, bool counted,
                                cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(b.nbrange, 0, sizeof(uint2) * (size_t)std::max<int64_t>(n, 1),
                                  stream);
  if (e != cudaSuccess) return e;
  if (q.m == 0 || n == 0) return cudaMemsetAsync(&b.header->nb_pairs, 0, sizeof(uint32_t), stream);
  HybArgs a = hyb_args(d, b, q, p, n);
  a.nbcnt = b.nbcnt;
  a.nbkey = b.nbkey[0];
  a.nbval = b.nbval[0];
  a.nb_max = d.nb_max;
  const bool psi = isfinite(p.r_max);
  // pairs per hit point, their offsets and total, the pairs themselves; the
  // heavy tiles split as in the forward: their parts count (then write) the
  // ball pairs of their share of the entries, the finish adds the counts
  // (then writes the kNN pairs of the points that fall back)
  if (counted) {
    // the forward's plan, counts and kNN ids
    a.knn_ids = b.nbknn;
    a.knn_stored = true;
    a.hparts = b.hparts;
    a.hitems = b.hitems;
    a.hunit = b.hunit;
    a.hsum = b.hsum;
  } else {
    if ((e = hyb_split_plan(a, d, b, q, stream)) != cudaSuccess) return e;
    a.phase = kHybSplitParts;
    if ((e = hyb_pass<kHybCount>(a, d.channels, psi, stream)) != cudaSuccess) return e;
    a.phase = kHybSplitFinish;
    if ((e = hyb_pass<kHybCount>(a, d.channels, psi, stream)) != cudaSuccess) return e;
  }
  if ((e = exclusive_scan_u32(b.nbcnt, b.nbcnt, q.m, &b.header->nb_pairs, b.scan_ws, stream)) !=
      cudaSuccess)
    return e;
  a.phase = kHybSplitParts;
  if ((e = hyb_pass<kHybEmit>(a, d.channels, psi, stream)) != cudaSuccess) return e;
  a.phase = kHybSplitFinish;
  if ((e = hyb_pass<kHybEmit>(a, d.channels, psi, stream)) != cudaSuccess) return e;
  // by Gaussian, stable: each Gaussian's hit points stay in increasing order
  e = radix_sort_pairs(b.nbkey[0], b.nbval[0], b.nbkey[1], b.nbval[1], d.nb_max,
                       &b.header->nb_pairs, d.grid.id_bits, b.nbsort_ws, &b.header->stalled,
                       stream);
  if (e != cudaSuccess) return e;
  nb_range_kernel<<<(unsigned)((d.nb_max + 255) / 256), 256, 0, stream>>>(
      b.nbkey[b.nbsorted], b.header, d.nb_max, b.nbrange);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace gpf
