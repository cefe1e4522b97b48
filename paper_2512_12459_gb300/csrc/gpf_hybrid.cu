// gpf_radiance_fwd with the paper's hybrid neighbourhood (GPF_NB_BALL_KNN;
// Sec. 4.2, Neighborhood Search; the query listing of Algorithm S3): the
// Gaussians whose mean lies within ball_r of the hit point, or, where fewer
// than k_min do, the k_min nearest means. The weights are the field's,
// exp(-Q/2) psi(|d|), without truncation; the output is summed or softly
// normalised as in the k-sigma forward.
//
// The means are listed once each under their cell on the centre level (cells
// of edge >= the index's ball_radius), hashed like the box lists under a
// separate key space. One warp per tile of 32 cell-sorted hit points, taking
// tiles from the work counter:
//   * ball: the warp walks the centre cells that the tile's box, grown by
//     ball_r, overlaps; each lane vets one listed Gaussian (its tag, its
//     centre cell, its mean's distance to the tile's box); survivors are
//     staged in shared memory and every lane tests and sums them for its own
//     hit point (a tile whose grown box meets more than kMaxTileCells cells
//     walks the 3 x 3 x 3 cells around each hit point lane by lane instead);
//   * kNN: a lane whose ball holds fewer than k_min Gaussians searches rings
//     of centre cells around its own cell for the k_min nearest means (ring R
//     can be closed once the k-th distance is at most R cells), then sums
//     those instead.
// The same selection serves the backward (Sec. 4.2, Differentiable
// Accumulation, with N(x) held fixed): a counting pass writes each hit
// point's number of selected Gaussians, their exclusive scan gives each
// point its offset, an emitting pass writes the (Gaussian, hit point) pairs
// there in the order the selection visits them, and a stable sort by
// Gaussian leaves every Gaussian's hit points in increasing order: the
// pairs, and so the backward's sums, do not depend on thread timing.
#include <cuda_runtime.h>
#include <math.h>
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
  uint32_t* nbkey;         // emit pass: Gaussian ids of the pairs
  uint32_t* nbval;         // emit pass: hit point positions of the pairs
  int64_t nb_max;          // capacity of nbkey / nbval
};

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

// The k_min nearest means by rings of centre cells around the lane's cell;
// then the sums over them (or their pairs from offset pos). Returns how many
// were found (k_min unless the field is smaller or the rings run out).
template <int C, bool PSI, int MODE>
__device__ int lane_knn(const HybArgs& a, float px, float py, float pz, float (&L)[C],
                        float& Z, uint32_t pos, int64_t k_pos) {
  constexpr int RS = rec_stride(C);
  const Grid& G = a.grid;
  const int Lb = G.blevel;
  const int k = a.k_min;
  float kd[GPF_MAX_KMIN];
  uint32_t kg[GPF_MAX_KMIN];
  int found = 0;
  const int hx = (int)(coord0(px, G.ox, G.inv_cell0, G.max0x) >> Lb);
  const int hy = (int)(coord0(py, G.oy, G.inv_cell0, G.max0y) >> Lb);
  const int hz = (int)(coord0(pz, G.oz, G.inv_cell0, G.max0z) >> Lb);
  const int mx = (int)(G.max0x >> Lb), my = (int)(G.max0y >> Lb), mz = (int)(G.max0z >> Lb);
  const int rmax = max(max(max(hx, mx - hx), max(hy, my - hy)), max(hz, mz - hz));
  const float cell = G.cell0 * (float)(1u << Lb);
  for (int R = 0; R <= min(rmax, kMaxRing); ++R) {
    // the cells of the shell max(|dx|, |dy|, |dz|) = R only, O(R^2) of them:
    // whole squares at dz = +-R; in between, whole rows at dy = +-R and the
    // two end cells dx = +-R of every other row
    for (int dz = -R; dz <= R; ++dz)
      for (int dy = -R; dy <= R; ++dy) {
        const bool full = dz == -R || dz == R || dy == -R || dy == R;
        const int dx_step = full || R == 0 ? 1 : 2 * R;
        for (int dx = -R; dx <= R; dx += dx_step) {
          const int cx = hx + dx, cy = hy + dy, cz = hz + dz;
          if (cx < 0 || cy < 0 || cz < 0 || cx > mx || cy > my || cz > mz) continue;
          const CellHash h = cell_hash(G, Lb, cx, cy, cz, kCentreSalt);
          const uint2 rg = __ldg(a.brange + h.bucket);
          for (uint32_t e = rg.x; e < rg.y; ++e) {
            const uint32_t v = __ldg(a.gval + e);
            if ((v & ~G.id_mask) != h.tag) continue;
            const uint32_t g = v & G.id_mask;
            float rr[4];
            const float4 t = __ldg(reinterpret_cast<const float4*>(a.rec + (int64_t)g * RS));
            rr[0] = t.x; rr[1] = t.y; rr[2] = t.z; rr[3] = t.w;
            if (!in_centre_cell(G, rr, cx, cy, cz)) continue;
            const float d2 = mean_d2(rr, px, py, pz);
            // insert (d2, g) into the sorted list of the k nearest (ties: smaller id)
            if (found == k && !(d2 < kd[k - 1] || (d2 == kd[k - 1] && g < kg[k - 1]))) continue;
            int pos = found < k ? found++ : k - 1;
            while (pos > 0 && (kd[pos - 1] > d2 || (kd[pos - 1] == d2 && kg[pos - 1] > g))) {
              kd[pos] = kd[pos - 1];
              kg[pos] = kg[pos - 1];
              --pos;
            }
            kd[pos] = d2;
            kg[pos] = g;
          }
        }
      }
    // every mean in rings beyond R lies at least R cells away
    const float reach = (float)R * cell;
    if (found == k && kd[k - 1] <= reach * reach) break;
  }
  for (int i = 0; i < found; ++i) {
    if (MODE == kHybSums) {
      float rr[RS];
      hyb_load_rec<RS>(a.rec, kg[i], rr);
      const float w = hyb_weight<PSI>(rr, px, py, pz, a);
#pragma unroll
      for (int c = 0; c < C; ++c) L[c] = fmaf(w, rr[13 + c], L[c]);
      Z += w;
    } else if (MODE == kHybEmit) {
      emit_pair(a, pos + (uint32_t)i, kg[i], k_pos);
    }
  }
  return found;
}

template <int C, bool PSI, int MODE>
__global__ void __launch_bounds__(kHybThreads)
hybrid_fwd_kernel(HybArgs a) {
  constexpr int RS = rec_stride(C);
  __shared__ __align__(16) float s_rec[kHybWarps][kWarp * RS];
  __shared__ uint32_t s_gid[kHybWarps][kWarp];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (index_unusable(a.header)) return;
  if (MODE == kHybEmit && (int64_t)a.header->nb_pairs > a.nb_max) {
    // more pairs than room: flag it once; every later kernel leaves its outputs
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(const_cast<uint32_t*>(&a.header->overflow), 1u);
    return;
  }
  const Grid& G = a.grid;
  const int Lb = G.blevel;
  const int64_t n_act = a.header->n_active;
  const int64_t n_tiles = (a.m + kWarp - 1) / kWarp;
  float* my_rec = s_rec[wib];
  for (;;) {
    __syncwarp();
    unsigned long long tile_u = 0;
    if (lane == 0) tile_u = atomicAdd(a.next_tile, 1ull);
    const int64_t tile = (int64_t)__shfl_sync(kFullMask, tile_u, 0);
    if (tile >= n_tiles) break;
    const int64_t k = tile * kWarp + lane;
    const bool in_range = k < a.m;
    const bool active = k < n_act;
    const uint32_t q = in_range ? a.qval[k] : 0u;
    if (MODE == kHybSums && in_range && !active) {
#pragma unroll
      for (int c = 0; c < C; ++c) a.out[(int64_t)c * a.m + q] = 0.0f;
      if (a.z) a.z[q] = 0.0f;
    }
    if (MODE == kHybCount && in_range && !active) a.nbcnt[k] = 0u;
    if (tile * kWarp >= n_act) continue;  // warp-uniform
    const uint32_t pos = MODE == kHybEmit && active ? a.nbcnt[k] : 0u;
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
    if (a.n == 0) {
      // no Gaussians: the build left no lists to read
    } else if (n_cells <= kMaxTileCells) {
      for (uint32_t cz = cz0; cz <= cz1; ++cz)
        for (uint32_t cy = cy0; cy <= cy1; ++cy)
          for (uint32_t cx = cx0; cx <= cx1; ++cx) {
            const CellHash h = cell_hash(G, Lb, cx, cy, cz, kCentreSalt);
            const uint2 rg = __ldg(a.brange + h.bucket);
            for (uint32_t e0 = rg.x; e0 < rg.y; e0 += kWarp) {
              const uint32_t e = e0 + lane;
              const uint32_t v = e < rg.y ? __ldg(a.gval + e) : 0u;
              bool keep = e < rg.y && (v & ~G.id_mask) == h.tag;
              float rr[RS];
              if (keep) {
                hyb_load_rec<RS>(a.rec, v & G.id_mask, rr);
                keep = in_centre_cell(G, rr, cx, cy, cz);
                if (keep) {
                  // the mean's distance to the tile's box, against ball_r
                  const float ex = fmaxf(fmaxf(b0 - rr[0], rr[0] - b3), 0.0f);
                  const float ey = fmaxf(fmaxf(b1 - rr[1], rr[1] - b4), 0.0f);
                  const float ez = fmaxf(fmaxf(b2 - rr[2], rr[2] - b5), 0.0f);
                  keep = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= a.ball_r2;
                }
              }
              const uint32_t kb = __ballot_sync(kFullMask, keep);
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
    // sparse neighbourhoods: the k_min nearest instead (in the emit pass they
    // take the slots the ball's pairs were written to: there are at least as
    // many of them, min(k_min, N) > cnt)
    if (active && a.n > 0 && cnt < a.k_min) {
#pragma unroll
      for (int c = 0; c < C; ++c) L[c] = 0.0f;
      Z = 0.0f;
      cnt = lane_knn<C, PSI, MODE>(a, px, py, pz, L, Z, pos, k);
    }
    if (MODE == kHybCount && active) a.nbcnt[k] = (uint32_t)cnt;
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

}  // namespace

cudaError_t launch_hybrid_forward(const IndexDims& d, const IndexBuffers& b,
                                  const gpf_queries& q, const gpf_query_params& p, int64_t n,
                                  float* out, float* z, const KernelEvents& ev,
                                  cudaStream_t stream) {
  if (q.m == 0) return cudaSuccess;
  HybArgs a = hyb_args(d, b, q, p, n);
  a.out = out;
  a.z = z;
  cudaError_t e;
  if (ev.start && (e = cudaEventRecord(ev.start, stream)) != cudaSuccess) return e;
  if ((e = hyb_pass<kHybSums>(a, d.channels, isfinite(p.r_max), stream)) != cudaSuccess) return e;
  return ev.stop ? cudaEventRecord(ev.stop, stream) : cudaSuccess;
}

cudaError_t launch_hybrid_pairs(const IndexDims& d, const IndexBuffers& b, const gpf_queries& q,
                                const gpf_query_params& p, int64_t n, cudaStream_t stream) {
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
  // pairs per hit point, their offsets and total, the pairs themselves
  if ((e = hyb_pass<kHybCount>(a, d.channels, psi, stream)) != cudaSuccess) return e;
  if ((e = exclusive_scan_u32(b.nbcnt, b.nbcnt, q.m, &b.header->nb_pairs, b.scan_ws, stream)) !=
      cudaSuccess)
    return e;
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
