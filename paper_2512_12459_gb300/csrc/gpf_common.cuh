// Shared device-side definitions of libgpf: the multi-level grid geometry and
// its cell hash, the per-Gaussian record and packed level box, the rotation
// and k-sigma bounds of a Gaussian, and the hardware exp2 wrapper used by the
// pair loops.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/gpf.h"

namespace gpf {

constexpr int kWarp = 32;
constexpr uint32_t kFullMask = 0xffffffffu;
constexpr uint32_t kIdMask = 0x7fffffffu;
constexpr int kMaxLevels = 16;
constexpr int kCoordBits = 20;                 // level-0 cell coordinates < 2^20
constexpr uint32_t kCoordMax = (1u << kCoordBits) - 1;

// Device counters at the head of the index workspace.
struct DeviceHeader {
  uint32_t n_pairs;      // (bucket, Gaussian) entries the last build needed
  uint32_t n_active;     // active hit points (valid and facing the viewer)
  uint32_t overflow;     // 1 if n_pairs > max_pairs or a box was too large
  uint32_t level_mask;   // bit L set when some Gaussian lives on level L
  uint32_t n_live;       // Gaussians whose level box holds a hit point
  uint32_t n_small;      // live Gaussians spanning <= 2 query-level cells per axis
  uint32_t n_huge;       // live large Gaussians of the two top size ranks (split in the backward)
  uint32_t stalled;      // 1 if a bounded wait of the build's sort gave up
  // work counters of the persistent pair loops (reset before each launch)
  unsigned long long next_tile;       // forward: next tile of 32 hit points
  unsigned long long next_work;       // backward: next work item
  uint32_t nonfinite;    // 1 if a Gaussian parameter or an active hit point is not finite
  uint32_t nb_pairs;     // (hit point, Gaussian) pairs of the last hybrid backward
  uint32_t n_xunits;     // work units of the split forward tiles (<= GPF_MAX_SPLIT_UNITS)
  uint32_t n_hunits;     // work units of the split hybrid forward tiles (same limit)
  uint32_t pad[48];
};
static_assert(sizeof(DeviceHeader) == 256, "header is one 256-byte block");

// The index of the last build cannot be used (a full pair buffer, a sort
// that gave up waiting, or a non-finite input): the kernels that read it
// return at once and leave their outputs untouched.
__device__ __forceinline__ bool index_unusable(const DeviceHeader* h) {
  return (h->overflow | h->stalled | h->nonfinite) != 0u;
}
// The flags word of gpf_index_flags_async (GPF_FLAG_* of gpf.h).
__device__ __forceinline__ uint32_t index_flags(const DeviceHeader* h) {
  return (h->overflow ? (uint32_t)GPF_FLAG_CAPACITY : 0u) |
         (h->stalled ? (uint32_t)GPF_FLAG_TIMEOUT : 0u) |
         (h->nonfinite ? (uint32_t)GPF_FLAG_NONFINITE : 0u);
}

// Per-Gaussian record read by the pair loops, float32, stride rec_stride(C):
//   [0..2]  mu
//   [3]     bounding-sphere radius of the k-sigma ellipsoid (k * max s_j),
//           rounded up to carry the Gaussian's grid level in its low
//           kLevelBits mantissa bits (rec_radius_with_level, rec_level)
//   [4..12] M = S^-1 R^T, row-major: M[j][k] = R[k][j] / s_j
//   [13..]  Phi[0..C-1], then zero padding to a multiple of 4 floats
// bfloat16 as the upper 16 bits of a float32: exact widening, and rounding
// to nearest with ties to even (the carry of the low half into the upper
// half, plus the upper half's last bit for ties); finite values.
__host__ __device__ __forceinline__ float bf16_to_f32(uint16_t h) {
#ifdef __CUDA_ARCH__
  return __uint_as_float((uint32_t)h << 16);
#else
  const uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
__device__ __forceinline__ uint16_t f32_to_bf16(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Bits of the backward's order key that rank the large Gaussians by size
// (largest first), between the class and the coarse cell of the mean.
constexpr int kOrderSizeBits = 3;
// The backward splits each Gaussian of the two top size ranks (bounds over
// at least 2^12 query-level cells), up to kSplitMax of them, into kSplitWays
// work units over its rows of cells, summing their partial sums in order.
constexpr int kSplitWays = GPF_BWD_SPLIT_WAYS;
constexpr int64_t kSplitMax = GPF_BWD_SPLIT_MAX;

constexpr int kLevelBits = 4;  // levels < 2^kLevelBits = kMaxLevels
constexpr uint32_t kLevelMask = (1u << kLevelBits) - 1u;
static_assert(kMaxLevels <= (1 << kLevelBits), "a level must fit in kLevelBits");

// A radius no smaller than r (finite, >= 0) whose low mantissa bits hold level.
__device__ __forceinline__ float rec_radius_with_level(float r, uint32_t level) {
  const uint32_t u = __float_as_uint(fminf(r, 1e30f));
  return __uint_as_float(((u + kLevelMask) & ~kLevelMask) | level);
}
__device__ __forceinline__ uint32_t rec_level(float r) { return __float_as_uint(r) & kLevelMask; }

__host__ __device__ constexpr int rec_stride(int channels) {
  return channels <= 3 ? 16 : 4 * ((13 + channels + 3) / 4);
}
// Packed hit point of the backward, float32, stride qrec_stride(C):
//   [0..2] x, [3] zeta = 1/max(Z,eps) (1 in SUM mode),
//   [4] kappa = sum_c g_c O_c (0 in SUM mode or when Z <= eps),
//   [5..] gamma_c = g_c rho_c, then zero padding to a multiple of 4 floats
__host__ __device__ constexpr int qrec_stride(int channels) {
  return 4 * ((5 + channels + 3) / 4);
}
// Per-Gaussian sums of the backward (A 6, B 3, D 3, dPhi C), zero padded.
__host__ __device__ constexpr int gacc_stride(int channels) {
  return 12 + channels <= 16 ? 16 : 32;
}

// Geometry of the multi-level grid, passed by value to kernels.
//   level L has cubic cells of edge cell0 * 2^L, all sharing the origin;
//   level-0 cell coordinates i0 = floor((v - origin) / cell0), clamped to
//   [0, 2^K * dims - 1]; the level-L coordinate is i0 >> L.
//   Hit points are sorted by their cell on the query level K, whose cells
//   have linear keys (iz * dy + iy) * dx + ix over dims[3].
//   Gaussian lists live in 2^hash_bits buckets keyed by (level, cell).
struct Grid {
  float ox, oy, oz;        // origin
  float inv_cell0;         // 1 / cell0
  float cell0;             // finest cell edge
  int levels;              // number of levels
  int max_span;            // cells per axis a Gaussian box may span on its level
  int qlevel;              // K
  int dx, dy, dz;          // query-level dims
  uint32_t n_keys;         // dx * dy * dz
  int qsub;                // sub-cell bits per axis of the hit-point order (0..2)
  uint32_t key_inactive;   // = n_keys << 3 qsub, after every active key
  int key_bits;            // bits of a query-level key including the inactive one
  int hash_bits;
  uint32_t n_buckets;      // 2^hash_bits
  uint32_t max0x, max0y, max0z;  // largest level-0 coordinate per axis
  int id_bits;             // low bits of an entry word holding the Gaussian id
  uint32_t id_mask;        // (1 << id_bits) - 1
  int oshift;              // level whose cells order the backward's Gaussians
  uint32_t odx, ody;       // cells per axis on that level
  int obits;               // bits of an order key (cell key and 2 class bits)
  int coop;                // forward: cooperative mode up to this many cells
  int blevel;              // centre level of the ball query (-1: no centre entries)
  int cshift;              // level of the coarse centre occupancy bits (>= blevel + 2)
  uint32_t cdx, cdy, cdz;  // cells per axis on that level
  uint32_t fwords;         // 32-bit words per x row of the fine (centre-level)
                           // occupancy bits (0: no fine bits)
  uint32_t fdy;            // centre-level cells along y
};

// Word of the fine centre occupancy bits holding centre cell (cx, cy, cz)
// (bit cx & 31 of it): rows along x, padded to whole words.
__device__ __forceinline__ uint32_t focc_word(const Grid& g, uint32_t cx, uint32_t cy,
                                              uint32_t cz) {
  return (cz * g.fdy + cy) * g.fwords + (cx >> 5);
}

// Bit of the centre occupancy map (one bit per cell of level cshift, set when
// some Gaussian mean lies in it) for the centre-level cell (cx, cy, cz).
__device__ __forceinline__ uint32_t cocc_bit(const Grid& g, uint32_t cx, uint32_t cy,
                                             uint32_t cz) {
  const int s = g.cshift - g.blevel;
  return ((cz >> s) * g.cdy + (cy >> s)) * g.cdx + (cx >> s);
}

// Level-0 cell coordinate of v along one axis: floor((v - o) / c0) in float32,
// clamped. Correctly rounded float ops and floor are monotone in v, so a point
// inside [a, b] lands in a cell between the cells of a and b on every level.
__device__ __forceinline__ uint32_t coord0(float v, float o, float inv_c, uint32_t cmax) {
  float t = floorf(__fmul_rn(__fsub_rn(v, o), inv_c));
  t = fminf(fmaxf(t, 0.0f), (float)cmax);
  return (uint32_t)t;
}

__host__ __device__ __forceinline__ uint32_t qkey_of(const Grid& g, uint32_t ix, uint32_t iy,
                                                     uint32_t iz) {
  return (iz * (uint32_t)g.dy + iy) * (uint32_t)g.dx + ix;
}

// Hash of the cell (ix, iy, iz) of level L: the 64-bit packed cell through
// the splitmix64 finaliser (Steele, Lea and Flood 2014). The top hash_bits
// bits pick the bucket; the low bits, shifted above the id bits, tag the
// entry words so that entries of other cells sharing the bucket are told
// apart without a memory access (a false match is caught by the box test).
struct CellHash {
  uint32_t bucket;
  uint32_t tag;     // entry word bits above id_bits
};
// Salt of the centre-cell keys (one entry per Gaussian, in the cell of its
// mean on the centre level): a key space apart from the box entries'.
constexpr uint64_t kCentreSalt = 0xd1b54a32d192ed03ull;

__host__ __device__ __forceinline__ CellHash cell_hash(const Grid& g, int L, uint32_t ix,
                                                       uint32_t iy, uint32_t iz,
                                                       uint64_t salt = 0) {
  uint64_t z = ((uint64_t)ix | ((uint64_t)iy << 20) | ((uint64_t)iz << 40) |
                ((uint64_t)L << 60)) ^ salt;
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  CellHash h;
  h.bucket = (uint32_t)(z >> (64 - g.hash_bits));
  h.tag = ((uint32_t)z) << g.id_bits;
  return h;
}
__host__ __device__ __forceinline__ uint32_t bucket_of(const Grid& g, int L, uint32_t ix,
                                                       uint32_t iy, uint32_t iz) {
  return cell_hash(g, L, ix, iy, iz).bucket;
}

// Level box of a Gaussian, packed in a uint4:
//   x = lo.x | level << 20, y = lo.y, z = lo.z (cell coordinates on that level),
//   w = span.x | span.y << 8 | span.z << 16 (hi = lo + span, each span <= 255).
struct LevelBox {
  int level;
  uint32_t lx, ly, lz, hx, hy, hz;
};
__device__ __forceinline__ LevelBox unpack_box(const uint4 b) {
  LevelBox r;
  r.level = (int)(b.x >> 20);
  r.lx = b.x & kCoordMax;
  r.ly = b.y;
  r.lz = b.z;
  r.hx = r.lx + (b.w & 0xffu);
  r.hy = r.ly + ((b.w >> 8) & 0xffu);
  r.hz = r.lz + ((b.w >> 16) & 0xffu);
  return r;
}
__device__ __forceinline__ bool box_holds(const LevelBox& b, uint32_t x, uint32_t y, uint32_t z) {
  return x >= b.lx && x <= b.hx && y >= b.ly && y <= b.hy && z >= b.lz && z <= b.hz;
}

// Rotation and scale of a Gaussian from its raw parameters: R(q/|q|) with
// column j = local axis j in world coordinates (Sec. 4.1), s = exp(l).
struct Frame {
  float R[3][3];
  float s[3];
  float qhat[4];
  float inv_qn;
};
__device__ __forceinline__ Frame gaussian_frame(const float* quat, const float* logscale,
                                                int64_t n, int64_t g) {
  Frame f;
  float qw = quat[g], qx = quat[n + g], qy = quat[2 * n + g], qz = quat[3 * n + g];
  const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  f.inv_qn = qn > 0.0f ? 1.0f / qn : 0.0f;
  qw *= f.inv_qn; qx *= f.inv_qn; qy *= f.inv_qn; qz *= f.inv_qn;
  f.qhat[0] = qw; f.qhat[1] = qx; f.qhat[2] = qy; f.qhat[3] = qz;
  f.R[0][0] = 1.0f - 2.0f * (qy * qy + qz * qz);
  f.R[0][1] = 2.0f * (qx * qy - qw * qz);
  f.R[0][2] = 2.0f * (qx * qz + qw * qy);
  f.R[1][0] = 2.0f * (qx * qy + qw * qz);
  f.R[1][1] = 1.0f - 2.0f * (qx * qx + qz * qz);
  f.R[1][2] = 2.0f * (qy * qz - qw * qx);
  f.R[2][0] = 2.0f * (qx * qz - qw * qy);
  f.R[2][1] = 2.0f * (qy * qz + qw * qx);
  f.R[2][2] = 1.0f - 2.0f * (qx * qx + qy * qy);
  f.s[0] = expf(logscale[g]);
  f.s[1] = expf(logscale[n + g]);
  f.s[2] = expf(logscale[2 * n + g]);
  return f;
}

// Level-0 cell range of the axis-aligned bounds of the ellipsoid Q <= k^2:
// half-extent k sqrt(sum_j R_kj^2 s_j^2) per axis, widened by 1e-4 relative
// and rounded outwards, so a pair with float32 Q <= k^2 lies inside.
__device__ __forceinline__ void gaussian_cells0(const Grid& g, const Frame& f, const float mu[3],
                                                float cutoff, uint32_t lo[3], uint32_t hi[3]) {
  const float o[3] = {g.ox, g.oy, g.oz};
  const uint32_t cm[3] = {g.max0x, g.max0y, g.max0z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float v = f.R[k][0] * f.R[k][0] * f.s[0] * f.s[0] +
                    f.R[k][1] * f.R[k][1] * f.s[1] * f.s[1] +
                    f.R[k][2] * f.R[k][2] * f.s[2] * f.s[2];
    const float e = cutoff * sqrtf(v) * 1.0001f + 1e-30f;
    lo[k] = coord0(__fsub_rd(mu[k], e), o[k], g.inv_cell0, cm[k]);
    hi[k] = coord0(__fadd_ru(mu[k], e), o[k], g.inv_cell0, cm[k]);
  }
}

// Query-level cell bounds of a Gaussian's k-sigma box (gaussian_cells0's
// level-0 bounds >> K), packed 10 bits per axis (query-level cells per axis
// are at most GPF_MAX_DIM = 1024): x = lo, y = hi, each ix | iy << 10 | iz << 20.
__device__ __forceinline__ uint2 pack_qbox(const uint32_t lo[3], const uint32_t hi[3], int K) {
  return make_uint2((lo[0] >> K) | ((lo[1] >> K) << 10) | ((lo[2] >> K) << 20),
                    (hi[0] >> K) | ((hi[1] >> K) << 10) | ((hi[2] >> K) << 20));
}
__device__ __forceinline__ void unpack_qbox(uint2 b, uint32_t lo[3], uint32_t hi[3]) {
  lo[0] = b.x & 1023u; lo[1] = (b.x >> 10) & 1023u; lo[2] = (b.x >> 20) & 1023u;
  hi[0] = b.y & 1023u; hi[1] = (b.y >> 10) & 1023u; hi[2] = (b.y >> 20) & 1023u;
}
static_assert(GPF_MAX_DIM <= 1024, "query-level cell coordinates fit 10 bits");

// 2^x on the special-function unit (ex2.approx.ftz.f32, relative error
// ~2^-22 over the range used here).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kLog2e = 1.4426950408889634f;

// Lower bound of sqrt(Q) = |M (x - mu)| over an axis-aligned box with centre
// c and half-extent h: |M(c - mu)| - |(|M| h)|, lowered by 4e-6 (|M(c-mu)| +
// |(|M| h)|) to cover float32 rounding. A pair inside the box with Q <= k^2
// implies the bound is <= k.
__device__ __forceinline__ float mahalanobis_lower_bound(const float* Mrow, float mx, float my,
                                                         float mz, float cx, float cy, float cz,
                                                         float hx, float hy, float hz) {
  float ex = cx - mx, ey = cy - my, ez = cz - mz;
  float v0 = fmaf(Mrow[0], ex, fmaf(Mrow[1], ey, Mrow[2] * ez));
  float v1 = fmaf(Mrow[3], ex, fmaf(Mrow[4], ey, Mrow[5] * ez));
  float v2 = fmaf(Mrow[6], ex, fmaf(Mrow[7], ey, Mrow[8] * ez));
  float s0 = fmaf(fabsf(Mrow[0]), hx, fmaf(fabsf(Mrow[1]), hy, fabsf(Mrow[2]) * hz));
  float s1 = fmaf(fabsf(Mrow[3]), hx, fmaf(fabsf(Mrow[4]), hy, fabsf(Mrow[5]) * hz));
  float s2 = fmaf(fabsf(Mrow[6]), hx, fmaf(fabsf(Mrow[7]), hy, fabsf(Mrow[8]) * hz));
  float vn = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
  float sn = sqrtf(fmaf(s0, s0, fmaf(s1, s1, s2 * s2)));
  return (vn - sn) - 4e-6f * (vn + sn);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace gpf
