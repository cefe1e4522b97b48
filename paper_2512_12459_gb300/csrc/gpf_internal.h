// Internal interfaces between the C ABI layer and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "gpf_common.cuh"

namespace gpf {

inline size_t align_up(size_t b, size_t a = 256) { return (b + a - 1) / a * a; }
// Words of the fine centre occupancy bits (Grid::fwords per row).
inline size_t focc_words(const Grid& g) {
  return (size_t)g.fwords * g.fdy * ((g.max0z >> g.blevel) + 1);
}

// Host-side count of the kernels this library has launched (gpf_launch_count).
void note_launches(uint64_t k);

// Blocks of a persistent launch of `kernel` (static shared memory only):
// the blocks that can be resident on all SMs of the current device at once,
// at most max_blocks and at least 1.
int64_t persistent_blocks(const void* kernel, int threads, int64_t max_blocks);

// ---- scan / sort (gpf_sort.cu)
int64_t scan_partials_count(int64_t n);
size_t scan_workspace_bytes(int64_t n_max);
// out[i] = sum_{j<i} in[j] for i < n (host-known n); *total_out = sum (device, may be null).
cudaError_t exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_out,
                               void* ws, cudaStream_t stream);
// The sort's element count limit: status words hold 30-bit counts.
constexpr int64_t kMaxSortN = int64_t(1) << 30;
int64_t radix_tiles(int64_t n_max);
size_t radix_sort_workspace_bytes(int64_t n_max);
int radix_sort_passes(int bits);
// Stable sort of min(*d_n, n_max) pairs (n_max pairs when d_n is null) by
// key bits [0, bits). The result is in (k0, v0) after an even number of
// passes, in (k1, v1) after an odd one. *stalled (device) is set to 1 if a
// bounded wait of the single-pass sort gave up (the output is then invalid).
// counted: the kernel that wrote the keys has already added their digit
// counts, digit d of pass p at radix_sort_counts(ws)[p * kSortBins + d],
// into counts that radix_sort_clear_counts zeroed before it ran.
constexpr int kSortBins = 256;
constexpr int kSortMaxPasses = 4;
cudaError_t radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                             int64_t n_max, const uint32_t* d_n, int bits, void* ws,
                             uint32_t* stalled, cudaStream_t stream, bool counted = false);
uint32_t* radix_sort_counts(void* ws);
cudaError_t radix_sort_clear_counts(void* ws, cudaStream_t stream);
// The failure-detection probe of the single-pass sort's bounded wait (a
// look-back whose predecessor tile is never processed): buffer size, launch.
size_t sort_wait_probe_bytes();
cudaError_t launch_sort_wait_probe(void* buf, uint32_t spin_limit, uint32_t* stalled,
                                   cudaStream_t stream);

// ---- index build (gpf_index.cu)
struct IndexBuffers {
  DeviceHeader* header;
  float* rec;           // [N_max * rec_stride] Gaussian records
  uint4* box;           // [N_max] level boxes
  uint32_t* gcount;     // [N_max] entries per Gaussian
  uint8_t* glive;       // [N_max] 1 if the backward visits the Gaussian (a hit point in reach)
  uint32_t* gmask;      // [N_max] occupied cells of the level box (boxes of <= 31 cells)
  uint2* qbox;          // [N_max] query-level cell bounds of each Gaussian (pack_qbox)
  uint32_t* goffset;    // [N_max] exclusive scan of gcount
  uint32_t* okey[2];    // [N_max] query-level key of each mean (sort ping-pong)
  uint32_t* oval[2];    // [N_max] Gaussian ids in that order
  uint32_t* qkey[2];    // [M_max] sort ping-pong of hit points
  uint32_t* qval[2];
  uint32_t* qstart;     // [n_keys + 2] per-cell start of the sorted hit points
  float* qrec;          // [M_max * qrec_stride] packed hit points of the backward
  float* gacc;          // [N_max * gacc_stride] per-Gaussian sums of the backward
                        // (room for float64 sums: the gradient-check build)
  float* bpart;         // [kSplitMax * kSplitWays * gacc_stride] partial sums of
                        // the backward's split Gaussians (room for float64)
  uint32_t* occ;        // [n_buckets / 32] occupancy bits of (level, cell) buckets
  uint32_t* gkey[2];    // [P_max] (bucket, Gaussian) entries, sort ping-pong
  uint32_t* gval[2];
  uint2* brange;        // [n_buckets] [start, end) of every bucket's list
  // the GPF_NB_BALL_KNN backward (nb_max > 0): selected pairs, per-point
  // counts / offsets, per-Gaussian ranges of the sorted pairs
  uint32_t* nbkey[2];   // [nb_max] Gaussian ids (sort ping-pong)
  uint32_t* nbval[2];   // [nb_max] sorted hit point positions
  uint32_t* nbcnt;      // [M_max + 1] pairs per hit point, then their offsets
  uint32_t* nbknn;      // [M_max * GPF_MAX_KMIN] the forward's kNN ids of each point
                        // that fell back (read by launch_hybrid_pairs(counted))
  uint2* nbrange;       // [N_max] [start, end) of each Gaussian's pairs
  void* nbsort_ws;
  int nbsorted;
  // forward tile splitting (split_items > 0)
  uint32_t* tparts;     // [tiles_max + 1] parts of each tile (1 = not split), then scanned
  uint32_t* xoff;       // [tiles_max + 1] parts of each split tile (0 otherwise), then scanned
  uint4* xunit;         // [GPF_MAX_SPLIT_UNITS] (tile, part, parts, valid) of every split unit
  float* xsum;          // [GPF_MAX_SPLIT_UNITS * (C + 1) * 32] partial sums of split units
  // a centre level (ball_radius > 0): occupancy bits of the centre cells'
  // coarse cells (Grid::cshift), and the hybrid forward's tile splitting
  uint32_t* cocc;       // [cdx * cdy * cdz / 32] set: some mean lies in the cell
  uint32_t* focc;       // [focc_words] the same per centre cell (Grid::fwords > 0)
  uint32_t* hparts;     // [tiles_max + 1] parts of each tile (1 = not split)
  uint32_t* hoff;       // [tiles_max + 1] parts of each split tile (0 otherwise), then scanned
  uint32_t* hitems;     // [tiles_max] listed entries of the centre cells of each tile's box
  uint4* hunit;         // [GPF_MAX_SPLIT_UNITS] (tile, part, parts, valid) of every split unit
  float* hsum;          // [GPF_MAX_SPLIT_UNITS * (C + 2) * 32] partial L, Z and count
  float* dec;           // GPF_BF16 fields: decoded float32 [(10 + C), n] (rows
                        // mean 3, quat 4, logscale 3, spectrum C; N_max room)
  void* scan_ws;
  void* qsort_ws;
  void* gsort_ws;
  void* osort_ws;
  int qsorted, gsorted, osorted;  // which ping-pong buffer holds the result
};

struct IndexDims {
  Grid grid;
  int channels;
  float cutoff;         // k (may be +INF)
  bool brute;           // no cell lists: every Gaussian against every hit point
  int storage;          // storage form of the fields (gpf_field.storage)
  bool bf16;            // a 16-bit form (decoded at build)
  int64_t n_max, m_max, p_max;
  int64_t nb_max;       // capacity of the GPF_NB_BALL_KNN backward's pairs
  int split_items;      // > 0: split forward tiles above this estimated work
};

// GPF_BF16 fields are decoded into b.dec first and the build reads that.
cudaError_t launch_build(const IndexDims& dims, const IndexBuffers& b, const gpf_field& f,
                         const gpf_queries& q, cudaStream_t stream);
// Forward tile splitting (split_items > 0), after the bucket ranges exist:
// each tile's estimated work, its parts, and the table of split units
// (gpf_fwd.cu).
// The unit list of split tiles: xoff (each tile's parts if split, else 0)
// is scanned in place, tile t's units are written at xunit[xoff[t] ...], and
// *n_units (device memory) receives their number; a tile whose units would
// not all fit under GPF_MAX_SPLIT_UNITS gets tparts = 1 and runs unsplit.
cudaError_t launch_split_units(int64_t n_tiles, uint32_t* tparts, uint32_t* xoff, uint4* xunit,
                               uint32_t* n_units, void* scan_ws, cudaStream_t stream);
cudaError_t launch_tile_split(const IndexDims& dims, const IndexBuffers& b, const gpf_queries& q,
                              cudaStream_t stream);
// The float32 field the pair loops read: f itself, or the decoded arrays of
// the last build when f is in GPF_BF16 storage.
gpf_field float32_view(const IndexDims& dims, const IndexBuffers& b, const gpf_field& f);
// gpf_field_quantize (gpf_index.cu).
cudaError_t launch_quantize(const gpf_field& src, const gpf_field& dst, cudaStream_t stream);

// ---- pair loops (gpf_fwd.cu, gpf_bwd.cu)
// Events recorded around a pair-loop kernel (either may be null).
struct KernelEvents {
  cudaEvent_t start = nullptr;
  cudaEvent_t stop = nullptr;
};
// With counts != null nothing is written but the pair counts (see gpf_count_pairs).
cudaError_t launch_forward(const IndexDims& dims, const IndexBuffers& b, const gpf_queries& q,
                           const gpf_query_params& p, int64_t n, float* out, float* z,
                           unsigned long long* counts, const KernelEvents& ev,
                           cudaStream_t stream);
// The GPF_NB_BALL_KNN forward (gpf_hybrid.cu).
// write_counts: also each hit point's number of selected pairs into nbcnt
// (and each split part's ball count), for launch_hybrid_pairs(counted).
cudaError_t launch_hybrid_forward(const IndexDims& dims, const IndexBuffers& b,
                                  const gpf_queries& q, const gpf_query_params& p, int64_t n,
                                  float* out, float* z, bool write_counts,
                                  const KernelEvents& ev, cudaStream_t stream);
// The selected (hit point, Gaussian) pairs of the GPF_NB_BALL_KNN query,
// sorted by Gaussian: b.nbval[b.nbsorted] holds the hit point positions of
// Gaussian g in [b.nbrange[g].x, b.nbrange[g].y) (gpf_hybrid.cu). Sets the
// capacity flag when they exceed dims.nb_max.
// counted: the last forward of this build wrote the counts for the same
// selection (launch_hybrid_forward with write_counts), so they are not
// computed again.
cudaError_t launch_hybrid_pairs(const IndexDims& dims, const IndexBuffers& b,
                                const gpf_queries& q, const gpf_query_params& p, int64_t n,
                                bool counted, cudaStream_t stream);
cudaError_t launch_backward(const IndexDims& dims, const IndexBuffers& b, const gpf_field& f,
                            const gpf_queries& q, const gpf_query_params& p,
                            const float* grad_out, const float* out, const float* z,
                            const gpf_field_grad& g, bool hyb_counted, const KernelEvents& ev,
                            cudaStream_t stream);

// ---- loss and optimiser (gpf_optim.cu)
size_t mse_workspace_bytes(int64_t m);
cudaError_t launch_mse(int64_t m, int channels, const float* out, const float* target,
                       const uint8_t* valid, float* loss, float* grad, void* ws,
                       cudaStream_t stream);
// The same three kernels on caller-placed scratch: psum / pcnt of
// ceil(m / mse_points_per_partial()) partials and one float scale.
int64_t mse_points_per_partial();
cudaError_t launch_mse_parts(int64_t m, int channels, const float* out, const float* target,
                             const uint8_t* valid, float* loss, float* grad, float* psum,
                             uint32_t* pcnt, float* scale, cudaStream_t stream);
// guard: the header of an index whose flags cancel the update (or null).
cudaError_t launch_adam(const gpf_field& params, const gpf_field_grad& g, const gpf_field_grad& m,
                        const gpf_field_grad& v, const gpf_adam_hparams& hp,
                        const DeviceHeader* guard, cudaStream_t stream);
// gpf_index_flags_async: the GPF_FLAG_* word of a header into *flags.
cudaError_t launch_index_flags(const DeviceHeader* header, uint32_t* flags, cudaStream_t stream);

// ---- throughput probes (gpf_probe.cu): which 0 = FP32 FMA (flop/s), 1 =
// ex2.approx (results/s); synchronous, on a stream of its own.
cudaError_t measure_alu_peak(int which, int iters, double* per_second, double* seconds);

// ---- loss without caller scratch (gpf_noalloc.cu)
int64_t noalloc_max_points();
cudaError_t launch_mse_noalloc(int64_t m, int channels, const float* out, const float* target,
                               const uint8_t* valid, float* loss, float* grad,
                               cudaStream_t stream);

}  // namespace gpf
