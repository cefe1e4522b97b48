// The C ABI of libgpf (include/gpf.h): argument validation, workspace
// layout, error reporting, and the launches of the kernel files.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>

#include "gpf_internal.h"

using namespace gpf;

namespace {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};

gpf_status fail(gpf_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
gpf_status fail(gpf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

gpf_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GPF_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

#define GPF_CHECK_PTR_AL(p, al, what)                                                       \
  do {                                                                                      \
    if ((p) == nullptr) return fail(GPF_ERR_INVALID_ARG, "%s is NULL", what);               \
    if (!aligned((p), (al)))                                                                \
      return fail(GPF_ERR_INVALID_ARG, "%s is not %d-byte aligned", what, (int)(al));       \
  } while (0)
#define GPF_CHECK_PTR(p, what) GPF_CHECK_PTR_AL(p, 4, what)

// The four arrays (and the anchors) of a field in its storage.
#define GPF_CHECK_FIELD_ARRAYS(f, name)                                                    \
  do {                                                                                      \
    const int al_ = (f)->storage == GPF_F32 ? 4 : 2;                                        \
    GPF_CHECK_PTR_AL((f)->mean, (f)->storage == GPF_BF16 ? 2 : 4, name ".mean");            \
    GPF_CHECK_PTR_AL((f)->quat, al_, name ".quat");                                         \
    GPF_CHECK_PTR_AL((f)->logscale, al_, name ".logscale");                                 \
    GPF_CHECK_PTR_AL((f)->spectrum, al_, name ".spectrum");                                 \
    if ((f)->storage != GPF_F32) GPF_CHECK_PTR_AL((f)->anchor, 16, name ".anchor");         \
  } while (0)

}  // namespace

void gpf::note_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

struct gpf_index {
  gpf_grid_config cfg;
  IndexDims dims;
  size_t ws_bytes;
  IndexBuffers buf;
  bool built;
  // identity of the last build
  gpf_field field;
  gpf_queries queries;
  // gpf_index_set_timing_events
  KernelEvents fwd_ev, bwd_ev;
  // the last GPF_NB_BALL_KNN forward on this build wrote each hit point's
  // number of selected pairs (and its split parts' ball counts) for these
  // ball_r and k_min: a backward with the same selection need not count
  struct {
    bool valid;
    float ball_r;
    int32_t k_min;
  } hyb_counts;
};

namespace {

// Carves the workspace; with base == nullptr only computes the size.
size_t layout(const gpf_index* ix, char* base, IndexBuffers* b) {
  const IndexDims& d = ix->dims;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align_up(bytes);
    return p;
  };
  IndexBuffers t{};
  const int64_t N = d.n_max, M = d.m_max, P = d.brute ? 0 : d.p_max;
  const size_t ncp = (size_t)d.grid.n_keys + 2;
  const size_t nb = d.brute ? 1 : (size_t)d.grid.n_buckets;
  t.header = reinterpret_cast<DeviceHeader*>(take(sizeof(DeviceHeader)));
  t.rec = reinterpret_cast<float*>(take(sizeof(float) * N * rec_stride(d.channels)));
  t.box = reinterpret_cast<uint4*>(take(sizeof(uint4) * N));
  t.gcount = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * N));
  t.glive = reinterpret_cast<uint8_t*>(take(sizeof(uint8_t) * N));
  t.gmask = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * N));
  t.qbox = reinterpret_cast<uint2*>(take(sizeof(uint2) * N));
  t.goffset = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * N));
  for (int k = 0; k < 2; ++k) {
    t.okey[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * N));
    t.oval[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * N));
  }
  for (int k = 0; k < 2; ++k) {
    t.qkey[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * M));
    t.qval[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * M));
  }
  t.qstart = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * ncp));
  t.qrec = reinterpret_cast<float*>(take(sizeof(float) * M * qrec_stride(d.channels)));
  // room for float64 sums (the gradient-check build of the backward)
  t.gacc = reinterpret_cast<float*>(take(sizeof(double) * N * gacc_stride(d.channels)));
  t.bpart = reinterpret_cast<float*>(take(sizeof(double) * std::min<int64_t>(N, kSplitMax) *
                                          kSplitWays * gacc_stride(d.channels)));
  for (int k = 0; k < 2; ++k) {
    t.gkey[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (P > 0 ? P : 1)));
    t.gval[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (P > 0 ? P : 1)));
  }
  t.occ = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * ((nb + 31) / 32)));
  t.brange = reinterpret_cast<uint2*>(take(sizeof(uint2) * nb));
  t.dec = d.bf16 ? reinterpret_cast<float*>(take(sizeof(float) * (10 + d.channels) * N)) : nullptr;
  if (d.split_items > 0) {
    const int64_t tiles = (M + kWarp - 1) / kWarp;
    t.tparts = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (tiles + 1)));
    t.xoff = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (tiles + 1)));
    t.xunit = reinterpret_cast<uint4*>(take(sizeof(uint4) * GPF_MAX_SPLIT_UNITS));
    t.xsum = reinterpret_cast<float*>(
        take(sizeof(float) * (size_t)GPF_MAX_SPLIT_UNITS * (d.channels + 1) * kWarp));
  }
  if (d.grid.blevel >= 0) {
    const int64_t tiles = (M + kWarp - 1) / kWarp;
    t.cocc = reinterpret_cast<uint32_t*>(
        take(sizeof(uint32_t) * (((size_t)d.grid.cdx * d.grid.cdy * d.grid.cdz + 31) / 32)));
    if (d.grid.fwords)
      t.focc = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * focc_words(d.grid)));
    t.hparts = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (tiles + 1)));
    t.hoff = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (tiles + 1)));
    t.hitems = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (tiles + 1)));
    t.hunit = reinterpret_cast<uint4*>(take(sizeof(uint4) * GPF_MAX_SPLIT_UNITS));
    t.hsum = reinterpret_cast<float*>(
        take(sizeof(float) * (size_t)GPF_MAX_SPLIT_UNITS * (d.channels + 2) * kWarp));
  }
  if (d.nb_max > 0) {
    for (int k = 0; k < 2; ++k) {
      t.nbkey[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * d.nb_max));
      t.nbval[k] = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * d.nb_max));
    }
    t.nbcnt = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * (M + 1)));
    t.nbknn = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * std::max<int64_t>(M, 1) *
                                               GPF_MAX_KMIN));
    t.nbrange = reinterpret_cast<uint2*>(take(sizeof(uint2) * std::max<int64_t>(N, 1)));
    t.nbsort_ws = take(radix_sort_workspace_bytes(d.nb_max));
    t.nbsorted = radix_sort_passes(d.grid.id_bits) % 2;
  }
  t.scan_ws = take(scan_workspace_bytes(
      std::max<int64_t>(std::max<int64_t>(std::max<int64_t>(N, 1), ncp), M + 2)));
  t.qsort_ws = take(radix_sort_workspace_bytes(M > 0 ? M : 1));
  t.gsort_ws = take(radix_sort_workspace_bytes(P > 0 ? P : 1));
  t.osort_ws = take(radix_sort_workspace_bytes(N > 0 ? N : 1));
  t.qsorted = radix_sort_passes(d.grid.key_bits) % 2;
  t.osorted = radix_sort_passes(d.grid.obits) % 2;
  t.gsorted = radix_sort_passes(d.grid.hash_bits) % 2;
  if (b) *b = t;
  return off;
}

gpf_status check_field(const gpf_index* ix, const gpf_field* f) {
  if (!f) return fail(GPF_ERR_INVALID_ARG, "field is NULL");
  if (f->n < 0) return fail(GPF_ERR_INVALID_ARG, "field.n = %lld < 0", (long long)f->n);
  if (f->n > ix->dims.n_max)
    return fail(GPF_ERR_INVALID_ARG, "field.n = %lld exceeds max_gaussians = %lld",
                (long long)f->n, (long long)ix->dims.n_max);
  if (f->n >= (int64_t)kIdMask) return fail(GPF_ERR_INVALID_ARG, "field.n too large");
  if (f->channels != ix->dims.channels)
    return fail(GPF_ERR_INVALID_ARG, "field.channels = %d but the index holds %d channels",
                f->channels, ix->dims.channels);
  if (f->storage != GPF_F32 && f->storage != GPF_BF16 && f->storage != GPF_BF16_MEAN32)
    return fail(GPF_ERR_INVALID_ARG, "field.storage = %d is not a storage form", f->storage);
  if (f->storage != ix->dims.storage)
    return fail(GPF_ERR_INVALID_ARG, "field.storage = %d but the index was created for %d",
                f->storage, ix->dims.storage);
  if (f->n > 0) GPF_CHECK_FIELD_ARRAYS(f, "field");
  return GPF_OK;
}

gpf_status check_queries(const gpf_index* ix, const gpf_queries* q) {
  if (!q) return fail(GPF_ERR_INVALID_ARG, "queries is NULL");
  if (q->m < 0) return fail(GPF_ERR_INVALID_ARG, "queries.m = %lld < 0", (long long)q->m);
  if (q->m > ix->dims.m_max)
    return fail(GPF_ERR_INVALID_ARG, "queries.m = %lld exceeds max_queries = %lld",
                (long long)q->m, (long long)ix->dims.m_max);
  if (q->m > 0) {
    GPF_CHECK_PTR(q->x, "queries.x");
    GPF_CHECK_PTR(q->normal, "queries.normal");
    GPF_CHECK_PTR(q->wo, "queries.wo");
    if (q->albedo && !aligned(q->albedo, 4))
      return fail(GPF_ERR_INVALID_ARG, "queries.albedo is not 4-byte aligned");
  }
  return GPF_OK;
}

gpf_status check_params(const gpf_query_params* p) {
  if (!p) return fail(GPF_ERR_INVALID_ARG, "params is NULL");
  if (p->mode != GPF_SUM && p->mode != GPF_NORMALIZED && p->mode != GPF_DISK_KDE)
    return fail(GPF_ERR_INVALID_ARG, "params.mode = %d is not a gpf_mode", p->mode);
  if (p->mode == GPF_DISK_KDE && !(p->r_max > 0.0f && isfinite(p->r_max)))
    return fail(GPF_ERR_INVALID_ARG, "GPF_DISK_KDE needs a finite gather radius r_max > 0");
  if (isnan(p->r_max) || p->r_max < 0.0f)
    return fail(GPF_ERR_INVALID_ARG, "params.r_max must be >= 0 or +INF");
  if (!(p->eps > 0.0f) || !isfinite(p->eps))
    return fail(GPF_ERR_INVALID_ARG, "params.eps must be finite and > 0");
  if (p->neighbourhood != GPF_NB_KSIGMA && p->neighbourhood != GPF_NB_BALL_KNN)
    return fail(GPF_ERR_INVALID_ARG, "params.neighbourhood = %d is unknown", p->neighbourhood);
  if (p->neighbourhood == GPF_NB_BALL_KNN) {
    if (p->mode == GPF_DISK_KDE)
      return fail(GPF_ERR_INVALID_ARG, "GPF_DISK_KDE gathers a disk, not GPF_NB_BALL_KNN");
    if (!(p->ball_r >= 0.0f) || !isfinite(p->ball_r))
      return fail(GPF_ERR_INVALID_ARG, "params.ball_r must be finite and >= 0");
    if (p->k_min < 0 || p->k_min > GPF_MAX_KMIN)
      return fail(GPF_ERR_INVALID_ARG, "params.k_min = %d outside 0..%d", p->k_min, GPF_MAX_KMIN);
  }
  if (p->f64_sums != 0 && p->f64_sums != 1)
    return fail(GPF_ERR_INVALID_ARG, "params.f64_sums must be 0 or 1");
  return GPF_OK;
}

gpf_status check_same(const gpf_index* ix, const gpf_field* f, const gpf_queries* q) {
  if (!ix->built) return fail(GPF_ERR_NOT_BUILT, "gpf_build_index has not run on this index");
  const gpf_field& a = ix->field;
  const gpf_queries& b = ix->queries;
  if (a.n != f->n || a.mean != f->mean || a.quat != f->quat || a.logscale != f->logscale ||
      a.spectrum != f->spectrum)
    return fail(GPF_ERR_MISMATCH, "field differs from the one given to gpf_build_index");
  if (b.m != q->m || b.x != q->x || b.normal != q->normal || b.wo != q->wo ||
      b.valid != q->valid)
    return fail(GPF_ERR_MISMATCH, "queries differ from the ones given to gpf_build_index");
  return GPF_OK;
}

}  // namespace

namespace gpf {
int64_t persistent_blocks(const void* kernel, int threads, int64_t max_blocks) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
      sms <= 0 || per_sm <= 0) {
    cudaGetLastError();  // clear; fall back to one block per work unit
    return max_blocks > 0 ? max_blocks : 1;
  }
  const int64_t resident = (int64_t)sms * per_sm;
  return std::max<int64_t>(1, std::min<int64_t>(resident, max_blocks));
}
}  // namespace gpf

extern "C" {

const char* gpf_version(void) { return "gpf 0.1 (sm_103a)"; }

const char* gpf_status_string(gpf_status s) {
  switch (s) {
    case GPF_OK: return "GPF_OK";
    case GPF_ERR_INVALID_ARG: return "GPF_ERR_INVALID_ARG";
    case GPF_ERR_CUDA: return "GPF_ERR_CUDA";
    case GPF_ERR_WORKSPACE_TOO_SMALL: return "GPF_ERR_WORKSPACE_TOO_SMALL";
    case GPF_ERR_CAPACITY: return "GPF_ERR_CAPACITY";
    case GPF_ERR_NOT_BUILT: return "GPF_ERR_NOT_BUILT";
    case GPF_ERR_MISMATCH: return "GPF_ERR_MISMATCH";
    case GPF_ERR_TIMEOUT: return "GPF_ERR_TIMEOUT";
    case GPF_ERR_NONFINITE: return "GPF_ERR_NONFINITE";
  }
  return "GPF_ERR_UNKNOWN";
}

const char* gpf_last_error(void) { return g_last_error.c_str(); }

gpf_status gpf_index_create(const gpf_grid_config* cfg, gpf_index** out) {
  if (!cfg || !out) return fail(GPF_ERR_INVALID_ARG, "cfg or out is NULL");
  *out = nullptr;
  if (!(cfg->cell_size > 0.0f) || !isfinite(cfg->cell_size))
    return fail(GPF_ERR_INVALID_ARG, "cell_size must be finite and > 0");
  if (cfg->levels < 1 || cfg->levels > GPF_MAX_LEVELS)
    return fail(GPF_ERR_INVALID_ARG, "levels = %d outside 1..%d", cfg->levels, GPF_MAX_LEVELS);
  if (cfg->max_span < 1 || cfg->max_span > 64)
    return fail(GPF_ERR_INVALID_ARG, "max_span = %d outside 1..64", cfg->max_span);
  if (cfg->query_level < 0 || cfg->query_level > 15)
    return fail(GPF_ERR_INVALID_ARG, "query_level = %d outside 0..15", cfg->query_level);
  if (cfg->hash_bits < 8 || cfg->hash_bits > 28)
    return fail(GPF_ERR_INVALID_ARG, "hash_bits = %d outside 8..28", cfg->hash_bits);
  for (int k = 0; k < 3; ++k) {
    if (!isfinite(cfg->origin[k])) return fail(GPF_ERR_INVALID_ARG, "origin must be finite");
    if (cfg->dims[k] < 1 || cfg->dims[k] > GPF_MAX_DIM)
      return fail(GPF_ERR_INVALID_ARG, "dims[%d] = %d outside 1..%d", k, cfg->dims[k],
                  GPF_MAX_DIM);
    if (((int64_t)cfg->dims[k] << cfg->query_level) > (int64_t(1) << kCoordBits))
      return fail(GPF_ERR_INVALID_ARG, "dims[%d] * 2^query_level exceeds 2^%d finest cells", k,
                  kCoordBits);
  }
  if (cfg->channels < 1 || cfg->channels > GPF_MAX_CHANNELS)
    return fail(GPF_ERR_INVALID_ARG, "channels = %d outside 1..%d", cfg->channels,
                GPF_MAX_CHANNELS);
  if (!(cfg->cutoff_sigma > 0.0f))
    return fail(GPF_ERR_INVALID_ARG, "cutoff_sigma must be > 0 (or +INF)");
  if (cfg->brute_force != 0 && cfg->brute_force != 1)
    return fail(GPF_ERR_INVALID_ARG, "brute_force must be 0 or 1");
  if (cfg->field_storage != GPF_F32 && cfg->field_storage != GPF_BF16 &&
      cfg->field_storage != GPF_BF16_MEAN32)
    return fail(GPF_ERR_INVALID_ARG, "field_storage = %d is not a storage form",
                cfg->field_storage);
  if (!(cfg->ball_radius >= 0.0f) || !isfinite(cfg->ball_radius))
    return fail(GPF_ERR_INVALID_ARG, "ball_radius must be finite and >= 0");
  if (cfg->ball_radius > 0.0f && (double)cfg->ball_radius > (double)cfg->cell_size * (1u << 19))
    return fail(GPF_ERR_INVALID_ARG, "ball_radius exceeds 2^19 finest cells");
  if (cfg->coop_cells < 0 || cfg->coop_cells > GPF_MAX_COOP_CELLS)
    return fail(GPF_ERR_INVALID_ARG, "coop_cells = %d outside 0..%d", cfg->coop_cells,
                GPF_MAX_COOP_CELLS);
  if (cfg->max_gaussians < 0 || cfg->max_queries < 0 || cfg->max_pairs < 0 ||
      cfg->max_nb_pairs < 0)
    return fail(GPF_ERR_INVALID_ARG, "capacities must be >= 0");
  if (cfg->max_gaussians >= kMaxSortN || cfg->max_queries >= kMaxSortN ||
      cfg->max_pairs >= kMaxSortN || cfg->max_nb_pairs >= kMaxSortN)
    return fail(GPF_ERR_INVALID_ARG, "capacities must be below 2^30");
  if (cfg->split_items < 0)
    return fail(GPF_ERR_INVALID_ARG, "split_items must be >= 0");
  if (cfg->tile_order < 0 || cfg->tile_order > 2 || cfg->tile_order > cfg->query_level)
    return fail(GPF_ERR_INVALID_ARG, "tile_order = %d outside 0..min(2, query_level = %d)",
                cfg->tile_order, cfg->query_level);
  if (cfg->max_nb_pairs > 0 && !(cfg->ball_radius > 0.0f))
    return fail(GPF_ERR_INVALID_ARG, "max_nb_pairs > 0 needs ball_radius > 0 (centre entries)");
  const uint64_t cells = (uint64_t)cfg->dims[0] * cfg->dims[1] * cfg->dims[2];
  if (cells > (1ull << 28))
    return fail(GPF_ERR_INVALID_ARG, "grid has %llu cells, more than 2^28",
                (unsigned long long)cells);
  if ((cells << (3 * cfg->tile_order)) >= (1ull << 32))
    return fail(GPF_ERR_INVALID_ARG, "tile_order = %d: %llu cells leave no room for %d sub-cell "
                "bits in a 32-bit sort key", cfg->tile_order, (unsigned long long)cells,
                3 * cfg->tile_order);
  gpf_index* ix = new (std::nothrow) gpf_index();
  if (!ix) return fail(GPF_ERR_INVALID_ARG, "out of host memory");
  ix->cfg = *cfg;
  IndexDims& d = ix->dims;
  d.grid.ox = cfg->origin[0];
  d.grid.oy = cfg->origin[1];
  d.grid.oz = cfg->origin[2];
  d.grid.cell0 = cfg->cell_size;
  d.grid.inv_cell0 = 1.0f / cfg->cell_size;
  d.grid.levels = cfg->levels;
  d.grid.max_span = cfg->max_span;
  d.grid.coop = cfg->coop_cells ? cfg->coop_cells : 4;
  d.grid.blevel = -1;
  if (cfg->ball_radius > 0.0f) {
    int L = 0;
    while ((double)cfg->cell_size * (double)(1u << L) < (double)cfg->ball_radius && L < 19) ++L;
    d.grid.blevel = L;
  }
  d.grid.qlevel = cfg->query_level;
  d.grid.hash_bits = cfg->hash_bits;
  d.grid.n_buckets = 1u << cfg->hash_bits;
  d.grid.max0x = ((uint32_t)cfg->dims[0] << cfg->query_level) - 1;
  d.grid.max0y = ((uint32_t)cfg->dims[1] << cfg->query_level) - 1;
  d.grid.max0z = ((uint32_t)cfg->dims[2] << cfg->query_level) - 1;
  {
    int ib = 1;
    while (ib < 31 && (int64_t(1) << ib) < cfg->max_gaussians) ++ib;
    d.grid.id_bits = ib;
    d.grid.id_mask = (uint32_t)((uint64_t(1) << ib) - 1);
  }
  if (d.grid.blevel >= 0) {
    // centre occupancy: cells of at least 4 x 4 x 4 centre cells, at most 2^20 bits
    int sh = d.grid.blevel + 2;
    auto n_cells = [&](int k) {
      return (uint64_t)((d.grid.max0x >> k) + 1) * ((d.grid.max0y >> k) + 1) *
             ((d.grid.max0z >> k) + 1);
    };
    while (sh < kCoordBits && n_cells(sh) > (1u << 20)) ++sh;
    d.grid.cshift = sh;
    d.grid.cdx = (d.grid.max0x >> sh) + 1;
    d.grid.cdy = (d.grid.max0y >> sh) + 1;
    d.grid.cdz = (d.grid.max0z >> sh) + 1;
    // fine centre occupancy: one bit per centre cell, rows along x in whole
    // words, when it takes at most 2^24 words (64 MB)
    const int L = d.grid.blevel;
    const uint64_t fw = ((uint64_t)(d.grid.max0x >> L) + 32) / 32;
    const uint64_t fr = (uint64_t)((d.grid.max0y >> L) + 1) * ((d.grid.max0z >> L) + 1);
    d.grid.fwords = fw * fr <= (1u << 24) ? (uint32_t)fw : 0u;
    d.grid.fdy = (d.grid.max0y >> L) + 1;
  }
  d.grid.dx = cfg->dims[0];
  d.grid.dy = cfg->dims[1];
  d.grid.dz = cfg->dims[2];
  d.grid.n_keys = (uint32_t)cells;
  // sort keys of the hit points: the query-level cell key, then 3 b bits of
  // the sub-cell Morton code (b = tile_order); inactive hit points sort last
  d.grid.qsub = cfg->tile_order;
  const int sub_bits = 3 * cfg->tile_order;
  int bits = 0;
  while ((1ull << bits) <= (cells << sub_bits)) ++bits;
  d.grid.key_inactive = (uint32_t)(cells << sub_bits);
  d.grid.key_bits = bits;
  // the backward walks Gaussians ordered by a cell 16 x coarser than the query level
  d.grid.oshift = std::min(cfg->query_level + 4, kCoordBits);
  d.grid.odx = (d.grid.max0x >> d.grid.oshift) + 1;
  d.grid.ody = (d.grid.max0y >> d.grid.oshift) + 1;
  {
    const uint64_t ocells = (uint64_t)d.grid.odx * d.grid.ody * ((d.grid.max0z >> d.grid.oshift) + 1);
    int ob = 1;
    while ((1ull << ob) < ocells) ++ob;
    d.grid.obits = ob + kOrderSizeBits + 2;
  }
  d.channels = cfg->channels;
  d.cutoff = cfg->cutoff_sigma;
  d.brute = isinf(cfg->cutoff_sigma) || cfg->brute_force == 1;
  d.storage = cfg->field_storage;
  d.bf16 = cfg->field_storage != GPF_F32;
  d.n_max = cfg->max_gaussians;
  d.m_max = cfg->max_queries;
  d.p_max = d.brute ? 0 : cfg->max_pairs;
  d.nb_max = cfg->max_nb_pairs;
  d.split_items = cfg->split_items;
  ix->ws_bytes = layout(ix, nullptr, nullptr);
  ix->built = false;
  *out = ix;
  return GPF_OK;
}

void gpf_index_destroy(gpf_index* index) { delete index; }

gpf_status gpf_index_workspace_size(const gpf_index* index, size_t* bytes) {
  if (!index || !bytes) return fail(GPF_ERR_INVALID_ARG, "index or bytes is NULL");
  *bytes = index->ws_bytes;
  return GPF_OK;
}

gpf_status gpf_build_index(gpf_index* index, const gpf_field* field, const gpf_queries* queries,
                           void* workspace, size_t workspace_bytes, gpf_stream stream) {
  if (!index) return fail(GPF_ERR_INVALID_ARG, "index is NULL");
  gpf_status s;
  if ((s = check_field(index, field)) != GPF_OK) return s;
  if ((s = check_queries(index, queries)) != GPF_OK) return s;
  if (!workspace) return fail(GPF_ERR_INVALID_ARG, "workspace is NULL");
  if (!aligned(workspace, 256)) return fail(GPF_ERR_INVALID_ARG, "workspace is not 256-byte aligned");
  if (workspace_bytes < index->ws_bytes)
    return fail(GPF_ERR_WORKSPACE_TOO_SMALL, "workspace has %zu bytes, needs %zu", workspace_bytes,
                index->ws_bytes);
  layout(index, static_cast<char*>(workspace), &index->buf);
  index->built = false;
  index->hyb_counts.valid = false;
  cudaError_t e = launch_build(index->dims, index->buf, *field, *queries,
                               reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_build_index");
  index->field = *field;
  index->queries = *queries;
  index->built = true;
  return GPF_OK;
}

gpf_status gpf_index_stats(const gpf_index* index, gpf_index_stats_t* stats, gpf_stream stream) {
  if (!index || !stats) return fail(GPF_ERR_INVALID_ARG, "index or stats is NULL");
  if (!index->built) return fail(GPF_ERR_NOT_BUILT, "gpf_build_index has not run on this index");
  DeviceHeader h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&h, index->buf.header, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "gpf_index_stats");
  memset(stats, 0, sizeof(*stats));
  stats->n_pairs = h.n_pairs;
  stats->n_active = h.n_active;
  stats->n_live = h.n_live;
  stats->n_small = h.n_small;
  stats->n_huge = h.n_huge;
  stats->n_split = std::min<int64_t>(h.n_huge, kSplitMax);
  stats->level_mask = h.level_mask;
  stats->flags = (h.overflow ? GPF_FLAG_CAPACITY : 0u) | (h.stalled ? GPF_FLAG_TIMEOUT : 0u) |
                 (h.nonfinite ? GPF_FLAG_NONFINITE : 0u);
  stats->overflow = (int32_t)h.overflow;
  stats->n_hybrid_units = (int32_t)h.n_hunits;
  stats->n_nb_pairs = h.nb_pairs;
  if (h.stalled)
    return fail(GPF_ERR_TIMEOUT, "a bounded wait of the index build's sort gave up");
  if (h.nonfinite)
    return fail(GPF_ERR_NONFINITE,
                "a Gaussian parameter or an active hit point of the last build is not finite");
  if (h.overflow)
    return fail(GPF_ERR_CAPACITY, "pair buffer overflow: %u entries needed, capacity %lld",
                h.n_pairs, (long long)index->dims.p_max);
  return GPF_OK;
}

gpf_status gpf_index_flags_async(const gpf_index* index, uint32_t* flags, gpf_stream stream) {
  if (!index) return fail(GPF_ERR_INVALID_ARG, "index is NULL");
  GPF_CHECK_PTR(flags, "flags");
  if (!index->built) return fail(GPF_ERR_NOT_BUILT, "gpf_build_index has not run on this index");
  const cudaError_t e = launch_index_flags(index->buf.header, flags,
                                           reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_index_flags_async");
  return GPF_OK;
}

gpf_status gpf_radiance_fwd(const gpf_index* index, const gpf_field* field,
                            const gpf_queries* queries, const gpf_query_params* params,
                            float* out, float* z_out, gpf_stream stream) {
  if (!index) return fail(GPF_ERR_INVALID_ARG, "index is NULL");
  gpf_status s;
  if ((s = check_field(index, field)) != GPF_OK) return s;
  if ((s = check_queries(index, queries)) != GPF_OK) return s;
  if ((s = check_params(params)) != GPF_OK) return s;
  if (params->f64_sums != 0)
    return fail(GPF_ERR_INVALID_ARG, "params.f64_sums applies to gpf_radiance_bwd only");
  if ((s = check_same(index, field, queries)) != GPF_OK) return s;
  if (params->neighbourhood == GPF_NB_BALL_KNN) {
    if (index->dims.grid.blevel < 0)
      return fail(GPF_ERR_INVALID_ARG, "the index has no centre entries (ball_radius = 0)");
    if (params->ball_r > index->cfg.ball_radius)
      return fail(GPF_ERR_INVALID_ARG, "params.ball_r = %g exceeds the index's ball_radius %g",
                  params->ball_r, index->cfg.ball_radius);
  }
  if (queries->m > 0) {
    GPF_CHECK_PTR(out, "out");
    if (z_out && !aligned(z_out, 4)) return fail(GPF_ERR_INVALID_ARG, "z_out is not aligned");
  }
  const bool hyb = params->neighbourhood == GPF_NB_BALL_KNN;
  const bool counts = hyb && index->dims.nb_max > 0;
  cudaError_t e =
      hyb ? launch_hybrid_forward(index->dims, index->buf, *queries, *params, field->n, out, z_out,
                                  counts, index->fwd_ev, reinterpret_cast<cudaStream_t>(stream))
          : launch_forward(index->dims, index->buf, *queries, *params, field->n, out, z_out,
                           nullptr, index->fwd_ev, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_radiance_fwd");
  if (hyb) {
    auto& hc = const_cast<gpf_index*>(index)->hyb_counts;
    hc.valid = counts;
    hc.ball_r = params->ball_r;
    hc.k_min = params->k_min;
  }
  return GPF_OK;
}

gpf_status gpf_count_pairs(const gpf_index* index, const gpf_field* field,
                           const gpf_queries* queries, uint64_t* counts, gpf_stream stream) {
  if (!index) return fail(GPF_ERR_INVALID_ARG, "index is NULL");
  gpf_status s;
  if ((s = check_field(index, field)) != GPF_OK) return s;
  if ((s = check_queries(index, queries)) != GPF_OK) return s;
  if ((s = check_same(index, field, queries)) != GPF_OK) return s;
  if (!counts || !aligned(counts, 8))
    return fail(GPF_ERR_INVALID_ARG, "counts is NULL or not 8-byte aligned");
  gpf_query_params p{GPF_SUM, INFINITY, 1e-6f, 0, 0.0f, 0, 0};
  cudaError_t e = launch_forward(index->dims, index->buf, *queries, p, field->n, nullptr, nullptr,
                                 reinterpret_cast<unsigned long long*>(counts), KernelEvents{},
                                 reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_count_pairs");
  return GPF_OK;
}

gpf_status gpf_index_set_timing_events(gpf_index* index, void* fwd_start, void* fwd_stop,
                                       void* bwd_start, void* bwd_stop) {
  if (!index) return fail(GPF_ERR_INVALID_ARG, "index is NULL");
  index->fwd_ev.start = static_cast<cudaEvent_t>(fwd_start);
  index->fwd_ev.stop = static_cast<cudaEvent_t>(fwd_stop);
  index->bwd_ev.start = static_cast<cudaEvent_t>(bwd_start);
  index->bwd_ev.stop = static_cast<cudaEvent_t>(bwd_stop);
  return GPF_OK;
}

uint64_t gpf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

gpf_status gpf_radiance_bwd(const gpf_index* index, const gpf_field* field,
                            const gpf_queries* queries, const gpf_query_params* params,
                            const float* grad_out, const float* out, const float* z,
                            const gpf_field_grad* grads, gpf_stream stream) {
  if (!index) return fail(GPF_ERR_INVALID_ARG, "index is NULL");
  gpf_status s;
  if ((s = check_field(index, field)) != GPF_OK) return s;
  if ((s = check_queries(index, queries)) != GPF_OK) return s;
  if ((s = check_params(params)) != GPF_OK) return s;
  if ((s = check_same(index, field, queries)) != GPF_OK) return s;
  if (params->mode == GPF_DISK_KDE)
    return fail(GPF_ERR_INVALID_ARG, "GPF_DISK_KDE (the photon density estimate) has no gradient");
  if (params->neighbourhood == GPF_NB_BALL_KNN) {
    if (index->dims.grid.blevel < 0)
      return fail(GPF_ERR_INVALID_ARG, "the index has no centre entries (ball_radius = 0)");
    if (params->ball_r > index->cfg.ball_radius)
      return fail(GPF_ERR_INVALID_ARG, "params.ball_r = %g exceeds the index's ball_radius %g",
                  params->ball_r, index->cfg.ball_radius);
    if (index->dims.nb_max <= 0)
      return fail(GPF_ERR_INVALID_ARG,
                  "the GPF_NB_BALL_KNN backward needs an index with max_nb_pairs > 0");
  }
  if (!grads) return fail(GPF_ERR_INVALID_ARG, "grads is NULL");
  if (grads->reserved != 0) return fail(GPF_ERR_INVALID_ARG, "grads.reserved must be 0");
  if (field->n > 0) {
    GPF_CHECK_PTR(grads->mean, "grads.mean");
    GPF_CHECK_PTR(grads->quat, "grads.quat");
    GPF_CHECK_PTR(grads->logscale, "grads.logscale");
    GPF_CHECK_PTR(grads->spectrum, "grads.spectrum");
  }
  if (queries->m > 0) {
    GPF_CHECK_PTR(grad_out, "grad_out");
    if (params->mode == GPF_NORMALIZED) {
      GPF_CHECK_PTR(out, "out");
      GPF_CHECK_PTR(z, "z");
    }
  }
  auto& hc = const_cast<gpf_index*>(index)->hyb_counts;
  const bool counted = params->neighbourhood == GPF_NB_BALL_KNN && hc.valid &&
                       hc.ball_r == params->ball_r && hc.k_min == params->k_min;
  cudaError_t e = launch_backward(index->dims, index->buf,
                                  float32_view(index->dims, index->buf, *field), *queries, *params,
                                  grad_out, out, z, *grads, counted, index->bwd_ev,
                                  reinterpret_cast<cudaStream_t>(stream));
  // the pair offsets have replaced the counts
  if (params->neighbourhood == GPF_NB_BALL_KNN) hc.valid = false;
  if (e != cudaSuccess) return cuda_fail(e, "gpf_radiance_bwd");
  return GPF_OK;
}

gpf_status gpf_mse_workspace_size(int64_t m, size_t* bytes) {
  if (m < 0 || !bytes) return fail(GPF_ERR_INVALID_ARG, "m < 0 or bytes is NULL");
  *bytes = mse_workspace_bytes(m);
  return GPF_OK;
}

gpf_status gpf_mse_loss_grad(int64_t m, int32_t channels, const float* out, const float* target,
                             const uint8_t* valid, float* loss, float* grad, void* workspace,
                             size_t workspace_bytes, gpf_stream stream) {
  if (m < 0) return fail(GPF_ERR_INVALID_ARG, "m < 0");
  if (channels < 1 || channels > GPF_MAX_CHANNELS)
    return fail(GPF_ERR_INVALID_ARG, "channels = %d outside 1..%d", channels, GPF_MAX_CHANNELS);
  GPF_CHECK_PTR(loss, "loss");
  if (m > 0) {
    GPF_CHECK_PTR(out, "out");
    GPF_CHECK_PTR(target, "target");
    GPF_CHECK_PTR(grad, "grad");
  }
  if (!workspace) return fail(GPF_ERR_INVALID_ARG, "workspace is NULL");
  if (!aligned(workspace, 256)) return fail(GPF_ERR_INVALID_ARG, "workspace is not 256-byte aligned");
  if (workspace_bytes < mse_workspace_bytes(m))
    return fail(GPF_ERR_WORKSPACE_TOO_SMALL, "workspace has %zu bytes, needs %zu", workspace_bytes,
                mse_workspace_bytes(m));
  cudaError_t e = launch_mse(m, channels, out, target, valid, loss, grad, workspace,
                             reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_mse_loss_grad");
  return GPF_OK;
}

gpf_status gpf_mse_loss_grad_noalloc(int64_t m, int32_t channels, const float* out,
                                     const float* target, const uint8_t* valid, float* loss,
                                     float* grad, gpf_stream stream) {
  if (m < 0) return fail(GPF_ERR_INVALID_ARG, "m < 0");
  if (m > noalloc_max_points())
    return fail(GPF_ERR_INVALID_ARG,
                "m = %lld exceeds GPF_NOALLOC_MAX_POINTS = %lld; use gpf_mse_loss_grad",
                (long long)m, (long long)noalloc_max_points());
  if (channels < 1 || channels > GPF_MAX_CHANNELS)
    return fail(GPF_ERR_INVALID_ARG, "channels = %d outside 1..%d", channels, GPF_MAX_CHANNELS);
  GPF_CHECK_PTR(loss, "loss");
  if (m > 0) {
    GPF_CHECK_PTR(out, "out");
    GPF_CHECK_PTR(target, "target");
    GPF_CHECK_PTR(grad, "grad");
  }
  cudaError_t e = launch_mse_noalloc(m, channels, out, target, valid, loss, grad,
                                     reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_mse_loss_grad_noalloc");
  return GPF_OK;
}

gpf_status gpf_adam_step(const gpf_field* params, const gpf_field_grad* grads,
                         const gpf_field_grad* m, const gpf_field_grad* v,
                         const gpf_adam_hparams* hp, gpf_stream stream) {
  if (!params || !grads || !m || !v || !hp)
    return fail(GPF_ERR_INVALID_ARG, "a pointer argument is NULL");
  if (params->n < 0) return fail(GPF_ERR_INVALID_ARG, "params.n < 0");
  if (params->storage != GPF_F32)
    return fail(GPF_ERR_INVALID_ARG, "Adam updates a GPF_F32 (master) field");
  if (params->channels < 1 || params->channels > GPF_MAX_CHANNELS)
    return fail(GPF_ERR_INVALID_ARG, "params.channels outside 1..%d", GPF_MAX_CHANNELS);
  if (hp->step_counter) {
    if (hp->step != 0) return fail(GPF_ERR_INVALID_ARG, "hp.step must be 0 with a step_counter");
    if (!aligned(hp->step_counter, 8))
      return fail(GPF_ERR_INVALID_ARG, "hp.step_counter is not 8-byte aligned");
  } else if (hp->step < 1) {
    return fail(GPF_ERR_INVALID_ARG, "hp.step = %d < 1", hp->step);
  }
  if (!(hp->beta1 >= 0.0f && hp->beta1 < 1.0f) || !(hp->beta2 >= 0.0f && hp->beta2 < 1.0f))
    return fail(GPF_ERR_INVALID_ARG, "betas must lie in [0, 1)");
  if (!(hp->eps >= 0.0f)) return fail(GPF_ERR_INVALID_ARG, "eps must be >= 0");
  const DeviceHeader* guard = nullptr;
  if (hp->guard) {
    if (!hp->guard->built)
      return fail(GPF_ERR_NOT_BUILT, "hp.guard: gpf_build_index has not run on that index");
    guard = hp->guard->buf.header;
  }
  for (int k = 0; k < 4; ++k)
    if (!isfinite(hp->lr[k]) || hp->lr[k] < 0.0f)
      return fail(GPF_ERR_INVALID_ARG, "lr[%d] must be finite and >= 0", k);
  if (params->n > 0) {
    const gpf_field_grad* gs[3] = {grads, m, v};
    const char* names[3] = {"grads", "m", "v"};
    GPF_CHECK_PTR(params->mean, "params.mean");
    GPF_CHECK_PTR(params->quat, "params.quat");
    GPF_CHECK_PTR(params->logscale, "params.logscale");
    GPF_CHECK_PTR(params->spectrum, "params.spectrum");
    for (int k = 0; k < 3; ++k) {
      if (!gs[k]->mean || !gs[k]->quat || !gs[k]->logscale || !gs[k]->spectrum)
        return fail(GPF_ERR_INVALID_ARG, "%s has a NULL array", names[k]);
    }
  }
  cudaError_t e =
      launch_adam(*params, *grads, *m, *v, *hp, guard, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_adam_step");
  return GPF_OK;
}

gpf_status gpf_field_quantize(const gpf_field* src, const gpf_field* dst, gpf_stream stream) {
  if (!src || !dst) return fail(GPF_ERR_INVALID_ARG, "src or dst is NULL");
  if (src->storage != GPF_F32) return fail(GPF_ERR_INVALID_ARG, "src must be GPF_F32");
  if (dst->storage != GPF_BF16 && dst->storage != GPF_BF16_MEAN32)
    return fail(GPF_ERR_INVALID_ARG, "dst must be GPF_BF16 or GPF_BF16_MEAN32");
  if (src->n < 0 || src->n != dst->n || src->channels != dst->channels)
    return fail(GPF_ERR_INVALID_ARG, "src and dst differ in n or channels");
  if (src->channels < 1 || src->channels > GPF_MAX_CHANNELS)
    return fail(GPF_ERR_INVALID_ARG, "channels outside 1..%d", GPF_MAX_CHANNELS);
  if (src->n > 0) {
    GPF_CHECK_FIELD_ARRAYS(src, "src");
    GPF_CHECK_FIELD_ARRAYS(dst, "dst");
  }
  const cudaError_t e = launch_quantize(*src, *dst, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "gpf_field_quantize");
  return GPF_OK;
}

gpf_status gpf_sort_pairs_workspace_size(int64_t n, size_t* bytes) {
  if (!bytes) return fail(GPF_ERR_INVALID_ARG, "bytes is NULL");
  if (n < 0 || n >= kMaxSortN)
    return fail(GPF_ERR_INVALID_ARG, "n = %lld outside [0, 2^30)", (long long)n);
  *bytes = 256 + radix_sort_workspace_bytes(n > 0 ? n : 1);
  return GPF_OK;
}

gpf_status gpf_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                          int64_t n, int32_t bits, void* workspace, size_t workspace_bytes,
                          int32_t* result_in_alt, gpf_stream stream) {
  if (!result_in_alt) return fail(GPF_ERR_INVALID_ARG, "result_in_alt is NULL");
  size_t need = 0;
  gpf_status s = gpf_sort_pairs_workspace_size(n, &need);
  if (s != GPF_OK) return s;
  if (bits < 0 || bits > 32) return fail(GPF_ERR_INVALID_ARG, "bits = %d outside 0..32", bits);
  GPF_CHECK_PTR_AL(workspace, 256, "workspace");
  if (workspace_bytes < need)
    return fail(GPF_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, %zu needed",
                workspace_bytes, need);
  if (n > 0) {
    GPF_CHECK_PTR(keys, "keys");
    GPF_CHECK_PTR(vals, "vals");
    GPF_CHECK_PTR(keys_alt, "keys_alt");
    GPF_CHECK_PTR(vals_alt, "vals_alt");
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* stalled = static_cast<uint32_t*>(workspace);
  cudaError_t e = cudaMemsetAsync(stalled, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess && n > 0)
    e = radix_sort_pairs(keys, vals, keys_alt, vals_alt, n, nullptr, bits,
                         static_cast<char*>(workspace) + 256, stalled, st);
  if (e != cudaSuccess) return cuda_fail(e, "gpf_sort_pairs");
  *result_in_alt = n > 0 ? radix_sort_passes(bits) % 2 : 0;
  return GPF_OK;
}

gpf_status gpf_sort_pairs_check(const void* workspace, gpf_stream stream) {
  GPF_CHECK_PTR_AL(workspace, 256, "workspace");
  uint32_t flag = 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&flag, workspace, sizeof(flag), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "gpf_sort_pairs_check");
  if (flag) return fail(GPF_ERR_TIMEOUT, "a bounded wait of the sort gave up");
  return GPF_OK;
}

gpf_status gpf_measure_alu_peak(int32_t which, int32_t iters, double* per_second,
                                double* seconds) {
  if (which != GPF_PEAK_FP32_FMA && which != GPF_PEAK_EX2)
    return fail(GPF_ERR_INVALID_ARG, "which = %d is not GPF_PEAK_FP32_FMA or GPF_PEAK_EX2", which);
  if (iters < 1 || iters > (1 << 20))
    return fail(GPF_ERR_INVALID_ARG, "iters = %d outside 1 .. 2^20", iters);
  if (!per_second || !seconds) return fail(GPF_ERR_INVALID_ARG, "per_second or seconds is NULL");
  const cudaError_t e = measure_alu_peak(which, iters, per_second, seconds);
  if (e != cudaSuccess) return cuda_fail(e, "gpf_measure_alu_peak");
  return GPF_OK;
}

gpf_status gpf_test_sort_wait_timeout(uint32_t spin_limit, gpf_stream stream) {
  if (spin_limit < 1 || spin_limit > (1u << 22))
    return fail(GPF_ERR_INVALID_ARG, "spin_limit = %u outside 1 .. 2^22", spin_limit);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* buf = nullptr;
  uint32_t* stalled = nullptr;
  cudaError_t e = cudaMalloc(&buf, sort_wait_probe_bytes());
  if (e == cudaSuccess) e = cudaMalloc(&stalled, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(stalled, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = launch_sort_wait_probe(buf, spin_limit, stalled, st);
  uint32_t flag = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flag, stalled, sizeof(flag), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (buf) cudaFree(buf);
  if (stalled) cudaFree(stalled);
  if (e != cudaSuccess) return cuda_fail(e, "gpf_test_sort_wait_timeout");
  if (flag) return fail(GPF_ERR_TIMEOUT, "the wait gave up after %u polls and set the flag",
                        spin_limit);
  return GPF_OK;
}

}  // extern "C"
