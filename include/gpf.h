/*
 * gpf.h - C ABI of the Gaussian Photon Field hit-point radiance library
 * (libgpf.so, CUDA, sm_103a).
 *
 * The library evaluates the radiance a Gaussian Photon Field (arxiv
 * 2512.12459) returns at camera-ray hit points, its gradient with respect to
 * every Gaussian parameter, the MSE loss that supervises it and the Adam step
 * that optimises it:
 *
 *   Gaussian i: mean mu_i, rotation q_i (quaternion (w,x,y,z), normalised by
 *   the library), log-scale l_i (scale s_i = exp(l_i)), spectral flux Phi_i
 *   (C channels). Sec. 4.1: Sigma_i = R S S^T R^T, contribution
 *   Phi_i exp(-1/2 d^T Sigma_i^-1 d).
 *
 *   Hit point x with normal n, direction to the viewer w_o, albedo rho:
 *     u_i = S_i^-1 R_i^T (x - mu_i),  Q_i = u_i . u_i
 *     psi = 1 if |x - mu_i| <= r else exp(-3 t^2), t = (|x - mu_i| - r)/max(r, 1e-6)
 *     w_i = exp(-Q_i / 2) psi                 (Sec. 4.2, aggregation)
 *     L = sum_{i : Q_i <= k^2} w_i Phi_i,  Z = sum_{i : Q_i <= k^2} w_i
 *     O = rho * L * [n.w_o > 0]                  (GPF_SUM)
 *     O = rho * L / max(Z, eps) * [n.w_o > 0]    (GPF_NORMALIZED; the soft
 *                                                  normalisation of the
 *                                                  query listing of Algorithm S3)
 *   k is the truncation in standard deviations (3: the 3-sigma ellipsoid; an
 *   infinite k sums every Gaussian).
 *
 *   GPF_DISK_KDE is the per-view photon density estimate the field replaces
 *   (Sec. 3.2, Eq. kde; the gather of Algorithm S1), on the same index: the
 *   field holds photons (mean = position, spectrum = flux) and
 *     O = rho * (1 / (pi r^2)) * sum_{i : |x - mu_i| <= r} Phi_i * [n.w_o > 0]
 *   with r = r_max. The index finds photon i through its k-sigma box, so
 *   every photon must have k * max scale >= r (e.g. isotropic log-scale
 *   log(r / k)); rotations do not matter.
 *
 * Conventions for every call:
 *   - Arrays are float32 structure-of-arrays, row-major [rows, count], one row
 *     per component (mean [3,N] = all x, then all y, then all z).
 *   - Every array pointer is a DEVICE pointer owned by the caller, contiguous
 *     and 4-byte aligned. The library never allocates device memory: scratch
 *     comes from a caller-provided workspace (256-byte aligned) whose size the
 *     library reports.
 *   - Every call that takes a stream enqueues its work on that stream and
 *     returns without synchronising (gpf_index_stats excepted). A NULL stream
 *     is the legacy default stream.
 *   - Every call returns a gpf_status. Arguments are validated on the host
 *     before anything is enqueued; on an error nothing is enqueued and
 *     gpf_last_error() describes it. No call aborts or throws.
 *   - Problems found on the device (a full pair buffer; a wait of the index
 *     build's single-pass sort that ran out of its poll limit; a non-finite
 *     Gaussian parameter or active hit point) set a flag in the index
 *     workspace. Every later kernel that reads the index (forward, backward,
 *     and an Adam step given the index as its guard) sees it and leaves its
 *     outputs untouched. gpf_index_stats() reads the flags back and reports
 *     GPF_ERR_CAPACITY, GPF_ERR_TIMEOUT or GPF_ERR_NONFINITE;
 *     gpf_index_flags_async() copies them to device memory without a
 *     synchronisation (for a step replayed as a CUDA graph).
 */
#ifndef GPF_H
#define GPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st *gpf_stream;

typedef enum gpf_status {
  GPF_OK = 0,
  GPF_ERR_INVALID_ARG = 1,        /* bad pointer, size, alignment or mode      */
  GPF_ERR_CUDA = 2,               /* a CUDA runtime call or launch failed      */
  GPF_ERR_WORKSPACE_TOO_SMALL = 3,/* workspace smaller than the reported size  */
  GPF_ERR_CAPACITY = 4,           /* the (cell, Gaussian) pair buffer was full */
  GPF_ERR_NOT_BUILT = 5,          /* index used before gpf_build_index         */
  GPF_ERR_MISMATCH = 6,           /* field/queries differ from those indexed   */
  GPF_ERR_TIMEOUT = 7,            /* a bounded device-side wait gave up        */
  GPF_ERR_NONFINITE = 8           /* a non-finite parameter or hit point       */
} gpf_status;

/* Bits of the device flags word (gpf_index_flags_async); 0 = usable. */
#define GPF_FLAG_CAPACITY 1u      /* the pair buffer was full                   */
#define GPF_FLAG_TIMEOUT 2u       /* a bounded wait of the build's sort gave up */
#define GPF_FLAG_NONFINITE 4u     /* a Gaussian parameter (mean, quat, logscale,
                                     spectrum) or the position of an active hit
                                     point was NaN or infinite                 */

typedef enum gpf_mode { GPF_SUM = 0, GPF_NORMALIZED = 1, GPF_DISK_KDE = 2 } gpf_mode;

/* Maximum number of spectral channels C. */
#define GPF_MAX_CHANNELS 8
/* Maximum cells per axis of the hit-point grid. */
#define GPF_MAX_DIM 1024
/* Maximum number of grid levels. */
#define GPF_MAX_LEVELS 16

/* Storage of a field's parameter arrays (gpf_field.storage). */
#define GPF_F32 0
#define GPF_BF16 1
#define GPF_BF16_MEAN32 2
/* Gaussians per anchor group of the GPF_BF16 storage. */
#define GPF_BF16_GROUP 16

/* The Gaussian Photon Field (Sec. 4.1). Arrays [rows, n].
 *
 * storage GPF_F32: float32 arrays as named; anchor NULL.
 * storage GPF_BF16 (16-bit storage, float32 arithmetic): the four arrays hold
 *   bfloat16 values (uint16, the upper half of a float32), and anchor holds
 *   float32 [ceil(N/16), 4], 16-byte aligned: for each group j of
 *   GPF_BF16_GROUP consecutive Gaussians (16j .. 16j+15) four consecutive
 *   floats, an origin (x, y, z) and a log-scale reference l_ref.
 *   The decoded float32 parameters are
 *     mu_k = origin_k + f32(mean_k)          (means as offsets from the origin)
 *     l_k  = l_ref + f32(logscale_k)         (log-scales as offsets)
 *     q, Phi = f32(quat), f32(spectrum)
 *   (float32 additions). gpf_build_index decodes them once per build; every
 *   later step computes in float32 on the decoded values, and gradients are
 *   with respect to the decoded values. A group should be compact in space
 *   (order the Gaussians spatially, e.g. by the Morton code of the means):
 *   the offsets then carry bfloat16's 8 significant bits on a small range.
 *   gpf_field_quantize writes this form from a float32 field.
 * storage GPF_BF16_MEAN32: as GPF_BF16, except that mean holds the float32
 *   means themselves (anchors still carry the log-scale references; their
 *   origins are unused). Eight significant bits cannot place a mean to the
 *   few 1e-4 of its own scale that a 1e-3 radiance error needs; this form
 *   keeps that precision and stores the rest in 16 bits. */
typedef struct gpf_field {
  int64_t n;             /* number of Gaussians N >= 0                       */
  int32_t channels;      /* C, 1..GPF_MAX_CHANNELS                           */
  int32_t storage;       /* GPF_F32, GPF_BF16 or GPF_BF16_MEAN32             */
  const void *mean;      /* [3,N] mu                                         */
  const void *quat;      /* [4,N] (w,x,y,z), any non-zero norm               */
  const void *logscale;  /* [3,N] l, scale s = exp(l)                        */
  const void *spectrum;  /* [C,N] Phi                                        */
  const float *anchor;   /* GPF_BF16: [ceil(N/16), 4]; GPF_F32: NULL         */
} gpf_field;

/* Camera-ray hit points (first diffuse hits, Sec. 4.2). */
typedef struct gpf_queries {
  int64_t m;             /* number of hit points M >= 0                      */
  const float *x;        /* [3,M] positions                                  */
  const float *normal;   /* [3,M] surface normals                            */
  const float *wo;       /* [3,M] directions towards the viewer              */
  const float *albedo;   /* [C,M] BSDF albedo rho, or NULL for rho = 1       */
  const uint8_t *valid;  /* [M] non-zero = supervised/valid, or NULL = all   */
} gpf_queries;

/* Query parameters. */
/* Neighbourhood of a hit point (gpf_query_params.neighbourhood). */
#define GPF_NB_KSIGMA 0    /* {i : Q_i <= k^2}, k = the index's cutoff_sigma   */
#define GPF_NB_BALL_KNN 1  /* the paper's hybrid query (Sec. 4.2, Neighborhood
                              Search; Algorithm S3): the Gaussians whose mean
                              lies within ball_r of x, or, when there are
                              fewer than k_min of them, the k_min nearest
                              means (ties: the smaller index). No truncation
                              of the weights. ball_r = 0: kNN only; k_min = 0:
                              ball only. The backward needs an index with
                              max_nb_pairs > 0.                              */
#define GPF_MAX_KMIN 16

typedef struct gpf_query_params {
  int32_t mode;          /* gpf_mode                                         */
  float r_max;           /* falloff radius r (paper: 0.02); +INF disables psi;
                            GPF_DISK_KDE: the gather radius (finite, > 0)    */
  float eps;             /* normalisation floor (paper: 1e-6)                */
  int32_t neighbourhood; /* GPF_NB_KSIGMA or GPF_NB_BALL_KNN                 */
  float ball_r;          /* GPF_NB_BALL_KNN: ball radius (paper: 0.02), at
                            most the index's ball_radius                     */
  int32_t k_min;         /* GPF_NB_BALL_KNN: 0..GPF_MAX_KMIN (paper: 3)      */
  int32_t f64_sums;      /* gpf_radiance_bwd only. 0: the per-Gaussian sums
                            and their reduction run in float32 (the product
                            path). 1: the gradient-check build: the same
                            float32 pair terms are summed, reduced and turned
                            into gradients in float64, so that summation
                            order no longer hides a wrong term (slow: GB300's
                            float64 rate is low). Must be 0 in the forward. */
} gpf_query_params;

/* Multi-level uniform grid and capacities of an index.
 * Level L (0 <= L < levels) has cubic cells of edge cell_size * 2^L, all
 * levels sharing the origin. A Gaussian is listed on the finest level on which
 * its k-sigma bounds span at most max_span cells per axis, in the cells of
 * that box which hold hit points. Hit points are sorted by their cell on
 * query_level, a dims[0] x dims[1] x dims[2] grid. Points outside the grid
 * are clamped into its border cells, which keeps the result exact (only
 * slower). */
#define GPF_MAX_COOP_CELLS 8

typedef struct gpf_grid_config {
  float origin[3];       /* lower corner shared by all levels                */
  float cell_size;       /* c0: cell edge on the finest level, > 0           */
  int32_t levels;        /* 1..GPF_MAX_LEVELS                                */
  int32_t max_span;      /* S, 1..64                                         */
  int32_t query_level;   /* K, 0..15; dims[k] * 2^K <= 2^20                  */
  int32_t dims[3];       /* hit-point grid cells per axis, 1..GPF_MAX_DIM    */
  int32_t hash_bits;     /* 2^hash_bits buckets hold the Gaussian lists, 8..28 */
  int32_t channels;      /* C of the fields this index will hold             */
  float cutoff_sigma;    /* truncation k: Q <= k^2 (3 = 3 sigma); +INF = no
                            truncation (every Gaussian, no cell lists)       */
  int32_t brute_force;   /* 1: no cell lists; every Gaussian is tested with
                            Q <= k^2 (used to check the culled path)         */
  int32_t coop_cells;    /* forward tile shape: a tile of 32 hit points walks
                            a level's lists together when its points fall in
                            at most this many cells of that level, else each
                            point's own list is pooled; 1..GPF_MAX_COOP_CELLS,
                            0 = 4                                            */
  int32_t field_storage; /* storage of the fields built from: GPF_F32,
                            GPF_BF16 or GPF_BF16_MEAN32 (the 16-bit forms
                            reserve float32 decode arrays)                   */
  float ball_radius;     /* > 0: also list every Gaussian once under the cell
                            of its mean on the first level whose cells are
                            >= ball_radius, for GPF_NB_BALL_KNN queries with
                            a ball of at most this radius; 0: none           */
  int64_t max_gaussians; /* capacity N_max (< 2^30)                          */
  int64_t max_queries;   /* capacity M_max (< 2^30)                          */
  int64_t max_pairs;     /* capacity of (cell, Gaussian) entries (< 2^30)    */
  int64_t max_nb_pairs;  /* capacity of (hit point, Gaussian) pairs of the
                            GPF_NB_BALL_KNN backward (< 2^30; 0: that
                            backward is refused). A backward whose
                            neighbourhoods hold more pairs sets the capacity
                            flag and leaves its gradients untouched.         */
  int32_t split_items;   /* forward load balance: 0 = every tile of 32 hit
                            points is one work unit; > 0 = the build
                            estimates each tile's work (the list entries its
                            points walk) and splits a tile above this many
                            into up to GPF_MAX_TILE_PARTS units over disjoint
                            chunks of its lists, whose partial sums a final
                            kernel adds in part order (results still
                            deterministic; they differ from the unsplit sums
                            by summation order only)                         */
  int32_t tile_order;    /* order of the hit points inside each query-level
                            cell, which shapes the forward's 32-point tiles:
                            0 = hit point index order; b = 1 or 2 = by the
                            Morton order of the 2^b x 2^b x 2^b sub-cells
                            (level query_level - b), then index order, so
                            that consecutive hit points form compact boxes.
                            Needs b <= query_level and at most 32 key bits
                            (3 b above the cell key). Results depend on it
                            through summation order only.                    */
} gpf_grid_config;
#define GPF_MAX_TILE_PARTS 64
#define GPF_MAX_SPLIT_UNITS 32768

/* Opaque host-side handle. It holds sizes and pointers into the workspace;
 * the device data live in the caller's workspace. */
typedef struct gpf_index gpf_index;

/* Counters read back by gpf_index_stats. The Gaussian classes are those of
 * the backward's work split: a live Gaussian has a hit point in a cell of its
 * k-sigma box; a small one's bounds span at most 2 query-level cells per
 * axis (one lane of a warp takes it); a large one is spread over a warp; the
 * large ones whose bounds cover at least 2^12 query-level cells ("huge") are
 * split, up to GPF_BWD_SPLIT_MAX of them, into GPF_BWD_SPLIT_WAYS work units
 * whose partial sums are added in a fixed order. */
#define GPF_BWD_SPLIT_WAYS 16
#define GPF_BWD_SPLIT_MAX 16384
typedef struct gpf_index_stats_t {
  int64_t n_pairs;       /* (cell, Gaussian) entries the last build needed   */
  int64_t n_active;      /* hit points that are valid and face the viewer    */
  int64_t n_live;        /* live Gaussians                                   */
  int64_t n_small;       /* live small Gaussians                             */
  int64_t n_huge;        /* live huge Gaussians                              */
  int64_t n_split;       /* huge Gaussians split: min(n_huge, GPF_BWD_SPLIT_MAX) */
  uint32_t level_mask;   /* bit L set when some Gaussian lives on level L    */
  uint32_t flags;        /* GPF_FLAG_* bits (0 = usable)                     */
  int32_t overflow;      /* 1 if n_pairs exceeded max_pairs                  */
  int32_t n_hybrid_units; /* work units of the tiles the last GPF_NB_BALL_KNN
                            forward split (tiles whose ball boxes list more
                            than 512 centre entries; 0: none split)          */
  int64_t n_nb_pairs;    /* (hit point, Gaussian) pairs the last GPF_NB_BALL_KNN
                            backward selected (above max_nb_pairs: the
                            capacity flag, and the room a rebuild needs)     */
} gpf_index_stats_t;

/* Gradients, each [rows, N] float32, device pointers owned by the caller. */
typedef struct gpf_field_grad {
  float *mean;           /* [3,N] d/d mu                                     */
  float *quat;           /* [4,N] d/d q (raw, through the normalisation)     */
  float *logscale;       /* [3,N] d/d l                                      */
  float *spectrum;       /* [C,N] d/d Phi                                    */
  int32_t accumulate;    /* 0: overwrite, 1: add to the existing values      */
  int32_t reserved;
} gpf_field_grad;

/* Adam hyper-parameters (Sec. A.2: Adam, learning rate 5e-4). */
typedef struct gpf_adam_hparams {
  float lr[4];           /* learning rate per group: mean, quat, logscale,
                            spectrum                                         */
  float beta1, beta2, eps;
  int32_t step;          /* 1-based index of the update being applied, or 0
                            when step_counter is given                        */
  int64_t *step_counter; /* NULL, or a device int64 holding the number of
                            updates applied so far: the update uses
                            t = *step_counter + 1 and then increments it, so
                            a captured CUDA graph replays correct steps       */
  const gpf_index *guard;/* NULL, or a built index (the one whose backward
                            produced the gradients): when its last build set
                            a device flag (GPF_FLAG_*), the update is skipped
                            on the device: parameters, moments and the step
                            counter stay untouched. The check happens when
                            the kernels run, so a captured graph keeps it.   */
} gpf_adam_hparams;

/* ------------------------------------------------------------------------ */

/* Version string of the library. */
const char *gpf_version(void);

/* Short name of a status code. Never NULL. */
const char *gpf_status_string(gpf_status s);

/* Message of the last failed call on this host thread ("" if none). */
const char *gpf_last_error(void);

/*
 * gpf_index_create - validate a grid configuration and make a handle.
 *   cfg  host pointer, read during the call only.
 *   out  receives the handle; release it with gpf_index_destroy.
 * Errors: GPF_ERR_INVALID_ARG (NULL pointer, cell_size <= 0 or not finite,
 * dims outside 1..GPF_MAX_DIM or more than 2^28 cells, channels outside
 * 1..GPF_MAX_CHANNELS, cutoff_sigma <= 0, brute_force not 0/1, negative
 * capacities).
 * Allocates host memory only.
 */
gpf_status gpf_index_create(const gpf_grid_config *cfg, gpf_index **out);

/* Release a handle (NULL is ignored). The workspace stays the caller's. */
void gpf_index_destroy(gpf_index *index);

/*
 * gpf_index_workspace_size - device bytes gpf_build_index needs.
 *   bytes receives the size for the handle's capacities.
 */
gpf_status gpf_index_workspace_size(const gpf_index *index, size_t *bytes);

/*
 * gpf_build_index - the spatial index of one (field, hit point set) pair.
 *
 * Preprocesses every Gaussian (normalised rotation, M = S^-1 R^T, the
 * axis-aligned bounds of its k-sigma ellipsoid: half-extent
 * k sqrt(sum_j R_kj^2 s_j^2) per axis), sorts the hit points by grid cell,
 * then emits one (cell, Gaussian) entry for every cell that the Gaussian's
 * bounds overlap and that holds at least one active hit point, and
 * radix-sorts the entries by cell into per-cell Gaussian lists. It replaces
 * the paper's periodically rebuilt KD-tree over the centres (Sec. A.2) and
 * bounds the neighbourhood by the k-sigma ellipsoid (Sec. 4.2, Neighborhood
 * Search, read as {i : Q_i <= k^2}).
 *
 *   index      handle from gpf_index_create.
 *   field      N <= max_gaussians, C = the handle's channels.
 *   queries    M <= max_queries; the set later passed to fwd/bwd.
 *   workspace  device buffer of at least gpf_index_workspace_size bytes,
 *              256-byte aligned, owned by the caller, kept alive and
 *              unmodified until the last fwd/bwd that uses this build.
 * With cutoff_sigma = +INF or brute_force = 1 no cell lists are built and
 * fwd/bwd test every Gaussian against every hit point.
 * The index records the field and query pointers and sizes; fwd/bwd given
 * others return GPF_ERR_MISMATCH. A pair count above max_pairs sets the
 * overflow flag (see gpf_index_stats).
 * Errors: GPF_ERR_INVALID_ARG, GPF_ERR_WORKSPACE_TOO_SMALL, GPF_ERR_CUDA.
 */
gpf_status gpf_build_index(gpf_index *index, const gpf_field *field,
                           const gpf_queries *queries, void *workspace,
                           size_t workspace_bytes, gpf_stream stream);

/*
 * gpf_index_stats - synchronise the stream and read the device counters of
 * the last build. The counters are filled in either way; the status is
 * GPF_ERR_TIMEOUT, GPF_ERR_NONFINITE or GPF_ERR_CAPACITY (in that order of
 * precedence) when the matching flag is set, else GPF_OK.
 */
gpf_status gpf_index_stats(const gpf_index *index, gpf_index_stats_t *stats,
                           gpf_stream stream);

/*
 * gpf_index_flags_async - enqueue on the stream a one-thread kernel that
 * writes the device flags of the index's last build (GPF_FLAG_* bits, 0 =
 * usable) to *flags, without synchronising: a step captured in a CUDA graph
 * can report an unusable build through it (copy the word to pinned host
 * memory in the same graph and read it once the replay has finished).
 *   flags  device uint32, 4-byte aligned, owned by the caller.
 * The paper has no counterpart: it is error reporting for graph replays.
 * Errors: GPF_ERR_INVALID_ARG, GPF_ERR_NOT_BUILT, GPF_ERR_CUDA.
 */
gpf_status gpf_index_flags_async(const gpf_index *index, uint32_t *flags, gpf_stream stream);

/*
 * gpf_radiance_fwd - radiance O at every hit point (Sec. 4.2, aggregation
 * equation; the soft falloff and normalisation of the query listing of
 * Algorithm S3; the BSDF modulation read as albedo times a hemisphere gate).
 *
 *   index, field, queries  as given to the last gpf_build_index.
 *   params  host pointer: mode, r_max (+INF: psi = 1), eps.
 *   out     [C,M] float32 device, written for every hit point (0 where the
 *           point is invalid or n.w_o <= 0).
 *   z_out   [M] float32 device or NULL: Z = sum_i w_i for active points, 0
 *           elsewhere (GPF_DISK_KDE: the number of photons gathered). Keep it
 *           for gpf_radiance_bwd in GPF_NORMALIZED mode.
 * Sums run in float32 in a fixed order: results are bitwise reproducible
 * for a given build.
 * The pair loop is a persistent kernel whose warps take tiles of hit points
 * from a work counter in the index: calls on one index must be ordered (one
 * stream, or events between streams).
 * Errors: GPF_ERR_INVALID_ARG, GPF_ERR_NOT_BUILT, GPF_ERR_MISMATCH, GPF_ERR_CUDA.
 */
gpf_status gpf_radiance_fwd(const gpf_index *index, const gpf_field *field,
                            const gpf_queries *queries,
                            const gpf_query_params *params, float *out,
                            float *z_out, gpf_stream stream);

/*
 * gpf_count_pairs - the work of gpf_radiance_fwd for the last build, without
 * computing radiance: counts[0] = (hit point, candidate Gaussian) pairs the
 * pair loop evaluates after culling, counts[1] = pairs with Q <= k^2 (the
 * neighbourhood of Sec. 4.2 read as the k-sigma ellipsoid; the algorithmic
 * work of the query).
 *   counts  device array of 2 uint64, 8-byte aligned, overwritten.
 * Errors: as gpf_radiance_fwd.
 */
gpf_status gpf_count_pairs(const gpf_index *index, const gpf_field *field,
                           const gpf_queries *queries, uint64_t *counts,
                           gpf_stream stream);

/*
 * gpf_index_set_timing_events - have later calls on this index record
 * caller-created CUDA events around their pair-loop kernels, for per-kernel
 * timing with cudaEventElapsedTime: fwd_start / fwd_stop around the kernel of
 * gpf_radiance_fwd, bwd_start / bwd_stop around the pair-loop kernel of
 * gpf_radiance_bwd (not its packing and gradient-epilogue kernels).
 *   each event  a cudaEvent_t passed as void*, created and owned by the
 *               caller, or NULL (not recorded). The handles are kept until
 *               the next call of this function and recorded on the stream of
 *               every later gpf_radiance_fwd / gpf_radiance_bwd call; the
 *               caller keeps them alive for as long as they are set.
 * The paper has no counterpart: it is an instrumentation hook.
 * Errors: GPF_ERR_INVALID_ARG (index NULL); a failed event record surfaces
 * as GPF_ERR_CUDA from the call that records it.
 */
gpf_status gpf_index_set_timing_events(gpf_index *index, void *fwd_start, void *fwd_stop,
                                       void *bwd_start, void *bwd_stop);

/*
 * gpf_launch_count - number of CUDA kernels this library has launched in the
 * process so far (host-side counter; memsets and copies are not counted).
 */
uint64_t gpf_launch_count(void);

/*
 * gpf_radiance_bwd - gradient of sum_{c,m} grad_out[c,m] O[c,m] with respect
 * to mu, q (raw), l and Phi (Sec. 4.2, Differentiable Accumulation). The
 * exponentials are recomputed, not stored. Contributions are reduced per
 * Gaussian inside one warp (no global atomics), so results are bitwise
 * reproducible.
 *
 *   grad_out  [C,M] device, upstream gradient d loss / d O.
 *   out, z    [C,M] and [M] device: the outputs of the matching forward
 *             (read only in GPF_NORMALIZED mode; may be NULL in GPF_SUM).
 *   grads     host struct of device pointers [3,N], [4,N], [3,N], [C,N];
 *             accumulate = 0 overwrites, 1 adds. Left untouched when the
 *             index's last build set a device flag.
 *   params    as gpf_radiance_fwd; f64_sums = 1 selects the float64
 *             gradient-check build of the sums.
 * With GPF_NB_BALL_KNN the selection N(x) is held fixed (it is piecewise
 * constant in the parameters): the library runs the forward's selection
 * again, writes every selected (hit point, Gaussian) pair at a per-point
 * offset, sorts the pairs by Gaussian (stable, so each Gaussian's hit points
 * stay in index order) and sums each Gaussian's pairs in one warp, without
 * atomics; the index needs max_nb_pairs at least the number of selected
 * pairs, and more sets the capacity flag. When the last GPF_NB_BALL_KNN
 * gpf_radiance_fwd on this build (and index) had the same ball_r and k_min,
 * it has already written each hit point's number of selected pairs and the
 * k_min nearest of the points that fell back, and the selection's ball part
 * runs once here instead of the whole selection twice; that forward must
 * then be ordered before this call (the same stream, or an event).
 * Errors: as gpf_radiance_fwd.
 */
gpf_status gpf_radiance_bwd(const gpf_index *index, const gpf_field *field,
                            const gpf_queries *queries,
                            const gpf_query_params *params,
                            const float *grad_out, const float *out,
                            const float *z, const gpf_field_grad *grads,
                            gpf_stream stream);

/*
 * gpf_mse_loss_grad - the MSE loss of Sec. 4.3 and its gradient:
 *   loss = (1/|V|) sum_{m valid} sum_c (out[c,m] - target[c,m])^2
 *   grad[c,m] = 2 (out - target) / |V| on valid points, 0 elsewhere.
 *   out, target  [C,M] float32 device; valid [M] uint8 device or NULL.
 *   loss         float32 device scalar (written); grad [C,M] device.
 *   workspace    device scratch of gpf_mse_workspace_size(m) bytes.
 * The reduction order is fixed (bitwise reproducible). |V| = 0 gives 0.
 */
gpf_status gpf_mse_workspace_size(int64_t m, size_t *bytes);
gpf_status gpf_mse_loss_grad(int64_t m, int32_t channels, const float *out,
                             const float *target, const uint8_t *valid,
                             float *loss, float *grad, void *workspace,
                             size_t workspace_bytes, gpf_stream stream);

/*
 * gpf_mse_loss_grad_noalloc - gpf_mse_loss_grad without a caller workspace.
 * (A library convenience; the paper has no counterpart.)
 *
 * For callers that cannot hand the library device memory of their own: code
 * where allocating is not permitted or not possible (a host framework that
 * owns every device allocation and offers no hook for it, a loop that must
 * never enter the allocator), or a plain C host without CUDA memory
 * management. The scratch that gpf_mse_loss_grad takes from its workspace
 * lives here in a fixed array inside the library (128 KiB of device memory on
 * every GPU that loads the library, held until the process exits).
 *   Arguments, outputs and results as gpf_mse_loss_grad (bitwise equal).
 *   m <= GPF_NOALLOC_MAX_POINTS, else GPF_ERR_INVALID_ARG and nothing runs.
 * Every call looks up the array's device address on the current device (a
 * host-side lookup, no allocation), so the address stays right after a
 * cudaDeviceReset reloads the library's device code; the first call on a
 * device (or after such a reset) also loads that code, so make it before any
 * stream capture. Allocates no memory. All calls share the one array, which keeps the
 * last call's partial sums; every call overwrites what it reads, but calls
 * whose kernels may overlap on the GPU race on it: order them.
 */
#define GPF_NOALLOC_MAX_POINTS ((int64_t)1 << 26)
gpf_status gpf_mse_loss_grad_noalloc(int64_t m, int32_t channels, const float *out,
                                     const float *target, const uint8_t *valid,
                                     float *loss, float *grad, gpf_stream stream);

/*
 * gpf_adam_step - one bias-corrected Adam update (Sec. A.2) of the four
 * parameter tensors in place:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2
 *   p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
 *   params  the field's arrays, written in place (the const pointers of
 *           gpf_field are cast away: pass writable buffers).
 *   grads   gradients from gpf_radiance_bwd.
 *   m, v    first and second moments, same layout as params (a gpf_field_grad
 *           each; zero them before step 1).
 *   hp      host struct; either hp->step >= 1 and hp->step_counter NULL, or
 *           hp->step == 0 and hp->step_counter a device int64 (8-byte
 *           aligned) that this call reads and increments on the stream.
 * One launch over all four tensors (plus one single-thread launch that
 * increments step_counter when it is given).
 */
gpf_status gpf_adam_step(const gpf_field *params, const gpf_field_grad *grads,
                         const gpf_field_grad *m, const gpf_field_grad *v,
                         const gpf_adam_hparams *hp, gpf_stream stream);

/*
 * gpf_field_quantize - the GPF_BF16 form of a float32 field (a facility of
 * the 16-bit storage; the paper keeps float32 parameters). Used after each
 * Adam update of a float32 master copy.
 *   src  GPF_F32 field of N Gaussians (device arrays, read).
 *   dst  GPF_BF16 or GPF_BF16_MEAN32 field with the same n and channels;
 *        its arrays (uint16, or float32 means for GPF_BF16_MEAN32) and its
 *        anchor array are written.
 * For every group of GPF_BF16_GROUP consecutive Gaussians: origin = midpoint
 * of the group's smallest and largest mean per axis, l_ref = midpoint of the
 * smallest and largest of its 3 x 16 log-scales (float32 (lo + hi) * 0.5);
 * offsets are float32 differences; every stored value is the float32 value
 * rounded to the nearest bfloat16, ties to even. One launch.
 * Errors: GPF_ERR_INVALID_ARG, GPF_ERR_CUDA.
 */
gpf_status gpf_field_quantize(const gpf_field *src, const gpf_field *dst, gpf_stream stream);

/*
 * gpf_sort_pairs_workspace_size / gpf_sort_pairs / gpf_sort_pairs_check -
 * the index build's stable LSD radix sort of (uint32 key, uint32 value)
 * pairs by key bits [0, bits), 8 bits per pass (a step of the cell-list
 * build, Sec. 4.2), exported for tests and reuse.
 *   keys, vals          device [n]: the pairs (input, and scratch)
 *   keys_alt, vals_alt  device [n]: the other half of the ping-pong
 *   n                   0 <= n < 2^30
 *   bits                0..32 (0: nothing to do)
 *   workspace           device, 256-byte aligned, at least
 *                       gpf_sort_pairs_workspace_size(n) bytes, owned by the
 *                       caller and kept until gpf_sort_pairs_check; its
 *                       first 4 bytes receive the stall flag
 *   *result_in_alt      (host, written) 1 if the sorted pairs end in
 *                       keys_alt / vals_alt (an odd number of passes), 0 if
 *                       in keys / vals
 * Equal keys keep their input order. Each pass is one single-pass kernel
 * whose tiles take their offsets from the earlier tiles (decoupled
 * look-back, every wait bounded). Asynchronous on stream.
 * gpf_sort_pairs_check synchronises the stream and returns GPF_ERR_TIMEOUT
 * if a wait gave up (the output is then invalid), else GPF_OK.
 * Errors: GPF_ERR_INVALID_ARG, GPF_ERR_WORKSPACE_TOO_SMALL, GPF_ERR_CUDA.
 */
gpf_status gpf_sort_pairs_workspace_size(int64_t n, size_t *bytes);
gpf_status gpf_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt,
                          uint32_t *vals_alt, int64_t n, int32_t bits, void *workspace,
                          size_t workspace_bytes, int32_t *result_in_alt, gpf_stream stream);
gpf_status gpf_sort_pairs_check(const void *workspace, gpf_stream stream);

/*
 * gpf_measure_alu_peak - measured throughput of the two pipes the pair loops
 * are bound by, for the roofline denominators: GPF_PEAK_FP32_FMA (float32
 * fused multiply-adds, reported in flop/s, one FMA = 2 flops) or GPF_PEAK_EX2
 * (the special-function unit's ex2.approx.ftz.f32, every included pair's
 * exponential, in results/s). Launches 8 blocks of 256 threads per SM, each
 * thread running 8 independent chains of iters x 16 operations, once untimed
 * and once timed with CUDA events, on a stream of its own; synchronous.
 *   per_second  host, receives the rate; seconds: host, the timed launch.
 * The paper has no counterpart: it is a measurement aid.
 * Errors: GPF_ERR_INVALID_ARG (which, iters outside 1 .. 2^20, NULL), GPF_ERR_CUDA.
 */
#define GPF_PEAK_FP32_FMA 0
#define GPF_PEAK_EX2 1
gpf_status gpf_measure_alu_peak(int32_t which, int32_t iters, double *per_second,
                                double *seconds);

/*
 * gpf_test_sort_wait_timeout - failure-detection test of the sort's bounded
 * wait, with no fault: one block of a single-pass sort kernel takes the
 * second of two tiles whose first tile no block processes, so its walk back
 * polls status words that nothing writes, spin_limit times (1 .. 2^22),
 * gives up, sets the stall flag and finishes. Synchronous (allocates and
 * frees its own device buffer). Returns GPF_ERR_TIMEOUT when the wait gave
 * up and said so (the expected outcome), GPF_OK if it did not.
 * Errors: GPF_ERR_INVALID_ARG (spin_limit outside 1 .. 2^22), GPF_ERR_CUDA.
 */
gpf_status gpf_test_sort_wait_timeout(uint32_t spin_limit, gpf_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GPF_H */
