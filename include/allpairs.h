/*
 * allpairs.h -- C ABI of the GB300 all-pairs library (libap.so).
 *
 * The library evaluates a pair function f(l(i), l(j)) for every unordered pair
 * 0 <= i < j < n of an item set (the problem statement of Sec. III), walking
 * the strict upper triangle in recursively blocked tiles (Sec. IV-B) with
 * persistent CUDA kernels that pop tiles from an atomic queue.
 *
 * General conventions
 *   - All compute is asynchronous on the caller's CUDA stream (`stream` is a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - The caller owns every input and output buffer.  The library owns what
 *     ap_create_items allocates and frees it in ap_destroy.
 *   - Arguments are validated before any launch: an error return leaves no
 *     partial write in caller memory.  Errors are returned as ap_status and
 *     never thrown across the ABI.
 *   - Packed pair layout: results for pair (i, j), i < j, live at
 *         p(i, j) = i*n - i*(i+1)/2 + (j - i - 1),     P = n(n-1)/2 entries,
 *     the row-major enumeration of the strict upper triangle.  n < 2 gives
 *     P = 0 and every call returns AP_OK without touching memory.
 *   - One handle is not thread-safe; different handles are independent.
 *   - Device waits inside the kernels are bounded; when one runs out the
 *     kernel records a code readable with ap_last_device_error() and the call
 *     that synchronises next reports AP_ERR_TIMEOUT.
 */
#ifndef ALLPAIRS_H
#define ALLPAIRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AP_OK = 0,
  AP_ERR_INVALID_ARG = 1,  /* bad pointer, size, kind or combination */
  AP_ERR_OOM = 2,          /* a device or pinned-host allocation failed */
  AP_ERR_CUDA = 3,         /* a CUDA runtime/driver call failed */
  AP_ERR_TIMEOUT = 4,      /* a bounded device wait ran out */
  AP_ERR_UNSUPPORTED = 5,  /* valid request this build does not implement */
  AP_ERR_STATE = 6         /* handle in the wrong state for the call */
} ap_status;

typedef enum {
  AP_ITEMS_CLOUD2D = 0,    /* weighted 2-D point clouds (microscopy particles, Sec. V-C) */
  AP_ITEMS_CLOUD3D = 1,    /* weighted 3-D point clouds */
  AP_ITEMS_VECTOR = 2,     /* dense FP32 vectors of one length (noise patterns, Sec. V-A) */
  AP_ITEMS_SPARSE = 3      /* sparse FP32 vectors over one index space (composition
                              vectors, Sec. V-B) */
} ap_item_kind;

typedef enum {
  /* Gaussian overlap cost between point clouds, the cross term of the GMM
   * L2 distance (Sec. V-C):
   *   f(i,j) = sum_a sum_b w_a w_b exp(-|x_a - (R x_b + t)|^2 / (2(s_a^2 + s_b^2)))
   * output float[P] */
  AP_FN_OVERLAP = 0,
  /* Pearson (normalised cross) correlation of dense vectors (Sec. V-A):
   *   r(i,j) = sum_k (x_ik - mu_i)(x_jk - mu_j) / sqrt(ss_i ss_j)
   * output double[P] */
  AP_FN_PEARSON = 1,
  /* debugging pair function: atomically adds 1 to int32 out[p(i,j)] for every
   * pair the schedule visits (coverage check: every i < j exactly once).
   * Works for any item kind; the caller zeroes out[] first. */
  AP_FN_COVERAGE = 2,
  /* the two particle scores of the microscopy application (Sec. V-C names
   * them; these are their standard forms), items as Gaussian mixtures with
   * components N(x; x_a, s_a^2 I), weights w_a, s2 = s_a^2 + s_b^2:
   * squared L2 distance between the mixtures, output float[P]:
   *   d(i,j) = S_i + S_j - 2 sum_a sum_b w_a w_b (2 pi s2)^(-dim/2)
   *                                     exp(-|x_a - (R x_b + t)|^2 / (2 s2)),
   *   S_i the same double sum over item i with itself (a = a' included) */
  AP_FN_GMM_L2 = 3,
  /* Bhattacharyya cost, output float[P]:
   *   f(i,j) = sum_a sum_b sqrt(w_a w_b) (2 s_a s_b / s2)^(dim/2)
   *                          exp(-|x_a - (R x_b + t)|^2 / (4 s2)) */
  AP_FN_BHATTACHARYYA = 4,
  /* cosine of sparse vectors (the composition-vector comparison of Sec. V-B,
   * "essentially the dot product between two sparse vectors"):
   *   c(i,j) = sum_k a_ik a_jk / sqrt(sum_k a_ik^2 sum_k a_jk^2)
   * FP32 products, FP64 sums and scaling; NaN for a row without non-zero
   * values; output double[P] */
  AP_FN_COSINE = 5
} ap_pair_fn;

typedef enum {
  AP_PREC_FP32 = 0,        /* plain FP32 CUDA-core path */
  AP_PREC_SPLIT_BF16 = 1   /* Pearson Gram as hi*hi + hi*lo + lo*hi BF16 products
                              on the tensor cores, FP32 accumulation */
} ap_precision;

typedef struct ap_items ap_items;   /* opaque, library-owned */

/* Description of an item set (the inputs of the load pipeline l, Sec. III). */
typedef struct ap_items_desc {
  int32_t kind;            /* ap_item_kind */
  int32_t data_on_host;    /* 1: x/y/z/sigma/weight/data are host pointers; 0: device */
  int64_t n_items;         /* n >= 0 */
  /* Point clouds (kind CLOUD2D/CLOUD3D), ragged structure-of-arrays.
   * offsets is ALWAYS a host pointer, int64[n_items + 1], non-decreasing,
   * offsets[0] == 0; the points of item i are [offsets[i], offsets[i+1]).
   * x, y, sigma: float[offsets[n]]; z: float[offsets[n]] for 3-D, ignored
   * for 2-D; weight: float[offsets[n]] or NULL (all weights 1).  sigma > 0,
   * weight >= 0 (zero-weight points contribute nothing).  Empty items are
   * allowed (their costs are 0). */
  const int64_t *offsets;
  const float *x, *y, *z, *sigma, *weight;
  /* Dense vectors (kind VECTOR): row-major float[n_items][ld], dim <= ld
   * values per row are used, dim >= 2. */
  const float *data;
  int64_t dim;
  int64_t ld;              /* row stride in elements; 0 means ld = dim */
  /* Vector representations to build, a bitmask of (1u << ap_precision);
   * 0 selects split-BF16 only. */
  uint32_t precisions;
  /* Vectors on the host only: 0 = copy everything to the device at creation
   * (the host buffer may be freed afterwards); > 0 = out-of-core mode, the
   * library keeps `data` (which must be page-locked and outlive the handle)
   * and streams items through an HBM slot cache of at most this many bytes
   * (the first-level device cache of Sec. IV-A). */
  uint64_t slot_cache_bytes;
  /* Sparse vectors (kind SPARSE), CSR: offsets (as above, a host pointer,
   * int64[n_items + 1]) delimit row i's entries; indices int32[offsets[n]]
   * strictly increasing within a row and in [0, dim); data float[offsets[n]]
   * the values.  indices and data are host or device pointers (data_on_host);
   * dim is the size of the index space (20^k for k-mers of k amino acids). */
  const int32_t *indices;
  /* Vectors given encoded (the parse stage of l, Sec. III stage 2): with
   * blobs != NULL (and data == NULL, data_on_host = 1, slot_cache_bytes > 0,
   * ld = 0), row i is the blob_bytes[i] bytes at host pointer blobs[i] in
   * `codec`; blobs and blob_bytes are host arrays that must outlive the
   * handle.  Host threads (parse_threads, 0 = one per core) decode 256-row
   * macros into page-locked host slots, host_cache_bytes of them (the
   * second-level cache of Sec. IV-A; 0 = two slots, i.e. decode on every
   * device-cache miss), from which the device cache is filled. */
  const uint8_t *const *blobs;
  const uint64_t *blob_bytes;
  int32_t codec;           /* ap_codec */
  int32_t parse_threads;
  uint64_t host_cache_bytes;
} ap_items_desc;

/* Encodings of vectors for ap_items_desc.blobs. */
typedef enum {
  AP_CODEC_NONE = 0,
  /* lossless: the bits of x_k XOR those of x_(k-1) (x_(-1) = +0) as an
   * unsigned LEB128 varint, 1-5 bytes a value */
  AP_CODEC_XOR_VARINT = 1
} ap_codec;

/* Run statistics of the last ap_run_pairs on a handle. */
typedef struct ap_run_stats {
  int64_t tiles;            /* tiles executed */
  int64_t item_loads;       /* item loads into the device cache (R * n in Sec. VI-A) */
  double reuse_R;           /* loads relative to the data set size, Eq. 1 */
  uint64_t h2d_bytes;       /* bytes copied host -> device */
  double slot_hit_rate;     /* fraction of item requests served by a resident slot */
  int32_t tile_m, tile_n;   /* tile shape used (items x items) */
  int32_t order;            /* 0 = recursive quadrant order, 1 = row panels,
                               2 = largest tiles first (point sets under 16 MB) */
  int32_t reserved;
  int64_t parsed_rows;      /* rows decoded by the parse stage during the run */
  double host_hit_rate;     /* second-level cache: requests served without decoding */
} ap_run_stats;

/* Tile plan of a point-cloud set: blocks of at most block_items items and
 * block_pts padded points (one block is staged in shared memory per tile),
 * reg_r a-points held per lane (chunks of 32*reg_r points).  sorted = items
 * stored largest first (decided at creation).  rate = point pairs per second
 * the tuner measured for the chosen plan. */
typedef struct ap_plan {
  int32_t block_items;
  int32_t block_pts;
  int32_t reg_r;
  int32_t sorted;
  double rate;
  /* vector sets only: 0 runs each 128 x 256 tile over all columns in one
   * unit; k >= 1 splits every tile's columns into k ranges and runs them
   * range by range inside waves of one tile per SM, so the tiles in flight
   * read the same columns and share them in L2; the partial Grams meet in
   * FP64 in the output, which a last pass scales by rs_i rs_j.  The default
   * (set at creation, and by ap_set_plan with k_split = -1): ranges of about
   * 16384 columns and at least two units per SM, at most one range per 64
   * columns; 0 where that gives one range */
  int32_t k_split;
  /* vector sets only: CTAs per tensor-core MMA.  2 (the default; 0 in
   * ap_set_plan asks for it): the units are 256 x 256 block pairs, each
   * computed by a cluster of two CTAs on neighbouring SMs with one
   * tcgen05.mma.cta_group::2 (each CTA stages its own 128 rows and half of
   * the other block); 1: one CTA per 128 x 256 tile.  Results agree to
   * rounding (the same products, chained the same way). */
  int32_t mma_ctas;
} ap_plan;

/*
 * ap_create_items -- run the load pipeline l(i) for every item (Sec. III:
 * transfer to the GPU and pre-process there) into library-owned storage.
 *   Clouds: points are padded per item to a multiple of 4 with zero weight
 *   and stored as (x, y[, z], sigma^2, log2 w) in device memory.
 *   Vectors: one pass over the rows: each row is centred on a shift s_i
 *   close to its mean (the mean of 1024 evenly strided values), c = x - s_i,
 *   stored as BF16 hi = rn(c), lo = rn(c - hi) for split-BF16 and/or as
 *   FP32 c for the FP32 path, rows padded with zeros, while FP64 sums of c
 *   and c^2 give delta_i = mu_i - s_i and ss_i = sum (x - mu_i)^2 exactly
 *   (the correlation subtracts D delta_i delta_j from the Gram in FP64); a
 *   row whose shift missed its mean by D delta^2 > ss / 64 is written again
 *   centred on its mean.
 *   Sparse vectors: the CSR arrays copied, FP64 squared norms per row, and
 *   per column chunk of 2048 codes the first entry of every row in it.
 * Host-side planning (block and tile lists, sorting) happens before the call
 * returns; every copy and kernel of the call is ordered on `stream`, for all
 * kinds (host sources: pageable memory is staged by the copy calls, pinned
 * memory is read by the GPU when the stream gets there).  Inputs may be
 * freed once that work has run (after a stream synchronise), except the
 * out-of-core host source (see slot_cache_bytes).
 * Errors: AP_ERR_INVALID_ARG (desc/out NULL, negative sizes, bad kind,
 * offsets not non-decreasing, missing arrays, sparse indices not strictly
 * increasing within a row or outside [0, dim)), AP_ERR_OOM, AP_ERR_CUDA.
 * On error *out is set to NULL and nothing is leaked.
 */
ap_status ap_create_items(const ap_items_desc *desc, void *stream, ap_items **out);

/*
 * ap_update_items -- re-run the load pipeline for vectors of the same shape
 * into the existing storage (no allocation).  data: row-major
 * float[n_items][ld] on the host (data_on_host = 1) or the device.
 * Errors: AP_ERR_INVALID_ARG, AP_ERR_STATE (not a resident vector set).
 */
ap_status ap_update_items(ap_items *items, const float *data, int32_t data_on_host,
                          void *stream);

/*
 * ap_run_pairs -- f(l(i), l(j)) for every pair i < j (Sec. III), written to
 * the packed device array `out` (layout above).
 *   fn = AP_FN_OVERLAP: clouds; out float[P]; params NULL (identity) or a
 *        device float[P][3] = (theta, tx, ty) per pair (2-D only), the
 *        transform applied to the second item j.
 *   fn = AP_FN_PEARSON: vectors; out double[P]; precision selects the Gram
 *        path (the representation must have been built at creation).
 *   fn = AP_FN_COVERAGE: any kind; out int32[P] is incremented.
 *   fn = AP_FN_COSINE: sparse vectors; out double[P].
 *   fn = AP_FN_GMM_L2, AP_FN_BHATTACHARYYA: clouds; out float[P]; params as
 *        for the overlap.  The first call of each builds a re-scaled copy of
 *        the storage (16 bytes a point, + 4 for 3-D weights) and, for the L2
 *        distance, the self terms S_i; later calls reuse them.
 * Errors: AP_ERR_INVALID_ARG (fn/kind mismatch, NULL out with P > 0, params
 * with 3-D clouds), AP_ERR_STATE (representation not built), AP_ERR_CUDA,
 * AP_ERR_TIMEOUT.
 */
ap_status ap_run_pairs(ap_items *items, int32_t fn, int32_t precision,
                       const float *params, void *out, void *stream);

/*
 * ap_run_pairs_list -- f(l(a), l(b)) for a chosen list of pairs only (the
 * comparison stage of Sec. III on a subset): out[k] = f(pi[k], pj[k]).
 *   pi, pj: HOST int32[n_pairs], original item ids, 0 <= a, b < n_items,
 *        a != b, either order, repeats allowed (copied before the call
 *        returns; the call synchronises `stream`).
 *   fn = AP_FN_OVERLAP, AP_FN_GMM_L2, AP_FN_BHATTACHARYYA: clouds; out
 *        device float[n_pairs]; params NULL or device float[n_pairs][3], the
 *        transform applied to item pj[k] (2-D only).  A pair listed as
 *        (a < b) gives the bits of ap_run_pairs at a's and b's packed index.
 *   fn = AP_FN_PEARSON: resident vector sets; out device double[n_pairs];
 *        precision selects the representation (built at creation); one warp
 *        per pair, the Gram's three products per column in FP32, FP64 sums.
 *        A list of at least 32 pairs per 128-item row block it touches first
 *        copies those blocks into row-major rows of one 4-byte word per
 *        column, in a buffer of n_items x dim words (padded to 64) that the
 *        first such call allocates and the handle keeps until ap_destroy;
 *        where that allocation fails, the call reads the blocked rows.
 *   fn = AP_FN_COSINE: sparse sets; out device double[n_pairs]; the two
 *        rows' codes merged (FP32 products, FP64 sums).
 * Errors: AP_ERR_INVALID_ARG (fn/kind mismatch, an index out of range or a
 * == b, NULL arrays with n_pairs > 0, params with other than 2-D clouds),
 * AP_ERR_STATE (representation not built), AP_ERR_UNSUPPORTED (out-of-core
 * sets, n_pairs > INT32_MAX), AP_ERR_CUDA.
 */
ap_status ap_run_pairs_list(ap_items *items, int32_t fn, int32_t precision, const int32_t *pi,
                            const int32_t *pj, int64_t n_pairs, const float *params, void *out,
                            void *stream);

/*
 * ap_load_and_run -- ap_update_items from host memory fused with
 * ap_run_pairs(AP_FN_PEARSON, AP_PREC_SPLIT_BF16) on a resident vector set:
 * the host rows travel in 256-item macros on the library's copy stream, each
 * macro is pre-processed as it lands, and every pair (a <= m, m) of macro m
 * is computed right away, so the transfers overlap the Gram (the
 * asynchronous, overlapped processing of Sec. IV-C; every item is loaded
 * once, R = 1).  host_data: float[n_items][ld] in host memory (page-locked for
 * the copies to overlap), read until the work on `stream` completes; out:
 * device double[P], overwritten.  The handle's stored items become the new
 * ones, as after ap_update_items.
 * Errors: AP_ERR_INVALID_ARG (not a vector set, NULL pointers with P > 0),
 * AP_ERR_STATE (out-of-core set, or no split-BF16 representation).
 */
ap_status ap_load_and_run(ap_items *items, const float *host_data, double *out, void *stream);

/*
 * ap_backward -- adjoint of the overlap cost (2-D clouds) with respect to the
 * per-pair transform (theta, tx, ty):
 *   grad_params[p][k] = grad_out[p] * d f_p / d param_k,
 *   d f / d t     = sum w_a w_b e d / s2,
 *   d f / d theta = sum w_a w_b e (d . J R x_b) / s2,  J = [[0,-1],[1,0]],
 * with d = x_a - (R x_b + t), s2 = s_a^2 + s_b^2, e = exp(-|d|^2 / (2 s2)),
 * the exponentials recomputed rather than stored.  params: device float[P][3]
 * or NULL (identity); grad_out: device float[P] or NULL (all ones);
 * grad_params: device float[P][3], overwritten; f_out: device float[P] or NULL.
 * Errors: AP_ERR_INVALID_ARG (not 2-D clouds, grad_params NULL with P > 0).
 */
ap_status ap_backward(ap_items *items, const float *params, const float *grad_out,
                      float *grad_params, float *f_out, void *stream);

/*
 * ap_ascent -- batched per-pair registration: n_steps fused steps of
 *   (f, g) = (f, grad f)(params);  if f >= fmin: params += eta * g / f
 * (gradient ascent on log f) for every pair at once.  params: device
 * float[P][3], updated in place; f_out: device float[P] or NULL, receives f
 * at the parameters of the last step (before its update); flags: device
 * int32[P] or NULL, set to 1 where some step was skipped (f < fmin).
 * Errors: AP_ERR_INVALID_ARG (not 2-D clouds, n_steps < 0, params NULL).
 */
ap_status ap_ascent(ap_items *items, float *params, int32_t n_steps, float eta,
                    float fmin, float *f_out, int32_t *flags, void *stream);

/*
 * ap_backward_list, ap_ascent_list -- ap_backward and ap_ascent on a chosen
 * list of pairs (registration of selected pairs, Sec. V-C): pi, pj as for
 * ap_run_pairs_list (host, original ids, the transform acting on pj[k]);
 * params, grad_out, grad_params, f_out and flags are device arrays of
 * n_pairs (x 3) entries indexed by list position.  Errors as for
 * ap_backward / ap_ascent and ap_run_pairs_list.
 */
ap_status ap_backward_list(ap_items *items, const int32_t *pi, const int32_t *pj,
                           int64_t n_pairs, const float *params, const float *grad_out,
                           float *grad_params, float *f_out, void *stream);
ap_status ap_ascent_list(ap_items *items, const int32_t *pi, const int32_t *pj, int64_t n_pairs,
                         float *params, int32_t n_steps, float eta, float fmin, float *f_out,
                         int32_t *flags, void *stream);

/* ap_destroy -- free everything the handle owns (its device slots, pinned
 * host cache, staging buffers, streams and plans: the storage levels of the
 * cache hierarchy of Sec. IV-A, released when the item set is done); NULL is
 * accepted.  Waits for the handle's outstanding work on its streams first.
 * Errors: none (always AP_OK). */
ap_status ap_destroy(ap_items *items);

/* Statistics of the last ap_run_pairs (host struct, caller-owned). */
ap_status ap_get_stats(const ap_items *items, ap_run_stats *out);

/*
 * ap_tune -- autotune the tile plan of a point-cloud set: the block size of
 * the recursively ordered upper triangle (Sec. IV-B) and the register
 * blocking.  Every candidate (block_items in {2, 4, 8, 16, 32}, block_pts in
 * {2048, 4096, 8192}, reg_r in {2, 4}) is timed on an even sample of its own
 * tiles (~2e10 point pairs, or all of them) and the fastest becomes the
 * handle's plan.  mode 0 tunes the overlap cost, mode 1 the adjoint / ascent
 * kernel (2-D only).  Synchronises `stream`; allocates temporary device
 * memory.  *out (may be NULL) receives the plan and its measured rate.
 * Errors: AP_ERR_INVALID_ARG, AP_ERR_UNSUPPORTED (vector sets), AP_ERR_CUDA.
 */
ap_status ap_tune(ap_items *items, int32_t mode, void *stream, ap_plan *out);

/* Current plan of a handle (vector sets report their fixed 128 x 256 tile). */
ap_status ap_get_plan(const ap_items *items, ap_plan *out);

/* Install a plan, e.g. a cached tuning result; `sorted`, `rate` and
 * `reserved` are ignored.  Synchronises the device.
 * Clouds: errors AP_ERR_INVALID_ARG (block_items outside 1..32, block_pts
 * outside 64..8192, reg_r not 2 or 4 or too small for the largest item:
 * 32 * reg_r * 128 points per item at most); k_split is ignored.
 * Vector sets: block_items must be 128 and block_pts 256 (the fixed tile),
 * reg_r is ignored and k_split (-1 for the default, or 0..AP_MAX_K_SPLIT)
 * chooses the schedule of the split-BF16 Gram; errors AP_ERR_INVALID_ARG, AP_ERR_STATE (out-of-core
 * or without the split-BF16 copy), AP_ERR_OOM. */
#define AP_MAX_K_SPLIT 256
ap_status ap_set_plan(ap_items *items, const ap_plan *plan);

/* Out-of-core schedules. */
typedef enum {
  /* the default: a resident set of macros plus groups streamed past it,
   * evicting the macro needed farthest ahead (the future is known) */
  AP_OOC_RESIDENT_STREAM = 0,
  /* the paper's policy: macro pairs in recursive quadrant order (Sec. IV-B),
   * a miss loads into the least recently used slot (Sec. IV-A-1) */
  AP_OOC_DC_LRU = 1,
  /* column slices: the same chunk of columns of every item resident at once
   * (one chunk buffer, plus a ring of raw pieces that lets the next chunk's
   * copy overlap this chunk's Gram), the Gram accumulated over the chunks in
   * FP64; each
   * item crosses the host link once (R = 1).  The Gram is a sum over
   * columns, so this schedule is open to the correlation only: rows are
   * centred on a shift (the mean of their first chunk) and the exact mean,
   * variance and centred Gram follow from the shifted sums at the end */
  AP_OOC_K_SLICED = 2
} ap_ooc_policy;

/* ap_set_out_of_core_policy -- rebuild an out-of-core handle's schedule with
 * another policy (synchronises the device).  Switching between the macro
 * schedules (0, 1) and the column slices (2) frees one kind of buffer and
 * allocates the other within the same slot_cache_bytes.  Errors:
 * AP_ERR_INVALID_ARG (not a vector set, unknown policy, cache too small for
 * a column chunk of 64 columns), AP_ERR_STATE (not out of core),
 * AP_ERR_OOM. */
ap_status ap_set_out_of_core_policy(ap_items *items, int32_t policy);

/*
 * ap_plan_out_of_core -- host-only preview of the out-of-core schedule for n
 * vectors of length dim and a slot cache of slot_cache_bytes (the device cache
 * of Sec. IV-A, here holding pre-processed 256-item macros of 256*Dp*4 bytes,
 * Dp = dim rounded up to 64) under `policy`.  Builds the schedule, checks that
 * every macro pair is computed exactly once with both macros resident, and
 * reports the slots, the macro loads (R = loads / ceil(n/256), Sec. VI-A) and
 * the steps.  AP_OOC_K_SLICED reports 2 slots (its two chunk buffers), one
 * load per macro and one step per column chunk.  Errors: AP_ERR_INVALID_ARG (bad
 * sizes or policy, NULL outputs, fewer than 3 slots while the set does not
 * fit), AP_ERR_STATE (schedule check failed).
 */
ap_status ap_plan_out_of_core(int64_t n_items, int64_t dim, uint64_t slot_cache_bytes,
                              int32_t policy, int64_t *n_slots, int64_t *n_loads,
                              int64_t *n_steps);

/* ap_encode_vector -- encode dim floats in `codec` (host memory).  out NULL:
 * *len = an upper bound of the encoded size.  Errors: AP_ERR_INVALID_ARG
 * (NULL arguments, unknown codec, cap too small). */
ap_status ap_encode_vector(const float *x, int64_t dim, int32_t codec, uint8_t *out,
                           uint64_t cap, uint64_t *len);

/* ap_decode_vector -- the parse stage's decoder for one row (host memory).
 * Errors: AP_ERR_INVALID_ARG (unknown codec, malformed or short input, or
 * input left over after dim values). */
ap_status ap_decode_vector(const uint8_t *in, uint64_t len, int32_t codec, int64_t dim, float *x);

/* Failure-path switches for testing the bounded device waits. */
typedef enum {
  AP_DEBUG_NONE = 0,
  /* the tensor-core Gram's producer withholds the first stage of every tile,
   * so the consumer's wait runs out: the kernel records a device error code
   * (read with ap_last_device_error), every role leaves, TMEM is freed and
   * the context stays usable */
  AP_DEBUG_WITHHOLD_STAGE = 1,
  /* as above, but the withheld stage is the sixth of each tile (its last when
   * it has fewer), so the wait runs out with tensor-core MMAs of the tile
   * already issued: they are drained before TMEM is freed */
  AP_DEBUG_WITHHOLD_LATER_STAGE = 2
} ap_debug_flags;

/* ap_set_debug -- set the failure-path switch and the wall-clock budget of
 * every bounded device wait (nanoseconds; 0 restores the 2 s default) for
 * the handle's later launches.  Errors: AP_ERR_INVALID_ARG (unknown flag). */
ap_status ap_set_debug(ap_items *items, int32_t flags, uint64_t wait_budget_ns);

/*
 * Task trace of the streamed pipelines (the optional profiling flag of
 * Sec. IV-C that traces the tasks each resource executes, shown as a
 * timeline in Fig. 4).  With tracing on, the out-of-core column-slice run
 * (ap_run_pairs on an out-of-core set) and ap_load_and_run record, on each of
 * their CUDA streams, when every task started and ended: host-to-device
 * copies (copy stream), pre-processing (pre-processing stream), the Gram and
 * the final scaling (the caller's stream).  Timing uses CUDA events, so the
 * traced call stays asynchronous; ap_get_trace waits for the recorded events.
 */
typedef enum {
  AP_STAGE_COPY = 0,        /* host -> device copy of one chunk / macro */
  AP_STAGE_PREPROCESS = 1,  /* centring and split-BF16 conversion */
  AP_STAGE_GRAM = 2,        /* tensor-core Gram over one chunk / macro column */
  AP_STAGE_FINALIZE = 3     /* the pass that scales the pairs */
} ap_stage;

typedef struct ap_trace_event {
  int32_t stream;           /* 0 the caller's stream, 1 copies, 2 pre-processing */
  int32_t stage;            /* ap_stage */
  int64_t index;            /* column chunk (slices) or 256-item macro (load-and-run) */
  uint64_t bytes;           /* bytes copied host -> device (AP_STAGE_COPY), else 0 */
  double start_ms, end_ms;  /* from the start of the traced call */
} ap_trace_event;

/* ap_set_trace -- turn the task trace of the handle's later calls on (1) or
 * off (0).  Each traced call replaces the previous call's trace.
 * Errors: AP_ERR_INVALID_ARG (NULL handle, on not 0/1). */
ap_status ap_set_trace(ap_items *items, int32_t on);

/* ap_get_trace -- the last traced call's tasks: waits until they have run,
 * writes min(cap, *count) events to out (host, caller-owned) in the order
 * they were issued and sets *count to the number recorded (0 when nothing was
 * traced).  Errors: AP_ERR_INVALID_ARG (NULL handle or count, out NULL with
 * cap > 0), AP_ERR_CUDA. */
ap_status ap_get_trace(ap_items *items, ap_trace_event *out, int64_t cap, int64_t *count);

/* Static, NUL-terminated description of a status code. */
const char *ap_status_string(ap_status s);

/* Name of the CUDA error behind the calling thread's most recent AP_ERR_CUDA
 * or AP_ERR_OOM return (e.g. "cudaErrorInvalidValue"); "" if there was none.
 * Static string; diagnostic only. */
const char *ap_last_cuda_error(void);

/* Code recorded by a bounded device wait that ran out during the handle's
 * last synchronised call (0 = none); also cleared by this call. */
int32_t ap_last_device_error(ap_items *items);

/* n(n-1)/2 (Sec. VI-A); 0 for n < 2. */
int64_t ap_pair_count(int64_t n);

/* Packed index of (i, j), 0 <= i < j < n; -1 otherwise. */
int64_t ap_pair_index(int64_t i, int64_t j, int64_t n);

/*
 * ap_plan_tiles -- host-side tile list of the schedule: the upper triangle of
 * an n x n item grid cut into square blocks of `block` items, the block pairs
 * (I, J) with I <= J listed in recursive quadrant order (Sec. IV-B: split into
 * four quadrants, recurse, skip empty quadrants).  Writes (I, J) pairs to
 * out[2k], out[2k+1] for k < *n_tiles when cap suffices.
 * Errors: AP_ERR_INVALID_ARG (n < 0, block < 1, n_tiles NULL, out NULL with
 * cap > 0); *n_tiles is always set to the required count.
 */
ap_status ap_plan_tiles(int64_t n, int32_t block, int32_t *out, int64_t cap,
                        int64_t *n_tiles);

/*
 * ap_pipe_rate -- measured issue rate of one SM pipe on the current device,
 * the denominator of the CUDA-core kernels' rooflines (measurement support;
 * the paper reports no kernel-level rates and has no counterpart).
 *   pipe 0: FP32 fused multiply-add (FMA results; 2 flops each),
 *   pipe 1: MUFU ex2.approx results, pipe 2: MUFU rcp.approx results,
 *   pipe 3: packed FP32x2 fused multiply-add (FMA results, two per
 *           instruction).
 * Every SM runs 64 warps of eight independent chains of the instruction for a
 * few milliseconds (synchronous, legacy default stream; one small temporary
 * device allocation).  Writes results per clock per SM (from the SMs' cycle
 * counters), results per second over the whole GPU (CUDA events) and, if
 * sm_mhz is not NULL, the SM clock seen during the run.  Changes no GPU
 * setting.  Errors: AP_ERR_INVALID_ARG (unknown pipe, NULL outputs),
 * AP_ERR_CUDA / AP_ERR_OOM.
 */
ap_status ap_pipe_rate(int32_t pipe, double *per_clk_per_sm, double *per_s, double *sm_mhz);

/*
 * ap_pearson_fp32_noalloc -- all-pairs Pearson correlation on the plain FP32
 * CUDA-core path, for callers that cannot let the library allocate GPU
 * memory: processes whose device memory is handed out by their own pool
 * allocator (a cudaMalloc behind its back can fail or fragment the pool), and
 * services with a hard per-request memory limit.  The paper has no
 * counterpart; this is an addition of this library.
 *   data: device float[n_items][ld] (row-major, dim <= ld values per row,
 *         ld = 0 means ld = dim), caller-owned, read only;
 *   out:  device double[n_items(n_items-1)/2], packed as above, written.
 * Same arithmetic as ap_run_pairs(AP_FN_PEARSON, AP_PREC_FP32): FP64 mean and
 * norm per item, FP32 centring and Gram, FP64 scaling.  It calls no
 * cudaMalloc, cudaFree or other allocating routine: its working memory (item
 * means, inverse norms, the tile-queue counter) is one file-scope
 * `static __device__` array of AP_NOALLOC_SCRATCH_BYTES bytes that every GPU
 * loading the library keeps until the process exits.
 *   - At most AP_NOALLOC_MAX_ITEMS items; more returns AP_ERR_UNSUPPORTED
 *     before any device work.  dim < 2, ld < dim, NULL data/out with n >= 2
 *     return AP_ERR_INVALID_ARG.  n < 2 returns AP_OK and touches nothing.
 *   - The first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array (its queue counter is reset at the start
 *     of every call): calls whose work overlaps on the GPU -- on different
 *     streams, or from different threads -- race and give wrong results.
 *     Serialise them, e.g. on one stream.
 */
#define AP_NOALLOC_MAX_ITEMS 65536
#define AP_NOALLOC_SCRATCH_BYTES (256 + 2 * 8 * AP_NOALLOC_MAX_ITEMS)
ap_status ap_pearson_fp32_noalloc(const float *data, int64_t n_items, int64_t dim, int64_t ld,
                                  double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* ALLPAIRS_H */
