// ap_internal.h -- internal declarations of the all-pairs library.
//
// Storage kept by a handle, the launch wrappers of each kernel family and the
// host planners.  Nothing here is part of the C ABI (see allpairs.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "allpairs.h"

namespace ap {

// ---------------------------------------------------------------------------
// status word written by bounded device waits (AP device error codes)
// ---------------------------------------------------------------------------
enum DeviceError : int32_t {
  DEV_OK = 0,
  DEV_TIMEOUT_FULL = 1,     // consumer gave up waiting for a stage to fill
  DEV_TIMEOUT_EMPTY = 2,    // producer gave up waiting for a stage to drain
  DEV_TIMEOUT_ACCUM = 3,    // epilogue gave up waiting for the accumulator
  DEV_TIMEOUT_STAGE = 4,    // a bulk copy of item data did not land
  DEV_TIMEOUT_SLOT = 5,     // a slot-ready flag was never raised
  DEV_TIMEOUT_UNIT = 6,     // a CTA pair's unit hand-out ring did not advance
};

// wall-clock budget of one device wait (nanoseconds, %globaltimer)
constexpr unsigned long long kWaitBudgetNs = 2000000000ull;   // 2 s

// ---------------------------------------------------------------------------
// packed upper-triangle index, p(i,j) = i*n - i(i+1)/2 + (j-i-1)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t pair_index(int64_t i, int64_t j, int64_t n) {
  return i * n - (i * (i + 1)) / 2 + (j - i - 1);
}

// ---------------------------------------------------------------------------
// point-cloud storage: items sorted by the planner, padded to a multiple of
// 4 points; 2-D points packed as float4 {x, y, s2k, lw}, 3-D as
// float4 {x, y, z, s2k} plus float lw[], where s2k = sigma^2 / (log2(e)/2)
// and lw = log2(weight) (-inf for padding), so that
//   w_b * exp(-d^2 / (2 (sa^2 + sb^2))) = 2^(lw_b - d^2 / (s2k_a + s2k_b)).
// ---------------------------------------------------------------------------
struct CloudStore {
  int dim = 2;
  int64_t n = 0;
  bool unit_weights = true;
  std::vector<int64_t> h_size;      // points per item (original order)
  std::vector<int32_t> h_perm;      // storage position -> original item id
  std::vector<int64_t> h_poff;      // padded offsets in storage order [n+1]
  int64_t total_pts = 0;            // padded
  float4 *d_pts = nullptr;          // [total_pts]
  float *d_lw = nullptr;            // [total_pts] (3-D with weights only)
  int64_t *d_poff = nullptr;        // [n+1]
  int32_t *d_cnt = nullptr;         // [n] real points per stored item
  int32_t *d_perm = nullptr;        // [n]
  // tile plan (rebuilt when the tuned parameters change)
  int32_t block_items = 0, block_pts = 0, reg_r = 0;
  int32_t max_rj = 0;               // most row jobs (chunks of 32 reg_r points) of a block
  bool sorted = false;
  // pair lists: tiles are listed pairs of one-item blocks, outputs by list
  // position (set only on the temporary copy a list run launches with)
  bool list_mode = false;
  std::vector<int32_t> h_iperm;     // original item id -> storage position
  int32_t *d_bstart_single = nullptr;   // [n + 1]: block b = item b
  int32_t *d_list_tiles = nullptr;  // [list_cap][2] storage positions
  int64_t list_cap = 0;
  std::vector<int32_t> h_bstart;    // block b = storage items [bstart[b], bstart[b+1])
  int32_t *d_bstart = nullptr;
  int32_t *d_tiles = nullptr;       // [n_tiles][2] block pairs (I <= J)
  int64_t n_tiles = 0;
  int64_t tiles_cap = 0;
  // particle scores: re-scaled storage per score (index score - 1), built on
  // first use, and the GMM L2 self terms per original item
  float4 *d_pts_score[2] = {nullptr, nullptr};
  float *d_lw_score[2] = {nullptr, nullptr};
  double *d_self = nullptr;
};

// one macro pair (a <= b) of an out-of-core batch and the slots holding them
struct OocPair { int32_t a, b, slot_a, slot_b; };
// one step of the out-of-core schedule: loads (macro, slot), then a Gram batch
struct OocStep {
  std::vector<std::pair<int32_t, int32_t>> loads;
  std::vector<OocPair> pairs;
  int64_t unit0 = 0, n_units = 0, cover0 = 0, n_cover = 0;
};

// ---------------------------------------------------------------------------
// dense-vector storage
// ---------------------------------------------------------------------------
constexpr int64_t kOocMacroItems = 256;   // items per device / host cache slot

// the second-level (host) cache of decoded macros and its parse threads
// (hostcache.cu)
struct HostCacheRelease;
struct HostCache {
  struct Impl;
  int64_t n = 0, dim = 0, n_slots = 0;
  size_t slot_floats = 0;
  const uint8_t *const *blobs = nullptr;
  const uint64_t *blob_bytes = nullptr;
  int32_t codec = 0;
  float *pinned = nullptr;                 // [n_slots][256][dim]
  Impl *impl = nullptr;
  HostCacheRelease *release_args = nullptr;
  // counters (under the lock)
  int64_t hits = 0, misses = 0, parsed_rows = 0;
  bool bad_input = false;
  ~HostCache();
  ap_status init(int64_t n_items, int64_t dim, const uint8_t *const *blobs,
                 const uint64_t *bytes, int32_t codec, int64_t slots, int threads);
  void announce(const std::vector<int64_t> &macros);   // the run's requests, in order
  int acquire(int64_t macro);                           // a ready slot, held
  void release(int slot);
  const float *slot_ptr(int slot) const { return pinned + (size_t)slot * slot_floats; }
  void *release_arg(int slot);
  static void CUDART_CB release_cb(void *arg);          // cudaLaunchHostFunc target
  void worker();
  void pump();
};
int64_t xor_varint_encode(const float *x, int64_t dim, uint8_t *out, uint64_t cap);
bool xor_varint_decode(const uint8_t *in, uint64_t len, int64_t dim, float *x);

struct VecStore {
  int64_t n = 0, D = 0, ld = 0;
  int64_t Dp = 0;                   // padded row length (multiple of 64)
  uint32_t precisions = 0;
  double *d_mu = nullptr, *d_ss = nullptr, *d_rs = nullptr;   // FP64 per item (d_mu: the shift)
  double *d_delta_all = nullptr;    // mean - shift per item
  double *d_partc = nullptr;        // [n][kSplitParts] partial sums of c
  int32_t *d_recentre = nullptr;    // [n + 1]: count, rows centred again
  double *d_part = nullptr;         // [n][kSplitParts] partial sums of c^2
  int64_t n_rows_alloc = 0;         // rows rounded up to the row block
  __nv_bfloat16 *d_hi = nullptr, *d_lo = nullptr;              // [n][Dp]
  float *d_c32 = nullptr;                                      // [n][Dp]
  uint32_t *d_rows = nullptr;       // [n][Dp] row-major copy for long pair lists
  float *d_stage = nullptr;         // raw rows staged from the host
  int64_t stage_rows = 0;
  // out-of-core mode: HBM slot cache of 256-item macros
  bool out_of_core = false;
  const float *h_src = nullptr;
  HostCache *host = nullptr;        // encoded items: decoded macros in pinned host slots
  uint64_t slot_cache_bytes = 0;
  int64_t n_macros = 0, n_slots = 0, group = 0, ring = 0;
  __nv_bfloat16 *d_pool_hi = nullptr, *d_pool_lo = nullptr;   // slot pool, blocked layout
  float *d_raw = nullptr;                                      // raw staging ring
  std::vector<cudaEvent_t> ev_raw_ready, ev_raw_free, ev_prepped;
  std::vector<int> ring_used;
  std::vector<OocStep> steps;
  int32_t *d_units = nullptr, *d_cover_units = nullptr;
  void *tmap_pool_hi = nullptr, *tmap_pool_lo = nullptr;
  int64_t ooc_loads = 0, ooc_uses = 0;
  // out-of-core, column-sliced schedule (AP_OOC_K_SLICED): every item's
  // chunk of slice_cols columns resident at once in one chunk buffer ([0])
  int32_t ooc_policy = 0;
  int64_t slice_cols = 0, n_slices = 0;
  __nv_bfloat16 *d_slice_hi[2] = {nullptr, nullptr}, *d_slice_lo[2] = {nullptr, nullptr};
  void *tmap_slice_hi[2] = {nullptr, nullptr}, *tmap_slice_lo[2] = {nullptr, nullptr};
  double *d_shift = nullptr, *d_part_c = nullptr, *d_delta = nullptr;
  int32_t *d_slice_units = nullptr; int64_t n_slice_units = 0;
  int32_t *d_slice_cover = nullptr; int64_t n_slice_cover = 0;   // one unit per tile
  cudaEvent_t ev_slice_ready[2] = {nullptr, nullptr}, ev_slice_done[2] = {nullptr, nullptr};
  // streamed load-and-run of a resident set: per macro column m, the split-K
  // units of the pairs (a <= m, m) on the resident blocked arrays
  // With stream_chunks > 1 the columns go in chunks of stream_chunk_cols,
  // and entry c * macros + m holds the units of macro column m over chunk c
  int32_t *d_stream_units = nullptr;
  std::vector<std::pair<int64_t, int64_t>> stream_cols;   // (first unit, units)
  int64_t stream_chunks = 0, stream_chunk_cols = 0;
  // tile plans
  int32_t *d_tiles_tc = nullptr;  int64_t n_tiles_tc = 0;
  // k_split > 0: the tiles run as split-K units in waves (panel_units)
  int32_t k_split = 0;
  int32_t *d_panel_units = nullptr; int64_t n_panel_units = 0;
  // mma_ctas = 2: the same schedule on CTA pairs (gram_tc2.cu): split-K units
  // in waves of tc2_pairs() macro pairs, and one unit per macro pair (whole
  // columns: k_split = 0 and coverage)
  int32_t mma_ctas = 2;
  int32_t *d_pair_units = nullptr; int64_t n_pair_units = 0;
  int32_t *d_pair_whole = nullptr; int64_t n_pair_whole = 0;
  std::vector<int32_t> h_tiles_tc;
  int32_t *d_tiles_f32 = nullptr; int64_t n_tiles_f32 = 0;
  void *tmap_hi = nullptr, *tmap_lo = nullptr;   // CUtensorMap (host copies)
  double *d_g64 = nullptr;          // FP64 partial sums of the tensor-core Gram
};

}  // namespace ap

namespace ap {
// task trace of a streamed pipeline (ap_set_trace): CUDA events at the start
// and end of every task, on the stream that runs it
struct TraceRec {
  int32_t stream = 0, stage = 0;
  int64_t index = 0;
  uint64_t bytes = 0;
  cudaEvent_t a = nullptr, b = nullptr;
};
struct Tracer {
  bool on = false;
  cudaEvent_t base = nullptr;
  std::vector<TraceRec> recs;
  void clear();
  // a new trace whose time zero is now on s (no-op when tracing is off)
  cudaError_t start(cudaStream_t s);
  // open a task on st; returns its record (-1 when off)
  int begin(int32_t stream, int32_t stage, int64_t index, uint64_t bytes, cudaStream_t st);
  void end(int rec, cudaStream_t st);
  ~Tracer() { clear(); }
};
// host-side range for tools that show NVTX (the enqueue of one stage)
struct NvtxRange {
  explicit NvtxRange(const char *name);
  ~NvtxRange();
};
}  // namespace ap

namespace ap {
// a captured launch sequence, replayed with cudaGraphLaunch
struct GraphKey {
  int32_t kind;                    // 1 overlap, 2 coverage, 3 ascent, 4 L2, 5 Bhattacharyya
  const void *a, *b, *c, *d;       // buffers the sequence reads / writes
  float eta, fmin;
  int32_t n;
  bool operator==(const GraphKey &o) const {
    return kind == o.kind && a == o.a && b == o.b && c == o.c && d == o.d && eta == o.eta &&
           fmin == o.fmin && n == o.n;
  }
};
struct GraphEntry {
  GraphKey key;
  uint64_t plan_version;
  cudaGraphExec_t exec;
};
}  // namespace ap

namespace ap {
// sparse vectors in CSR form over an index space of `dim` codes, cut into
// chunks of kSparseChunk codes; cptr[c][i] = first entry of row i with a
// code >= c * kSparseChunk, relative to the row's start (chunk-major, so the
// bounds of 32 consecutive rows in one chunk are one coalesced load)
constexpr int kSparseChunk = 4096;
constexpr int kSparseBlock = 32;     // items i of a tile
constexpr int kSparseBlockJ = 64;    // items j of a tile
struct SparseStore {
  int64_t n = 0, dim = 0, nnz = 0, n_chunks = 0;
  int64_t *d_off = nullptr;
  int32_t *d_idx = nullptr;
  float *d_val = nullptr;
  int32_t *d_cptr = nullptr;        // [n_chunks + 1][n]
  double *d_rs = nullptr;           // 1 / sqrt(sum of squares), NaN for none
  int32_t *d_tiles = nullptr;       // block pairs (I <= J) of 32 items
  int64_t n_tiles = 0;
  // per block of 32 items: the item (0..31) each row slot j of a tile takes;
  // slots w and w + 16 (one warp) pair a heavy row with a light one
  int32_t *d_jperm = nullptr;
};
}  // namespace ap

struct ap_items {
  int32_t kind = 0;
  int device = 0;
  ap::CloudStore cl;
  ap::VecStore vec;
  ap::SparseStore sp;
  int32_t *d_status = nullptr;      // [0] device error code, [1..] scratch
  int32_t *d_queue = nullptr;       // tile-queue heads (one per launch slot)
  float *d_scratch = nullptr;       // generic scratch
  int64_t scratch_bytes = 0;
  ap_run_stats stats{};
  int32_t last_dev_error = 0;
  cudaStream_t copy_stream = nullptr;
  cudaStream_t prep_stream = nullptr;    // pre-processing of streamed macros (load-and-run)
  cudaStream_t graph_stream = nullptr;   // private stream the graphs are captured on
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  uint64_t plan_version = 0;
  uint64_t wait_budget_ns = 0;          // 0 = the default budget
  int32_t debug = 0;                    // failure-path testing switches
  ap::Tracer trace;                     // task trace of the streamed pipelines
  std::vector<ap::GraphEntry> graphs;
};

namespace ap {

// ---------------------------------------------------------------------------
// host planners (plan.cpp)
// ---------------------------------------------------------------------------
// Upper-triangle block pairs (I <= J) of an nb x nb block grid in recursive
// quadrant order (split in four, recurse, skip empty quadrants).
void dc_block_pairs(int64_t nb, std::vector<int32_t> &out);
// Group storage-ordered items into blocks of at most max_items items and
// max_pts padded points (an item larger than max_pts forms its own block).
// Blocks also respect max_chunks = sum over items of ceil(cnt / chunk).
void make_blocks(const std::vector<int64_t> &poff, const std::vector<int64_t> &cnt,
                 int32_t max_items, int64_t max_pts, int64_t chunk, int64_t max_chunks,
                 std::vector<int32_t> &bstart);

// ---------------------------------------------------------------------------
// kernel launchers
// ---------------------------------------------------------------------------
// vectors (vec.cu)
// Blocked layout of the pre-processed copies: rows in blocks of 128 items,
// columns in blocks of kblk; one (row block, column block) tile is a
// contiguous 128 x kblk array, so every tile load is one contiguous run.
constexpr int kRowBlock = 128;
constexpr int kTcKBlock = 32;     // bf16 columns per block (64 bytes per row)
constexpr int kF32KBlock = 16;    // fp32 columns per block (64 bytes per row)
constexpr int kSplitParts = 16;   // FP64 partials of sum c^2 and sum c per row
__host__ __device__ __forceinline__ size_t blocked_offset(int64_t row, int64_t k, int64_t nkb,
                                                          int kblk) {
  return ((size_t)(row / kRowBlock) * nkb + (size_t)(k / kblk)) * ((size_t)kRowBlock * kblk) +
         (size_t)(row % kRowBlock) * kblk + (size_t)(k % kblk);
}
cudaError_t launch_vec_mean(const float *X, int64_t n, int64_t D, int64_t ld, double *mu,
                            cudaStream_t s);
// the single-pass load pipeline of vectors: per row a shift (the mean of
// evenly spread samples), then the centred split / FP32 copies and the FP64
// sums of c and c^2 in one pass, then delta = mean - shift, ss and rs; rows
// whose shift missed the mean by D delta^2 > ss / 64 are redone from the
// exact mean.  recentre: device int32 [n + 1] scratch (count, rows).
cudaError_t launch_vec_prep(const float *X, int64_t row0, int64_t out_row0, int64_t n, int64_t D,
                            int64_t ld, int64_t Dp, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                            float *c32, double *shift, double *part, double *part_c,
                            double *delta, double *ss, double *rs, int32_t *recentre,
                            cudaStream_t s);
// out[p] -= (D delta_i rs_i)(delta_j rs_j) over the packed triangle: the
// mean correction of pairs the Gram kernel already scaled by rs_i rs_j
cudaError_t launch_pair_correct(double *out, const double *rs, const double *delta, int64_t n,
                                int64_t D, cudaStream_t s);
// out[p] = (out[p] - D delta_i delta_j) rs_i rs_j over the packed triangle
cudaError_t launch_pair_finalize(double *out, const double *rs, const double *delta, int64_t n,
                                 int64_t D, cudaStream_t s);
// columns [col0, col0 + width) of rows row0.. (cols of them real, staged
// with leading dimension ld) centred on per-row shifts and split into blocked
// copies Dl columns wide; FP64 partials of c and c^2 accumulated per row
cudaError_t launch_vec_split_cols(const float *X, int64_t row0, int64_t n, int64_t cols,
                                  int64_t ld, int64_t width, int64_t col0, int64_t Dl,
                                  const double *shift, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                  float *c32, double *part, double *part_c, int first_chunk,
                                  cudaStream_t s);
// per-row shifts of rows read where they are (X may be pinned host memory
// the device can address): the mean of 32 evenly spaced runs of 32 values
cudaError_t launch_vec_shift_runs(const float *X, int64_t n, int64_t D, int64_t ld,
                                  double *shift, cudaStream_t s);
// one column chunk [.., cols) of rows row0.., centred on per-row shifts (the
// rows' blocked copies hold cols_p >= cols columns); FP64 partials of
// sum c^2 and sum c are set (first_chunk) or accumulated per row
cudaError_t launch_vec_split_slice(const float *X, int64_t row0, int64_t n, int64_t cols,
                                   int64_t ld, int64_t cols_p, const double *shift,
                                   __nv_bfloat16 *hi, __nv_bfloat16 *lo, double *part,
                                   double *part_c, int first_chunk, cudaStream_t s);
// after the last chunk: delta_i = mu_i - s_i, ss, rs, and
// out[p] = (out[p] - D delta_i delta_j) rs_i rs_j
cudaError_t launch_slice_finalize(const double *part, const double *part_c, int64_t n,
                                  int64_t D, double *delta, double *ss, double *rs, double *out,
                                  cudaStream_t s);
cudaError_t launch_gram_f32(const float *C, int64_t n, int64_t Dp, const double *rs,
                            const int32_t *tiles, int64_t n_tiles, int32_t *queue,
                            void *out, int coverage, int64_t row0, int64_t n_total,
                            cudaStream_t s, const double *delta = nullptr,
                            int64_t D = 0);
// tensor-core split-BF16 Gram (gram_tc.cu)
constexpr int kTcTileM = 128;    // rows of the I block per tile
constexpr int kTcTileN = 256;    // rows of the J block per tile
cudaError_t make_tc_tensor_maps(const __nv_bfloat16 *hi, const __nv_bfloat16 *lo,
                                int64_t n, int64_t Dp, void **tmap_hi, void **tmap_lo);
cudaError_t launch_gram_tc(const void *tmap_hi, const void *tmap_lo, int64_t n, int64_t Dp,
                           const double *rs, const int32_t *tiles, int64_t n_tiles,
                           int32_t *queue, int32_t *status, double *g64, void *out,
                           int coverage, int ooc, uint64_t budget, int32_t debug,
                           cudaStream_t s);
// split-BF16 Gram on CTA pairs (gram_tc2.cu): units of kOocTileInts int32
// {A row block of CTA 0, of CTA 1, B row block of CTA 0, of CTA 1, first row
// block (128 items) of the I block, J block (256 items), first chunk, end
// chunk}; atomic = 1 adds partial Grams into FP64 out, 0 writes G rs_i rs_j
// of whole block pairs, coverage = 1 counts pairs into int32 out.
cudaError_t launch_gram_tc2(const void *tmap_hi, const void *tmap_lo, int64_t n, const double *rs,
                            const int32_t *units, int64_t n_units, int32_t *queue,
                            int32_t *status, double *g64, void *out, int coverage, int atomic,
                            uint64_t budget, int32_t debug, cudaStream_t s);
// CTA pairs of one launch (clusters of two that fit on the device at once)
int64_t tc2_pairs();
// units of the CTA-pair Gram over the resident set: macro pairs (I <= J, 256
// items each) in recursive quadrant order, in waves of `group` macro pairs,
// k_split column ranges of the nchunks 64-column chunks per wave (k_split <= 1:
// one unit per macro pair over all columns)
void pair_units(int64_t n, int64_t nchunks, int64_t group, int64_t k_split,
                std::vector<int32_t> &units);
// the same for a given list of macro pairs (I, J) in the order to run them
void pair_units_of(const std::vector<int32_t> &macro_pairs, int64_t nchunks, int64_t group,
                   int64_t k_split, std::vector<int32_t> &units);
// out-of-core unit: {A row block, B row blocks (2), I block, J block, chunk
// begin, chunk end, unused}; chunks are 64 columns of D
constexpr int kOocTileInts = 8;
constexpr int kOocChunkCols = 64;
constexpr int kMaxKSplit = AP_MAX_K_SPLIT;
constexpr int64_t kKSplitCols = 16384;   // target columns per split-K unit
// CTAs of one Gram launch and the FP64 scratch (doubles) it needs: one
// 128 x 256 FP64 partial-sum tile per CTA
int64_t tc_grid(int64_t n_tiles);
size_t tc_scratch_doubles(int64_t n_tiles);
void free_tc_tensor_maps(void *tmap_hi, void *tmap_lo);
void tc_tiles(int64_t n, std::vector<int32_t> &tiles);   // (I-block of 128, J-block of 256)
// cloud tiles of a set whose points take under 16 MB: reordered largest
// first (point pairs per tile); returns whether it reordered
bool order_cloud_tiles(const std::vector<int32_t> &bstart, const std::vector<int64_t> &cnt,
                       int64_t total_pts, std::vector<int32_t> &tiles);
// the most row jobs (chunks of `chunk` points) any block of a cloud plan has
int32_t max_row_jobs(const std::vector<int32_t> &bstart, const std::vector<int64_t> &cnt,
                     int64_t chunk);
// split-K units of the tiles: waves of `group` tiles, column range-major
// inside each wave (k_split ranges of the nchunks 64-column chunks)
void panel_units(const std::vector<int32_t> &tiles, int64_t nchunks, int64_t group,
                 int64_t k_split, std::vector<int32_t> &units);
// the split-K schedule of a vector set's split-BF16 Gram: k_split column
// ranges per tile (0 whole tiles, -1 the default rule of default_k_split)
int32_t default_k_split(int64_t n_tiles, int64_t Dp);
ap_status set_vector_plan(ap_items *it, int32_t k_split, int32_t mma_ctas = 0);

// the particle scores' re-scaled cloud storage and L2 self terms, built on
// first use (api.cu)
ap_status ensure_score_storage(ap_items *it, int score, cudaStream_t s);
// pair lists (pairlist.cu): Pearson of listed pairs over the resident rows
// (pairs sorted by row block, pos = each result's position in the caller's
// list; blocks = the n_blocks distinct row blocks the list touches)
cudaError_t launch_pearson_list(VecStore &v, bool split, const int32_t *pi,
                                const int32_t *pj, const int32_t *pos, int64_t n_pairs,
                                const int32_t *blocks, int64_t n_blocks, double *out,
                                cudaStream_t s);

// clouds (overlap.cu)
cudaError_t launch_overlap(const CloudStore &cs, const float *params, float *out,
                           int coverage, int32_t *queue, cudaStream_t s);
// adjoint (params_io == NULL: grad_params = grad_out * grad f) or one fused
// ascent step (params_io != NULL: params_io += eta grad f / f where f >= fmin)
cudaError_t launch_overlap_grad_q(const CloudStore &cs, int32_t *queue, const float *params,
                                  const float *grad_out, float *grad_params, float *f_out,
                                  float eta, float fmin, float *params_io, int32_t *flags,
                                  cudaStream_t s);
// particle scores (score 1 GMM L2 distance, 2 Bhattacharyya cost) on the
// re-scaled storage pts / lw; self = the L2 self terms (score 1)
cudaError_t launch_score(const CloudStore &cs, int score, const float4 *pts, const float *lw,
                         const double *self, const float *params, float *out, int32_t *queue,
                         cudaStream_t s);
cudaError_t launch_cloud_rescore(const CloudStore &cs, int score, float4 *pts_out, float *lw_out,
                                 cudaStream_t s);
cudaError_t launch_cloud_self(const CloudStore &cs, const float4 *pts, const float *lw,
                              double *self, cudaStream_t s);
// sparse vectors (sparse.cu)
ap_status create_sparse(const ap_items_desc *d, ap_items *it, cudaStream_t s);
void free_sparse(SparseStore &sp);
cudaError_t launch_sparse_cosine(const SparseStore &sp, double *out, int coverage,
                                 int32_t *queue, cudaStream_t s);
constexpr int kOverlapMaxRowJobs = 128;   // chunks of one I block
constexpr int kOverlapMaxBlockItems = 32;
cudaError_t launch_cloud_pack(const float *x, const float *y, const float *z,
                              const float *sigma, const float *w, const int64_t *src_off,
                              const int32_t *perm, const int64_t *poff, int64_t n, int dim,
                              float4 *pts, float *lw, cudaStream_t s);

int num_sms();

// ---------------------------------------------------------------------------
// shared host helpers (api.cu, tune.cu)
// ---------------------------------------------------------------------------
ap_status from_cuda(cudaError_t e);
// propagate an ap_status
#define AP_TRY_ST(expr)                            \
  do {                                             \
    ap_status _s = (expr);                         \
    if (_s != AP_OK) return _s;                    \
  } while (0)

#define AP_TRY(expr)                               \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) return ::ap::from_cuda(_e); \
  } while (0)
template <typename T>
cudaError_t dmalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
}
template <typename T>
void dfree(T *&p) {
  if (p) cudaFree(reinterpret_cast<void *>(p));
  p = nullptr;
}

struct CloudPlanChoice { int32_t block_items, block_pts, reg_r; bool sorted; };
CloudPlanChoice choose_cloud_plan(const CloudStore &c);
ap_status build_cloud_plan(ap_items *it, const CloudPlanChoice &ch, cudaStream_t s = nullptr);
// smallest a-points-per-lane that keeps the largest item within the row jobs
int32_t min_reg_r(const CloudStore &c);

// Launch `seq` on `s` through a cached CUDA graph captured on the handle's
// private stream (direct launch when `s` is itself being captured).
ap_status run_graphed(ap_items *it, const GraphKey &key, cudaStream_t s,
                      const std::function<cudaError_t(cudaStream_t)> &seq);
void clear_graphs(ap_items *it);

// out-of-core vector sets (slotcache.cu)
ap_status create_out_of_core(const ap_items_desc *d, ap_items *it);
ap_status run_out_of_core(ap_items *it, void *out, int coverage, cudaStream_t s);
void free_out_of_core(VecStore &v);
// host source streamed macro by macro into a resident set, each macro's pairs
// computed as soon as it is pre-processed (slotcache.cu)
ap_status stream_load_and_run(ap_items *it, const float *h, double *out, cudaStream_t s);

}  // namespace ap
