// slotcache.cu -- out-of-core vector sets: an HBM slot cache refilled
// asynchronously from page-locked host memory (the first-level device cache
// of Sec. IV-A with the asynchronous, overlapped loading of Sec. IV-C).
//
// Unit of caching: a "macro" of 256 consecutive items, stored pre-processed
// (split-BF16 hi/lo, blocked layout) in one slot of a pool; the Gram's tile
// (128 items x 256 items) reads its A half-macro and its B macro straight out
// of the pool through 4-D tensor maps whose row-block coordinate is
// 2*slot + half.
//
// Schedule (host, computed once, the future fully known): a resident set A
// of S - g macros is loaded and its pairs computed, then the remaining
// macros stream through the other g slots in groups; every pair of A with
// the streamed groups is done on the way, and the remaining macros are
// handled the same way.  A slot is given up by the macro needed farthest in
// the future (or never again), which is the schedule-aware form of the
// paper's least-recently-used eviction.  A load is: copy the macro's raw FP32
// rows from the host into a staging ring (copy stream), then pre-process them
// into the slot on the compute stream.  Copies for the next group run while
// the current group's Gram runs; the compute stream only waits for its own
// loads.  Each batch's tiles are split along D into units so even a small
// batch fills every SM; units add their FP64 partial Gram into the packed
// output, and a final pass scales by 1 / sqrt(ss_i ss_j).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <numeric>
#include <set>
#include <vector>

#include "ap_internal.h"

namespace ap {

namespace {

constexpr int64_t kMacro = 2 * kRowBlock;   // items per slot

}  // namespace


static void free_raw_ring(VecStore &v) {
  dfree(v.d_raw);
  for (cudaEvent_t e : v.ev_raw_ready) cudaEventDestroy(e);
  for (cudaEvent_t e : v.ev_raw_free) cudaEventDestroy(e);
  for (cudaEvent_t e : v.ev_prepped) cudaEventDestroy(e);
  v.ev_raw_ready.clear();
  v.ev_raw_free.clear();
  v.ev_prepped.clear();
  v.ring_used.clear();
  v.ring = 0;
}

static ap_status alloc_raw_ring(VecStore &v, int64_t ring, size_t floats_each) {
  v.ring = ring;
  AP_TRY(dmalloc(&v.d_raw, (size_t)ring * floats_each));
  for (int64_t b = 0; b < ring; ++b) {
    cudaEvent_t a, f;
    AP_TRY(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    v.ev_raw_ready.push_back(a);
    AP_TRY(cudaEventCreateWithFlags(&f, cudaEventDisableTiming));
    v.ev_raw_free.push_back(f);
  }
  v.ring_used.assign(ring, 0);
  return AP_OK;
}

static void free_pool(VecStore &v) {
  dfree(v.d_pool_hi);
  dfree(v.d_pool_lo);
  dfree(v.d_units);
  dfree(v.d_cover_units);
  free_tc_tensor_maps(v.tmap_pool_hi, v.tmap_pool_lo);
  v.tmap_pool_hi = v.tmap_pool_lo = nullptr;
  v.steps.clear();
}

static void free_slices(VecStore &v) {
  for (int b = 0; b < 2; ++b) {
    dfree(v.d_slice_hi[b]);
    dfree(v.d_slice_lo[b]);
    free_tc_tensor_maps(v.tmap_slice_hi[b], v.tmap_slice_lo[b]);
    v.tmap_slice_hi[b] = v.tmap_slice_lo[b] = nullptr;
    if (v.ev_slice_ready[b]) cudaEventDestroy(v.ev_slice_ready[b]);
    if (v.ev_slice_done[b]) cudaEventDestroy(v.ev_slice_done[b]);
    v.ev_slice_ready[b] = v.ev_slice_done[b] = nullptr;
  }
  dfree(v.d_shift);
  dfree(v.d_part_c);
  dfree(v.d_delta);
  dfree(v.d_slice_units);
  dfree(v.d_slice_cover);
  v.n_slice_units = v.n_slice_cover = 0;
}

void free_out_of_core(VecStore &v) {
  delete v.host;
  v.host = nullptr;
  free_pool(v);
  free_slices(v);
  free_raw_ring(v);
  dfree(v.d_stream_units);
  v.stream_cols.clear();
}

// Build the load / compute schedule for M macros and S slots.
static void build_schedule(VecStore &v) {
  const int64_t M = v.n_macros, S = v.n_slots, g = v.group;
  std::vector<int64_t> slot_of(M, -1), macro_in(S, -1);
  std::vector<int64_t> undone(M);
  std::iota(undone.begin(), undone.end(), 0);
  v.steps.clear();

  // position of each macro in the remaining order (for farthest-next-use eviction)
  auto load = [&](int64_t m, const std::set<int64_t> &keep, const std::vector<int64_t> &order,
                  OocStep &st) {
    if (slot_of[m] >= 0) return;
    int64_t victim = -1, best_rank = -1;
    std::vector<int64_t> rank(M, -1);
    for (size_t k = 0; k < order.size(); ++k) rank[order[k]] = (int64_t)k;
    for (int64_t s = 0; s < S; ++s) {
      const int64_t o = macro_in[s];
      if (o < 0) { victim = s; break; }                  // a free slot
      if (keep.count(o)) continue;
      const int64_t r = rank[o] < 0 ? INT64_MAX : rank[o];  // never needed again: best
      if (r > best_rank) { best_rank = r; victim = s; }
    }
    if (macro_in[victim] >= 0) slot_of[macro_in[victim]] = -1;
    macro_in[victim] = m;
    slot_of[m] = victim;
    st.loads.push_back({(int32_t)m, (int32_t)victim});
  };
  auto pairs_among = [&](const std::vector<int64_t> &a, const std::vector<int64_t> &b,
                         bool same, OocStep &st) {
    for (size_t x = 0; x < a.size(); ++x)
      for (size_t y = same ? x : 0; y < b.size(); ++y) {
        const int64_t p = std::min(a[x], b[y]), q = std::max(a[x], b[y]);
        st.pairs.push_back({(int32_t)p, (int32_t)q, (int32_t)slot_of[p], (int32_t)slot_of[q]});
      }
  };

  while (!undone.empty()) {
    // resident macros first: they cost no load
    std::stable_partition(undone.begin(), undone.end(),
                          [&](int64_t m) { return slot_of[m] >= 0; });
    if ((int64_t)undone.size() <= S) {
      OocStep st;
      std::set<int64_t> keep(undone.begin(), undone.end());
      for (int64_t m : undone) load(m, keep, undone, st);
      pairs_among(undone, undone, true, st);
      v.steps.push_back(st);
      break;
    }
    std::vector<int64_t> A(undone.begin(), undone.begin() + (S - g));
    std::vector<int64_t> rest(undone.begin() + (S - g), undone.end());
    std::vector<int64_t> order = A;
    order.insert(order.end(), rest.begin(), rest.end());
    {
      OocStep st;
      std::set<int64_t> keep(A.begin(), A.end());
      for (int64_t m : A) load(m, keep, order, st);
      pairs_among(A, A, true, st);
      v.steps.push_back(st);
    }
    for (size_t k = 0; k < rest.size(); k += g) {
      std::vector<int64_t> G(rest.begin() + k, rest.begin() + std::min(rest.size(), k + g));
      OocStep st;
      std::set<int64_t> keep(A.begin(), A.end());
      keep.insert(G.begin(), G.end());
      std::vector<int64_t> later(rest.begin() + k, rest.end());
      for (int64_t m : G) load(m, keep, later, st);
      pairs_among(A, G, false, st);     // pairs among `rest` are left to the next phase
      v.steps.push_back(st);
    }
    undone = rest;
  }
}

// Expand each step's macro pairs into split-K tile units.
static void build_units(VecStore &v, std::vector<int32_t> &units, std::vector<int32_t> &cover) {
  const int64_t nch = v.Dp / kOocChunkCols;
  for (OocStep &st : v.steps) {
    std::vector<std::array<int32_t, 5>> tiles;   // rb_a, rb_b, ib, jb
    for (const OocPair &pp : st.pairs) {
      for (int h = 0; h < 2; ++h) {
        const int64_t ib = 2LL * pp.a + h, i0 = ib * kRowBlock;
        const int64_t jmax = std::min<int64_t>((int64_t)pp.b * kMacro + kMacro, v.n) - 1;
        if (i0 >= v.n || i0 >= jmax) continue;
        tiles.push_back({2 * pp.slot_a + h, 2 * pp.slot_b, (int32_t)ib, pp.b, 0});
      }
    }
    const int64_t T = (int64_t)tiles.size();
    int64_t ks = T > 0 ? (2LL * num_sms() + T - 1) / T : 1;
    ks = std::max<int64_t>(1, std::min<int64_t>(ks, std::min<int64_t>(32, nch)));
    st.unit0 = (int64_t)units.size() / kOocTileInts;
    st.cover0 = (int64_t)cover.size() / kOocTileInts;
    for (const auto &t : tiles) {
      for (int64_t k = 0; k < ks; ++k) {
        const int32_t c0 = (int32_t)(k * nch / ks), c1 = (int32_t)((k + 1) * nch / ks);
        const int32_t u[kOocTileInts] = {t[0], t[1], t[1] + 1, t[2], t[3], c0, c1, 0};
        units.insert(units.end(), u, u + kOocTileInts);
        if (k == 0) {
          const int32_t cu[kOocTileInts] = {t[0], t[1], t[1] + 1, t[2], t[3], 0, 0, 0};
          cover.insert(cover.end(), cu, cu + kOocTileInts);
        }
      }
    }
    st.n_units = (int64_t)units.size() / kOocTileInts - st.unit0;
    st.n_cover = (int64_t)cover.size() / kOocTileInts - st.cover0;
  }
}

// The paper's policy, for comparison: macro pairs in recursive quadrant
// order (Sec. IV-B), each job loading what it misses into the least recently
// used slot not needed by the job itself (Sec. IV-A-1).  A step ends at every
// miss, so batches are as long as the run of hits.
static void build_schedule_lru(VecStore &v) {
  const int64_t M = v.n_macros, S = v.n_slots;
  std::vector<int64_t> slot_of(M, -1), macro_in(S, -1), last_use(S, -1);
  std::vector<int32_t> order;
  dc_block_pairs(M, order);
  v.steps.clear();
  OocStep cur;
  int64_t clock = 0;
  for (size_t t = 0; t < order.size(); t += 2) {
    const int64_t a = order[t], b = order[t + 1];
    const bool miss = slot_of[a] < 0 || slot_of[b] < 0;
    if (miss && !cur.pairs.empty()) {
      v.steps.push_back(cur);
      cur = OocStep();
    }
    for (int64_t m : {a, b}) {
      if (slot_of[m] >= 0) continue;
      int64_t victim = -1;
      for (int64_t s = 0; s < S; ++s) {
        const int64_t o = macro_in[s];
        if (o < 0) { victim = s; break; }
        if (o == a || o == b) continue;
        if (victim < 0 || last_use[s] < last_use[victim]) victim = s;
      }
      if (macro_in[victim] >= 0) slot_of[macro_in[victim]] = -1;
      macro_in[victim] = m;
      slot_of[m] = victim;
      cur.loads.push_back({(int32_t)m, (int32_t)victim});
    }
    ++clock;
    last_use[slot_of[a]] = clock;
    last_use[slot_of[b]] = clock;
    cur.pairs.push_back({(int32_t)a, (int32_t)b, (int32_t)slot_of[a], (int32_t)slot_of[b]});
  }
  if (!cur.pairs.empty() || !cur.loads.empty()) v.steps.push_back(cur);
}

// Upload the units of v.steps (replacing earlier ones) and count loads/uses.
static ap_status install_schedule(VecStore &v) {
  std::vector<int32_t> units, cover;
  build_units(v, units, cover);
  dfree(v.d_units);
  dfree(v.d_cover_units);
  AP_TRY(dmalloc(&v.d_units, std::max<size_t>(units.size(), kOocTileInts)));
  AP_TRY(dmalloc(&v.d_cover_units, std::max<size_t>(cover.size(), kOocTileInts)));
  if (!units.empty())
    AP_TRY(cudaMemcpy(v.d_units, units.data(), units.size() * 4, cudaMemcpyHostToDevice));
  if (!cover.empty())
    AP_TRY(cudaMemcpy(v.d_cover_units, cover.data(), cover.size() * 4, cudaMemcpyHostToDevice));
  v.ooc_loads = 0;
  v.ooc_uses = 0;
  for (const OocStep &st : v.steps) {
    v.ooc_loads += (int64_t)st.loads.size();
    std::set<int32_t> used;
    for (const OocPair &pp : st.pairs) { used.insert(pp.a); used.insert(pp.b); }
    v.ooc_uses += (int64_t)used.size();
  }
  return AP_OK;
}

// the slot pool of the macro schedules (AP_OOC_RESIDENT_STREAM, AP_OOC_DC_LRU)
static ap_status alloc_pool(VecStore &v) {
  const int64_t pool_rows = 2 * kRowBlock * v.n_slots;
  AP_TRY(dmalloc(&v.d_pool_hi, (size_t)pool_rows * v.Dp));
  AP_TRY(dmalloc(&v.d_pool_lo, (size_t)pool_rows * v.Dp));
  AP_TRY(cudaMemset(v.d_pool_hi, 0, (size_t)pool_rows * v.Dp * 2));
  AP_TRY(cudaMemset(v.d_pool_lo, 0, (size_t)pool_rows * v.Dp * 2));
  AP_TRY_ST(alloc_raw_ring(v, std::max<int64_t>(2, v.group), (size_t)kMacro * v.ld));
  AP_TRY(make_tc_tensor_maps(v.d_pool_hi, v.d_pool_lo, pool_rows, v.Dp, &v.tmap_pool_hi,
                             &v.tmap_pool_lo));
  return AP_OK;
}

// Column slices.  The Gram's CTAs leave no room on an SM for the
// pre-processing kernels, which therefore run between Gram launches; what
// overlaps the Gram of one chunk is the copy of the next.  So: two hi/lo
// chunk buffers of all rows (chunk c + 1 is pre-processed while the Gram of
// chunk c reads the other one) and a raw ring of kMacro-row pieces, a whole
// chunk when the cache allows (at least 64K columns per chunk), else four
// pieces.  Chunk width is a multiple of 64; chunks of equal width cover Dp.
// The link idles only before the first chunk lands and nothing overlaps the
// last chunk's pre-processing and Gram, so more, narrower chunks shorten the
// part of the run that is not copy-bound.
constexpr int64_t kMinSlices = 12;
constexpr int64_t kMinSliceCols = 262144;
static bool slice_geometry(int64_t n, int64_t Dp, uint64_t budget, int64_t *cols,
                           int64_t *count, int64_t *ring) {
  if (n < 1) return false;
  const int64_t rows = (n + kRowBlock - 1) / kRowBlock * kRowBlock;
  const int64_t pieces = (n + kMacro - 1) / kMacro;
  for (int64_t r : {pieces, std::min<int64_t>(pieces, 4)}) {
    const uint64_t per_col = 2ull * 4ull * rows + 4ull * kMacro * r;
    const int64_t cmax = (int64_t)(budget / per_col) / kOocChunkCols * kOocChunkCols;
    const bool last = r == std::min<int64_t>(pieces, 4);
    if (cmax >= std::min<int64_t>(Dp, 65536) || (last && cmax >= kOocChunkCols)) {
      // at least kMinSlices chunks while every row's piece of a chunk stays
      // 1 MiB (256K columns): the last chunk's Gram is the part of the run
      // no copy overlaps, and strided host-to-device copies of shorter row
      // pieces fall below the link rate (256 KiB pieces: 140 GB/s against
      // 211 GB/s for 1 MiB and contiguous copies, measured on GB300)
      *count = std::max<int64_t>((Dp + cmax - 1) / cmax,
                                 std::min<int64_t>(kMinSlices, Dp / kMinSliceCols));
      *cols = ((Dp + *count - 1) / *count + kOocChunkCols - 1) / kOocChunkCols * kOocChunkCols;
      *ring = r;
      return true;
    }
  }
  return false;
}

static ap_status alloc_slices(VecStore &v) {
  int64_t ring = 0;
  if (!slice_geometry(v.n, v.Dp, v.slot_cache_bytes, &v.slice_cols, &v.n_slices, &ring))
    return AP_ERR_INVALID_ARG;
  const int64_t rows = (v.n + kRowBlock - 1) / kRowBlock * kRowBlock;
  const size_t elems = (size_t)rows * v.slice_cols;
  for (int b = 0; b < 2; ++b) {
    AP_TRY(dmalloc(&v.d_slice_hi[b], elems));
    AP_TRY(dmalloc(&v.d_slice_lo[b], elems));
    AP_TRY(cudaMemset(v.d_slice_hi[b], 0, elems * 2));
    AP_TRY(cudaMemset(v.d_slice_lo[b], 0, elems * 2));
    AP_TRY(make_tc_tensor_maps(v.d_slice_hi[b], v.d_slice_lo[b], v.n, v.slice_cols,
                               &v.tmap_slice_hi[b], &v.tmap_slice_lo[b]));
    AP_TRY(cudaEventCreateWithFlags(&v.ev_slice_ready[b], cudaEventDisableTiming));
    AP_TRY(cudaEventCreateWithFlags(&v.ev_slice_done[b], cudaEventDisableTiming));
  }
  AP_TRY(dmalloc(&v.d_shift, (size_t)v.n));
  AP_TRY(dmalloc(&v.d_delta, (size_t)v.n));
  AP_TRY(dmalloc(&v.d_part_c, (size_t)v.n * kSplitParts));
  AP_TRY_ST(alloc_raw_ring(v, ring, (size_t)kMacro * v.slice_cols));
  // every block pair of the triangle on CTA pairs, split-K units in waves
  // over one chunk
  std::vector<int32_t> tiles, units;
  tc_tiles(v.n, tiles);
  const int64_t nt = (int64_t)tiles.size() / 2;
  const int64_t nch = v.slice_cols / kOocChunkCols;
  pair_units(v.n, nch, tc2_pairs(), std::max<int32_t>(1, default_k_split(nt, v.slice_cols)),
             units);
  v.n_slice_units = (int64_t)units.size() / kOocTileInts;
  AP_TRY(dmalloc(&v.d_slice_units, std::max<size_t>(units.size(), kOocTileInts)));
  if (!units.empty())
    AP_TRY(cudaMemcpy(v.d_slice_units, units.data(), units.size() * 4, cudaMemcpyHostToDevice));
  std::vector<int32_t> cover;
  pair_units(v.n, nch, tc2_pairs(), 1, cover);
  v.n_slice_cover = (int64_t)cover.size() / kOocTileInts;
  AP_TRY(dmalloc(&v.d_slice_cover, std::max<size_t>(cover.size(), kOocTileInts)));
  if (!cover.empty())
    AP_TRY(cudaMemcpy(v.d_slice_cover, cover.data(), cover.size() * 4, cudaMemcpyHostToDevice));
  return AP_OK;
}

// The column-sliced run: chunk c of every row is copied (strided, in pieces
// of kMacro rows) on the copy stream, centred on a per-row shift (the mean of
// 32 runs of 32 values spread over the whole row, so that a trend or a period
// does not leave the shift far from the row's mean) and split on the prep stream into chunk buffer c % 2
// once the Gram of chunk c - 2 has finished with it, and the Gram of all
// block pairs over chunk c adds its FP64 partials on s; each item crosses the
// host link once (R = 1).  The shifted-data identities turn the accumulated
// sums into the centred Gram at the end.
static ap_status run_slices(ap_items *it, void *out, int coverage, cudaStream_t s) {
  VecStore &v = it->vec;
  const int64_t P = v.n * (v.n - 1) / 2;
  if (coverage) {
    AP_TRY(launch_gram_tc2(v.tmap_slice_hi[0], v.tmap_slice_lo[0], v.n, v.d_rs, v.d_slice_cover,
                           v.n_slice_cover, it->d_queue, it->d_status, v.d_g64, out, 1, 0,
                           it->wait_budget_ns, it->debug, s));
    it->stats.tiles = v.n_slice_cover;
    it->stats.item_loads = 0;
    it->stats.reuse_R = 0.0;
    it->stats.h2d_bytes = 0;
    it->stats.slot_hit_rate = 1.0;
    return AP_OK;
  }
  if (!it->prep_stream)
    AP_TRY(cudaStreamCreateWithFlags(&it->prep_stream, cudaStreamNonBlocking));
  NvtxRange range("out-of-core column slices");
  Tracer &tr = it->trace;
  AP_TRY(tr.start(s));
  AP_TRY(cudaMemsetAsync(out, 0, (size_t)P * sizeof(double), s));
  AP_TRY(cudaEventRecord(it->ev_a, s));
  AP_TRY(cudaStreamWaitEvent(it->copy_stream, it->ev_a, 0));
  AP_TRY(cudaStreamWaitEvent(it->prep_stream, it->ev_a, 0));
  // per-row shifts from samples spread over each whole row, read from the
  // page-locked source where it is; where the source is not mapped into the
  // device's address space, the mean of the row's first chunk
  const float *d_src = nullptr;
  if (cudaHostGetDevicePointer((void **)&d_src, (void *)v.h_src, 0) != cudaSuccess) {
    cudaGetLastError();
    d_src = nullptr;
  }
  if (d_src) AP_TRY(launch_vec_shift_runs(d_src, v.n, v.D, v.ld, v.d_shift, it->prep_stream));
  std::fill(v.ring_used.begin(), v.ring_used.end(), 0);
  int64_t seq = 0;
  for (int64_t c = 0; c < v.n_slices; ++c) {
    const int b = (int)(c & 1);             // the chunk buffer
    const int64_t c0 = c * v.slice_cols;
    const int64_t cols = std::max<int64_t>(0, std::min<int64_t>(v.slice_cols, v.D - c0));
    NvtxRange chunk_range("chunk: copy + pre-process + Gram");
    if (c >= 2) AP_TRY(cudaStreamWaitEvent(it->prep_stream, v.ev_slice_done[b], 0));
    int t_copy = -1, t_prep = -1;
    for (int64_t r0 = 0; r0 < v.n; r0 += kMacro) {
      const int64_t rows = std::min<int64_t>(kMacro, v.n - r0);
      const int64_t rb = seq++ % v.ring;
      float *raw = v.d_raw + (size_t)rb * kMacro * v.slice_cols;
      if (v.ring_used[rb]) AP_TRY(cudaStreamWaitEvent(it->copy_stream, v.ev_raw_free[rb], 0));
      if (r0 == 0)
        t_copy = tr.begin(1, AP_STAGE_COPY, c, (uint64_t)v.n * cols * 4, it->copy_stream);
      if (cols > 0)
        AP_TRY(cudaMemcpy2DAsync(raw, (size_t)v.slice_cols * 4, v.h_src + (size_t)r0 * v.ld + c0,
                                 (size_t)v.ld * 4, (size_t)cols * 4, (size_t)rows,
                                 cudaMemcpyHostToDevice, it->copy_stream));
      AP_TRY(cudaEventRecord(v.ev_raw_ready[rb], it->copy_stream));
      AP_TRY(cudaStreamWaitEvent(it->prep_stream, v.ev_raw_ready[rb], 0));
      if (r0 == 0) t_prep = tr.begin(2, AP_STAGE_PREPROCESS, c, 0, it->prep_stream);
      if (c == 0 && !d_src)
        AP_TRY(launch_vec_mean(raw, rows, std::max<int64_t>(cols, 1), v.slice_cols,
                               v.d_shift + r0, it->prep_stream));
      AP_TRY(launch_vec_split_slice(raw, r0, rows, cols, v.slice_cols, v.slice_cols, v.d_shift,
                                    v.d_slice_hi[b], v.d_slice_lo[b], v.d_part, v.d_part_c,
                                    c == 0 ? 1 : 0, it->prep_stream));
      AP_TRY(cudaEventRecord(v.ev_raw_free[rb], it->prep_stream));
      v.ring_used[rb] = 1;
    }
    tr.end(t_copy, it->copy_stream);
    tr.end(t_prep, it->prep_stream);
    AP_TRY(cudaEventRecord(v.ev_slice_ready[b], it->prep_stream));
    AP_TRY(cudaStreamWaitEvent(s, v.ev_slice_ready[b], 0));
    const int t_gram = tr.begin(0, AP_STAGE_GRAM, c, 0, s);
    AP_TRY(launch_gram_tc2(v.tmap_slice_hi[b], v.tmap_slice_lo[b], v.n, v.d_rs, v.d_slice_units,
                           v.n_slice_units, it->d_queue, it->d_status, v.d_g64, out, 0, 1,
                           it->wait_budget_ns, it->debug, s));
    tr.end(t_gram, s);
    AP_TRY(cudaEventRecord(v.ev_slice_done[b], s));
  }
  const int t_fin = tr.begin(0, AP_STAGE_FINALIZE, 0, 0, s);
  AP_TRY(launch_slice_finalize(v.d_part, v.d_part_c, v.n, v.D, v.d_delta, v.d_ss, v.d_rs,
                               reinterpret_cast<double *>(out), s));
  tr.end(t_fin, s);
  it->stats.tiles = v.n_slice_units * v.n_slices;
  it->stats.tile_m = 2 * kTcTileM;
  it->stats.tile_n = kTcTileN;
  it->stats.item_loads = v.n;
  it->stats.reuse_R = 1.0;
  it->stats.h2d_bytes = (uint64_t)v.n * v.D * 4;
  it->stats.slot_hit_rate = 1.0;
  return AP_OK;
}

ap_status create_out_of_core(const ap_items_desc *d, ap_items *it) {
  VecStore &v = it->vec;
  if (!d->data_on_host) return AP_ERR_INVALID_ARG;
  if (v.precisions != (1u << AP_PREC_SPLIT_BF16)) return AP_ERR_UNSUPPORTED;
  v.out_of_core = true;
  v.h_src = d->data;
  v.slot_cache_bytes = d->slot_cache_bytes;
  if (d->blobs) {
    v.host = new (std::nothrow) HostCache();
    if (!v.host) return AP_ERR_OOM;
    const uint64_t macro_bytes = (uint64_t)kMacro * v.D * 4;
    AP_TRY_ST(v.host->init(v.n, v.D, d->blobs, d->blob_bytes, d->codec,
                           (int64_t)(d->host_cache_bytes / macro_bytes), d->parse_threads));
  }
  v.n_macros = (v.n + kMacro - 1) / kMacro;
  const uint64_t slot_bytes = (uint64_t)kMacro * v.Dp * 2 * sizeof(__nv_bfloat16);
  v.n_slots = (int64_t)std::min<uint64_t>(d->slot_cache_bytes / slot_bytes, (uint64_t)v.n_macros);
  if (v.n_slots < 3 && v.n_slots < v.n_macros) return AP_ERR_INVALID_ARG;   // cache too small
  v.group = std::max<int64_t>(1, std::min<int64_t>(4, v.n_slots / 4));
  AP_TRY(dmalloc(&v.d_g64, tc_scratch_doubles(num_sms())));
  v.ooc_policy = AP_OOC_RESIDENT_STREAM;
  AP_TRY_ST(alloc_pool(v));
  build_schedule(v);
  return install_schedule(v);
}

ap_status run_out_of_core(ap_items *it, void *out, int coverage, cudaStream_t s) {
  VecStore &v = it->vec;
  if (v.ooc_policy == AP_OOC_K_SLICED) return run_slices(it, out, coverage, s);
  int64_t hits0 = 0, misses0 = 0, parsed0 = 0;
  if (v.host && !coverage) {
    // the macro loads in order: the parse threads decode ahead of the copies
    std::vector<int64_t> plan;
    for (const OocStep &st : v.steps)
      for (const auto &ld : st.loads) plan.push_back(ld.first);
    hits0 = v.host->hits;
    misses0 = v.host->misses;
    parsed0 = v.host->parsed_rows;
    v.host->announce(plan);
  }
  const int64_t P = v.n * (v.n - 1) / 2;
  if (!coverage) AP_TRY(cudaMemsetAsync(out, 0, (size_t)P * sizeof(double), s));
  // copies must follow whatever the caller queued before this call
  AP_TRY(cudaEventRecord(it->ev_a, s));
  AP_TRY(cudaStreamWaitEvent(it->copy_stream, it->ev_a, 0));
  uint64_t h2d = 0;
  int64_t item_loads = 0;
  int64_t ring_pos = 0;
  for (const OocStep &st : v.steps) {
    if (!coverage) {
      for (const auto &ld : st.loads) {
        const int64_t m = ld.first, slot = ld.second;
        const int64_t b = ring_pos++ % v.ring;
        const int64_t r0 = m * kMacro, rows = std::min<int64_t>(kMacro, v.n - r0);
        float *raw = v.d_raw + (size_t)b * kMacro * v.ld;
        if (v.ring_used[b]) AP_TRY(cudaStreamWaitEvent(it->copy_stream, v.ev_raw_free[b], 0));
        if (v.host) {
          // from the host cache (decoding the macro first on a miss); the
          // slot is released once the copy has run
          const int hs = v.host->acquire(m);
          AP_TRY(cudaMemcpyAsync(raw, v.host->slot_ptr(hs), (size_t)rows * v.ld * 4,
                                 cudaMemcpyHostToDevice, it->copy_stream));
          AP_TRY(cudaLaunchHostFunc(it->copy_stream, HostCache::release_cb,
                                    v.host->release_arg(hs)));
        } else {
          AP_TRY(cudaMemcpyAsync(raw, v.h_src + (size_t)r0 * v.ld, (size_t)rows * v.ld * 4,
                                 cudaMemcpyHostToDevice, it->copy_stream));
        }
        AP_TRY(cudaEventRecord(v.ev_raw_ready[b], it->copy_stream));
        AP_TRY(cudaStreamWaitEvent(s, v.ev_raw_ready[b], 0));
        const size_t slot_off = (size_t)slot * kMacro * v.Dp;
        AP_TRY(launch_vec_prep(raw, r0, 0, rows, v.D, v.ld, v.Dp, v.d_pool_hi + slot_off,
                               v.d_pool_lo + slot_off, nullptr, v.d_mu, v.d_part, v.d_partc,
                               v.d_delta_all, v.d_ss, v.d_rs, v.d_recentre, s));
        AP_TRY(cudaEventRecord(v.ev_raw_free[b], s));
        v.ring_used[b] = 1;
        h2d += (uint64_t)rows * v.ld * 4;
        item_loads += rows;
      }
    }
    const int32_t *units = coverage ? v.d_cover_units + st.cover0 * kOocTileInts
                                    : v.d_units + st.unit0 * kOocTileInts;
    const int64_t nu = coverage ? st.n_cover : st.n_units;
    AP_TRY(launch_gram_tc(v.tmap_pool_hi, v.tmap_pool_lo, v.n, v.Dp, v.d_rs, units, nu,
                          it->d_queue, it->d_status, v.d_g64, out, coverage, 1,
                          it->wait_budget_ns, it->debug, s));
  }
  if (!coverage)
    AP_TRY(launch_pair_finalize(reinterpret_cast<double *>(out), v.d_rs, v.d_delta_all, v.n, v.D,
                                s));
  it->stats.tiles = 0;
  for (const OocStep &st : v.steps) it->stats.tiles += coverage ? st.n_cover : st.n_units;
  it->stats.tile_m = kTcTileM;
  it->stats.tile_n = kTcTileN;
  it->stats.item_loads = coverage ? 0 : item_loads;
  it->stats.reuse_R = coverage ? 0.0 : (double)item_loads / (double)v.n;
  it->stats.h2d_bytes = h2d;
  it->stats.slot_hit_rate =
      v.ooc_uses > 0 ? 1.0 - (double)v.ooc_loads / (double)v.ooc_uses : 1.0;
  it->stats.parsed_rows = 0;
  it->stats.host_hit_rate = 0.0;
  if (v.host && !coverage) {
    // the counters of this run (every request is enqueued by now)
    const int64_t h = v.host->hits - hits0, m = v.host->misses - misses0;
    it->stats.parsed_rows = v.host->parsed_rows - parsed0;
    it->stats.host_hit_rate = h + m > 0 ? (double)h / (double)(h + m) : 0.0;
    if (v.host->bad_input) return AP_ERR_INVALID_ARG;
  }
  return AP_OK;
}

}  // namespace ap

using namespace ap;

extern "C" ap_status ap_set_out_of_core_policy(ap_items *items, int32_t policy) {
  if (!items || items->kind != AP_ITEMS_VECTOR) return AP_ERR_INVALID_ARG;
  if (policy != AP_OOC_RESIDENT_STREAM && policy != AP_OOC_DC_LRU && policy != AP_OOC_K_SLICED)
    return AP_ERR_INVALID_ARG;
  VecStore &v = items->vec;
  if (!v.out_of_core) return AP_ERR_STATE;
  const cudaError_t e = cudaDeviceSynchronize();     // the old buffers may be in use
  if (e != cudaSuccess) return from_cuda(e);
  const bool was_sliced = v.ooc_policy == AP_OOC_K_SLICED;
  const bool sliced = policy == AP_OOC_K_SLICED;
  if (sliced && v.host) return AP_ERR_UNSUPPORTED;    // slices need raw column ranges
  if (sliced) {
    // validate before giving up the slot pool
    int64_t cols, count, ring;
    if (!slice_geometry(v.n, v.Dp, v.slot_cache_bytes, &cols, &count, &ring))
      return AP_ERR_INVALID_ARG;
  }
  if (sliced != was_sliced) {
    // the two kinds of schedule keep different buffers within the same budget
    free_pool(v);
    free_slices(v);
    free_raw_ring(v);
  }
  v.ooc_policy = policy;
  if (sliced) return was_sliced ? AP_OK : alloc_slices(v);
  if (was_sliced) AP_TRY_ST(alloc_pool(v));
  if (policy == AP_OOC_DC_LRU) build_schedule_lru(v);
  else build_schedule(v);
  return install_schedule(v);
}

extern "C" ap_status ap_plan_out_of_core(int64_t n_items, int64_t dim, uint64_t slot_cache_bytes,
                                         int32_t policy, int64_t *n_slots, int64_t *n_loads,
                                         int64_t *n_steps) {
  if (n_items < 0 || dim < 2 || !n_slots || !n_loads || !n_steps) return AP_ERR_INVALID_ARG;
  if (policy != AP_OOC_RESIDENT_STREAM && policy != AP_OOC_DC_LRU && policy != AP_OOC_K_SLICED)
    return AP_ERR_INVALID_ARG;
  if (policy == AP_OOC_K_SLICED) {
    // two chunk buffers; every macro loaded once; one step per column chunk
    int64_t cols, count, ring;
    if (!slice_geometry(n_items, (dim + 63) / 64 * 64, slot_cache_bytes, &cols, &count, &ring))
      return AP_ERR_INVALID_ARG;
    *n_slots = 2;
    *n_loads = (n_items + kMacro - 1) / kMacro;
    *n_steps = count;
    return AP_OK;
  }
  VecStore v;
  v.n = n_items;
  v.D = dim;
  v.Dp = (dim + 63) / 64 * 64;
  v.n_macros = (n_items + 255) / 256;
  const uint64_t slot_bytes = 256ull * v.Dp * 4;
  v.n_slots = (int64_t)std::min<uint64_t>(slot_cache_bytes / slot_bytes, (uint64_t)v.n_macros);
  if (v.n_slots < 3 && v.n_slots < v.n_macros) return AP_ERR_INVALID_ARG;
  v.group = std::max<int64_t>(1, std::min<int64_t>(4, v.n_slots / 4));
  if (policy == AP_OOC_DC_LRU) build_schedule_lru(v);
  else build_schedule(v);
  // every macro pair (a <= b) exactly once, both macros resident in the slots named
  std::vector<int32_t> seen((size_t)v.n_macros * v.n_macros, 0);
  std::vector<int64_t> holder(v.n_slots, -1);
  int64_t loads = 0;
  for (const OocStep &st : v.steps) {
    for (const auto &ld : st.loads) { holder[ld.second] = ld.first; ++loads; }
    for (const OocPair &pp : st.pairs) {
      if (pp.a > pp.b || holder[pp.slot_a] != pp.a || holder[pp.slot_b] != pp.b) return AP_ERR_STATE;
      seen[(size_t)pp.a * v.n_macros + pp.b] += 1;
    }
  }
  for (int64_t a = 0; a < v.n_macros; ++a)
    for (int64_t b = a; b < v.n_macros; ++b)
      if (seen[(size_t)a * v.n_macros + b] != 1) return AP_ERR_STATE;
  *n_slots = v.n_slots;
  *n_loads = loads;
  *n_steps = (int64_t)v.steps.size();
  return AP_OK;
}

namespace ap {

// Units of the streamed run: column m holds the pairs (a <= m, m) of macros,
// addressed directly in the resident arrays (row block = item block), as
// CTA-pair units in waves like the resident schedule (column ranges of
// ~16384 columns, two units per SM at least).  With C column chunks, each
// (chunk, column) entry holds those pairs over the chunk's columns only.
static ap_status build_stream_units(VecStore &v, int64_t C) {
  const int64_t M = (v.n + kMacro - 1) / kMacro;
  const int64_t ccols = C > 1 ? (v.Dp + C - 1) / C : v.Dp;
  v.stream_chunk_cols = (ccols + kOocChunkCols - 1) / kOocChunkCols * kOocChunkCols;
  v.stream_chunks = C;
  std::vector<int32_t> units;
  v.stream_cols.clear();
  for (int64_t c = 0; c < C; ++c) {
    const int64_t c0 = c * v.stream_chunk_cols;
    const int64_t w = std::min<int64_t>(v.stream_chunk_cols, v.Dp - c0);
    const int64_t nch = w / kOocChunkCols, off = c0 / kOocChunkCols;
    for (int64_t m = 0; m < M; ++m) {
      std::vector<int32_t> macro, col_units;
      for (int64_t a = 0; a <= m; ++a) {
        macro.push_back((int32_t)a);
        macro.push_back((int32_t)m);
      }
      // split-K: the rule of the single-CTA tiles (two 128-row tiles per pair)
      const int64_t ks = std::max<int32_t>(1, default_k_split(2 * (m + 1), w));
      pair_units_of(macro, nch, tc2_pairs(), ks, col_units);
      for (size_t u = 0; u < col_units.size(); u += kOocTileInts) {
        col_units[u + 6] += (int32_t)off;
        col_units[u + 7] += (int32_t)off;
      }
      const int64_t u0 = (int64_t)units.size() / kOocTileInts;
      units.insert(units.end(), col_units.begin(), col_units.end());
      v.stream_cols.push_back({u0, (int64_t)units.size() / kOocTileInts - u0});
    }
  }
  dfree(v.d_stream_units);
  AP_TRY(dmalloc(&v.d_stream_units, std::max<size_t>(units.size(), kOocTileInts)));
  if (!units.empty())
    AP_TRY(cudaMemcpy(v.d_stream_units, units.data(), units.size() * 4, cudaMemcpyHostToDevice));
  return AP_OK;
}

// Column chunks for the streamed run: rows of 2 MiB or more go in chunks of
// whole 1 MiB pieces (at most 8), so that each chunk's Gram is spread over
// its copies and only the last chunk's last columns follow the last copy;
// strided pieces of 1 MiB copy at the link's full rate, shorter ones do not.
static int64_t stream_chunks_for(const VecStore &v) {
  constexpr int64_t kPieceCols = (1 << 20) / 4;
  if (v.D < 2 * kPieceCols) return 1;
  return std::min<int64_t>(8, v.D / kPieceCols);
}

ap_status stream_load_and_run(ap_items *it, const float *h, double *out, cudaStream_t s) {
  VecStore &v = it->vec;
  // column chunks need the shifts before the first chunk: sampled over the
  // whole rows from the page-locked source, where the device can read it
  const float *d_src = nullptr;
  if (cudaHostGetDevicePointer((void **)&d_src, (void *)h, 0) != cudaSuccess) {
    cudaGetLastError();
    d_src = nullptr;
  }
  const int64_t C = d_src ? stream_chunks_for(v) : 1;
  if (!v.d_stream_units || v.stream_chunks != C) {
    ap_status st = build_stream_units(v, C);
    if (st != AP_OK) return st;
  }
  if (!v.d_raw) {
    // raw staging ring: up to 8 GiB of macros, so the copies run ahead of
    // the Gram instead of waiting for each column's compute
    const int64_t macro_bytes = kMacro * v.ld * 4;
    v.ring = std::max<int64_t>(2, std::min<int64_t>({(8LL << 30) / macro_bytes, 16,
                                                     (int64_t)v.stream_cols.size()}));
    AP_TRY(dmalloc(&v.d_raw, (size_t)v.ring * kMacro * v.ld));
    for (int64_t b = 0; b < v.ring; ++b) {
      cudaEvent_t a, f, p;
      AP_TRY(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
      v.ev_raw_ready.push_back(a);
      AP_TRY(cudaEventCreateWithFlags(&f, cudaEventDisableTiming));
      v.ev_raw_free.push_back(f);
      AP_TRY(cudaEventCreateWithFlags(&p, cudaEventDisableTiming));
      v.ev_prepped.push_back(p);
    }
    v.ring_used.assign(v.ring, 0);
  }
  if (!it->prep_stream)
    AP_TRY(cudaStreamCreateWithFlags(&it->prep_stream, cudaStreamNonBlocking));
  const int64_t P = v.n * (v.n - 1) / 2;
  NvtxRange range("load and run");
  Tracer &tr = it->trace;
  AP_TRY(tr.start(s));
  AP_TRY(cudaMemsetAsync(out, 0, (size_t)P * sizeof(double), s));
  // earlier work on s may still read the rows about to be overwritten
  AP_TRY(cudaEventRecord(it->ev_a, s));
  AP_TRY(cudaStreamWaitEvent(it->copy_stream, it->ev_a, 0));
  AP_TRY(cudaStreamWaitEvent(it->prep_stream, it->ev_a, 0));
  const bool split = v.d_hi != nullptr, f32 = v.d_c32 != nullptr;
  if (C > 1) {
    // chunk c of macro m: a strided copy of its rows' columns, split into
    // the resident arrays at those columns (FP64 sums of c and c^2 added up
    // over the chunks), then the pairs (a <= m, m) over the chunk
    AP_TRY(launch_vec_shift_runs(d_src, v.n, v.D, v.ld, v.d_mu, it->prep_stream));
    const int64_t M = (v.n + kMacro - 1) / kMacro;
    int64_t seq = 0;
    for (int64_t c = 0; c < C; ++c) {
      const int64_t c0 = c * v.stream_chunk_cols;
      const int64_t w = std::min<int64_t>(v.stream_chunk_cols, v.Dp - c0);
      const int64_t cols = std::max<int64_t>(0, std::min<int64_t>(w, v.D - c0));
      for (int64_t m = 0; m < M; ++m, ++seq) {
        const int64_t b = seq % v.ring;
        const int64_t r0 = m * kMacro, rows = std::min<int64_t>(kMacro, v.n - r0);
        float *raw = v.d_raw + (size_t)b * kMacro * v.ld;
        if (v.ring_used[b]) AP_TRY(cudaStreamWaitEvent(it->copy_stream, v.ev_raw_free[b], 0));
        const int t_copy = tr.begin(1, AP_STAGE_COPY, seq, (uint64_t)rows * cols * 4,
                                    it->copy_stream);
        if (cols > 0)
          AP_TRY(cudaMemcpy2DAsync(raw, (size_t)w * 4, h + (size_t)r0 * v.ld + c0,
                                   (size_t)v.ld * 4, (size_t)cols * 4, (size_t)rows,
                                   cudaMemcpyHostToDevice, it->copy_stream));
        tr.end(t_copy, it->copy_stream);
        AP_TRY(cudaEventRecord(v.ev_raw_ready[b], it->copy_stream));
        AP_TRY(cudaStreamWaitEvent(it->prep_stream, v.ev_raw_ready[b], 0));
        const int t_prep = tr.begin(2, AP_STAGE_PREPROCESS, seq, 0, it->prep_stream);
        AP_TRY(launch_vec_split_cols(raw, r0, rows, cols, w, w, c0, v.Dp, v.d_mu,
                                     split ? v.d_hi : nullptr, split ? v.d_lo : nullptr,
                                     f32 ? v.d_c32 : nullptr, v.d_part, v.d_partc, c == 0 ? 1 : 0,
                                     it->prep_stream));
        tr.end(t_prep, it->prep_stream);
        AP_TRY(cudaEventRecord(v.ev_raw_free[b], it->prep_stream));
        AP_TRY(cudaEventRecord(v.ev_prepped[b], it->prep_stream));
        v.ring_used[b] = 1;
        AP_TRY(cudaStreamWaitEvent(s, v.ev_prepped[b], 0));
        const auto &uc = v.stream_cols[(size_t)(c * M + m)];
        const int t_gram = tr.begin(0, AP_STAGE_GRAM, seq, 0, s);
        AP_TRY(launch_gram_tc2(v.tmap_hi, v.tmap_lo, v.n, v.d_rs,
                               v.d_stream_units + uc.first * kOocTileInts, uc.second,
                               it->d_queue, it->d_status, v.d_g64, out, 0, 1, it->wait_budget_ns,
                               it->debug, s));
        tr.end(t_gram, s);
      }
    }
    // the rows' statistics from the chunks' sums, then r from the Gram
    const int t_fin = tr.begin(0, AP_STAGE_FINALIZE, 0, 0, s);
    AP_TRY(launch_slice_finalize(v.d_part, v.d_partc, v.n, v.D, v.d_delta_all, v.d_ss, v.d_rs,
                                 out, s));
    tr.end(t_fin, s);
    it->stats.item_loads = v.n;
    it->stats.reuse_R = 1.0;
    it->stats.h2d_bytes = (uint64_t)v.n * v.D * 4;
    it->stats.slot_hit_rate = 1.0;
    return AP_OK;
  }
  // three streams: copies (copy_stream) -> pre-processing (prep_stream) ->
  // Gram column m (s), linked by per-slot events
  for (size_t m = 0; m < v.stream_cols.size(); ++m) {
    const int64_t b = (int64_t)(m % v.ring);
    const int64_t r0 = (int64_t)m * kMacro, rows = std::min<int64_t>(kMacro, v.n - r0);
    float *raw = v.d_raw + (size_t)b * kMacro * v.ld;
    if (v.ring_used[b]) AP_TRY(cudaStreamWaitEvent(it->copy_stream, v.ev_raw_free[b], 0));
    const int t_copy = tr.begin(1, AP_STAGE_COPY, (int64_t)m, (uint64_t)rows * v.ld * 4,
                                it->copy_stream);
    AP_TRY(cudaMemcpyAsync(raw, h + (size_t)r0 * v.ld, (size_t)rows * v.ld * 4,
                           cudaMemcpyHostToDevice, it->copy_stream));
    tr.end(t_copy, it->copy_stream);
    AP_TRY(cudaEventRecord(v.ev_raw_ready[b], it->copy_stream));
    AP_TRY(cudaStreamWaitEvent(it->prep_stream, v.ev_raw_ready[b], 0));
    const int t_prep = tr.begin(2, AP_STAGE_PREPROCESS, (int64_t)m, 0, it->prep_stream);
    AP_TRY(launch_vec_prep(raw, r0, r0, rows, v.D, v.ld, v.Dp, split ? v.d_hi : nullptr,
                           split ? v.d_lo : nullptr, f32 ? v.d_c32 : nullptr, v.d_mu, v.d_part,
                           v.d_partc, v.d_delta_all, v.d_ss, v.d_rs, v.d_recentre,
                           it->prep_stream));
    tr.end(t_prep, it->prep_stream);
    AP_TRY(cudaEventRecord(v.ev_raw_free[b], it->prep_stream));
    AP_TRY(cudaEventRecord(v.ev_prepped[b], it->prep_stream));
    v.ring_used[b] = 1;
    AP_TRY(cudaStreamWaitEvent(s, v.ev_prepped[b], 0));
    const int t_gram = tr.begin(0, AP_STAGE_GRAM, (int64_t)m, 0, s);
    AP_TRY(launch_gram_tc2(v.tmap_hi, v.tmap_lo, v.n, v.d_rs,
                           v.d_stream_units + v.stream_cols[m].first * kOocTileInts,
                           v.stream_cols[m].second, it->d_queue, it->d_status, v.d_g64, out, 0,
                           1, it->wait_budget_ns, it->debug, s));
    tr.end(t_gram, s);
  }
  const int t_fin = tr.begin(0, AP_STAGE_FINALIZE, 0, 0, s);
  AP_TRY(launch_pair_finalize(out, v.d_rs, v.d_delta_all, v.n, v.D, s));
  tr.end(t_fin, s);
  it->stats.item_loads = v.n;
  it->stats.reuse_R = 1.0;
  it->stats.h2d_bytes = (uint64_t)v.n * v.ld * 4;
  it->stats.slot_hit_rate = 1.0;
  return AP_OK;
}

}  // namespace ap

extern "C" ap_status ap_load_and_run(ap_items *items, const float *host_data, double *out,
                                     void *stream) {
  if (!items || items->kind != AP_ITEMS_VECTOR) return AP_ERR_INVALID_ARG;
  if (items->vec.out_of_core || !items->vec.d_hi) return AP_ERR_STATE;
  if (items->vec.n < 2) return AP_OK;
  if (!host_data || !out) return AP_ERR_INVALID_ARG;
  return stream_load_and_run(items, host_data, out, reinterpret_cast<cudaStream_t>(stream));
}
