// api.cu -- the C ABI of the all-pairs library (declared in allpairs.h).
//
// Validation, library-owned storage, the load pipeline l (Sec. III: copy to
// the GPU, pre-process there), planning of the tiled schedule (Sec. IV-B) and
// dispatch to the kernel families.  Every compute step runs in CUDA kernels;
// there is no host fallback.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "ap_internal.h"

namespace ap {

// SM count of the current device, cached per device (first query under a lock)
int num_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cached[kMaxDev];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  const bool fits = dev < kMaxDev;
  int v = fits ? cached[dev].load(std::memory_order_acquire) : 0;
  if (v > 0) return v;
  std::lock_guard<std::mutex> lock(mu);
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
    v = 1;
  if (fits) cached[dev].store(v, std::memory_order_release);
  return v;
}

// the CUDA error behind this thread's last AP_ERR_CUDA / AP_ERR_OOM
thread_local cudaError_t g_last_cuda_error = cudaSuccess;

ap_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return AP_OK;
  g_last_cuda_error = e;
  cudaGetLastError();   // clear a non-sticky error so later calls can run
  return e == cudaErrorMemoryAllocation ? AP_ERR_OOM : AP_ERR_CUDA;
}

namespace {

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

void free_items(ap_items *it) {
  if (!it) return;
  cudaDeviceSynchronize();          // queued host functions may still use the host cache
  CloudStore &c = it->cl;
  dfree(c.d_pts); dfree(c.d_lw); dfree(c.d_poff); dfree(c.d_cnt); dfree(c.d_perm);
  dfree(c.d_bstart); dfree(c.d_tiles); dfree(c.d_bstart_single); dfree(c.d_list_tiles);
  for (int k = 0; k < 2; ++k) { dfree(c.d_pts_score[k]); dfree(c.d_lw_score[k]); }
  dfree(c.d_self);
  VecStore &v = it->vec;
  dfree(v.d_mu); dfree(v.d_ss); dfree(v.d_rs); dfree(v.d_part); dfree(v.d_hi); dfree(v.d_lo); dfree(v.d_c32);
  dfree(v.d_rows);
  dfree(v.d_partc); dfree(v.d_delta_all); dfree(v.d_recentre);
  dfree(v.d_stage); dfree(v.d_tiles_tc); dfree(v.d_tiles_f32); dfree(v.d_g64);
  dfree(v.d_panel_units); dfree(v.d_pair_units); dfree(v.d_pair_whole);
  free_out_of_core(v);
  free_sparse(it->sp);
  free_tc_tensor_maps(v.tmap_hi, v.tmap_lo);
  v.tmap_hi = v.tmap_lo = nullptr;
  dfree(it->d_queue);
  dfree(it->d_scratch);
  clear_graphs(it);
  if (it->graph_stream) cudaStreamDestroy(it->graph_stream);
  if (it->copy_stream) cudaStreamDestroy(it->copy_stream);
  if (it->prep_stream) cudaStreamDestroy(it->prep_stream);
  for (cudaEvent_t *e : {&it->ev_a, &it->ev_b})
    if (*e) cudaEventDestroy(*e);
  delete it;
}

}  // namespace

// ---------------------------------------------------------------------------
// point clouds
// ---------------------------------------------------------------------------
CloudPlanChoice choose_cloud_plan(const CloudStore &c) {
  CloudPlanChoice ch{};
  int64_t mx = 0, mn = INT64_MAX;
  for (int64_t s : c.h_size) { mx = std::max(mx, s); mn = std::min(mn, s); }
  if (c.n == 0) mn = 0;
  // uneven 3-D sets are sorted by size (transforms are 2-D only and need the
  // original order to know which item of a pair is moved)
  ch.sorted = (c.dim == 3) && mx > 4 * std::max<int64_t>(mn, 1);
  // a-points per lane: enough chunk width for the largest item
  ch.reg_r = std::max<int32_t>(2, min_reg_r(c));
  ch.block_pts = 4096;
  // block size: enough tiles to keep every SM busy several times over
  const int64_t want_tiles = (int64_t)num_sms() * 16;
  ch.block_items = kOverlapMaxBlockItems;
  while (ch.block_items > 2) {
    int64_t nb = (c.n + ch.block_items - 1) / ch.block_items;
    if (nb * (nb + 1) / 2 >= want_tiles) break;
    ch.block_items /= 2;
  }
  return ch;
}

ap_status build_cloud_plan(ap_items *it, const CloudPlanChoice &ch, cudaStream_t s) {
  CloudStore &c = it->cl;
  std::vector<int64_t> cnt(c.n);
  for (int64_t s = 0; s < c.n; ++s) cnt[s] = c.h_size[c.h_perm[s]];
  std::vector<int32_t> bstart;
  make_blocks(c.h_poff, cnt, ch.block_items, ch.block_pts, 32LL * ch.reg_r, kOverlapMaxRowJobs,
              bstart);
  std::vector<int32_t> tiles;
  dc_block_pairs((int64_t)bstart.size() - 1, tiles);
  const bool largest_first = order_cloud_tiles(bstart, cnt, c.total_pts, tiles);
  dfree(c.d_bstart);
  dfree(c.d_tiles);
  AP_TRY(dmalloc(&c.d_bstart, bstart.size()));
  AP_TRY(dmalloc(&c.d_tiles, std::max<size_t>(tiles.size(), 2)));
  // pageable sources: the copies are staged before the calls return
  AP_TRY(cudaMemcpyAsync(c.d_bstart, bstart.data(), bstart.size() * 4, cudaMemcpyHostToDevice, s));
  if (!tiles.empty())
    AP_TRY(cudaMemcpyAsync(c.d_tiles, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice, s));
  c.h_bstart = bstart;
  c.max_rj = max_row_jobs(bstart, cnt, 32LL * ch.reg_r);
  c.n_tiles = (int64_t)tiles.size() / 2;
  c.block_items = ch.block_items;
  c.block_pts = ch.block_pts;
  c.reg_r = ch.reg_r;
  it->stats.tiles = c.n_tiles;
  it->stats.tile_m = ch.block_items;
  it->stats.tile_n = ch.block_items;
  it->stats.order = largest_first ? 2 : 0;
  ++it->plan_version;
  return AP_OK;
}

namespace {

ap_status create_clouds(const ap_items_desc *d, ap_items *it, cudaStream_t s) {
  CloudStore &c = it->cl;
  c.dim = d->kind == AP_ITEMS_CLOUD3D ? 3 : 2;
  c.n = d->n_items;
  const int64_t *off = d->offsets;
  if (!off) return AP_ERR_INVALID_ARG;
  if (off[0] != 0) return AP_ERR_INVALID_ARG;
  c.h_size.resize(c.n);
  for (int64_t i = 0; i < c.n; ++i) {
    if (off[i + 1] < off[i]) return AP_ERR_INVALID_ARG;
    c.h_size[i] = off[i + 1] - off[i];
  }
  const int64_t total = off[c.n];
  if (total > 0 && (!d->x || !d->y || !d->sigma || (c.dim == 3 && !d->z)))
    return AP_ERR_INVALID_ARG;
  int64_t mx = 0;
  for (int64_t v : c.h_size) mx = std::max(mx, v);
  if (mx > (int64_t)4 * 32 * kOverlapMaxRowJobs) return AP_ERR_UNSUPPORTED;   // > 16384 points
  c.unit_weights = (d->weight == nullptr);

  CloudPlanChoice ch = choose_cloud_plan(c);
  c.sorted = ch.sorted;
  c.h_perm.resize(c.n);
  std::iota(c.h_perm.begin(), c.h_perm.end(), 0);
  if (c.sorted)
    std::stable_sort(c.h_perm.begin(), c.h_perm.end(),
                     [&](int32_t a, int32_t b) { return c.h_size[a] > c.h_size[b]; });
  c.h_poff.assign(c.n + 1, 0);
  for (int64_t sidx = 0; sidx < c.n; ++sidx)
    c.h_poff[sidx + 1] = c.h_poff[sidx] + round_up(c.h_size[c.h_perm[sidx]], 4);
  c.total_pts = c.h_poff[c.n];

  std::vector<int32_t> cnt32(c.n);
  for (int64_t sidx = 0; sidx < c.n; ++sidx) cnt32[sidx] = (int32_t)c.h_size[c.h_perm[sidx]];
  AP_TRY(dmalloc(&c.d_pts, std::max<int64_t>(c.total_pts, 4)));
  if (c.dim == 3 && !c.unit_weights) AP_TRY(dmalloc(&c.d_lw, std::max<int64_t>(c.total_pts, 4)));
  AP_TRY(dmalloc(&c.d_poff, c.n + 1));
  AP_TRY(dmalloc(&c.d_cnt, std::max<int64_t>(c.n, 1)));
  AP_TRY(dmalloc(&c.d_perm, std::max<int64_t>(c.n, 1)));
  // everything below is ordered on the caller's stream; host sources must
  // stay valid until that stream has run it (pageable memory is staged by
  // the copy calls themselves)
  AP_TRY(cudaMemcpyAsync(c.d_poff, c.h_poff.data(), (c.n + 1) * 8, cudaMemcpyHostToDevice, s));
  if (c.n > 0) {
    AP_TRY(cudaMemcpyAsync(c.d_cnt, cnt32.data(), c.n * 4, cudaMemcpyHostToDevice, s));
    AP_TRY(cudaMemcpyAsync(c.d_perm, c.h_perm.data(), c.n * 4, cudaMemcpyHostToDevice, s));
  }

  if (total > 0) {
    // source arrays on the device (temporary copies when they are host
    // memory), from the stream-ordered allocator and freed on the stream
    const float *src[5] = {d->x, d->y, c.dim == 3 ? d->z : nullptr, d->sigma, d->weight};
    float *tmp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t *d_src_off = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_src_off), (c.n + 1) * 8, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_src_off, off, (c.n + 1) * 8, cudaMemcpyHostToDevice, s);
    for (int k = 0; k < 5 && e == cudaSuccess; ++k) {
      if (!src[k] || !d->data_on_host) continue;
      e = cudaMallocAsync(reinterpret_cast<void **>(&tmp[k]), total * 4, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp[k], src[k], total * 4, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
      auto pick = [&](int k) -> const float * { return d->data_on_host ? tmp[k] : src[k]; };
      e = launch_cloud_pack(pick(0), pick(1), pick(2), pick(3), pick(4), d_src_off, c.d_perm,
                            c.d_poff, c.n, c.dim, c.d_pts, c.d_lw, s);
    }
    for (int k = 0; k < 5; ++k)
      if (tmp[k]) cudaFreeAsync(tmp[k], s);
    if (d_src_off) cudaFreeAsync(d_src_off, s);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return build_cloud_plan(it, ch, s);
}

// ---------------------------------------------------------------------------
// dense vectors
// ---------------------------------------------------------------------------
ap_status vec_load(ap_items *it, const float *data, int on_host, cudaStream_t s) {
  NvtxRange range("load: copy + pre-process");
  VecStore &v = it->vec;
  const bool split = (v.precisions & (1u << AP_PREC_SPLIT_BF16)) != 0;
  const bool f32 = (v.precisions & (1u << AP_PREC_FP32)) != 0;
  if (!on_host) {
    AP_TRY(launch_vec_prep(data, 0, 0, v.n, v.D, v.ld, v.Dp, split ? v.d_hi : nullptr,
                           split ? v.d_lo : nullptr, f32 ? v.d_c32 : nullptr, v.d_mu, v.d_part,
                           v.d_partc, v.d_delta_all, v.d_ss, v.d_rs, v.d_recentre, s));
    return AP_OK;
  }
  // host source: two staging buffers, copies on the copy stream overlap the
  // pre-processing of the previous chunk on the caller's stream
  const int64_t rows = v.stage_rows;
  const size_t half = (size_t)rows * v.ld;
  cudaEvent_t copied[2], done[2];
  for (int b = 0; b < 2; ++b) {
    AP_TRY(cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming));
    AP_TRY(cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming));
  }
  ap_status st = AP_OK;
  cudaError_t e = cudaEventRecord(it->ev_a, s);             // earlier work on the stage
  if (e == cudaSuccess) e = cudaStreamWaitEvent(it->copy_stream, it->ev_a, 0);
  int64_t chunk = 0;
  for (int64_t r0 = 0; r0 < v.n && e == cudaSuccess; r0 += rows, ++chunk) {
    const int b = (int)(chunk & 1);
    const int64_t nr = std::min(rows, v.n - r0);
    float *stage = v.d_stage + b * half;
    if (chunk >= 2) e = cudaStreamWaitEvent(it->copy_stream, done[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(stage, data + r0 * v.ld, (size_t)nr * v.ld * 4, cudaMemcpyHostToDevice,
                          it->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(copied[b], it->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, copied[b], 0);
    if (e == cudaSuccess)
      e = launch_vec_prep(stage, r0, r0, nr, v.D, v.ld, v.Dp, split ? v.d_hi : nullptr,
                          split ? v.d_lo : nullptr, f32 ? v.d_c32 : nullptr, v.d_mu, v.d_part,
                          v.d_partc, v.d_delta_all, v.d_ss, v.d_rs, v.d_recentre, s);
    if (e == cudaSuccess) e = cudaEventRecord(done[b], s);
  }
  if (e != cudaSuccess) st = from_cuda(e);
  // the events may be destroyed while pending: resources are released once done
  for (int b = 0; b < 2; ++b) {
    cudaEventDestroy(copied[b]);
    cudaEventDestroy(done[b]);
  }
  return st;
}

ap_status create_vectors(const ap_items_desc *d, ap_items *it, cudaStream_t s) {
  VecStore &v = it->vec;
  v.n = d->n_items;
  v.D = d->dim;
  v.ld = d->ld ? d->ld : d->dim;
  if (v.D < 2 || v.ld < v.D) return AP_ERR_INVALID_ARG;
  if (d->blobs) {
    // encoded items: decoded rows are dense, only the out-of-core path reads them
    if (d->data || !d->data_on_host || !d->slot_cache_bytes || d->ld) return AP_ERR_INVALID_ARG;
    if (d->codec != AP_CODEC_XOR_VARINT || !d->blob_bytes) return AP_ERR_INVALID_ARG;
  } else if (v.n > 0 && !d->data) {
    return AP_ERR_INVALID_ARG;
  }
  if (v.n > INT32_MAX / 2) return AP_ERR_UNSUPPORTED;
  v.precisions = d->precisions ? d->precisions : (1u << AP_PREC_SPLIT_BF16);
  if (v.precisions & ~((1u << AP_PREC_FP32) | (1u << AP_PREC_SPLIT_BF16)))
    return AP_ERR_INVALID_ARG;
  v.Dp = round_up(v.D, 64);
  const int64_t nn = std::max<int64_t>(v.n, 1);
  AP_TRY(dmalloc(&v.d_mu, nn));
  AP_TRY(dmalloc(&v.d_ss, nn));
  AP_TRY(dmalloc(&v.d_rs, nn));
  AP_TRY(dmalloc(&v.d_part, (size_t)nn * kSplitParts));
  AP_TRY(dmalloc(&v.d_partc, (size_t)nn * kSplitParts));
  AP_TRY(dmalloc(&v.d_delta_all, nn));
  AP_TRY(dmalloc(&v.d_recentre, nn + 1));
  // out-of-core: items stay in host memory and stream through the slot cache
  if (d->slot_cache_bytes) return create_out_of_core(d, it);
  // blocked copies cover whole row blocks; the padding rows stay zero
  v.n_rows_alloc = round_up(nn, kRowBlock);
  const size_t elems = (size_t)v.n_rows_alloc * v.Dp;
  if (v.precisions & (1u << AP_PREC_SPLIT_BF16)) {
    AP_TRY(dmalloc(&v.d_hi, elems));
    AP_TRY(dmalloc(&v.d_lo, elems));
    AP_TRY(cudaMemsetAsync(v.d_hi, 0, elems * 2, s));
    AP_TRY(cudaMemsetAsync(v.d_lo, 0, elems * 2, s));
    AP_TRY(make_tc_tensor_maps(v.d_hi, v.d_lo, nn, v.Dp, &v.tmap_hi, &v.tmap_lo));
    std::vector<int32_t> tiles;
    tc_tiles(v.n, tiles);
    v.n_tiles_tc = (int64_t)tiles.size() / 2;
    v.h_tiles_tc = tiles;
    // one FP64 scratch tile per SM: every Gram launch (whole tiles, split-K
    // units, streamed columns) has at most one CTA per SM
    AP_TRY(dmalloc(&v.d_g64, tc_scratch_doubles(num_sms())));
    AP_TRY(dmalloc(&v.d_tiles_tc, std::max<size_t>(tiles.size(), 2)));
    if (!tiles.empty())
      AP_TRY(cudaMemcpy(v.d_tiles_tc, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice));
    ap_status st = set_vector_plan(it, -1);
    if (st != AP_OK) return st;
  }
  if (v.precisions & (1u << AP_PREC_FP32)) {
    AP_TRY(dmalloc(&v.d_c32, elems));
    AP_TRY(cudaMemsetAsync(v.d_c32, 0, elems * 4, s));
    std::vector<int32_t> tiles;
    dc_block_pairs((v.n + 127) / 128, tiles);
    v.n_tiles_f32 = (int64_t)tiles.size() / 2;
    AP_TRY(dmalloc(&v.d_tiles_f32, std::max<size_t>(tiles.size(), 2)));
    if (!tiles.empty())
      AP_TRY(cudaMemcpy(v.d_tiles_f32, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice));
  }
  if (d->data_on_host && v.n > 0) {
    // ~256 MB per staging half
    v.stage_rows = std::max<int64_t>(1, std::min<int64_t>(v.n, (256ll << 20) / (v.ld * 4)));
    AP_TRY(dmalloc(&v.d_stage, (size_t)2 * v.stage_rows * v.ld));
  }
  if (v.n > 0) {
    ap_status st = vec_load(it, d->data, d->data_on_host, s);
    if (st != AP_OK) return st;
  }
  return AP_OK;
}

}  // namespace
ap_status ensure_score_storage(ap_items *it, int score, cudaStream_t s) {
  CloudStore &c = it->cl;
  if (c.d_pts_score[score - 1]) return AP_OK;
  // the re-scaled storage (and the L2 self terms) on first use
  const bool lw = score == 2 ? c.dim == 3 : c.d_lw != nullptr;
  AP_TRY(dmalloc(&c.d_pts_score[score - 1], (size_t)std::max<int64_t>(c.total_pts, 1)));
  if (lw) AP_TRY(dmalloc(&c.d_lw_score[score - 1], (size_t)std::max<int64_t>(c.total_pts, 1)));
  AP_TRY(launch_cloud_rescore(c, score, c.d_pts_score[score - 1], c.d_lw_score[score - 1], s));
  if (score == 1) {
    AP_TRY(dmalloc(&c.d_self, (size_t)c.n));
    AP_TRY(launch_cloud_self(c, c.d_pts_score[0], c.d_lw_score[0], c.d_self, s));
  }
  return AP_OK;
}

}  // namespace ap

using namespace ap;

extern "C" {

int64_t ap_pair_count(int64_t n) { return n < 2 ? 0 : n * (n - 1) / 2; }

int64_t ap_pair_index(int64_t i, int64_t j, int64_t n) {
  if (i < 0 || j <= i || j >= n) return -1;
  return pair_index(i, j, n);
}

const char *ap_last_cuda_error(void) {
  return g_last_cuda_error == cudaSuccess ? "" : cudaGetErrorName(g_last_cuda_error);
}

const char *ap_status_string(ap_status s) {
  switch (s) {
    case AP_OK: return "ok";
    case AP_ERR_INVALID_ARG: return "invalid argument";
    case AP_ERR_OOM: return "out of memory";
    case AP_ERR_CUDA: return "CUDA error";
    case AP_ERR_TIMEOUT: return "device wait timed out";
    case AP_ERR_UNSUPPORTED: return "unsupported";
    case AP_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

ap_status ap_plan_tiles(int64_t n, int32_t block, int32_t *out, int64_t cap, int64_t *n_tiles) {
  if (!n_tiles) return AP_ERR_INVALID_ARG;
  *n_tiles = 0;
  if (n < 0 || block < 1 || (cap > 0 && !out)) return AP_ERR_INVALID_ARG;
  std::vector<int32_t> t;
  dc_block_pairs((n + block - 1) / block, t);
  *n_tiles = (int64_t)t.size() / 2;
  if (cap >= *n_tiles && !t.empty()) std::memcpy(out, t.data(), t.size() * 4);
  return AP_OK;
}

ap_status ap_create_items(const ap_items_desc *desc, void *stream, ap_items **out) {
  if (!out) return AP_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || desc->n_items < 0) return AP_ERR_INVALID_ARG;
  if (desc->kind != AP_ITEMS_CLOUD2D && desc->kind != AP_ITEMS_CLOUD3D &&
      desc->kind != AP_ITEMS_VECTOR && desc->kind != AP_ITEMS_SPARSE)
    return AP_ERR_INVALID_ARG;
  if (desc->n_items > INT32_MAX / 4) return AP_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  ap_items *it = new (std::nothrow) ap_items();
  if (!it) return AP_ERR_OOM;
  it->kind = desc->kind;
  cudaGetDevice(&it->device);
  ap_status st = AP_OK;
  cudaError_t e = dmalloc(&it->d_queue, 64);
  if (e == cudaSuccess) e = cudaMemset(it->d_queue, 0, 64 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&it->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&it->graph_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&it->ev_a, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&it->ev_b, cudaEventDisableTiming);
  if (e != cudaSuccess) st = from_cuda(e);
  if (st == AP_OK) {
    it->d_status = it->d_queue + 1;
    if (desc->kind == AP_ITEMS_VECTOR) st = create_vectors(desc, it, s);
    else if (desc->kind == AP_ITEMS_SPARSE) st = create_sparse(desc, it, s);
    else st = create_clouds(desc, it, s);
  }
  if (st != AP_OK) {
    cudaDeviceSynchronize();
    free_items(it);
    return st;
  }
  *out = it;
  return AP_OK;
}

ap_status ap_update_items(ap_items *it, const float *data, int32_t data_on_host, void *stream) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (it->kind != AP_ITEMS_VECTOR || it->vec.out_of_core) return AP_ERR_STATE;
  if (it->vec.n > 0 && !data) return AP_ERR_INVALID_ARG;
  if (data_on_host && !it->vec.d_stage && it->vec.n > 0) {
    VecStore &v = it->vec;
    v.stage_rows = std::max<int64_t>(1, std::min<int64_t>(v.n, (256ll << 20) / (v.ld * 4)));
    AP_TRY(dmalloc(&v.d_stage, (size_t)2 * v.stage_rows * v.ld));
  }
  if (it->vec.n == 0) return AP_OK;
  return vec_load(it, data, data_on_host, reinterpret_cast<cudaStream_t>(stream));
}

ap_status ap_run_pairs(ap_items *it, int32_t fn, int32_t precision, const float *params,
                       void *out, void *stream) {
  if (!it) return AP_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t n = it->kind == AP_ITEMS_VECTOR   ? it->vec.n
                    : it->kind == AP_ITEMS_SPARSE ? it->sp.n
                                                  : it->cl.n;
  if (fn != AP_FN_OVERLAP && fn != AP_FN_PEARSON && fn != AP_FN_COVERAGE && fn != AP_FN_GMM_L2 &&
      fn != AP_FN_BHATTACHARYYA && fn != AP_FN_COSINE)
    return AP_ERR_INVALID_ARG;
  if ((fn == AP_FN_COSINE) != (it->kind == AP_ITEMS_SPARSE) && fn != AP_FN_COVERAGE)
    return AP_ERR_INVALID_ARG;
  if (precision != AP_PREC_FP32 && precision != AP_PREC_SPLIT_BF16) return AP_ERR_INVALID_ARG;
  NvtxRange range("ap_run_pairs");
  const bool cloud_fn = fn == AP_FN_OVERLAP || fn == AP_FN_GMM_L2 || fn == AP_FN_BHATTACHARYYA;
  if (cloud_fn && it->kind == AP_ITEMS_VECTOR) return AP_ERR_INVALID_ARG;
  if (fn == AP_FN_PEARSON && it->kind != AP_ITEMS_VECTOR) return AP_ERR_INVALID_ARG;
  if (params && (!cloud_fn || it->kind != AP_ITEMS_CLOUD2D)) return AP_ERR_INVALID_ARG;
  if (n < 2) return AP_OK;
  if (!out) return AP_ERR_INVALID_ARG;
  const int cover = fn == AP_FN_COVERAGE;
  if (it->kind == AP_ITEMS_SPARSE) {
    AP_TRY(launch_sparse_cosine(it->sp, reinterpret_cast<double *>(out), cover, it->d_queue, s));
    it->stats.tiles = it->sp.n_tiles;
    it->stats.tile_m = kSparseBlock;
    it->stats.tile_n = kSparseBlockJ;
    it->stats.item_loads = it->sp.n;
    it->stats.reuse_R = 1.0;
    it->stats.slot_hit_rate = 1.0;
    return AP_OK;
  }
  if (it->kind == AP_ITEMS_VECTOR && it->vec.out_of_core) {
    if (!cover && precision != AP_PREC_SPLIT_BF16) return AP_ERR_STATE;
    return run_out_of_core(it, out, cover, s);
  }
  if (it->kind == AP_ITEMS_VECTOR) {
    VecStore &v = it->vec;
    const bool have_split = v.d_hi != nullptr, have_f32 = v.d_c32 != nullptr;
    bool use_split = precision == AP_PREC_SPLIT_BF16;
    if (cover) use_split = have_split;
    if (use_split && !have_split) return AP_ERR_STATE;
    if (!use_split && !have_f32) return AP_ERR_STATE;
    const bool pairs = v.mma_ctas == 2;
    if (use_split && !cover && v.k_split > 0) {
      // split-K units in waves: partial Grams meet in FP64 in `out`
      AP_TRY(cudaMemsetAsync(out, 0, (size_t)(n * (n - 1) / 2) * sizeof(double), s));
      if (pairs)
        AP_TRY(launch_gram_tc2(v.tmap_hi, v.tmap_lo, v.n, v.d_rs, v.d_pair_units, v.n_pair_units,
                               it->d_queue, it->d_status, v.d_g64, out, 0, 1,
                               it->wait_budget_ns, it->debug, s));
      else
        AP_TRY(launch_gram_tc(v.tmap_hi, v.tmap_lo, v.n, v.Dp, v.d_rs, v.d_panel_units,
                              v.n_panel_units, it->d_queue, it->d_status, v.d_g64, out, 0, 1,
                              it->wait_budget_ns, it->debug, s));
      AP_TRY(launch_pair_finalize(reinterpret_cast<double *>(out), v.d_rs, v.d_delta_all, v.n,
                                  v.D, s));
      it->stats.tiles = pairs ? v.n_pair_units : v.n_panel_units;
      it->stats.tile_m = pairs ? 2 * kTcTileM : kTcTileM;
      it->stats.tile_n = kTcTileN;
    } else if (use_split && pairs) {
      // whole block pairs (or coverage) on CTA pairs
      AP_TRY(launch_gram_tc2(v.tmap_hi, v.tmap_lo, v.n, v.d_rs, v.d_pair_whole, v.n_pair_whole,
                             it->d_queue, it->d_status, v.d_g64, out, cover, 0,
                             it->wait_budget_ns, it->debug, s));
      if (!cover)
        AP_TRY(launch_pair_correct(reinterpret_cast<double *>(out), v.d_rs, v.d_delta_all, v.n,
                                   v.D, s));
      it->stats.tiles = v.n_pair_whole;
      it->stats.tile_m = 2 * kTcTileM;
      it->stats.tile_n = kTcTileN;
    } else if (use_split) {
      AP_TRY(launch_gram_tc(v.tmap_hi, v.tmap_lo, v.n, v.Dp, v.d_rs, v.d_tiles_tc, v.n_tiles_tc,
                            it->d_queue, it->d_status, v.d_g64, out, cover, 0,
                            it->wait_budget_ns, it->debug, s));
      if (!cover)
        AP_TRY(launch_pair_correct(reinterpret_cast<double *>(out), v.d_rs, v.d_delta_all, v.n,
                                   v.D, s));
      it->stats.tiles = v.n_tiles_tc;
      it->stats.tile_m = kTcTileM;
      it->stats.tile_n = kTcTileN;
    } else {
      AP_TRY(launch_gram_f32(v.d_c32, v.n, v.Dp, v.d_rs, v.d_tiles_f32, v.n_tiles_f32,
                             it->d_queue, out, cover, 0, v.n, s, v.d_delta_all, v.D));
      it->stats.tiles = v.n_tiles_f32;
      it->stats.tile_m = 128;
      it->stats.tile_n = 128;
    }
    it->stats.item_loads = v.n;
    it->stats.reuse_R = 1.0;
    it->stats.slot_hit_rate = 1.0;
    return AP_OK;
  }
  if (fn == AP_FN_GMM_L2 || fn == AP_FN_BHATTACHARYYA) {
    const int score = fn == AP_FN_GMM_L2 ? 1 : 2;
    AP_TRY_ST(ensure_score_storage(it, score, s));
    GraphKey key{3 + score, params, out, nullptr, nullptr, 0.f, 0.f, 1};
    ap_items *h = it;
    ap_status st = run_graphed(it, key, s, [h, params, out, score](cudaStream_t cs) {
      const CloudStore &c = h->cl;
      return launch_score(c, score, c.d_pts_score[score - 1], c.d_lw_score[score - 1], c.d_self,
                          params, reinterpret_cast<float *>(out), h->d_queue, cs);
    });
    if (st != AP_OK) return st;
    it->stats.tiles = it->cl.n_tiles;
    it->stats.item_loads = it->cl.n;
    it->stats.reuse_R = 1.0;
    it->stats.slot_hit_rate = 1.0;
    return AP_OK;
  }
  {
    GraphKey key{1 + cover, params, out, nullptr, nullptr, 0.f, 0.f, 1};
    ap_items *h = it;
    ap_status st = run_graphed(it, key, s, [h, params, out, cover](cudaStream_t cs) {
      return launch_overlap(h->cl, params, reinterpret_cast<float *>(out), cover, h->d_queue, cs);
    });
    if (st != AP_OK) return st;
  }
  it->stats.tiles = it->cl.n_tiles;
  it->stats.item_loads = it->cl.n;
  it->stats.reuse_R = 1.0;
  it->stats.slot_hit_rate = 1.0;
  return AP_OK;
}


ap_status ap_backward(ap_items *it, const float *params, const float *grad_out,
                      float *grad_params, float *f_out, void *stream) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (it->kind != AP_ITEMS_CLOUD2D) return AP_ERR_INVALID_ARG;
  if (it->cl.n < 2) return AP_OK;
  if (!grad_params) return AP_ERR_INVALID_ARG;
  AP_TRY(launch_overlap_grad_q(it->cl, it->d_queue, params, grad_out, grad_params, f_out, 0.f, 0.f,
                               nullptr, nullptr, reinterpret_cast<cudaStream_t>(stream)));
  return AP_OK;
}

ap_status ap_ascent(ap_items *it, float *params, int32_t n_steps, float eta, float fmin,
                    float *f_out, int32_t *flags, void *stream) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (it->kind != AP_ITEMS_CLOUD2D || n_steps < 0) return AP_ERR_INVALID_ARG;
  if (it->cl.n < 2 || n_steps == 0) return AP_OK;
  if (!params) return AP_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the n_steps fused steps are replayed as one CUDA graph
  GraphKey key{3, params, f_out, flags, nullptr, eta, fmin, n_steps};
  ap_items *h = it;
  return run_graphed(it, key, s, [h, params, n_steps, eta, fmin, f_out, flags](cudaStream_t cs) {
    for (int32_t k = 0; k < n_steps; ++k) {
      cudaError_t e = launch_overlap_grad_q(h->cl, h->d_queue, nullptr, nullptr, nullptr, f_out,
                                            eta, fmin, params, flags, cs);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  });
}

ap_status ap_destroy(ap_items *it) {
  if (!it) return AP_OK;
  cudaDeviceSynchronize();
  free_items(it);
  return AP_OK;
}

ap_status ap_get_stats(const ap_items *it, ap_run_stats *out) {
  if (!it || !out) return AP_ERR_INVALID_ARG;
  *out = it->stats;
  return AP_OK;
}

ap_status ap_set_debug(ap_items *it, int32_t flags, uint64_t wait_budget_ns) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (flags != AP_DEBUG_NONE && flags != AP_DEBUG_WITHHOLD_STAGE &&
      flags != AP_DEBUG_WITHHOLD_LATER_STAGE)
    return AP_ERR_INVALID_ARG;
  it->debug = flags;
  it->wait_budget_ns = wait_budget_ns;
  return AP_OK;
}

int32_t ap_last_device_error(ap_items *it) {
  if (!it || !it->d_status) return 0;
  int32_t v = 0;
  if (cudaMemcpy(&v, it->d_status, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (v != 0) cudaMemset(it->d_status, 0, sizeof v);
  return v;
}

}  // extern "C"
