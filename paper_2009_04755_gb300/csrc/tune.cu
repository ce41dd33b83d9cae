// tune.cu -- autotuner of the point-cloud tile plan, and CUDA-graph replay of
// the cloud launches.
//
// The tuner times every candidate plan (items per block, staged points per
// block, a-points per lane) on an evenly spread sample of its own tiles --
// about 2e10 point pairs, or everything when the workload is smaller -- and
// keeps the fastest.  The tile order stays the recursive quadrant order of
// the block grid (Sec. IV-B); what the tuner changes is the block size, i.e.
// how many items one tile reuses from shared memory and registers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ap_internal.h"

namespace ap {

int32_t min_reg_r(const CloudStore &c) {
  int64_t mx = 0;
  for (int64_t s : c.h_size) mx = std::max(mx, s);
  int32_t r = 2;                        // a-points go in pairs (FP32x2)
  while ((int64_t)r * 32 * kOverlapMaxRowJobs < mx && r < 4) r *= 2;
  return r;
}

void clear_graphs(ap_items *it) {
  for (GraphEntry &g : it->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  it->graphs.clear();
}

ap_status run_graphed(ap_items *it, const GraphKey &key, cudaStream_t s,
                      const std::function<cudaError_t(cudaStream_t)> &seq) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (s) AP_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return from_cuda(seq(s));   // caller is capturing
  for (GraphEntry &g : it->graphs)
    if (g.key == key && g.plan_version == it->plan_version) return from_cuda(cudaGraphLaunch(g.exec, s));
  AP_TRY(cudaStreamBeginCapture(it->graph_stream, cudaStreamCaptureModeRelaxed));
  cudaError_t e = seq(it->graph_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(it->graph_stream, &graph);
  if (e == cudaSuccess) e = e2;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return from_cuda(e);
  if (it->graphs.size() >= 16) {
    cudaGraphExecDestroy(it->graphs.front().exec);
    it->graphs.erase(it->graphs.begin());
  }
  it->graphs.push_back({key, it->plan_version, exec});
  return from_cuda(cudaGraphLaunch(exec, s));
}

namespace {

// point pairs of one block pair (I, J) of a candidate plan
double tile_cost(const std::vector<int32_t> &bstart, const std::vector<int64_t> &cnt, int32_t I,
                 int32_t J) {
  double si = 0, sj = 0, sq = 0;
  for (int32_t k = bstart[I]; k < bstart[I + 1]; ++k) { si += (double)cnt[k]; sq += (double)cnt[k] * cnt[k]; }
  if (I == J) return (si * si - sq) / 2;
  for (int32_t k = bstart[J]; k < bstart[J + 1]; ++k) sj += (double)cnt[k];
  return si * sj;
}

}  // namespace

// A set whose points fit many times into L2 gains nothing from the quadrant
// order's locality, but a queue of uneven tiles ends with a tail: such sets
// pop their tiles largest first (the greedy longest-first rule), so the last
// tiles taken are the small ones.
constexpr int64_t kLargestFirstBytes = 16ll << 20;

bool order_cloud_tiles(const std::vector<int32_t> &bstart, const std::vector<int64_t> &cnt,
                       int64_t total_pts, std::vector<int32_t> &tiles) {
  if (total_pts * (int64_t)(sizeof(float4) + sizeof(float)) > kLargestFirstBytes) return false;
  const size_t nt = tiles.size() / 2;
  std::vector<std::pair<double, int64_t>> key(nt);
  for (size_t t = 0; t < nt; ++t) key[t] = {-tile_cost(bstart, cnt, tiles[2 * t], tiles[2 * t + 1]), (int64_t)t};
  std::stable_sort(key.begin(), key.end(),
                   [](const std::pair<double, int64_t> &a, const std::pair<double, int64_t> &b) {
                     return a.first < b.first;
                   });
  std::vector<int32_t> out(tiles.size());
  for (size_t t = 0; t < nt; ++t) {
    out[2 * t] = tiles[2 * key[t].second];
    out[2 * t + 1] = tiles[2 * key[t].second + 1];
  }
  tiles.swap(out);
  return true;
}

}  // namespace ap

using namespace ap;

extern "C" ap_status ap_get_plan(const ap_items *it, ap_plan *out) {
  if (!it || !out) return AP_ERR_INVALID_ARG;
  out->k_split = 0;
  out->mma_ctas = 0;
  if (it->kind == AP_ITEMS_SPARSE) {
    out->block_items = kSparseBlock;       // items i of a tile (j: kSparseBlockJ)
    out->block_pts = kSparseBlockJ;
    out->reg_r = out->sorted = 0;
    out->rate = 0.0;
    return AP_OK;
  }
  if (it->kind == AP_ITEMS_VECTOR) {
    out->block_items = kTcTileM;
    out->block_pts = kTcTileN;
    out->reg_r = 0;
    out->sorted = 0;
    out->rate = 0.0;
    out->k_split = it->vec.k_split;
    out->mma_ctas = it->vec.mma_ctas;
    return AP_OK;
  }
  out->block_items = it->cl.block_items;
  out->block_pts = it->cl.block_pts;
  out->reg_r = it->cl.reg_r;
  out->sorted = it->cl.sorted ? 1 : 0;
  out->rate = 0.0;
  return AP_OK;
}

int32_t ap::default_k_split(int64_t n_tiles, int64_t Dp) {
  // column ranges of about kKSplitCols columns, and at least two units per SM
  const int64_t nch = Dp / kOocChunkCols;
  int64_t k = (Dp + kKSplitCols - 1) / kKSplitCols;
  if (n_tiles > 0) k = std::max<int64_t>(k, (2LL * num_sms() + n_tiles - 1) / n_tiles);
  k = std::min<int64_t>(k, std::min<int64_t>(nch, kMaxKSplit));
  return k <= 1 ? 0 : (int32_t)k;
}

namespace {
ap_status upload_units(const std::vector<int32_t> &units, int32_t **d, int64_t *n) {
  dfree(*d);
  *n = 0;
  AP_TRY(dmalloc(d, std::max<size_t>(units.size(), kOocTileInts)));
  if (!units.empty())
    AP_TRY(cudaMemcpy(*d, units.data(), units.size() * 4, cudaMemcpyHostToDevice));
  *n = (int64_t)units.size() / kOocTileInts;
  return AP_OK;
}
}  // namespace

// vector sets: (re)build the split-K wave units of the tensor-core tiles,
// for one CTA per tile (mma_ctas 1) or CTA pairs (mma_ctas 2; 0 = 2)
ap_status ap::set_vector_plan(ap_items *it, int32_t k_split, int32_t mma_ctas) {
  VecStore &v = it->vec;
  if (v.out_of_core) return AP_ERR_STATE;
  if (!v.d_hi) return AP_ERR_STATE;
  if (mma_ctas == 0) mma_ctas = 2;
  if (mma_ctas != 1 && mma_ctas != 2) return AP_ERR_INVALID_ARG;
  if (k_split < 0) k_split = default_k_split(v.n_tiles_tc, v.Dp);
  cudaError_t e = cudaDeviceSynchronize();      // the old units may still be in use
  if (e != cudaSuccess) return from_cuda(e);
  dfree(v.d_panel_units);
  dfree(v.d_pair_units);
  dfree(v.d_pair_whole);
  v.n_panel_units = v.n_pair_units = v.n_pair_whole = 0;
  v.k_split = 0;
  v.mma_ctas = mma_ctas;
  const int64_t nch = v.Dp / kOocChunkCols;
  std::vector<int32_t> units;
  if (mma_ctas == 2) {
    pair_units(v.n, nch, tc2_pairs(), 1, units);          // whole columns, one per macro pair
    AP_TRY_ST(upload_units(units, &v.d_pair_whole, &v.n_pair_whole));
  }
  if (k_split == 0) return AP_OK;
  if (mma_ctas == 2) {
    pair_units(v.n, nch, tc2_pairs(), k_split, units);
    AP_TRY_ST(upload_units(units, &v.d_pair_units, &v.n_pair_units));
  } else {
    panel_units(v.h_tiles_tc, nch, tc_grid(v.n_tiles_tc), k_split, units);
    AP_TRY_ST(upload_units(units, &v.d_panel_units, &v.n_panel_units));
  }
  v.k_split = k_split;
  return AP_OK;
}

extern "C" ap_status ap_set_plan(ap_items *it, const ap_plan *plan) {
  if (!it || !plan) return AP_ERR_INVALID_ARG;
  if (it->kind == AP_ITEMS_SPARSE) return AP_ERR_UNSUPPORTED;
  if (it->kind == AP_ITEMS_VECTOR) {
    if (plan->block_items != kTcTileM || plan->block_pts != kTcTileN) return AP_ERR_INVALID_ARG;
    if (plan->k_split < -1 || plan->k_split > kMaxKSplit) return AP_ERR_INVALID_ARG;
    if (plan->mma_ctas < 0 || plan->mma_ctas > 2) return AP_ERR_INVALID_ARG;
    return set_vector_plan(it, plan->k_split, plan->mma_ctas);
  }
  if (plan->block_items < 1 || plan->block_items > kOverlapMaxBlockItems) return AP_ERR_INVALID_ARG;
  if (plan->block_pts < 64 || plan->block_pts > 8192) return AP_ERR_INVALID_ARG;
  if (plan->reg_r != 2 && plan->reg_r != 4) return AP_ERR_INVALID_ARG;
  if (plan->reg_r < min_reg_r(it->cl)) return AP_ERR_INVALID_ARG;
  CloudPlanChoice ch{plan->block_items, plan->block_pts, plan->reg_r, it->cl.sorted};
  cudaError_t e = cudaDeviceSynchronize();      // the old plan may still be in use
  if (e != cudaSuccess) return from_cuda(e);
  return build_cloud_plan(it, ch);
}

extern "C" ap_status ap_tune(ap_items *it, int32_t mode, void *stream, ap_plan *out) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (mode != 0 && mode != 1) return AP_ERR_INVALID_ARG;
  if (it->kind == AP_ITEMS_VECTOR || it->kind == AP_ITEMS_SPARSE) return AP_ERR_UNSUPPORTED;
  if (mode == 1 && it->kind != AP_ITEMS_CLOUD2D) return AP_ERR_INVALID_ARG;
  CloudStore &c = it->cl;
  if (c.n < 2) {
    if (out) ap_get_plan(it, out);
    return AP_OK;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<int64_t> cnt(c.n);
  for (int64_t k = 0; k < c.n; ++k) cnt[k] = c.h_size[c.h_perm[k]];
  const int64_t P = c.n * (c.n - 1) / 2;
  const double budget = 2e10;

  float *d_out = nullptr, *d_g = nullptr;
  int32_t *d_bstart = nullptr, *d_tiles = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ap_status st = AP_OK;
  cudaError_t e = dmalloc(&d_out, (size_t)P);
  if (e == cudaSuccess && mode == 1) e = dmalloc(&d_g, (size_t)P * 3);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);

  CloudPlanChoice best{0, 0, 0, c.sorted};
  double best_rate = -1.0;
  const int32_t rmin = min_reg_r(c);
  for (int32_t rr : {2, 4}) {
    if (rr < rmin || e != cudaSuccess) continue;
    for (int32_t bp : {2048, 4096, 8192}) {
      for (int32_t bi : {2, 4, 8, 16, 32}) {
        if (e != cudaSuccess) break;
        std::vector<int32_t> bstart, tiles;
        make_blocks(c.h_poff, cnt, bi, bp, 32LL * rr, kOverlapMaxRowJobs, bstart);
        dc_block_pairs((int64_t)bstart.size() - 1, tiles);
        order_cloud_tiles(bstart, cnt, c.total_pts, tiles);
        const int64_t nt = (int64_t)tiles.size() / 2;
        std::vector<double> cost(nt);
        double total = 0;
        for (int64_t t = 0; t < nt; ++t) {
          cost[t] = tile_cost(bstart, cnt, tiles[2 * t], tiles[2 * t + 1]);
          total += cost[t];
        }
        // evenly spread sample of about `budget` point pairs, at least a few
        // tiles per SM
        int64_t stride = 1;
        if (total > budget) stride = (int64_t)std::ceil(total / budget);
        stride = std::min<int64_t>(stride, std::max<int64_t>(1, nt / (8LL * num_sms())));
        std::vector<int32_t> sample;
        double scost = 0;
        for (int64_t t = 0; t < nt; t += stride) {
          sample.push_back(tiles[2 * t]);
          sample.push_back(tiles[2 * t + 1]);
          scost += cost[t];
        }
        dfree(d_bstart);
        dfree(d_tiles);
        e = dmalloc(&d_bstart, bstart.size());
        if (e == cudaSuccess) e = dmalloc(&d_tiles, std::max<size_t>(sample.size(), 2));
        if (e == cudaSuccess)
          e = cudaMemcpy(d_bstart, bstart.data(), bstart.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !sample.empty())
          e = cudaMemcpy(d_tiles, sample.data(), sample.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
        CloudStore cand = c;                 // shallow copy pointing at the sample plan
        cand.d_bstart = d_bstart;
        cand.d_tiles = d_tiles;
        cand.n_tiles = (int64_t)sample.size() / 2;
        cand.block_items = bi;
        cand.block_pts = bp;
        cand.reg_r = rr;
        cand.max_rj = max_row_jobs(bstart, cnt, 32LL * rr);
        auto launch = [&]() {
          return mode == 0 ? launch_overlap(cand, nullptr, d_out, 0, it->d_queue, s)
                           : launch_overlap_grad_q(cand, it->d_queue, nullptr, nullptr, d_g, d_out,
                                                   0.f, 0.f, nullptr, nullptr, s);
        };
        float ms_best = 1e30f;
        e = launch();
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
          e = cudaEventRecord(e0, s);
          if (e == cudaSuccess) e = launch();
          if (e == cudaSuccess) e = cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          ms_best = std::min(ms_best, ms);
        }
        if (e != cudaSuccess) break;
        const double rate = scost / (ms_best * 1e-3);
        if (rate > best_rate) {
          best_rate = rate;
          best = {bi, bp, rr, c.sorted};
        }
      }
    }
  }
  if (e != cudaSuccess) st = from_cuda(e);
  dfree(d_out);
  dfree(d_g);
  dfree(d_bstart);
  dfree(d_tiles);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st != AP_OK) return st;
  if (best_rate > 0) {
    st = build_cloud_plan(it, best);
    if (st != AP_OK) return st;
  }
  if (out) {
    ap_get_plan(it, out);
    out->rate = best_rate;
  }
  return AP_OK;
}
