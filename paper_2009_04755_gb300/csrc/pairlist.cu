// pairlist.cu -- the pair function over a chosen list of pairs instead of the
// whole upper triangle: the comparison stage of Sec. III on a subset, and the
// per-pair registration of chosen pairs (Sec. V-C).
//
// Clouds reuse the all-pairs kernel: each listed pair (a, b) becomes a tile
// of two one-item blocks (storage positions of a and b), and the kernel's
// list mode puts tile t's transform and outputs at index t; the transform
// acts on b, as it acts on the second item of a packed pair.  A pair listed
// in packed order (a < b) therefore gets exactly the operations, and the
// bits, of the all-pairs run.
//
// Vectors use one warp per listed pair over the resident centred rows (split
// BF16 or FP32 copy), the same three products per column as the tensor-core
// Gram, summed in FP32 over 64 column blocks per lane and in FP64 after:
//   r_k = (sum_c c_a c_b - D delta_a delta_b) rs_a rs_b.
// The blocked layout puts a row's 32-column pieces 8 KB apart, so a row is
// read as scattered 64-byte pieces; the list is therefore run sorted by the
// row blocks of its two items (smaller item first: r is symmetric), so that
// the warps in flight read pieces of the same 8 KB blocks, and each result
// goes back to its list position.
// Sparse rows merge their sorted codes (one CTA per pair).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ap_internal.h"

namespace ap {

namespace {

constexpr int kListThreads = 256;

template <bool SPLIT>
__global__ void __launch_bounds__(kListThreads)
pearson_list_kernel(const __nv_bfloat16 *__restrict__ hi, const __nv_bfloat16 *__restrict__ lo,
                    const float *__restrict__ c32, int64_t Dp, const int32_t *__restrict__ pi,
                    const int32_t *__restrict__ pj, const int32_t *__restrict__ pos,
                    int64_t n_pairs, const double *__restrict__ rs,
                    const double *__restrict__ delta, int64_t D, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n_pairs;
       k += warps) {
    const int64_t a = pi[k], b = pj[k];
    double acc = 0.0;
    float part = 0.f;
    if (SPLIT) {
      // lane l takes column l of every 32-column block (64 contiguous bytes
      // per row and block for the warp)
      // four blocks per trip, all sixteen loads issued before any product
      // (Dp is a multiple of 64, so the block count is even, not always a
      // multiple of four: the last trip may hold two)
      const int64_t nkb = Dp / kTcKBlock;
      constexpr size_t kBlock = (size_t)kRowBlock * kTcKBlock;   // elements per block
      const size_t ra = blocked_offset(a, lane, nkb, kTcKBlock);
      const size_t rb = blocked_offset(b, lane, nkb, kTcKBlock);
      for (int64_t kb = 0; kb < nkb; kb += 4) {
        float ha[4], la[4], hb[4], lb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = kb + u < nkb;
          const size_t o = (size_t)(kb + u) * kBlock;
          ha[u] = in ? __bfloat162float(hi[ra + o]) : 0.f;
          la[u] = in ? __bfloat162float(lo[ra + o]) : 0.f;
          hb[u] = in ? __bfloat162float(hi[rb + o]) : 0.f;
          lb[u] = in ? __bfloat162float(lo[rb + o]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          part = fmaf(ha[u], hb[u], part);
          part = fmaf(ha[u], lb[u], part);
          part = fmaf(la[u], hb[u], part);
        }
        if ((kb & 63) == 60) {                     // 64 blocks per FP32 partial
          acc += (double)part;
          part = 0.f;
        }
      }
    } else {
      const int64_t nkb = Dp / kF32KBlock;
      for (int64_t col = lane, m = 0; col < Dp; col += 32, ++m) {
        const float ca = c32[blocked_offset(a, col, nkb, kF32KBlock)];
        const float cb = c32[blocked_offset(b, col, nkb, kF32KBlock)];
        part = fmaf(ca, cb, part);
        if ((m & 63) == 63) {
          acc += (double)part;
          part = 0.f;
        }
      }
    }
    acc += (double)part;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[pos[k]] = (acc - (double)D * delta[a] * delta[b]) * rs[a] * rs[b];
  }
}

// Sparse rows (strictly increasing codes): one CTA per listed pair, each
// thread merging an even slice of row a's entries against row b from the
// first code of b at or after its slice (a binary search), so a pair costs
// about nnz_a + nnz_b reads; FP32 products summed per thread in FP64.
constexpr int kMergeThreads = 256;
__global__ void __launch_bounds__(kMergeThreads)
cosine_list_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                   const float *__restrict__ val, const double *__restrict__ rs,
                   const int32_t *__restrict__ pi, const int32_t *__restrict__ pj,
                   int64_t n_pairs, double *__restrict__ out) {
  __shared__ double red[kMergeThreads / 32];
  for (int64_t k = blockIdx.x; k < n_pairs; k += gridDim.x) {
    const int64_t a = pi[k], b = pj[k];
    const int64_t a0 = off[a], na = off[a + 1] - a0, b0 = off[b], nb = off[b + 1] - b0;
    const int64_t per = (na + blockDim.x - 1) / blockDim.x;
    const int64_t s0 = (int64_t)threadIdx.x * per, s1 = s0 + per < na ? s0 + per : na;
    double acc = 0.0;
    if (s0 < s1) {
      // first entry of b whose code is >= the slice's first code
      const int32_t c0 = idx[a0 + s0];
      int64_t lo = 0, hi = nb;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (idx[b0 + mid] < c0) lo = mid + 1;
        else hi = mid;
      }
      int64_t q = lo;
      for (int64_t e = s0; e < s1 && q < nb; ++e) {
        const int32_t code = idx[a0 + e];
        while (q < nb && idx[b0 + q] < code) ++q;
        if (q < nb && idx[b0 + q] == code) acc += (double)(val[a0 + e] * val[b0 + q]);
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      out[k] = t * rs[a] * rs[b];
    }
    __syncthreads();
  }
}

// host checks shared by every list call: indices in range, a != b
ap_status check_list(const ap_items *it, const int32_t *pi, const int32_t *pj, int64_t n_pairs,
                     int64_t n) {
  if (n_pairs < 0 || (n_pairs > 0 && (!pi || !pj))) return AP_ERR_INVALID_ARG;
  if (n_pairs > INT32_MAX) return AP_ERR_UNSUPPORTED;   // tile indices are int32
  for (int64_t k = 0; k < n_pairs; ++k)
    if (pi[k] < 0 || pj[k] < 0 || pi[k] >= n || pj[k] >= n || pi[k] == pj[k])
      return AP_ERR_INVALID_ARG;
  (void)it;
  return AP_OK;
}

// the temporary list plan of a cloud set: one-item blocks, the listed pairs
// as tiles (storage positions), copied to the handle's list buffer on `s`
ap_status cloud_list_plan(ap_items *it, const int32_t *pi, const int32_t *pj, int64_t n_pairs,
                          cudaStream_t s, CloudStore &lc) {
  CloudStore &c = it->cl;
  if (c.h_iperm.size() != (size_t)c.n) {
    c.h_iperm.assign((size_t)c.n, 0);
    for (int64_t p = 0; p < c.n; ++p) c.h_iperm[c.h_perm[p]] = (int32_t)p;
  }
  std::vector<int32_t> single((size_t)c.n + 1);
  for (int64_t b = 0; b <= c.n; ++b) single[b] = (int32_t)b;
  if (!c.d_bstart_single) {
    AP_TRY(dmalloc(&c.d_bstart_single, single.size()));
    AP_TRY(cudaMemcpy(c.d_bstart_single, single.data(), single.size() * 4,
                      cudaMemcpyHostToDevice));
  }
  if (c.list_cap < n_pairs) {
    AP_TRY(cudaStreamSynchronize(s));              // the old list may still be read
    dfree(c.d_list_tiles);
    c.list_cap = 0;
    AP_TRY(dmalloc(&c.d_list_tiles, (size_t)n_pairs * 2));
    c.list_cap = n_pairs;
  } else {
    AP_TRY(cudaStreamSynchronize(s));
  }
  std::vector<int32_t> tiles((size_t)n_pairs * 2);
  for (int64_t k = 0; k < n_pairs; ++k) {
    tiles[2 * k] = c.h_iperm[pi[k]];
    tiles[2 * k + 1] = c.h_iperm[pj[k]];
  }
  AP_TRY(cudaMemcpy(c.d_list_tiles, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice));
  std::vector<int64_t> cnt((size_t)c.n);
  for (int64_t p = 0; p < c.n; ++p) cnt[p] = c.h_size[c.h_perm[p]];
  lc = c;
  lc.list_mode = true;
  lc.d_bstart = c.d_bstart_single;
  lc.d_tiles = c.d_list_tiles;
  lc.n_tiles = n_pairs;
  lc.block_items = 1;
  lc.max_rj = max_row_jobs(single, cnt, 32LL * c.reg_r);
  // a J block is one item: stage as many points as the largest item has
  int64_t most = 4;
  for (int64_t p = 0; p < c.n; ++p) most = std::max(most, c.h_poff[p + 1] - c.h_poff[p]);
  lc.block_pts = (int32_t)std::min<int64_t>(most, c.block_pts);
  return AP_OK;
}

// the listed pairs' indices on the device (host arrays in, stream-ordered)
ap_status device_pairs(const int32_t *pi, const int32_t *pj, int64_t n_pairs, cudaStream_t s,
                       int32_t **d_idx) {
  AP_TRY(dmalloc(d_idx, (size_t)n_pairs * 2));
  AP_TRY(cudaMemcpyAsync(*d_idx, pi, (size_t)n_pairs * 4, cudaMemcpyHostToDevice, s));
  AP_TRY(cudaMemcpyAsync(*d_idx + n_pairs, pj, (size_t)n_pairs * 4, cudaMemcpyHostToDevice, s));
  return AP_OK;
}

// the listed vector pairs sorted by the row blocks of their items (smaller
// item first), with their list positions: [a...][b...][position...] on the
// device (the host copy goes through a pageable buffer, staged by the call)
ap_status device_pairs_by_block(const int32_t *pi, const int32_t *pj, int64_t n_pairs,
                                cudaStream_t s, int32_t **d_idx) {
  std::vector<uint64_t> key((size_t)n_pairs);
  for (int64_t k = 0; k < n_pairs; ++k) {
    const uint32_t a = (uint32_t)std::min(pi[k], pj[k]), b = (uint32_t)std::max(pi[k], pj[k]);
    const uint64_t blocks = ((uint64_t)(a / kRowBlock) << 16) | (uint64_t)(b / kRowBlock);
    key[k] = (blocks << 32) | (uint64_t)k;     // row blocks < 2^16 (n <= INT32_MAX / 2)
  }
  std::sort(key.begin(), key.end());
  std::vector<int32_t> h((size_t)n_pairs * 3);
  for (int64_t q = 0; q < n_pairs; ++q) {
    const int64_t k = (int64_t)(key[q] & 0xffffffffu);
    h[q] = std::min(pi[k], pj[k]);
    h[n_pairs + q] = std::max(pi[k], pj[k]);
    h[2 * n_pairs + q] = (int32_t)k;
  }
  AP_TRY(dmalloc(d_idx, h.size()));
  AP_TRY(cudaMemcpyAsync(*d_idx, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s));
  return AP_OK;
}

}  // namespace

cudaError_t launch_pearson_list(const VecStore &v, bool split, const int32_t *pi,
                                const int32_t *pj, const int32_t *pos, int64_t n_pairs,
                                double *out, cudaStream_t s) {
  if (n_pairs <= 0) return cudaSuccess;
  const int64_t need = (n_pairs + (kListThreads / 32) - 1) / (kListThreads / 32);
  const int grid = (int)std::min<int64_t>(need, (int64_t)num_sms() * 8);
  if (split)
    pearson_list_kernel<true><<<grid, kListThreads, 0, s>>>(v.d_hi, v.d_lo, nullptr, v.Dp, pi, pj,
                                                            pos, n_pairs, v.d_rs, v.d_delta_all,
                                                            v.D, out);
  else
    pearson_list_kernel<false><<<grid, kListThreads, 0, s>>>(nullptr, nullptr, v.d_c32, v.Dp, pi,
                                                             pj, pos, n_pairs, v.d_rs,
                                                             v.d_delta_all, v.D, out);
  return cudaGetLastError();
}

}  // namespace ap

using namespace ap;

extern "C" ap_status ap_run_pairs_list(ap_items *it, int32_t fn, int32_t precision,
                                       const int32_t *pi, const int32_t *pj, int64_t n_pairs,
                                       const float *params, void *out, void *stream) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (precision != AP_PREC_FP32 && precision != AP_PREC_SPLIT_BF16) return AP_ERR_INVALID_ARG;
  const bool cloud_fn = fn == AP_FN_OVERLAP || fn == AP_FN_GMM_L2 || fn == AP_FN_BHATTACHARYYA;
  const bool cloud = it->kind == AP_ITEMS_CLOUD2D || it->kind == AP_ITEMS_CLOUD3D;
  const bool ok_kind = cloud ? cloud_fn
                             : (it->kind == AP_ITEMS_VECTOR && fn == AP_FN_PEARSON) ||
                                   (it->kind == AP_ITEMS_SPARSE && fn == AP_FN_COSINE);
  if (!ok_kind) return AP_ERR_INVALID_ARG;
  if (params && it->kind != AP_ITEMS_CLOUD2D) return AP_ERR_INVALID_ARG;
  const int64_t n = cloud ? it->cl.n : it->kind == AP_ITEMS_SPARSE ? it->sp.n : it->vec.n;
  AP_TRY_ST(check_list(it, pi, pj, n_pairs, n));
  if (n_pairs == 0) return AP_OK;
  if (!out) return AP_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!cloud) {
    const bool sparse = it->kind == AP_ITEMS_SPARSE;
    const bool split = precision == AP_PREC_SPLIT_BF16;
    if (!sparse) {
      const VecStore &v = it->vec;
      if (v.out_of_core) return AP_ERR_UNSUPPORTED;   // rows are not resident
      if ((split && !v.d_hi) || (!split && !v.d_c32)) return AP_ERR_STATE;
    }
    int32_t *d_idx = nullptr;
    ap_status st = sparse ? device_pairs(pi, pj, n_pairs, s, &d_idx)
                          : device_pairs_by_block(pi, pj, n_pairs, s, &d_idx);
    cudaError_t e = cudaSuccess;
    if (st == AP_OK) {
      if (sparse) {
        const SparseStore &sp = it->sp;
        const int grid = (int)std::min<int64_t>(n_pairs, (int64_t)num_sms() * 8);
        cosine_list_kernel<<<grid, kMergeThreads, 0, s>>>(sp.d_off, sp.d_idx, sp.d_val, sp.d_rs,
                                                           d_idx, d_idx + n_pairs, n_pairs,
                                                           reinterpret_cast<double *>(out));
        e = cudaGetLastError();
      } else {
        e = launch_pearson_list(it->vec, split, d_idx, d_idx + n_pairs, d_idx + 2 * n_pairs,
                                n_pairs, reinterpret_cast<double *>(out), s);
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // before the index buffer goes
      st = e == cudaSuccess ? AP_OK : from_cuda(e);
    }
    dfree(d_idx);
    return st;
  }
  CloudStore lc;
  AP_TRY_ST(cloud_list_plan(it, pi, pj, n_pairs, s, lc));
  if (fn == AP_FN_OVERLAP)
    AP_TRY(launch_overlap(lc, params, reinterpret_cast<float *>(out), 0, it->d_queue, s));
  else {
    const int score = fn == AP_FN_GMM_L2 ? 1 : 2;
    AP_TRY_ST(ensure_score_storage(it, score, s));
    const CloudStore &c = it->cl;
    AP_TRY(launch_score(lc, score, c.d_pts_score[score - 1], c.d_lw_score[score - 1], c.d_self,
                        params, reinterpret_cast<float *>(out), it->d_queue, s));
  }
  return AP_OK;
}

extern "C" ap_status ap_backward_list(ap_items *it, const int32_t *pi, const int32_t *pj,
                                      int64_t n_pairs, const float *params,
                                      const float *grad_out, float *grad_params, float *f_out,
                                      void *stream) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (it->kind != AP_ITEMS_CLOUD2D) return AP_ERR_INVALID_ARG;
  AP_TRY_ST(check_list(it, pi, pj, n_pairs, it->cl.n));
  if (n_pairs == 0) return AP_OK;
  if (!grad_params) return AP_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CloudStore lc;
  AP_TRY_ST(cloud_list_plan(it, pi, pj, n_pairs, s, lc));
  AP_TRY(launch_overlap_grad_q(lc, it->d_queue, params, grad_out, grad_params, f_out, 0.f, 0.f,
                               nullptr, nullptr, s));
  return AP_OK;
}

extern "C" ap_status ap_ascent_list(ap_items *it, const int32_t *pi, const int32_t *pj,
                                    int64_t n_pairs, float *params, int32_t n_steps, float eta,
                                    float fmin, float *f_out, int32_t *flags, void *stream) {
  if (!it) return AP_ERR_INVALID_ARG;
  if (it->kind != AP_ITEMS_CLOUD2D || n_steps < 0) return AP_ERR_INVALID_ARG;
  AP_TRY_ST(check_list(it, pi, pj, n_pairs, it->cl.n));
  if (n_pairs == 0 || n_steps == 0) return AP_OK;
  if (!params) return AP_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CloudStore lc;
  AP_TRY_ST(cloud_list_plan(it, pi, pj, n_pairs, s, lc));
  for (int32_t k = 0; k < n_steps; ++k)
    AP_TRY(launch_overlap_grad_q(lc, it->d_queue, nullptr, nullptr, nullptr, f_out, eta, fmin,
                                 params, flags, s));
  return AP_OK;
}
