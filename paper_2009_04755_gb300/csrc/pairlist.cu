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

// Long lists read a row-major copy instead.  Scattered 64-byte pieces reach
// about a quarter of the HBM copy rate; when the list reads the rows it
// touches several times over, the call first copies the touched row blocks
// into a row-major buffer of one 4-byte word per column (a split column's hi
// and lo bf16 packed, hi in the low half; or the FP32 value), streaming the
// blocked arrays once, and each pair then reads two contiguous rows.
constexpr int kRowsCols = 128;                  // columns per relayout item
constexpr int kRowsSlot = kRowBlock * 64 + 64;  // one staged 8 KB block + 64 B,
                                                // so slots start 16 banks apart
constexpr int kRowsSmem = 8 * kRowsSlot;
constexpr int kRowsThreads = 256;

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

// Item (row block rb, column group g): the 128 columns from g * 128 of every
// row of the block.  SPLIT: slots 0-3 hold hi's 32-column blocks, 4-7 lo's;
// FP32: slots 0-7 hold 16-column blocks.  Each warp then writes whole rows'
// 512-byte pieces.
template <bool SPLIT>
__global__ void __launch_bounds__(kRowsThreads, 3)
list_rows_kernel(const __nv_bfloat16 *__restrict__ hi, const __nv_bfloat16 *__restrict__ lo,
                 const float *__restrict__ c32, int64_t n, int64_t Dp,
                 const int32_t *__restrict__ blocks, int64_t n_blocks,
                 uint32_t *__restrict__ rows) {
  extern __shared__ __align__(16) uint8_t st[];
  const int64_t groups = (Dp + kRowsCols - 1) / kRowsCols;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kblk = SPLIT ? kTcKBlock : kF32KBlock;
  const int64_t nkb = Dp / kblk;
  for (int64_t w = blockIdx.x; w < n_blocks * groups; w += gridDim.x) {
    const int64_t rb = blocks[w / groups], col0 = (w % groups) * kRowsCols;
    const int cols = (int)(Dp - col0 < kRowsCols ? Dp - col0 : kRowsCols);   // 128 or 64
    const int per_slot = cols / kblk;            // staged blocks per array
    // 512 16-byte chunks per staged block
    for (int c = threadIdx.x; c < 8 * 512; c += kRowsThreads) {
      const int slot = c >> 9, off = (c & 511) * 16;
      const int kbl = SPLIT ? (slot & 3) : slot;
      if (kbl >= per_slot) continue;
      const int64_t kb = col0 / kblk + kbl;
      const uint8_t *src;
      if (SPLIT) {
        const __nv_bfloat16 *arr = slot < 4 ? hi : lo;
        src = reinterpret_cast<const uint8_t *>(arr + (size_t)(rb * nkb + kb) * kRowBlock * kblk);
      } else {
        src = reinterpret_cast<const uint8_t *>(c32 + (size_t)(rb * nkb + kb) * kRowBlock * kblk);
      }
      cp_async16(st + slot * kRowsSlot + off, src + off);
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const int c4 = lane * 4;                     // this lane's four columns
    if (c4 < cols) {
      for (int r = warp; r < kRowBlock; r += kRowsThreads / 32) {
        const int64_t row = rb * kRowBlock + r;
        if (row >= n) break;
        uint4 o;
        if (SPLIT) {
          const int kbl = c4 / kTcKBlock, c = c4 % kTcKBlock;
          const uint2 h = *reinterpret_cast<const uint2 *>(st + kbl * kRowsSlot +
                                                           (r * kTcKBlock + c) * 2);
          const uint2 l = *reinterpret_cast<const uint2 *>(st + (4 + kbl) * kRowsSlot +
                                                           (r * kTcKBlock + c) * 2);
          o.x = __byte_perm(h.x, l.x, 0x5410);
          o.y = __byte_perm(h.x, l.x, 0x7632);
          o.z = __byte_perm(h.y, l.y, 0x5410);
          o.w = __byte_perm(h.y, l.y, 0x7632);
        } else {
          const int kbl = c4 / kF32KBlock, c = c4 % kF32KBlock;
          o = *reinterpret_cast<const uint4 *>(st + kbl * kRowsSlot + (r * kF32KBlock + c) * 4);
        }
        *reinterpret_cast<uint4 *>(rows + (size_t)row * Dp + col0 + c4) = o;
      }
    }
    __syncthreads();                             // before the slots are refilled
  }
}

// One warp per listed pair over the row-major copy: lane l takes four
// consecutive columns of every 128, four such loads per row in flight; FP32
// partials over 64 columns per lane, then FP64, as the blocked kernel.
template <bool SPLIT>
__global__ void __launch_bounds__(kListThreads)
pearson_rows_kernel(const uint32_t *__restrict__ rows, int64_t Dp, const int32_t *__restrict__ pi,
                    const int32_t *__restrict__ pj, const int32_t *__restrict__ pos,
                    int64_t n_pairs, const double *__restrict__ rs,
                    const double *__restrict__ delta, int64_t D, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nq = Dp / 4;                     // 16-byte words per row
  for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n_pairs;
       k += warps) {
    const int64_t a = pi[k], b = pj[k];
    const uint4 *ra = reinterpret_cast<const uint4 *>(rows + (size_t)a * Dp);
    const uint4 *rb = reinterpret_cast<const uint4 *>(rows + (size_t)b * Dp);
    double acc = 0.0;
    float part = 0.f;
    for (int64_t q0 = 0, t = 0; q0 < nq; q0 += 128, ++t) {
      uint4 va[4], vb[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t q = q0 + u * 32 + lane;
        const bool in = q < nq;
        va[u] = in ? __ldg(ra + q) : make_uint4(0u, 0u, 0u, 0u);
        vb[u] = in ? __ldg(rb + q) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t wa[4] = {va[u].x, va[u].y, va[u].z, va[u].w};
        const uint32_t wb[4] = {vb[u].x, vb[u].y, vb[u].z, vb[u].w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (SPLIT) {
            const float ha = __uint_as_float(wa[e] << 16), la = __uint_as_float(wa[e] & 0xffff0000u);
            const float hb = __uint_as_float(wb[e] << 16), lb = __uint_as_float(wb[e] & 0xffff0000u);
            part = fmaf(ha, hb, part);
            part = fmaf(ha, lb, part);
            part = fmaf(la, hb, part);
          } else {
            part = fmaf(__uint_as_float(wa[e]), __uint_as_float(wb[e]), part);
          }
        }
      }
      if ((t & 3) == 3) {                        // 64 columns per lane
        acc += (double)part;
        part = 0.f;
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
// item first), with their list positions, then the distinct row blocks the
// list touches: [a...][b...][position...][block...] on the device (the host
// copy goes through a pageable buffer, staged by the call)
ap_status device_pairs_by_block(const int32_t *pi, const int32_t *pj, int64_t n_pairs,
                                int64_t n, cudaStream_t s, int32_t **d_idx,
                                int64_t *n_blocks) {
  std::vector<uint64_t> key((size_t)n_pairs);
  for (int64_t k = 0; k < n_pairs; ++k) {
    const uint32_t a = (uint32_t)std::min(pi[k], pj[k]), b = (uint32_t)std::max(pi[k], pj[k]);
    const uint64_t blocks = ((uint64_t)(a / kRowBlock) << 16) | (uint64_t)(b / kRowBlock);
    key[k] = (blocks << 32) | (uint64_t)k;     // row blocks < 2^16 (n <= INT32_MAX / 2)
  }
  std::sort(key.begin(), key.end());
  std::vector<int32_t> h((size_t)n_pairs * 3);
  std::vector<uint8_t> touched((size_t)((n + kRowBlock - 1) / kRowBlock), 0);
  for (int64_t q = 0; q < n_pairs; ++q) {
    const int64_t k = (int64_t)(key[q] & 0xffffffffu);
    h[q] = std::min(pi[k], pj[k]);
    h[n_pairs + q] = std::max(pi[k], pj[k]);
    h[2 * n_pairs + q] = (int32_t)k;
    touched[h[q] / kRowBlock] = touched[h[n_pairs + q] / kRowBlock] = 1;
  }
  for (size_t r = 0; r < touched.size(); ++r)
    if (touched[r]) h.push_back((int32_t)r);
  *n_blocks = (int64_t)h.size() - n_pairs * 3;
  AP_TRY(dmalloc(d_idx, h.size()));
  AP_TRY(cudaMemcpyAsync(*d_idx, h.data(), h.size() * 4, cudaMemcpyHostToDevice, s));
  return AP_OK;
}

}  // namespace

cudaError_t launch_pearson_list(VecStore &v, bool split, const int32_t *pi,
                                const int32_t *pj, const int32_t *pos, int64_t n_pairs,
                                const int32_t *blocks, int64_t n_blocks, double *out,
                                cudaStream_t s) {
  if (n_pairs <= 0) return cudaSuccess;
  const int64_t need = (n_pairs + (kListThreads / 32) - 1) / (kListThreads / 32);
  const int grid = (int)std::min<int64_t>(need, (int64_t)num_sms() * 8);
  // the copy streams 2 x 128 rows per touched block at about the HBM rate;
  // it pays once the list reads those rows, in 64-byte pieces at about a
  // quarter of that rate, more than kRowsPairsPerBlock pairs per block
  constexpr int64_t kRowsPairsPerBlock = 32;
  if (n_pairs >= kRowsPairsPerBlock * n_blocks) {
    if (!v.d_rows && dmalloc(&v.d_rows, (size_t)v.n * v.Dp) != cudaSuccess) {
      cudaGetLastError();                       // no room: the blocked kernel
      v.d_rows = nullptr;
    }
  }
  if (v.d_rows && n_pairs >= kRowsPairsPerBlock * n_blocks) {
    const cudaError_t e =
        split ? cudaFuncSetAttribute(list_rows_kernel<true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kRowsSmem)
              : cudaFuncSetAttribute(list_rows_kernel<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kRowsSmem);
    if (e != cudaSuccess) return e;
    const int64_t items = n_blocks * ((v.Dp + kRowsCols - 1) / kRowsCols);
    const int rgrid = (int)std::min<int64_t>(items, (int64_t)num_sms() * 3 * 16);
    if (split) {
      list_rows_kernel<true><<<rgrid, kRowsThreads, kRowsSmem, s>>>(
          v.d_hi, v.d_lo, nullptr, v.n, v.Dp, blocks, n_blocks, v.d_rows);
      pearson_rows_kernel<true><<<grid, kListThreads, 0, s>>>(v.d_rows, v.Dp, pi, pj, pos, n_pairs,
                                                              v.d_rs, v.d_delta_all, v.D, out);
    } else {
      list_rows_kernel<false><<<rgrid, kRowsThreads, kRowsSmem, s>>>(
          nullptr, nullptr, v.d_c32, v.n, v.Dp, blocks, n_blocks, v.d_rows);
      pearson_rows_kernel<false><<<grid, kListThreads, 0, s>>>(v.d_rows, v.Dp, pi, pj, pos,
                                                               n_pairs, v.d_rs, v.d_delta_all,
                                                               v.D, out);
    }
    return cudaGetLastError();
  }
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
    int64_t n_blocks = 0;
    ap_status st = sparse ? device_pairs(pi, pj, n_pairs, s, &d_idx)
                          : device_pairs_by_block(pi, pj, n_pairs, n, s, &d_idx, &n_blocks);
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
                                n_pairs, d_idx + 3 * n_pairs, n_blocks,
                                reinterpret_cast<double *>(out), s);
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
