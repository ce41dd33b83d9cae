// sparse.cu -- cosine of sparse composition vectors, the comparison of the
// bioinformatics application (Sec. V-B: "essentially the dot product between
// two sparse vectors"):
//
//   c(i,j) = sum_k a_ik a_jk / sqrt(sum_k a_ik^2 sum_k a_jk^2)
//
// Rows are CSR (strictly increasing int32 codes, FP32 values) over an index
// space of `dim` codes (20^k k-mers), cut into chunks of kSparseChunk codes.
// Schedule: persistent CTAs pop tiles (a block of 32 items I x a block of 64
// items J, every block pair holding a pair i < j, Sec. IV-B) from an atomic
// queue.  The 16 warps walk the chunks together, for 8 rows of I at a time:
// per chunk warps 0-7 each scatter one row i into the dense form of the
// chunk in shared memory, and after a barrier every lane reads its share of
// the chunk's entries of the warp's four rows j (once, into registers) and
// multiplies each against the 8 rows i.  The dense form is code-major, the 8
// rows' values of one code side by side (32 bytes), so one 16-byte load
// gathers four rows; the two 16-byte groups of a code are XOR-swizzled by
// code bit 1, which spreads the loads of random codes over the bank groups.
// The barriers pace every chunk step by its busiest warp, so the rows j of a
// block are dealt to the warps by entry count in a snake (heavy and light
// rows alternate).  Each warp copies the next chunk's entries of its rows (up
// to 64 per row) into a two-stage shared-memory ring with cp.async while it
// works on the current one, so the chunk loop does not wait on DRAM.  Per
// lane the FP32 products are summed over up to 64 chunks, then folded into
// FP64 pair sums in shared memory.  (Tiles of 32 x 32 items with 16 rows i
// per pass over chunks of 2048 codes ran 2.99 s on the 2500-item set, these
// 2.89 s: the lookups, not the chunk steps, set the pace.)
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ap_internal.h"

namespace ap {

namespace {

constexpr int kWarps = 16;                   // warps per CTA
constexpr int kThreads = 32 * kWarps;
constexpr int kRows = 8;                     // rows i per pass: the dense form's rows
constexpr int kGroups = kRows / 4;           // 16-byte groups of a code in the dense form
constexpr int BI = kSparseBlock;             // items i of a tile
constexpr int BJ = kSparseBlockJ;            // items j of a tile
constexpr int kJ = BJ / kWarps;              // rows j per warp
constexpr int kStage = 64;                   // staged entries per row and chunk
constexpr int W = kSparseChunk;
constexpr int kFoldChunks = 64;

// word of row q (0..kRows-1) at chunk code k in the swizzled dense form
__device__ __forceinline__ int dense_at(int k, int q) {
  return k * kRows + ((((q >> 2) ^ (k >> 1)) & (kGroups - 1)) << 2) + (q & 3);
}

// asynchronous 4-byte copy global -> shared; src_bytes 0 writes zeros and
// reads nothing
__device__ __forceinline__ void cp_async4(void *dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// One warp's staging of a chunk: up to kStage entries (2 per lane) of its row
// i (dense-row owners) and of its kJ rows j, filled by cp.async one chunk
// ahead.
struct WarpStage {
  int32_t code[1 + kJ][kStage];
  float val[1 + kJ][kStage];
};

template <int COVER>
__global__ void __launch_bounds__(kThreads, 1)
sparse_cos_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                  const float *__restrict__ val, const int32_t *__restrict__ cptr,
                  const double *__restrict__ rs, int64_t n, int64_t n_chunks,
                  const int32_t *__restrict__ tiles, int64_t n_tiles,
                  const int32_t *__restrict__ jperm, int32_t *queue, void *out) {
  extern __shared__ __align__(16) uint8_t smem[];
  float *dense = reinterpret_cast<float *>(smem);                     // [W][kRows], swizzled
  double *s_g = reinterpret_cast<double *>(dense + kRows * W);        // [BI][BJ]
  WarpStage *stage = reinterpret_cast<WarpStage *>(s_g + BI * BJ);    // [kWarps][2]
  __shared__ int s_tile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warps 0..kRows-1 each own one dense row (scatter and clear it, so the
  // clearing of a chunk and the next chunk's scatter stay in program order)
  const int wr = warp % kRows;
  const bool owner = warp < kRows;
  for (int k = threadIdx.x; k < kRows * W; k += kThreads) dense[k] = 0.f;
  WarpStage *my_stage = stage + warp * 2;

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t t = s_tile;
    if (t >= n_tiles) break;
    const int64_t i0 = (int64_t)tiles[2 * t] * BI, j0 = (int64_t)tiles[2 * t + 1] * BJ;
    const int32_t *jslot = jperm + (int64_t)tiles[2 * t + 1] * BJ;   // item of each row slot of J
    for (int q = threadIdx.x; q < BI * BJ; q += kThreads) s_g[q] = 0.0;
    __syncthreads();

    if (!COVER) {
      for (int pass = 0; pass < BI / kRows; ++pass) {
        // the warp's rows: r = 0 its row i (owners only: dense row wr),
        // r = 1.. its rows j (slots warp + (r - 1) * kWarps)
        int64_t row[1 + kJ], base[1 + kJ];
        bool valid[1 + kJ];
        row[0] = i0 + pass * kRows + wr;
#pragma unroll
        for (int h = 0; h < kJ; ++h) row[1 + h] = j0 + jslot[warp + h * kWarps];
        // pairs need j > i: a row j at or before every row i of the pass has none
        const int64_t i_first = i0 + pass * kRows;
#pragma unroll
        for (int r = 0; r <= kJ; ++r) {
          valid[r] = row[r] < n && (r == 0 ? owner : row[r] > i_first);
          base[r] = valid[r] ? off[row[r]] : 0;
        }
        float acc[kJ][kRows];
#pragma unroll
        for (int h = 0; h < kJ; ++h)
#pragma unroll
          for (int q = 0; q < kRows; ++q) acc[h][q] = 0.f;
        // one entry (code k of the chunk, value v) of a row j against the
        // kRows rows i: kGroups 16-byte loads of the dense form
        auto product = [&](int32_t k, float v, float (&a)[kRows]) {
          const float4 *dk = reinterpret_cast<const float4 *>(dense + k * kRows);
#pragma unroll
          for (int g = 0; g < kGroups; ++g) {
            const float4 d = dk[(g ^ (k >> 1)) & (kGroups - 1)];
            a[4 * g + 0] = fmaf(d.x, v, a[4 * g + 0]);
            a[4 * g + 1] = fmaf(d.y, v, a[4 * g + 1]);
            a[4 * g + 2] = fmaf(d.z, v, a[4 * g + 2]);
            a[4 * g + 3] = fmaf(d.w, v, a[4 * g + 3]);
          }
        };
        int since = 0;
        // chunk starts b0..b3 = cptr of chunks c .. c + 3 (relative to the row)
        int32_t b0[1 + kJ], b1[1 + kJ], b2[1 + kJ], b3[1 + kJ];
        auto bound = [&](int r, int64_t cn, bool in_range) -> int32_t {
          return (valid[r] && in_range) ? cptr[cn + row[r]] : 0;   // cn = c * n
        };
        // copies of chunk c's first kStage entries of every row into stage s;
        // slots past a row's entries are not copied (nothing reads them)
        auto stage_copy = [&](int64_t c, const int32_t *lo, const int32_t *hi, int s) {
#pragma unroll
          for (int r = 0; r <= kJ; ++r) {
#pragma unroll
            for (int u = 0; u < kStage / 32; ++u) {
              const int32_t e = lo[r] + u * 32 + lane;
              if (c < n_chunks && e < hi[r]) {
                const int64_t g = base[r] + e;
                cp_async4(&my_stage[s].code[r][u * 32 + lane], idx + g, 4u);
                cp_async4(&my_stage[s].val[r][u * 32 + lane], val + g, 4u);
              }
            }
          }
          cp_async_commit();
        };
#pragma unroll
        for (int r = 0; r <= kJ; ++r) {
          b0[r] = bound(r, 0, true);
          b1[r] = bound(r, n, 1 <= n_chunks);
          b2[r] = bound(r, 2 * n, 2 <= n_chunks);
        }
        stage_copy(0, b0, b1, 0);
        for (int64_t c = 0; c < n_chunks; ++c) {
          const int32_t code0 = (int32_t)(c * W);
          const int s = (int)(c & 1);
          const int64_t cn3 = (c + 3) * n;
#pragma unroll
          for (int r = 0; r <= kJ; ++r) b3[r] = bound(r, cn3, c + 3 <= n_chunks);
          stage_copy(c + 1, b1, b2, s ^ 1);            // the next chunk, in flight
          cp_async_wait_prev();                        // this chunk's copies landed
          const WarpStage &st = my_stage[s];
          // scatter row i (staged entries, then any beyond the stage)
          const int32_t ni = b1[0] - b0[0];
#pragma unroll
          for (int u = 0; u < kStage / 32; ++u)
            if (u * 32 + lane < ni)
              dense[dense_at(st.code[0][u * 32 + lane] - code0, wr)] = st.val[0][u * 32 + lane];
          for (int32_t e = kStage + lane; e < ni; e += 32) {
            const int64_t g = base[0] + b0[0] + e;
            dense[dense_at(__ldg(idx + g) - code0, wr)] = __ldg(val + g);
          }
          __syncthreads();
          // every entry of the warp's rows j in this chunk against the
          // kRows rows i held in the dense arrays
#pragma unroll
          for (int h = 0; h < kJ; ++h) {
            if (!valid[1 + h]) continue;
            const int32_t nj = b1[1 + h] - b0[1 + h];
#pragma unroll
            for (int u = 0; u < kStage / 32; ++u) {
              if (u * 32 + lane < nj)
                product(st.code[1 + h][u * 32 + lane] - code0, st.val[1 + h][u * 32 + lane],
                        acc[h]);
            }
            for (int32_t e = kStage + lane; e < nj; e += 32) {
              const int64_t g = base[1 + h] + b0[1 + h] + e;
              product(__ldg(idx + g) - code0, __ldg(val + g), acc[h]);
            }
          }
          __syncthreads();
#pragma unroll
          for (int u = 0; u < kStage / 32; ++u)
            if (u * 32 + lane < ni) dense[dense_at(st.code[0][u * 32 + lane] - code0, wr)] = 0.f;
          for (int32_t e = kStage + lane; e < ni; e += 32)
            dense[dense_at(__ldg(idx + base[0] + b0[0] + e) - code0, wr)] = 0.f;
#pragma unroll
          for (int r = 0; r <= kJ; ++r) { b0[r] = b1[r]; b1[r] = b2[r]; b2[r] = b3[r]; }
          if (++since == kFoldChunks || c + 1 == n_chunks) {
            since = 0;
            // fold the lanes' FP32 sums into the FP64 pair sums
#pragma unroll
            for (int h = 0; h < kJ; ++h)
#pragma unroll
              for (int q = 0; q < kRows; ++q) {
                double v = (double)acc[h][q];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) s_g[(pass * kRows + q) * BJ + warp + h * kWarps] += v;
                acc[h][q] = 0.f;
              }
          }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");   // the last (empty) group
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < BI * BJ; q += kThreads) {
      const int il = q / BJ, slot = q - il * BJ;
      const int64_t i = i0 + il, j = j0 + jslot[slot];
      if (i >= n || j >= n || j <= i) continue;
      const int64_t p = pair_index(i, j, n);
      if (COVER) atomicAdd(reinterpret_cast<int32_t *>(out) + p, 1);
      else reinterpret_cast<double *>(out)[p] = s_g[q] * rs[i] * rs[j];
    }
    __syncthreads();
  }
}

// row checks (strictly increasing codes in [0, dim)), FP64 squared norms
__global__ void sparse_rows_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                                   const float *__restrict__ val, int64_t n, int64_t dim,
                                   double *__restrict__ rs, int32_t *bad) {
  __shared__ double red[8];
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    double s = 0.0;
    for (int64_t e = off[i] + threadIdx.x; e < off[i + 1]; e += blockDim.x) {
      const int32_t k = idx[e];
      if (k < 0 || k >= dim || (e > off[i] && idx[e - 1] >= k)) atomicExch(bad, 1);
      s += (double)val[e] * (double)val[e];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      rs[i] = t > 0.0 ? 1.0 / sqrt(t) : __longlong_as_double(0x7ff8000000000000ll);
    }
    __syncthreads();
  }
}

// cptr[c][i] = lower bound of c * W in row i's codes, relative to the row
__global__ void sparse_cptr_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                                   int64_t n, int64_t n_chunks, int32_t *__restrict__ cptr) {
  const int64_t total = (n_chunks + 1) * n;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / n, i = q - c * n;
    const int64_t lo0 = off[i], hi0 = off[i + 1];
    const int64_t key = c * (int64_t)W;
    int64_t lo = lo0, hi = hi0;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)idx[mid] < key) lo = mid + 1;
      else hi = mid;
    }
    cptr[q] = (int32_t)(lo - lo0);
  }
}

}  // namespace

void free_sparse(SparseStore &sp) {
  dfree(sp.d_off);
  dfree(sp.d_idx);
  dfree(sp.d_val);
  dfree(sp.d_cptr);
  dfree(sp.d_rs);
  dfree(sp.d_tiles);
  dfree(sp.d_jperm);
}

ap_status create_sparse(const ap_items_desc *d, ap_items *it, cudaStream_t s) {
  SparseStore &sp = it->sp;
  const int64_t *off = d->offsets;
  if (!off || off[0] != 0 || d->dim < 1 || d->dim > INT32_MAX) return AP_ERR_INVALID_ARG;
  sp.n = d->n_items;
  sp.dim = d->dim;
  for (int64_t i = 0; i < sp.n; ++i) {
    if (off[i + 1] < off[i]) return AP_ERR_INVALID_ARG;
    if (off[i + 1] - off[i] > d->dim) return AP_ERR_INVALID_ARG;   // more entries than codes
  }
  sp.nnz = off[sp.n];
  if (sp.nnz > 0 && (!d->indices || !d->data)) return AP_ERR_INVALID_ARG;
  sp.n_chunks = (sp.dim + kSparseChunk - 1) / kSparseChunk;
  AP_TRY(dmalloc(&sp.d_off, (size_t)sp.n + 1));
  AP_TRY(dmalloc(&sp.d_idx, (size_t)std::max<int64_t>(sp.nnz, 1)));
  AP_TRY(dmalloc(&sp.d_val, (size_t)std::max<int64_t>(sp.nnz, 1)));
  AP_TRY(dmalloc(&sp.d_cptr, (size_t)(sp.n_chunks + 1) * std::max<int64_t>(sp.n, 1)));
  AP_TRY(dmalloc(&sp.d_rs, (size_t)std::max<int64_t>(sp.n, 1)));
  AP_TRY(cudaMemcpyAsync(sp.d_off, off, (size_t)(sp.n + 1) * 8, cudaMemcpyHostToDevice, s));
  const cudaMemcpyKind kind = d->data_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (sp.nnz > 0) {
    AP_TRY(cudaMemcpyAsync(sp.d_idx, d->indices, (size_t)sp.nnz * 4, kind, s));
    AP_TRY(cudaMemcpyAsync(sp.d_val, d->data, (size_t)sp.nnz * 4, kind, s));
  }
  int32_t *d_bad = it->d_queue + 2;              // scratch word of the handle
  AP_TRY(cudaMemsetAsync(d_bad, 0, 4, s));
  if (sp.n > 0) {
    const int g = (int)std::min<int64_t>(sp.n, 65535);
    sparse_rows_kernel<<<g, 256, 0, s>>>(sp.d_off, sp.d_idx, sp.d_val, sp.n, sp.dim, sp.d_rs,
                                         d_bad);
    AP_TRY(cudaGetLastError());
    const int64_t total = (sp.n_chunks + 1) * sp.n;
    const int g2 = (int)std::min<int64_t>((total + 255) / 256, 65535);
    sparse_cptr_kernel<<<g2, 256, 0, s>>>(sp.d_off, sp.d_idx, sp.n, sp.n_chunks, sp.d_cptr);
    AP_TRY(cudaGetLastError());
  }
  // row slots of each J block of BJ items, dealt to the warps by entry
  // count in a snake (warp w takes slots w, w + kWarps, ...: the w-th
  // heaviest row, the w-th lightest of the next kWarps, ...), so every
  // warp's rows j weigh about the same (rows past n count as empty)
  const int64_t nbi = (sp.n + BI - 1) / BI, nbj = (sp.n + BJ - 1) / BJ;
  std::vector<int32_t> jperm((size_t)std::max<int64_t>(nbj, 1) * BJ);
  for (int64_t b = 0; b < nbj; ++b) {
    int32_t order[BJ];
    auto cnt = [&](int32_t l) {
      const int64_t i = b * BJ + l;
      return i < sp.n ? off[i + 1] - off[i] : (int64_t)-1;
    };
    for (int32_t l = 0; l < BJ; ++l) order[l] = l;
    std::stable_sort(order, order + BJ, [&](int32_t a, int32_t c) { return cnt(a) > cnt(c); });
    for (int h = 0; h < kJ; ++h)
      for (int w = 0; w < kWarps; ++w)
        jperm[(size_t)b * BJ + w + h * kWarps] = order[h * kWarps + ((h & 1) ? kWarps - 1 - w : w)];
  }
  AP_TRY(dmalloc(&sp.d_jperm, jperm.size()));
  AP_TRY(cudaMemcpyAsync(sp.d_jperm, jperm.data(), jperm.size() * 4, cudaMemcpyHostToDevice, s));
  // tiles (I block of BI items, J block of BJ items) holding a pair i < j,
  // the J blocks in order and within each its I blocks
  std::vector<int32_t> tiles;
  for (int64_t bj = 0; bj < nbj; ++bj)
    for (int64_t bi = 0; bi < nbi && bi * BI < (bj + 1) * BJ - 1; ++bi) {
      tiles.push_back((int32_t)bi);
      tiles.push_back((int32_t)bj);
    }
  sp.n_tiles = (int64_t)tiles.size() / 2;
  AP_TRY(dmalloc(&sp.d_tiles, std::max<size_t>(tiles.size(), 2)));
  if (!tiles.empty())
    AP_TRY(cudaMemcpyAsync(sp.d_tiles, tiles.data(), tiles.size() * 4, cudaMemcpyHostToDevice, s));
  int32_t bad = 0;
  AP_TRY(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, s));
  AP_TRY(cudaStreamSynchronize(s));
  if (bad) return AP_ERR_INVALID_ARG;
  it->stats.tiles = sp.n_tiles;
  it->stats.tile_m = BI;
  it->stats.tile_n = BJ;
  return AP_OK;
}

cudaError_t launch_sparse_cosine(const SparseStore &sp, double *out, int coverage,
                                 int32_t *queue, cudaStream_t s) {
  if (sp.n_tiles <= 0) return cudaSuccess;
  const size_t smem = (size_t)kRows * W * 4 + (size_t)BI * BJ * 8 +
                      (size_t)kWarps * 2 * sizeof(WarpStage);
  void (*kern)(const int64_t *, const int32_t *, const float *, const int32_t *, const double *,
               int64_t, int64_t, const int32_t *, int64_t, const int32_t *, int32_t *, void *) =
      coverage ? sparse_cos_kernel<1> : sparse_cos_kernel<0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  const int64_t grid = std::min<int64_t>((int64_t)num_sms(), sp.n_tiles);
  kern<<<(int)grid, kThreads, smem, s>>>(sp.d_off, sp.d_idx, sp.d_val, sp.d_cptr, sp.d_rs, sp.n,
                                         sp.n_chunks, sp.d_tiles, sp.n_tiles, sp.d_jperm, queue,
                                         out);
  return cudaGetLastError();
}

}  // namespace ap
