// vec.cu -- dense-vector kernels: the load pipeline's GPU pre-processing
// (Sec. III, stage 4 of l) and the plain FP32 Gram path of the Pearson
// correlation (the normalised cross correlation of Sec. V-A).
//
//   mu_i = (1/D) sum_k x_ik,  ss_i = sum_k (x_ik - mu_i)^2       (FP64 result)
//   c_ik = x_ik - mu_i,  hi = bf16_rn(c),  lo = bf16_rn(c - hi)   (split-BF16)
//   r_ij = sum_k c_ik c_jk / sqrt(ss_i ss_j)                       (FP64 scaling)
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the
// per-element work stays in FP32: short FP32 partial sums (64 elements per
// thread) are folded into FP64 accumulators, and the centring subtracts the
// FP64 mean as a two-float pair (x - mu_hi) - mu_lo, which keeps c accurate
// to a few ulps of c itself even when |mu| >> |c|.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ap_internal.h"

namespace ap {

namespace {

constexpr int kStatsThreads = 512;
constexpr int kSplitThreads = 256;

__device__ __forceinline__ double block_sum_f64(double v, double *red) {
  // warp shuffle tree, then one warp over the per-warp sums
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) red[32] = v;
  __syncthreads();
  double r = red[32];
  __syncthreads();
  return r;
}

// Pass 1 of the load pipeline: one CTA per row, FP64 mean (FP32 partial sums
// of 64 elements per thread folded into FP64).
template <bool VEC4>
__global__ void __launch_bounds__(kStatsThreads)
vec_mean_kernel(const float *__restrict__ X, int64_t n, int64_t D, int64_t ld,
                double *__restrict__ mu_out) {
  __shared__ double red[33];
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
    const float *x = X + row * ld;
    double acc = 0.0;
    float part = 0.f;
    int cnt = 0;
    if (VEC4) {
      const float4 *x4 = reinterpret_cast<const float4 *>(x);
      const int64_t n4 = D >> 2, st = blockDim.x;
      int64_t k = threadIdx.x;
      // four independent 16-byte loads in flight per thread
      for (; k + 3 * st < n4; k += 4 * st) {
        const float4 v0 = __ldg(x4 + k), v1 = __ldg(x4 + k + st);
        const float4 v2 = __ldg(x4 + k + 2 * st), v3 = __ldg(x4 + k + 3 * st);
        part += ((v0.x + v0.y) + (v0.z + v0.w)) + ((v1.x + v1.y) + (v1.z + v1.w)) +
                (((v2.x + v2.y) + (v2.z + v2.w)) + ((v3.x + v3.y) + (v3.z + v3.w)));
        if (++cnt == 4) { acc += (double)part; part = 0.f; cnt = 0; }
      }
      for (; k < n4; k += st) {
        const float4 v = __ldg(x4 + k);
        part += (v.x + v.y) + (v.z + v.w);
      }
      for (int64_t e = (n4 << 2) + threadIdx.x; e < D; e += blockDim.x) part += x[e];
    } else {
      for (int64_t k = threadIdx.x; k < D; k += blockDim.x) {
        part += __ldg(x + k);
        if (++cnt == 64) { acc += (double)part; part = 0.f; cnt = 0; }
      }
    }
    acc += (double)part;
    const double mu = block_sum_f64(acc, red) / (double)D;
    if (threadIdx.x == 0) mu_out[row] = mu;
  }
}

// Pass 2: centre each row against its FP64 mean (as the two-float pair
// mu_hi + mu_lo), write the blocked split-BF16 and/or FP32 copies (zero
// padded to Dp columns) and this CTA's FP64 partial of sum_k c_k^2.
// Grid: x = kSplitParts column ranges of a row, y = rows (strided).
// SLICE: one column chunk of the rows, centred on a per-row shift instead of
// the mean; the CTA's partials of sum c^2 and sum c are added to `part` and
// `part_c` (set when first_chunk) so they accumulate over the chunks.
template <bool VEC4, bool SLICE>
__global__ void __launch_bounds__(kSplitThreads)
vec_split_kernel(const float *__restrict__ X, int64_t row0, int64_t out_row0, int64_t n,
                 int64_t D, int64_t ld, int64_t Dp, const double *__restrict__ mu,
                 __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                 float *__restrict__ c32, double *__restrict__ part,
                 double *__restrict__ part_c, int first_chunk) {
  __shared__ double red[33];
  const int64_t q4 = Dp >> 2;                  // float4 groups per padded row
  const int64_t nkb_tc = Dp / kTcKBlock, nkb_32 = Dp / kF32KBlock;
  for (int64_t lr = blockIdx.y; lr < n; lr += gridDim.y) {
    const int64_t row = row0 + lr;             // global item index (statistics)
    const int64_t orow = out_row0 + lr;        // row of the blocked copies
    const float *x = X + lr * ld;
    const double m = mu[row];
    const float mh = (float)m;
    const float ml = (float)(m - (double)mh);
    double acc = 0.0, acc_c = 0.0;
    float psum = 0.f, psum_c = 0.f;
    const int64_t stq = (int64_t)gridDim.x * blockDim.x;
    int iter = 0;
    // two float4 groups per trip, both loads issued before either is used
    for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q0 < q4; q0 += 2 * stq) {
      float vv[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t k = (q0 + u * stq) << 2;
        if (VEC4 && k + 3 < D) {
          const float4 t = __ldg(reinterpret_cast<const float4 *>(x + k));
          vv[u][0] = t.x; vv[u][1] = t.y; vv[u][2] = t.z; vv[u][3] = t.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) vv[u][e] = (k + e < D) ? __ldg(x + k + e) : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
      const int64_t q = q0 + u * stq;
      if (q >= q4) break;
      const int64_t k = q << 2;
      const float *v = vv[u];
      float c[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) c[e] = (k + e < D) ? (v[e] - mh) - ml : 0.f;
      psum += (c[0] * c[0] + c[1] * c[1]) + (c[2] * c[2] + c[3] * c[3]);
      if (SLICE) psum_c += (c[0] + c[1]) + (c[2] + c[3]);
      if (hi) {
        __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          h[e] = __float2bfloat16_rn(c[e]);
          l[e] = __float2bfloat16_rn(c[e] - __bfloat162float(h[e]));   // c - hi is exact
        }
        uint2 hv, lv;
        hv.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
        hv.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
        lv.x = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
        lv.y = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
        const size_t o = blocked_offset(orow, k, nkb_tc, kTcKBlock);
        *reinterpret_cast<uint2 *>(hi + o) = hv;
        *reinterpret_cast<uint2 *>(lo + o) = lv;
      }
      if (c32) {
        const size_t o = blocked_offset(orow, k, nkb_32, kF32KBlock);
        *reinterpret_cast<float4 *>(c32 + o) = make_float4(c[0], c[1], c[2], c[3]);
      }
      }
      // fold every 16 float4 (64 elements) into FP64
      if ((++iter & 7) == 0) {
        acc += (double)psum;
        psum = 0.f;
        if (SLICE) { acc_c += (double)psum_c; psum_c = 0.f; }
      }
    }
    acc += (double)psum;
    const double s = block_sum_f64(acc, red);
    const size_t slot = (size_t)row * gridDim.x + blockIdx.x;
    if (SLICE) {
      acc_c += (double)psum_c;
      const double sc = block_sum_f64(acc_c, red);
      if (threadIdx.x == 0) {
        part[slot] = first_chunk ? s : part[slot] + s;
        part_c[slot] = first_chunk ? sc : part_c[slot] + sc;
      }
    } else if (threadIdx.x == 0) {
      part[slot] = s;
    }
  }
}

// ss_i = sum of the row's partials in a fixed order; rs_i = 1 / sqrt(ss_i)
__global__ void vec_finalize_kernel(const double *__restrict__ part, int64_t row0, int64_t n,
                                    int nparts, double *__restrict__ ss,
                                    double *__restrict__ rs) {
  for (int64_t lr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lr < n;
       lr += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = row0 + lr;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[row * nparts + b];
    ss[row] = s;
    // zero variance: correlation undefined, propagate NaN
    rs[row] = s > 0.0 ? 1.0 / sqrt(s) : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// Column-sliced rows centred on shifts s_i: with S1 = sum_k c_ik and
// S2 = sum_k c_ik^2 over all D columns (c = x - s), delta_i = mu_i - s_i =
// S1 / D and ss_i = S2 - S1 delta_i (the shifted-data form of the variance).
__global__ void slice_stats_kernel(const double *__restrict__ part,
                                   const double *__restrict__ part_c, int64_t n, int nparts,
                                   int64_t D, double *__restrict__ delta,
                                   double *__restrict__ ss, double *__restrict__ rs) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    double s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nparts; ++b) {
      s1 += part_c[row * nparts + b];
      s2 += part[row * nparts + b];
    }
    const double d = s1 / (double)D, v = s2 - s1 * d;
    delta[row] = d;
    ss[row] = v;
    rs[row] = v > 0.0 ? 1.0 / sqrt(v) : __longlong_as_double(0x7ff8000000000000ll);
  }
}

// r_ij = (G_ij - D delta_i delta_j) rs_i rs_j over the packed upper triangle,
// G the Gram of the shifted rows (the centred Gram is G - D delta_i delta_j)
__global__ void slice_finalize_kernel(double *__restrict__ out, const double *__restrict__ rs,
                                      const double *__restrict__ delta, int64_t n, int64_t D) {
  for (int64_t i = blockIdx.x; i < n - 1; i += gridDim.x) {
    const double ri = rs[i], di = (double)D * delta[i];
    const int64_t p0 = pair_index(i, i + 1, n);
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x)
      out[p0 + (j - i - 1)] = (out[p0 + (j - i - 1)] - di * delta[j]) * (ri * rs[j]);
  }
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core Gram over upper-triangle tiles of 128 x 128 items.
// 256 threads, 8 x 8 outputs per thread, K staged 16 at a time through
// registers into transposed, double-buffered shared memory.
// ---------------------------------------------------------------------------
constexpr int kF32Tile = 128;
constexpr int kF32K = 16;
constexpr int kF32Pad = 4;

template <int COVER>
__global__ void __launch_bounds__(256, 1)
gram_f32_kernel(const float *__restrict__ C, int64_t n, int64_t Dp,
                const double *__restrict__ rs, const int32_t *__restrict__ tiles,
                int64_t n_tiles, int32_t *queue, void *out) {
  __shared__ __align__(16) float As[2][kF32K][kF32Tile + kF32Pad];
  __shared__ __align__(16) float Bs[2][kF32K][kF32Tile + kF32Pad];
  __shared__ int s_tile;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t nk = Dp / kF32K;

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t t = s_tile;
    __syncthreads();
    if (t >= n_tiles) break;
    const int64_t i0 = (int64_t)tiles[2 * t] * kF32Tile;
    const int64_t j0 = (int64_t)tiles[2 * t + 1] * kF32Tile;
    // blocked copy: block (row block, k block) = 128 rows x 16 columns, contiguous
    const int64_t nkb = Dp / kF32KBlock;
    const float4 *ablk = reinterpret_cast<const float4 *>(C + (size_t)(i0 >> 7) * nkb * 2048);
    const float4 *bblk = reinterpret_cast<const float4 *>(C + (size_t)(j0 >> 7) * nkb * 2048);

    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    float4 ra[2], rb[2];
    auto gload = [&](int64_t kb) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        ra[h] = __ldg(ablk + kb * 512 + tid + 256 * h);
        rb[h] = __ldg(bblk + kb * 512 + tid + 256 * h);
      }
    };
    auto sstore = [&](int buf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int f = tid + 256 * h, r = f >> 2, kq = (f & 3) * 4;
        As[buf][kq + 0][r] = ra[h].x; As[buf][kq + 1][r] = ra[h].y;
        As[buf][kq + 2][r] = ra[h].z; As[buf][kq + 3][r] = ra[h].w;
        Bs[buf][kq + 0][r] = rb[h].x; Bs[buf][kq + 1][r] = rb[h].y;
        Bs[buf][kq + 2][r] = rb[h].z; Bs[buf][kq + 3][r] = rb[h].w;
      }
    };

    gload(0);
    sstore(0);
    __syncthreads();
    for (int64_t kb = 0; kb < nk; ++kb) {
      const int buf = (int)(kb & 1);
      if (kb + 1 < nk) gload(kb + 1);
#pragma unroll
      for (int k = 0; k < kF32K; ++k) {
        float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
        float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      }
      if (kb + 1 < nk) sstore(buf ^ 1);
      __syncthreads();
    }

    // epilogue: r = G * rs_i * rs_j in FP64, strict upper triangle only
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t i = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + (a - 4));
      if (i >= n) continue;
      const double ri = COVER ? 0.0 : rs[i];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int64_t j = j0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
        if (j >= n || j <= i) continue;
        const int64_t p = pair_index(i, j, n);
        if (COVER) atomicAdd(reinterpret_cast<int32_t *>(out) + p, 1);
        else reinterpret_cast<double *>(out)[p] = (double)acc[a][b] * ri * rs[j];
      }
    }
  }
}

}  // namespace

cudaError_t launch_vec_mean(const float *X, int64_t n, int64_t D, int64_t ld, double *mu,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int grid = (int)(n < 65535 ? n : 65535);
  const bool vec4 = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (vec4) vec_mean_kernel<true><<<grid, kStatsThreads, 0, s>>>(X, n, D, ld, mu);
  else vec_mean_kernel<false><<<grid, kStatsThreads, 0, s>>>(X, n, D, ld, mu);
  return cudaGetLastError();
}

cudaError_t launch_vec_split(const float *X, int64_t row0, int64_t out_row0, int64_t n, int64_t D, int64_t ld,
                             int64_t Dp, const double *mu, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                             float *c32, double *part, double *ss, double *rs, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(kSplitParts, (unsigned)(n < 65535 ? n : 65535));
  const bool vec4 = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (vec4)
    vec_split_kernel<true, false><<<grid, kSplitThreads, 0, s>>>(
        X, row0, out_row0, n, D, ld, Dp, mu, hi, lo, c32, part, nullptr, 1);
  else
    vec_split_kernel<false, false><<<grid, kSplitThreads, 0, s>>>(
        X, row0, out_row0, n, D, ld, Dp, mu, hi, lo, c32, part, nullptr, 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int fg = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  vec_finalize_kernel<<<fg, 256, 0, s>>>(part, row0, n, kSplitParts, ss, rs);
  return cudaGetLastError();
}

cudaError_t launch_vec_split_slice(const float *X, int64_t row0, int64_t n, int64_t cols,
                                   int64_t ld, int64_t cols_p, const double *shift,
                                   __nv_bfloat16 *hi, __nv_bfloat16 *lo, double *part,
                                   double *part_c, int first_chunk, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(kSplitParts, (unsigned)(n < 65535 ? n : 65535));
  const bool vec4 = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (vec4)
    vec_split_kernel<true, true><<<grid, kSplitThreads, 0, s>>>(
        X, row0, row0, n, cols, ld, cols_p, shift, hi, lo, nullptr, part, part_c, first_chunk);
  else
    vec_split_kernel<false, true><<<grid, kSplitThreads, 0, s>>>(
        X, row0, row0, n, cols, ld, cols_p, shift, hi, lo, nullptr, part, part_c, first_chunk);
  return cudaGetLastError();
}

cudaError_t launch_slice_finalize(const double *part, const double *part_c, int64_t n,
                                  int64_t D, double *delta, double *ss, double *rs, double *out,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int fg = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  slice_stats_kernel<<<fg, 256, 0, s>>>(part, part_c, n, kSplitParts, D, delta, ss, rs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n < 2) return e;
  const int grid = (int)(n - 1 < 65535 ? n - 1 : 65535);
  slice_finalize_kernel<<<grid, 256, 0, s>>>(out, rs, delta, n, D);
  return cudaGetLastError();
}

cudaError_t launch_gram_f32(const float *C, int64_t n, int64_t Dp, const double *rs,
                            const int32_t *tiles, int64_t n_tiles, int32_t *queue, void *out,
                            int coverage, int64_t, int64_t, cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  int64_t grid = (int64_t)num_sms();
  if (grid > n_tiles) grid = n_tiles;
  if (coverage)
    gram_f32_kernel<1><<<(int)grid, 256, 0, s>>>(C, n, Dp, rs, tiles, n_tiles, queue, out);
  else
    gram_f32_kernel<0><<<(int)grid, 256, 0, s>>>(C, n, Dp, rs, tiles, n_tiles, queue, out);
  return cudaGetLastError();
}

}  // namespace ap
