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

// One CTA per row: FP64 mean, then FP64 centred sum of squares.
template <bool VEC4>
__global__ void __launch_bounds__(kStatsThreads)
vec_stats_kernel(const float *__restrict__ X, int64_t n, int64_t D, int64_t ld,
                 double *__restrict__ mu_out, double *__restrict__ ss_out,
                 double *__restrict__ rs_out) {
  __shared__ double red[33];
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
    const float *x = X + row * ld;
    // pass 1: sum
    double acc = 0.0;
    float part = 0.f;
    int cnt = 0;
    if (VEC4) {
      const float4 *x4 = reinterpret_cast<const float4 *>(x);
      int64_t n4 = D >> 2;
      for (int64_t k = threadIdx.x; k < n4; k += blockDim.x) {
        float4 v = __ldg(x4 + k);
        part += (v.x + v.y) + (v.z + v.w);
        if (++cnt == 16) { acc += (double)part; part = 0.f; cnt = 0; }
      }
      for (int64_t k = (n4 << 2) + threadIdx.x; k < D; k += blockDim.x) part += x[k];
    } else {
      for (int64_t k = threadIdx.x; k < D; k += blockDim.x) {
        part += __ldg(x + k);
        if (++cnt == 64) { acc += (double)part; part = 0.f; cnt = 0; }
      }
    }
    acc += (double)part;
    double mu = block_sum_f64(acc, red) / (double)D;
    // pass 2: centred sum of squares
    float mh = (float)mu;
    float ml = (float)(mu - (double)mh);
    acc = 0.0;
    part = 0.f;
    cnt = 0;
    if (VEC4) {
      const float4 *x4 = reinterpret_cast<const float4 *>(x);
      int64_t n4 = D >> 2;
      for (int64_t k = threadIdx.x; k < n4; k += blockDim.x) {
        float4 v = __ldg(x4 + k);
        float c0 = (v.x - mh) - ml, c1 = (v.y - mh) - ml;
        float c2 = (v.z - mh) - ml, c3 = (v.w - mh) - ml;
        part += (c0 * c0 + c1 * c1) + (c2 * c2 + c3 * c3);
        if (++cnt == 16) { acc += (double)part; part = 0.f; cnt = 0; }
      }
      for (int64_t k = (n4 << 2) + threadIdx.x; k < D; k += blockDim.x) {
        float c = (x[k] - mh) - ml;
        part += c * c;
      }
    } else {
      for (int64_t k = threadIdx.x; k < D; k += blockDim.x) {
        float c = (__ldg(x + k) - mh) - ml;
        part += c * c;
        if (++cnt == 64) { acc += (double)part; part = 0.f; cnt = 0; }
      }
    }
    acc += (double)part;
    double ss = block_sum_f64(acc, red);
    if (threadIdx.x == 0) {
      mu_out[row] = mu;
      ss_out[row] = ss;
      // zero variance: correlation undefined, propagate NaN
      rs_out[row] = ss > 0.0 ? 1.0 / sqrt(ss) : __longlong_as_double(0x7ff8000000000000ll);
    }
  }
}

// Centre each row and write the split-BF16 (and optionally FP32) copies,
// zero-padded to Dp columns.  Each thread handles 4 consecutive columns.
template <bool VEC4>
__global__ void __launch_bounds__(256)
vec_split_kernel(const float *__restrict__ X, int64_t n, int64_t D, int64_t ld, int64_t Dp,
                 const double *__restrict__ mu, __nv_bfloat16 *__restrict__ hi,
                 __nv_bfloat16 *__restrict__ lo, float *__restrict__ c32) {
  int64_t q4 = Dp >> 2;                       // float4 groups per padded row
  for (int64_t row = blockIdx.y; row < n; row += gridDim.y) {
    const float *x = X + row * ld;
    double m = mu[row];
    float mh = (float)m;
    float ml = (float)(m - (double)mh);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q4;
         q += (int64_t)gridDim.x * blockDim.x) {
      int64_t k = q << 2;
      float v[4];
      if (VEC4 && k + 3 < D) {
        float4 t = __ldg(reinterpret_cast<const float4 *>(x + k));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (k + e < D) ? __ldg(x + k + e) : 0.f;
      }
      float c[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) c[e] = (k + e < D) ? (v[e] - mh) - ml : 0.f;
      size_t o = (size_t)row * Dp + k;
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
        *reinterpret_cast<uint2 *>(hi + o) = hv;
        *reinterpret_cast<uint2 *>(lo + o) = lv;
      }
      if (c32) *reinterpret_cast<float4 *>(c32 + o) = make_float4(c[0], c[1], c[2], c[3]);
    }
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
  const int lrow = tid & 127, lh = tid >> 7;     // loader: row, k-quad pair
  const int64_t nk = Dp / kF32K;

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t t = s_tile;
    __syncthreads();
    if (t >= n_tiles) break;
    const int64_t i0 = (int64_t)tiles[2 * t] * kF32Tile;
    const int64_t j0 = (int64_t)tiles[2 * t + 1] * kF32Tile;
    const bool a_ok = i0 + lrow < n, b_ok = j0 + lrow < n;
    const float *arow = C + (a_ok ? (i0 + lrow) : 0) * Dp;
    const float *brow = C + (b_ok ? (j0 + lrow) : 0) * Dp;

    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    float4 ra[2], rb[2];
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    auto gload = [&](int64_t kb) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int64_t k = kb * kF32K + (lh + 2 * h) * 4;
        ra[h] = a_ok ? __ldg(reinterpret_cast<const float4 *>(arow + k)) : z4;
        rb[h] = b_ok ? __ldg(reinterpret_cast<const float4 *>(brow + k)) : z4;
      }
    };
    auto sstore = [&](int buf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int kq = (lh + 2 * h) * 4;
        As[buf][kq + 0][lrow] = ra[h].x; As[buf][kq + 1][lrow] = ra[h].y;
        As[buf][kq + 2][lrow] = ra[h].z; As[buf][kq + 3][lrow] = ra[h].w;
        Bs[buf][kq + 0][lrow] = rb[h].x; Bs[buf][kq + 1][lrow] = rb[h].y;
        Bs[buf][kq + 2][lrow] = rb[h].z; Bs[buf][kq + 3][lrow] = rb[h].w;
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

cudaError_t launch_vec_stats(const float *X, int64_t n, int64_t D, int64_t ld, double *mu,
                             double *ss, double *rs, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)(n < 65535 ? n : 65535);
  bool vec4 = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (vec4) vec_stats_kernel<true><<<grid, kStatsThreads, 0, s>>>(X, n, D, ld, mu, ss, rs);
  else vec_stats_kernel<false><<<grid, kStatsThreads, 0, s>>>(X, n, D, ld, mu, ss, rs);
  return cudaGetLastError();
}

cudaError_t launch_vec_split(const float *X, int64_t n, int64_t D, int64_t ld, int64_t Dp,
                             const double *mu, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                             float *c32, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t q4 = Dp >> 2;
  int gx = (int)((q4 + 255) / 256);
  if (gx > 1024) gx = 1024;
  dim3 grid(gx, (unsigned)(n < 65535 ? n : 65535));
  bool vec4 = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (vec4) vec_split_kernel<true><<<grid, 256, 0, s>>>(X, n, D, ld, Dp, mu, hi, lo, c32);
  else vec_split_kernel<false><<<grid, 256, 0, s>>>(X, n, D, ld, Dp, mu, hi, lo, c32);
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
