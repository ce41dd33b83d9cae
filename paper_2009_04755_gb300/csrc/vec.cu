// vec.cu -- dense-vector kernels: the load pipeline's GPU pre-processing
// (Sec. III, stage 4 of l) and the plain FP32 Gram path of the Pearson
// correlation (the normalised cross correlation of Sec. V-A).
//
//   s_i: a shift close to the mean (the mean of 1024 strided samples)
//   c_ik = x_ik - s_i,  hi = bf16_rn(c),  lo = bf16_rn(c - hi)    (split-BF16)
//   delta_i = (1/D) sum_k c_ik = mu_i - s_i,
//   ss_i = sum_k c_ik^2 - delta_i sum_k c_ik = sum_k (x_ik - mu_i)^2 (FP64)
//   r_ij = (sum_k c_ik c_jk - D delta_i delta_j) / sqrt(ss_i ss_j)  (FP64)
//
// One read of the rows does it all; rows whose shift missed the mean by
// D delta^2 > ss / 64 are written again centred on the exact mean.
// GB300 executes FP64 at a small fraction of its FP32 rate, so the
// per-element work stays in FP32: short FP32 partial sums (64 elements per
// thread) are folded into FP64 accumulators, and the centring subtracts the
// FP64 shift as a two-float pair (x - s_hi) - s_lo, which keeps c accurate
// to a few ulps of c itself even when |s| >> |c|.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

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

// The FP64 mean of each row's columns (the shift of column slices, taken
// from their first chunk): one CTA per row, FP32 partial sums of 64 elements
// per thread folded into FP64.
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

// Centre each row on its shift s (the two-float pair s_hi + s_lo), write the
// blocked split-BF16 and/or FP32 copies (zero padded to Dp columns) and this
// CTA's FP64 partials of sum_k c_k^2 and sum_k c_k into slot blockIdx.x of
// the row (set when first_chunk, else added, so column chunks accumulate).
// Grid: x = column ranges of a row (thread t of CTA b takes the float4
// groups b * blockDim + t + m * stride), y = rows (strided), or only the rows
// of list = [count, rows...].
//
// Blocked offsets advance by constants: the group stride is a multiple of 8
// float4 (one 32-column block), so a thread's column within a block is fixed
// and its block index grows by stride / 8 per step.
__device__ __forceinline__ void split_store(const float c[4], __nv_bfloat16 *hi,
                                            __nv_bfloat16 *lo, float *c32, size_t o_tc,
                                            size_t o_32) {
  if (hi) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(c[0], c[1]);
    const __nv_bfloat162 h23 = __floats2bfloat162_rn(c[2], c[3]);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    // c - hi is exact in FP32; its rounding to BF16 is the low part
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(c[0] - f01.x, c[1] - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(c[2] - f23.x, c[3] - f23.y);
    uint2 hv, lv;
    hv.x = *reinterpret_cast<const uint32_t *>(&h01);
    hv.y = *reinterpret_cast<const uint32_t *>(&h23);
    lv.x = *reinterpret_cast<const uint32_t *>(&l01);
    lv.y = *reinterpret_cast<const uint32_t *>(&l23);
    *reinterpret_cast<uint2 *>(hi + o_tc) = hv;
    *reinterpret_cast<uint2 *>(lo + o_tc) = lv;
  }
  if (c32) *reinterpret_cast<float4 *>(c32 + o_32) = make_float4(c[0], c[1], c[2], c[3]);
}

template <bool VEC4>
__global__ void __launch_bounds__(kSplitThreads, 4)
vec_split_kernel(const float *__restrict__ X, int64_t row0, int64_t out_row0, int64_t n,
                 int64_t D, int64_t ld, int64_t Dp, const double *__restrict__ mu,
                 __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                 float *__restrict__ c32, double *__restrict__ part,
                 double *__restrict__ part_c, int first_chunk,
                 const int32_t *__restrict__ list, int64_t col0, int64_t Dl) {
  // Dp columns (D of them real) of each row go to columns col0.. (a multiple
  // of 32) of blocked copies Dl columns wide
  __shared__ double2 red[kSplitThreads];
  const int64_t q4 = Dp >> 2;                  // float4 groups per padded row
  const int64_t qf = VEC4 ? (D >> 2) : 0;      // groups wholly inside the row
  const int64_t nkb_tc = Dl / kTcKBlock, nkb_32 = Dl / kF32KBlock;
  const int64_t kb0_tc = col0 / kTcKBlock, kb0_32 = col0 / kF32KBlock;
  const int64_t stq = (int64_t)gridDim.x * blockDim.x;
  const int64_t qa = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  constexpr size_t kTileTc = (size_t)kRowBlock * kTcKBlock, kTile32 = (size_t)kRowBlock * kF32KBlock;
  const size_t d_tc = (size_t)(stq >> 3) * kTileTc, d_32 = (size_t)(stq >> 2) * kTile32;
  const int64_t nrows = list ? (int64_t)list[0] : n;
  for (int64_t t = blockIdx.y; t < nrows; t += gridDim.y) {
    const int64_t lr = list ? (int64_t)list[1 + t] : t;
    const int64_t row = row0 + lr;             // global item index (statistics)
    const int64_t orow = out_row0 + lr;        // row of the blocked copies
    const float *x = X + lr * ld;
    const double m = mu[row];
    const float mh = (float)m;
    const float ml = (float)(m - (double)mh);
    const int64_t rb = orow / kRowBlock, ri = orow % kRowBlock;
    size_t o_tc = ((size_t)rb * nkb_tc + (size_t)(kb0_tc + (qa >> 3))) * kTileTc +
                  (size_t)ri * kTcKBlock + 4 * (size_t)(qa & 7);
    size_t o_32 = ((size_t)rb * nkb_32 + (size_t)(kb0_32 + (qa >> 2))) * kTile32 +
                  (size_t)ri * kF32KBlock + 4 * (size_t)(qa & 3);
    double acc = 0.0, acc_c = 0.0;
    float psum = 0.f, psum_c = 0.f;
    int64_t q = qa;
    // four groups per trip, all loads issued before any is used
    for (int trips = 0; q + 3 * stq < qf; q += 4 * stq) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(reinterpret_cast<const float4 *>(x) + q + u * stq);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float c[4] = {(v[u].x - mh) - ml, (v[u].y - mh) - ml, (v[u].z - mh) - ml,
                            (v[u].w - mh) - ml};
        psum += (c[0] * c[0] + c[1] * c[1]) + (c[2] * c[2] + c[3] * c[3]);
        psum_c += (c[0] + c[1]) + (c[2] + c[3]);
        split_store(c, hi, lo, c32, o_tc, o_32);
        o_tc += d_tc;
        o_32 += d_32;
      }
      if (++trips == 4) {                      // 64 elements per FP32 partial
        acc += (double)psum;
        acc_c += (double)psum_c;
        psum = psum_c = 0.f;
        trips = 0;
      }
    }
    // the rest one group at a time, bounds checked (ragged end, padding)
    for (; q < q4; q += stq) {
      const int64_t k = q << 2;
      float c[4];
      if (VEC4 && k + 3 < D) {
        const float4 t4 = __ldg(reinterpret_cast<const float4 *>(x + k));
        c[0] = (t4.x - mh) - ml; c[1] = (t4.y - mh) - ml;
        c[2] = (t4.z - mh) - ml; c[3] = (t4.w - mh) - ml;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) c[e] = (k + e < D) ? (__ldg(x + k + e) - mh) - ml : 0.f;
      }
      psum += (c[0] * c[0] + c[1] * c[1]) + (c[2] * c[2] + c[3] * c[3]);
      psum_c += (c[0] + c[1]) + (c[2] + c[3]);
      split_store(c, hi, lo, c32, o_tc, o_32);
      o_tc += d_tc;
      o_32 += d_32;
    }
    acc += (double)psum;
    acc_c += (double)psum_c;
    // FP64 runs at a small fraction of the FP32 rate: one warp adds the
    // CTA's partials from shared memory instead of a shuffle tree per warp
    red[threadIdx.x] = make_double2(acc, acc_c);
    __syncthreads();
    if (threadIdx.x < 32) {
      double s2 = 0.0, s1 = 0.0;
      for (int k = threadIdx.x; k < kSplitThreads; k += 32) {
        s2 += red[k].x;
        s1 += red[k].y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
      }
      if (threadIdx.x == 0) {
        const size_t slot = (size_t)row * gridDim.x + blockIdx.x;
        part[slot] = first_chunk ? s2 : part[slot] + s2;
        part_c[slot] = first_chunk ? s1 : part_c[slot] + s1;
      }
    }
    __syncthreads();
  }
}


// The shift of each row: the FP64 mean of up to kShiftSamples values spread
// evenly over the row; rows are centred on it in the single pass that
// follows, and the exact mean enters at the end (delta_i = mu_i - s_i from
// the same pass's sums).  One warp per row.
constexpr int kShiftSamples = 1024;
__global__ void vec_shift_kernel(const float *__restrict__ X, int64_t n, int64_t D, int64_t ld,
                                 double *__restrict__ shift) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t count = D < kShiftSamples ? D : kShiftSamples, stride = D / count;
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
       row += warps) {
    const float *x = X + row * ld;
    double acc = 0.0;
    for (int64_t k = lane; k < count; k += 32) acc += (double)__ldg(x + k * stride);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) shift[row] = acc / (double)count;
  }
}

// The shift of rows read straight from pinned host memory (column slices,
// before any chunk is copied): the mean of kShiftRuns evenly spaced runs of 32
// consecutive values, so that each warp load is one 128-byte request across
// the host link; a trend or a period is averaged over the whole row, not
// only over its first chunk.  One warp per row; D < 1024: every value.
constexpr int kShiftRuns = 32;
__global__ void vec_shift_runs_kernel(const float *__restrict__ X, int64_t n, int64_t D,
                                     int64_t ld, double *__restrict__ shift) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const bool all = D < 32 * kShiftRuns;
  const int64_t gap = all ? 32 : D / kShiftRuns;            // >= 32 when sampling
  const int64_t runs = all ? (D + 31) / 32 : kShiftRuns;
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
       row += warps) {
    const float *x = X + row * ld;
    double acc = 0.0;
    int64_t cnt = 0;
#pragma unroll 8
    for (int64_t r = 0; r < runs; ++r) {
      const int64_t k = r * gap + lane;
      if (k < D) { acc += (double)x[k]; ++cnt; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_xor_sync(0xffffffffu, acc, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) shift[row] = acc / (double)cnt;
  }
}

// A row whose shift misses its mean by D delta^2 > ss / 64 is centred again
// on the exact mean: the shifted rows' common part D delta_i delta_j then
// stays below 1/64 of sqrt(ss_i ss_j), so it adds nothing measurable to the
// rounding of the Gram's FP32 chains.
constexpr double kRecentreRatio = 1.0 / 64.0;

// Column-sliced rows centred on shifts s_i: with S1 = sum_k c_ik and
// S2 = sum_k c_ik^2 over all D columns (c = x - s), delta_i = mu_i - s_i =
// S1 / D and ss_i = S2 - S1 delta_i (the shifted-data form of the variance).
// list (optional): rows beyond kRecentreRatio get shift += delta and are
// appended to list = [count, rows...].
__global__ void slice_stats_kernel(const double *__restrict__ part,
                                   const double *__restrict__ part_c, int64_t n, int nparts,
                                   int64_t D, double *__restrict__ delta,
                                   double *__restrict__ ss, double *__restrict__ rs,
                                   double *__restrict__ shift, int32_t *__restrict__ list) {
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
    if (list && v > 0.0 && (double)D * d * d > kRecentreRatio * v) {
      shift[row] += d;
      list[1 + atomicAdd(list, 1)] = (int32_t)row;
    }
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

// r_ij -= (D delta_i rs_i)(delta_j rs_j): the same correction for pairs that
// the whole-tile Gram epilogue already scaled by rs_i rs_j
__global__ void pair_correct_kernel(double *__restrict__ out, const double *__restrict__ rs,
                                    const double *__restrict__ delta, int64_t n, int64_t D) {
  for (int64_t i = blockIdx.x; i < n - 1; i += gridDim.x) {
    const double ei = (double)D * delta[i] * rs[i];
    const int64_t p0 = pair_index(i, i + 1, n);
    for (int64_t j = i + 1 + threadIdx.x; j < n; j += blockDim.x)
      out[p0 + (j - i - 1)] -= ei * (delta[j] * rs[j]);
  }
}

// ---------------------------------------------------------------------------
// FP32 CUDA-core Gram over upper-triangle tiles of 128 x 128 items.
// 256 threads, 8 x 8 outputs per thread (FP32x2 FMAs), K staged 16 at a
// time through registers into transposed, double-buffered shared memory.
// ---------------------------------------------------------------------------
constexpr int kF32Tile = 128;
constexpr int kF32K = 16;
constexpr int kF32Pad = 4;

template <int COVER>
__global__ void __launch_bounds__(256, 2)
gram_f32_kernel(const float *__restrict__ C, int64_t n, int64_t Dp,
                const double *__restrict__ rs, const int32_t *__restrict__ tiles,
                int64_t n_tiles, int32_t *queue, void *out, const double *__restrict__ delta,
                double dcorr) {
  __shared__ __align__(16) float As[2][kF32K][kF32Tile + kF32Pad];
  __shared__ __align__(16) float Bs[2][kF32K][kF32Tile + kF32Pad];
  __shared__ int s_tile;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int nk = (int)(Dp / kF32K);          // < 2^27 k-blocks (int32 keeps registers free)

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

    // outputs (a, b) as packed pairs over b: one FP32x2 FMA per two outputs,
    // so the FMA pipe, not the issue slot, bounds the loop
    float2 acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);

    float4 ra[2], rb[2];
    auto gload = [&](int kb) {
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
    for (int kb = 0; kb < nk; ++kb) {
      const int buf = kb & 1;
      if (kb + 1 < nk) gload(kb + 1);
#pragma unroll
      for (int k = 0; k < kF32K; ++k) {
        float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
        float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
        float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
        float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float2 bv[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                              make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const float2 aa = make_float2(av[a], av[a]);
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = __ffma2_rn(aa, bv[b], acc[a][b]);
        }
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
      const double di = (COVER || !delta) ? 0.0 : dcorr * delta[i];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int64_t j = j0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
        if (j >= n || j <= i) continue;
        const int64_t p = pair_index(i, j, n);
        if (COVER) atomicAdd(reinterpret_cast<int32_t *>(out) + p, 1);
        else
          reinterpret_cast<double *>(out)[p] =
              ((double)((b & 1) ? acc[a][b >> 1].y : acc[a][b >> 1].x) -
               (delta ? di * delta[j] : 0.0)) * ri * rs[j];
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

cudaError_t launch_vec_shift_runs(const float *X, int64_t n, int64_t D, int64_t ld,
                                  double *shift, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int sg = (int)std::min<int64_t>((n + 7) / 8, 65535);
  vec_shift_runs_kernel<<<sg, 256, 0, s>>>(X, n, D, ld, shift);
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
    vec_split_kernel<true><<<grid, kSplitThreads, 0, s>>>(
        X, row0, row0, n, cols, ld, cols_p, shift, hi, lo, nullptr, part, part_c, first_chunk,
        nullptr, 0, cols_p);
  else
    vec_split_kernel<false><<<grid, kSplitThreads, 0, s>>>(
        X, row0, row0, n, cols, ld, cols_p, shift, hi, lo, nullptr, part, part_c, first_chunk,
        nullptr, 0, cols_p);
  return cudaGetLastError();
}

cudaError_t launch_vec_split_cols(const float *X, int64_t row0, int64_t n, int64_t cols,
                                  int64_t ld, int64_t width, int64_t col0, int64_t Dl,
                                  const double *shift, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                  float *c32, double *part, double *part_c, int first_chunk,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  dim3 grid(kSplitParts, (unsigned)(n < 65535 ? n : 65535));
  const bool vec4 = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  if (vec4)
    vec_split_kernel<true><<<grid, kSplitThreads, 0, s>>>(
        X, row0, row0, n, cols, ld, width, shift, hi, lo, c32, part, part_c, first_chunk, nullptr,
        col0, Dl);
  else
    vec_split_kernel<false><<<grid, kSplitThreads, 0, s>>>(
        X, row0, row0, n, cols, ld, width, shift, hi, lo, c32, part, part_c, first_chunk, nullptr,
        col0, Dl);
  return cudaGetLastError();
}

cudaError_t launch_vec_prep(const float *X, int64_t row0, int64_t out_row0, int64_t n, int64_t D,
                            int64_t ld, int64_t Dp, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                            float *c32, double *shift, double *part, double *part_c,
                            double *delta, double *ss, double *rs, int32_t *recentre,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int sg = (int)std::min<int64_t>((n + 7) / 8, 65535);
  vec_shift_kernel<<<sg, 256, 0, s>>>(X, n, D, ld, shift + row0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool vec4 = (ld % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  auto split = [&](dim3 grid, const int32_t *list) {
    if (vec4)
      vec_split_kernel<true><<<grid, kSplitThreads, 0, s>>>(
          X, row0, out_row0, n, D, ld, Dp, shift, hi, lo, c32, part, part_c, 1, list, 0, Dp);
    else
      vec_split_kernel<false><<<grid, kSplitThreads, 0, s>>>(
          X, row0, out_row0, n, D, ld, Dp, shift, hi, lo, c32, part, part_c, 1, list, 0, Dp);
    return cudaGetLastError();
  };
  const int fg = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  auto stats = [&](int32_t *list) {
    slice_stats_kernel<<<fg, 256, 0, s>>>(part + row0 * kSplitParts, part_c + row0 * kSplitParts,
                                          n, kSplitParts, D, delta + row0, ss + row0, rs + row0,
                                          shift + row0, list);
    return cudaGetLastError();
  };
  if ((e = split(dim3(kSplitParts, (unsigned)(n < 65535 ? n : 65535)), nullptr)) != cudaSuccess)
    return e;
  if ((e = cudaMemsetAsync(recentre, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
  if ((e = stats(recentre)) != cudaSuccess) return e;
  // the rows the sampled shift served badly, again from the exact mean (the
  // list is normally empty and the CTAs return at once)
  if ((e = split(dim3(kSplitParts, (unsigned)(n < 256 ? n : 256)), recentre)) != cudaSuccess)
    return e;
  return stats(nullptr);
}

cudaError_t launch_pair_correct(double *out, const double *rs, const double *delta, int64_t n,
                                int64_t D, cudaStream_t s) {
  if (n < 2) return cudaSuccess;
  const int grid = (int)(n - 1 < 65535 ? n - 1 : 65535);
  pair_correct_kernel<<<grid, 256, 0, s>>>(out, rs, delta, n, D);
  return cudaGetLastError();
}

cudaError_t launch_pair_finalize(double *out, const double *rs, const double *delta, int64_t n,
                                 int64_t D, cudaStream_t s) {
  if (n < 2) return cudaSuccess;
  const int grid = (int)(n - 1 < 65535 ? n - 1 : 65535);
  slice_finalize_kernel<<<grid, 256, 0, s>>>(out, rs, delta, n, D);
  return cudaGetLastError();
}

cudaError_t launch_slice_finalize(const double *part, const double *part_c, int64_t n,
                                  int64_t D, double *delta, double *ss, double *rs, double *out,
                                  cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int fg = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  slice_stats_kernel<<<fg, 256, 0, s>>>(part, part_c, n, kSplitParts, D, delta, ss, rs, nullptr,
                                        nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n < 2) return e;
  const int grid = (int)(n - 1 < 65535 ? n - 1 : 65535);
  slice_finalize_kernel<<<grid, 256, 0, s>>>(out, rs, delta, n, D);
  return cudaGetLastError();
}

cudaError_t launch_gram_f32(const float *C, int64_t n, int64_t Dp, const double *rs,
                            const int32_t *tiles, int64_t n_tiles, int32_t *queue, void *out,
                            int coverage, int64_t, int64_t, cudaStream_t s, const double *delta,
                            int64_t D) {
  if (n_tiles <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  // as many persistent CTAs as fit (two per SM: 16 warps keep the FMA pipe
  // issuing where 8 left it idle a third of the time)
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, coverage ? gram_f32_kernel<1> : gram_f32_kernel<0>, 256, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > n_tiles) grid = n_tiles;
  if (coverage)
    gram_f32_kernel<1><<<(int)grid, 256, 0, s>>>(C, n, Dp, rs, tiles, n_tiles, queue, out, delta,
                                                 (double)D);
  else
    gram_f32_kernel<0><<<(int)grid, 256, 0, s>>>(C, n, Dp, rs, tiles, n_tiles, queue, out, delta,
                                                 (double)D);
  return cudaGetLastError();
}

}  // namespace ap
