// noalloc.cu -- all-pairs Pearson correlation on the plain FP32 CUDA-core
// path without any device allocation by the library.
//
// Some callers cannot let a library allocate GPU memory: hosts whose GPU
// memory is carved up up front by a pool allocator that the library must not
// bypass, or services with hard limits on what a request may allocate.  This
// entry point takes the caller's raw vectors and output buffer and keeps its
// own working memory (per-item means, inverse norms and the tile-queue
// counter) in one fixed, statically sized device array, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array lives in this file as a `static __device__` object: every GPU
// that loads the library holds AP_NOALLOC_SCRATCH_BYTES of it until the
// process exits.  Host code cannot use the array's name as a device address,
// so its address is looked up once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <mutex>

#include "ap_internal.h"

namespace ap {
namespace {

constexpr int64_t kMaxItems = AP_NOALLOC_MAX_ITEMS;
constexpr size_t kHeaderBytes = 256;                       // queue counter, padded
constexpr size_t kScratchBytes = kHeaderBytes + 2 * sizeof(double) * kMaxItems;
static_assert(kScratchBytes == AP_NOALLOC_SCRATCH_BYTES, "scratch size out of sync");

// [0]: int32 tile-queue head (bytes 4..255 unused),
// [256 ...): double mu[kMaxItems], double rs[kMaxItems]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on
// the first call for that device).
cudaError_t scratch_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (warp == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) red[32] = v;
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// One CTA per row: FP64 mean, then the FP64 centred sum of squares.
__global__ void __launch_bounds__(512)
noalloc_stats_kernel(const float *__restrict__ X, int64_t n, int64_t D, int64_t ld,
                     double *__restrict__ mu_out, double *__restrict__ rs_out) {
  __shared__ double red[33];
  for (int64_t row = blockIdx.x; row < n; row += gridDim.x) {
    const float *x = X + row * ld;
    double acc = 0.0;
    float part = 0.f;
    int cnt = 0;
    for (int64_t k = threadIdx.x; k < D; k += blockDim.x) {
      part += __ldg(x + k);
      if (++cnt == 64) { acc += (double)part; part = 0.f; cnt = 0; }
    }
    const double mu = block_sum(acc + (double)part, red) / (double)D;
    const float mh = (float)mu, ml = (float)(mu - (double)mh);
    acc = 0.0;
    part = 0.f;
    cnt = 0;
    for (int64_t k = threadIdx.x; k < D; k += blockDim.x) {
      const float c = (__ldg(x + k) - mh) - ml;
      part += c * c;
      if (++cnt == 64) { acc += (double)part; part = 0.f; cnt = 0; }
    }
    const double ss = block_sum(acc + (double)part, red);
    if (threadIdx.x == 0) {
      mu_out[row] = mu;
      rs_out[row] = ss > 0.0 ? 1.0 / sqrt(ss) : __longlong_as_double(0x7ff8000000000000ll);
    }
  }
}

// Upper-triangle tile t of an nb x nb block grid in row-major order:
// row I holds nb - I tiles (J = I .. nb-1).
__device__ __forceinline__ void tri_tile(int64_t t, int64_t nb, int64_t &I, int64_t &J) {
  // tiles before row I: I*nb - I(I-1)/2; start from the real root, fix up
  const double b = 2.0 * (double)nb + 1.0;
  int64_t r = (int64_t)floor((b - sqrt(b * b - 8.0 * (double)t)) / 2.0);
  if (r < 0) r = 0;
  if (r > nb - 1) r = nb - 1;
  auto before = [&](int64_t i) { return i * nb - (i * (i - 1)) / 2; };
  while (r > 0 && before(r) > t) --r;
  while (r + 1 < nb && before(r + 1) <= t) ++r;
  I = r;
  J = r + (t - before(r));
}

// The FP32 Gram of the library's CUDA-core path (128 x 128 tiles, 8 x 8
// outputs per thread, K staged 16 at a time), reading the caller's row-major
// vectors and centring them on the fly; r = G * rs_i * rs_j in FP64.
__global__ void __launch_bounds__(256, 1)
noalloc_gram_f32_kernel(const float *__restrict__ X, int64_t n, int64_t D, int64_t ld,
                        const double *__restrict__ mu, const double *__restrict__ rs,
                        int64_t nb, int64_t n_tiles, int32_t *queue, double *__restrict__ out) {
  __shared__ __align__(16) float As[2][16][132];
  __shared__ __align__(16) float Bs[2][16][132];
  __shared__ int64_t s_tile;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t nk = (D + 15) / 16;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(queue, 1);
    __syncthreads();
    const int64_t t = s_tile;
    __syncthreads();
    if (t >= n_tiles) break;
    int64_t I, J;
    tri_tile(t, nb, I, J);
    const int64_t i0 = I * 128, j0 = J * 128;
    // loader: per K block of 16, each thread stages 8 consecutive columns of
    // one A row and one B row
    const int lrow = tid & 127, lq = tid >> 7;
    const int64_t ar = i0 + lrow, br = j0 + lrow;
    const bool a_ok = ar < n, b_ok = br < n;
    float amh = 0.f, aml = 0.f, bmh = 0.f, bml = 0.f;
    if (a_ok) { const double m = mu[ar]; amh = (float)m; aml = (float)(m - (double)amh); }
    if (b_ok) { const double m = mu[br]; bmh = (float)m; bml = (float)(m - (double)bmh); }
    const float *xa = X + (a_ok ? ar : 0) * ld, *xb = X + (b_ok ? br : 0) * ld;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    float ra[8], rb[8];
    auto gload = [&](int64_t kb) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t k = kb * 16 + lq * 8 + e;
        ra[e] = (a_ok && k < D) ? (__ldg(xa + k) - amh) - aml : 0.f;
        rb[e] = (b_ok && k < D) ? (__ldg(xb + k) - bmh) - bml : 0.f;
      }
    };
    auto sstore = [&](int buf) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        As[buf][lq * 8 + e][lrow] = ra[e];
        Bs[buf][lq * 8 + e][lrow] = rb[e];
      }
    };
    gload(0);
    sstore(0);
    __syncthreads();
    for (int64_t kb = 0; kb < nk; ++kb) {
      const int buf = (int)(kb & 1);
      if (kb + 1 < nk) gload(kb + 1);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      }
      if (kb + 1 < nk) sstore(buf ^ 1);
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t i = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + (a - 4));
      if (i >= n) continue;
      const double ri = rs[i];
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int64_t j = j0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + (b - 4));
        if (j >= n || j <= i) continue;
        out[pair_index(i, j, n)] = (double)acc[a][b] * ri * rs[j];
      }
    }
  }
}

}  // namespace
}  // namespace ap

using namespace ap;

extern "C" ap_status ap_pearson_fp32_noalloc(const float *data, int64_t n_items, int64_t dim,
                                             int64_t ld, double *out, void *stream) {
  if (n_items < 0 || dim < 2) return AP_ERR_INVALID_ARG;
  if (ld == 0) ld = dim;
  if (ld < dim) return AP_ERR_INVALID_ARG;
  if (n_items > kMaxItems) return AP_ERR_UNSUPPORTED;      // beyond the scratch array
  if (n_items < 2) return AP_OK;
  if (!data || !out) return AP_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? AP_ERR_OOM : AP_ERR_CUDA;
  int32_t *queue = reinterpret_cast<int32_t *>(base);
  double *mu = reinterpret_cast<double *>(base + kHeaderBytes);
  double *rs = mu + kMaxItems;
  // the queue head must start at zero on every call
  e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return AP_ERR_CUDA;
  const int sgrid = (int)(n_items < 65535 ? n_items : 65535);
  noalloc_stats_kernel<<<sgrid, 512, 0, s>>>(data, n_items, dim, ld, mu, rs);
  if (cudaGetLastError() != cudaSuccess) return AP_ERR_CUDA;
  const int64_t nb = (n_items + 127) / 128;
  const int64_t n_tiles = nb * (nb + 1) / 2;
  int64_t grid = num_sms();
  if (grid > n_tiles) grid = n_tiles;
  noalloc_gram_f32_kernel<<<(int)grid, 256, 0, s>>>(data, n_items, dim, ld, mu, rs, nb, n_tiles,
                                                    queue, out);
  return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}
