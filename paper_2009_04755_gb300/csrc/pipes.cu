// pipes.cu -- issue-rate probes of the SM pipes that bound the CUDA-core
// kernels of the library: the FP32 FMA pipe (the FP32 comparator Gram) and
// the MUFU (XU) pipe's ex2 and rcp (the overlap kernels spend one of each per
// point pair).  Measurement support for the rooflines the benchmark reports;
// nothing of the method runs here.
//
// Each probe fills every SM with 64 warps whose threads run eight independent
// dependency chains of one instruction, so the pipe, not latency, sets the
// rate.  The kernel has no waits and no memory traffic beyond one store per
// thread; it changes no GPU setting.  Results per clock come from the SM's
// own cycle counter against %globaltimer, so they do not depend on the clock
// the GPU happened to run at.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ap_internal.h"

namespace ap {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ float op_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}
__device__ __forceinline__ float op_rcp(float x) {
  float y;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// PIPE 0: fmaf chains; 1: ex2 chains (x -> 2^-x stays in [0.5, 1]);
// 2: rcp chains x -> 1 / (x + c) (the add keeps two reciprocals in a row from
// cancelling; it runs on the FMA pipe, eight times wider than the MUFU's
// reciprocal); 3: packed FP32x2 fma chains (two results per instruction,
// counted as two)
template <int PIPE>
__global__ void __launch_bounds__(kThreads, kBlocksPerSm)
pipe_probe_kernel(int iters, float *sink, unsigned long long *cycles, unsigned long long *ns) {
  float a[kChains];
  float2 a2[kChains / 2];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 0.5f + 1e-4f * (float)(threadIdx.x + 37 * k);
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) a2[k] = make_float2(a[2 * k], a[2 * k + 1]);
  const float m = 0.9999f, c = 1e-4f;
  const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
  __syncthreads();
  const unsigned long long c0 = clock64();
  const uint64_t t0 = gtimer();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      if (PIPE == 3) {
        // half as many instructions of two results each: the same results
        // per thread as the scalar probe
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) a2[k] = __ffma2_rn(a2[k], m2, c2);
      } else {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
          if (PIPE == 0) a[k] = fmaf(a[k], m, c);
          else if (PIPE == 1) a[k] = op_ex2(a[k]);
          else a[k] = op_rcp(a[k] + c);
        }
      }
    }
  }
  __syncthreads();
  const unsigned long long c1 = clock64();
  const uint64_t t1 = gtimer();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) s += a2[k].x + a2[k].y;
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) {
    cycles[blockIdx.x] = c1 - c0;
    ns[blockIdx.x] = t1 - t0;
  }
}

}  // namespace
}  // namespace ap

using namespace ap;

extern "C" ap_status ap_pipe_rate(int32_t pipe, double *per_clk_per_sm, double *per_s,
                                  double *sm_mhz) {
  if (pipe < 0 || pipe > 3 || !per_clk_per_sm || !per_s) return AP_ERR_INVALID_ARG;
  const int sms = num_sms();
  const int grid = sms * kBlocksPerSm;
  const int iters = (pipe == 0 || pipe == 3) ? 8192 : 1024;
  float *sink = nullptr;
  unsigned long long *cyc = nullptr, *ns = nullptr;
  AP_TRY(dmalloc(&sink, (size_t)grid * kThreads));
  cudaError_t e = dmalloc(&cyc, (size_t)grid);
  if (e == cudaSuccess) e = dmalloc(&ns, (size_t)grid);
  void (*k)(int, float *, unsigned long long *, unsigned long long *) =
      pipe == 0 ? pipe_probe_kernel<0>
      : pipe == 1 ? pipe_probe_kernel<1>
      : pipe == 2 ? pipe_probe_kernel<2> : pipe_probe_kernel<3>;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  // one launch to warm up, one timed
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      k<<<grid, kThreads>>>(iters, sink, cyc, ns);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  std::vector<unsigned long long> hc(grid), hn(grid);
  if (e == cudaSuccess) e = cudaMemcpy(hc.data(), cyc, grid * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hn.data(), ns, grid * 8, cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(sink);
  dfree(cyc);
  dfree(ns);
  if (e != cudaSuccess) return from_cuda(e);
  // every block runs on one SM at a time with kBlocksPerSm of them resident:
  // ops per SM = kBlocksPerSm blocks' ops, over that SM's cycles
  const double ops_block = (double)kThreads * iters * 16 * kChains;
  double cyc_max = 0.0, mhz_sum = 0.0;
  for (int b = 0; b < grid; ++b) {
    cyc_max = hc[b] > cyc_max ? (double)hc[b] : cyc_max;
    mhz_sum += hn[b] > 0 ? (double)hc[b] / (double)hn[b] * 1e3 : 0.0;
  }
  *per_clk_per_sm = ops_block * kBlocksPerSm / cyc_max;
  *per_s = ops_block * grid / (ms * 1e-3);
  if (sm_mhz) *sm_mhz = mhz_sum / grid;
  return AP_OK;
}
