// gram_tc.cu -- split-BF16 Gram of centred vectors on the 5th-generation
// tensor cores (tcgen05), the contraction inside the Pearson correlation
// (normalised cross correlation, Sec. V-A):
//
//   G_ij ~= Hi_i . Hi_j + Hi_i . Lo_j + Lo_i . Hi_j      (FP32 accumulation)
//   r_ij  = G_ij * rs_i * rs_j,  rs = 1 / sqrt(ss)        (FP64 epilogue)
//
// One persistent CTA per SM pops tiles (a block of 128 items I x a block of
// 256 items J, upper triangle only, recursive quadrant order) from an atomic
// queue.  Warp roles inside the CTA:
//   warp 0      one thread issues TMA tile loads (hi/lo of both blocks, 32
//               columns per stage, 64-byte swizzle) into a 4-stage ring;
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32 accumulators);
//               one thread issues the three tcgen05.mma products per 16
//               columns into one accumulator per 256-column chain and commits
//               each stage back to the producer;
//   warps 2-9   epilogue: tcgen05.ld of each finished chain into FP32
//               register sums (FP64 every 16384 columns), then FP64 scaling
//               and packed upper-triangle stores once per tile.
// Every wait is bounded (a per-launch budget, 2 s by default); when one runs
// out the CTA records a device error code, drains its in-flight copies and
// the MMAs it has issued, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ap_internal.h"
#include "tc_ptx.cuh"

namespace ap {

namespace {

using namespace tc;

constexpr int BM = kTcTileM;                 // 128 rows of the I block
constexpr int BN = kTcTileN;                 // 256 rows of the J block
constexpr int BK = kTcKBlock;                // bf16 columns per stage (64 bytes)
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;         // 8 KB
constexpr int B_BYTES = BN * BK * 2;         // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // 48 KB
constexpr int TMEM_COLS = 2 * BN;            // two 128 x 256 FP32 accumulators
constexpr int kEpiWarps = 8;                 // two per TMEM lane quarter
constexpr int NUM_THREADS = 32 * (2 + kEpiWarps);
constexpr int kChainStages = 8;              // one accumulation chain = 256 columns of D
constexpr int kHeadStages = 2;               // the first two chains of a unit: 64 columns
constexpr float kSeedBeta = 0.9f;            // seed damping (see the epilogue)
constexpr int kFlushCols = 16384;            // FP32 register sums -> FP64 every ~16384 columns
constexpr int kFlushKb = kFlushCols / BK;
constexpr int kUnitChunkStages = kOocChunkCols / BK;   // k-blocks per chunk of a split-K unit
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                           ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// Chains of a unit's nkb k-blocks: two head chains of kHeadStages, then
// chains of kChainStages; the last one may be shorter.
__device__ __forceinline__ int64_t chain_first(int64_t c) {
  return c < 2 ? c * kHeadStages : 2 * kHeadStages + (c - 2) * kChainStages;
}
__device__ __forceinline__ int64_t chain_stages(int64_t c, int64_t nkb) {
  const int64_t len = c < 2 ? kHeadStages : kChainStages, left = nkb - chain_first(c);
  return left < len ? left : len;
}
__device__ __forceinline__ int64_t chain_count(int64_t nkb) {
  return nkb <= 2 * kHeadStages ? (nkb + kHeadStages - 1) / kHeadStages
                                : 2 + (nkb - 2 * kHeadStages + kChainStages - 1) / kChainStages;
}

// Accumulate one 256-column chain of D (eight stages) per TMEM accumulator
// (two accumulators, double-buffered), so the tensor core never carries a
// long FP32 chain; eight epilogue warps drain each chain into FP32 register
// sums and fold those into FP64 scratch every kFlushCols columns.  Chain
// length trades the drain's cost against the accumulator's rounding: at
// 8192 x 2^20, chains of 64 / 128 / 256 / 512 / 1024 columns took 183 / 165
// / 156 / - / - ms (whole tiles) and 191 / 153 / 144 / 142 / 140 ms (64
// column ranges per tile), while the bias on strongly correlated items
// grows in proportion to the length (seeded chains, below, offset it).
//
// OOC = 1 (out-of-core units): each entry of `tiles` is kOocTileInts int32
// {row block of A, row blocks of B (two), I block, J block, first chunk, end
// chunk} (chunks of kOocChunkCols columns) -- row blocks index the slot pool the tensor maps cover, I/J the
// item grid -- and the epilogue adds the unit's partial Gram into FP64
// `out` (atomically: several K ranges of one tile may run at once).
template <int COVER, int OOC>
__global__ void __launch_bounds__(NUM_THREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
               int64_t n, int64_t Dp, const double *__restrict__ rs,
               const int32_t *__restrict__ tiles, int64_t n_tiles, int32_t *queue,
               int32_t *status, double *__restrict__ g64, void *out, uint64_t budget,
               int32_t debug) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], drain
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
  volatile int *s_abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  int *s_tile = reinterpret_cast<int *>(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem_base = smem_u32(smem);
  auto full_bar = [&](int s) { return smem_u32(&bars[s]); };
  auto empty_bar = [&](int s) { return smem_u32(&bars[STAGES + s]); };
  auto tfull_bar = [&](int a) { return smem_u32(&bars[2 * STAGES + a]); };
  auto tempty_bar = [&](int a) { return smem_u32(&bars[2 * STAGES + 2 + a]); };
  const uint32_t drain_bar = smem_u32(&bars[2 * STAGES + 4]);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), kEpiWarps);
    }
    mbar_init(drain_bar, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // pipeline state (each role keeps its own copy)
  uint32_t p_stage = 0, p_phase = 0, m_stage = 0, m_phase = 0;
  uint32_t cc = 0;                          // chains consumed so far (accumulator ring)
  uint32_t issued_mask = 0, parity_mask = 0;   // stages with copies issued, and their phase
  const int64_t nk = Dp / BK;
  double *my_g64 = g64 + (size_t)blockIdx.x * (BN * BM);

  for (;;) {
    if (threadIdx.x == 0) {
      int t = atomicAdd(queue, 1);
      if (*s_abort || *reinterpret_cast<volatile int32_t *>(status) != 0) t = (int)n_tiles;
      *s_tile = t;
    }
    __syncthreads();
    const int64_t t = *s_tile;
    if (t >= n_tiles) break;
    int32_t i0, j0, rb_a, rb_b, rb_b1;
    // this tile's (or unit's) k-blocks [kb0, kb0 + nkb) and its chains of
    // kChainStages k-blocks (the last one may be shorter)
    int64_t kb0 = 0, nkb = COVER ? 0 : nk;
    if (OOC) {
      const int32_t *u = tiles + (size_t)kOocTileInts * t;
      rb_a = u[0]; rb_b = u[1]; rb_b1 = u[2];
      i0 = u[3] * BM;
      j0 = u[4] * BN;
      kb0 = (int64_t)u[5] * kUnitChunkStages;
      nkb = COVER ? 0 : (int64_t)(u[6] - u[5]) * kUnitChunkStages;
    } else {
      i0 = tiles[2 * t] * BM;
      j0 = tiles[2 * t + 1] * BN;
      rb_a = tiles[2 * t];
      rb_b = tiles[2 * t + 1] * (BN / BM);
      rb_b1 = rb_b + 1;
    }

    const int64_t nchains = chain_count(nkb);
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer ----------------
      for (int64_t kb = kb0; kb < kb0 + nkb; ++kb) {
        if (!mbar_wait(empty_bar(p_stage), p_phase ^ 1, s_abort, budget)) {
          atomicCAS(status, 0, DEV_TIMEOUT_EMPTY);
          *s_abort = 1;
          break;
        }
        const uint32_t fb = full_bar(p_stage);
        const uint32_t sb = smem_base + p_stage * STAGE_BYTES;
        // debug 1 withholds the first stage of every tile, debug 2 its sixth
        // (or last) stage, after MMAs of the tile have been issued: the
        // consumer's bounded wait must run out and report (failure-path
        // testing only)
        if ((debug == 1 && kb == kb0) ||
            (debug == 2 && kb == kb0 + (nkb > 5 ? 5 : nkb - 1))) {
          if (++p_stage == STAGES) { p_stage = 0; p_phase ^= 1; }
          continue;
        }
        mbar_expect_tx(fb, STAGE_BYTES);
        const int32_t k = (int32_t)kb;
        tma_load_block(sb, &tm_hi, fb, k, rb_a);
        tma_load_block(sb + A_BYTES, &tm_lo, fb, k, rb_a);
        tma_load_block(sb + 2 * A_BYTES, &tm_hi, fb, k, rb_b);
        tma_load_block(sb + 2 * A_BYTES + A_BYTES, &tm_hi, fb, k, rb_b1);
        tma_load_block(sb + 2 * A_BYTES + B_BYTES, &tm_lo, fb, k, rb_b);
        tma_load_block(sb + 2 * A_BYTES + B_BYTES + A_BYTES, &tm_lo, fb, k, rb_b1);
        issued_mask |= 1u << p_stage;
        parity_mask = (parity_mask & ~(1u << p_stage)) | (p_phase << p_stage);
        if (++p_stage == STAGES) { p_stage = 0; p_phase ^= 1; }
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer ----------------
      uint32_t mc = cc;
      for (int64_t c = 0; c < nchains && !*s_abort; ++c, ++mc) {
        const uint32_t a = mc & 1, use = mc >> 1;
        if (!mbar_wait(tempty_bar(a), (use & 1) ^ 1, s_abort, budget)) {
          atomicCAS(status, 0, DEV_TIMEOUT_ACCUM);
          *s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + a * BN;
        bool ok = true;
        // chains 0 and 1 start from zero; later ones from the seed the
        // epilogue left in this accumulator
        const int64_t stages = chain_stages(c, nkb);
        const uint32_t seeded = c >= 2 ? 1u : 0u;
        for (int s = 0; s < stages; ++s) {
          if (!mbar_wait(full_bar(m_stage), m_phase, s_abort, budget)) {
            atomicCAS(status, 0, DEV_TIMEOUT_FULL);
            *s_abort = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = smem_base + m_stage * STAGE_BYTES;
          const uint32_t a_hi = sb, a_lo = sb + A_BYTES;
          const uint32_t b_hi = sb + 2 * A_BYTES, b_lo = sb + 2 * A_BYTES + B_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t off = kk * 32;    // 16 bf16 = 32 bytes inside the swizzle atom
            const uint64_t dah = sw64_desc(a_hi + off), dal = sw64_desc(a_lo + off);
            const uint64_t dbh = sw64_desc(b_hi + off), dbl = sw64_desc(b_lo + off);
            umma_bf16(dt, dah, dbh, (seeded | s | kk) != 0 ? 1u : 0u);
            umma_bf16(dt, dah, dbl, 1u);
            umma_bf16(dt, dal, dbh, 1u);
          }
          umma_commit(empty_bar(m_stage));
          if (++m_stage == STAGES) { m_stage = 0; m_phase ^= 1; }
        }
        if (!ok) break;
        umma_commit(tfull_bar(a));          // fires when this chain's MMAs have landed
      }
    } else if (warp >= 2) {
      // ---------------- epilogue ----------------
      const int q = warp & 3;                // TMEM lane quarter this warp may access
      const int h = (warp - 2) >> 2;         // column half of the 256-wide tile
      const int row = q * 32 + lane;
      const int64_t i = (int64_t)i0 + row;
      float sum[BN / 2];
#pragma unroll
      for (int c = 0; c < BN / 2; ++c) sum[c] = 0.f;
      bool flushed = false, ok = true;
      uint32_t ec = cc;
      int64_t kb_since = 0;                  // k-blocks summed since the last flush
      for (int64_t c = 0; c < nchains; ++c, ++ec) {
        const uint32_t a = ec & 1, use = ec >> 1;
        if (!mbar_wait(tfull_bar(a), use & 1, s_abort, budget)) {
          if (lane == 0) atomicCAS(status, 0, DEV_TIMEOUT_ACCUM);
          *s_abort = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + a * BN + h * (BN / 2);
        const int64_t len = chain_stages(c, nkb);
        kb_since += len;
        // The tensor core aligns the addends of each accumulate step to the
        // largest exponent, truncating what falls below a few guard bits,
        // and rounds the sum toward zero; a chain whose sum grows one way
        // (correlated items) therefore comes out short by an amount growing
        // with its length and with |accumulator|.  Chain c + 2 in this
        // accumulator starts from -g, g = kSeedBeta x R_c (this chain's
        // drained value, scaled to the next chain's length), and the register
        // sum takes +g: the seeds settle near g = 0.47 S (S a chain's sum), so
        // the accumulator runs from about -S/2 to +S/2, the round-toward-zero
        // errors of its two halves cancel and the alignment losses, which
        // scale with |accumulator|, halve.  Correlated pairs (r ~ 0.99) at
        // 16384 columns per unit, measured with unseeded chains and modelled
        // with the adder above: chains of 64 columns -2.4e-7, 256 columns
        // -8.7e-7, 256 seeded -1.3e-7.
        const bool seed = c + 2 < nchains;
        const float ratio =
            seed ? kSeedBeta * (float)chain_stages(c + 2, nkb) / (float)len : 0.f;
#pragma unroll
        for (int m = 0; m < BN / 2 / 16; ++m) {
          uint32_t v[16];
          tmem_ld16(taddr + m * 16, v);
#pragma unroll
          for (int e = 0; e < 16; ++e) {     // ratio 0 (no seed): g = 0, sum += r
            const float r = __uint_as_float(v[e]), g = r * ratio;
            sum[m * 16 + e] += r + g;
            v[e] = __float_as_uint(-g);
          }
          if (seed) tmem_st16(taddr + m * 16, v);
        }
        if (seed) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty_bar(a)) : "memory");
        if (kb_since >= kFlushKb && c + 1 < nchains) {
          kb_since = 0;
          // fold the FP32 partial sums into FP64 scratch ([col][row] layout)
#pragma unroll
          for (int e = 0; e < BN / 2; ++e) {
            double *gp = my_g64 + (size_t)(h * (BN / 2) + e) * BM + row;
            const double prev = flushed ? *gp : 0.0;
            *gp = prev + (double)sum[e];
            sum[e] = 0.f;
          }
          flushed = true;
        }
      }
      ok = ok && !*s_abort;
      if (ok && i < n) {
        const double ri = (COVER || OOC) ? 0.0 : rs[i];
        const int64_t jb = (int64_t)j0 + h * (BN / 2);
        int64_t p = pair_index(i, jb > i ? jb : i + 1, n);
#pragma unroll
        for (int e = 0; e < BN / 2; ++e) {
          const int64_t j = jb + e;
          if (j > i && j < n) {
            if (COVER) {
              atomicAdd(reinterpret_cast<int32_t *>(out) + p, 1);
            } else {
              double g = (double)sum[e];
              if (flushed) g += my_g64[(size_t)(h * (BN / 2) + e) * BM + row];
              if (OOC) atomicAdd(reinterpret_cast<double *>(out) + p, g);
              else reinterpret_cast<double *>(out)[p] = g * ri * rs[j];
            }
            ++p;
          }
        }
      }
    }
    cc += (uint32_t)nchains;
    __syncthreads();
  }

  // teardown: the producer drains copies still in flight after an abort
  if (warp == 0 && lane == 0 && *s_abort) {
    for (int s = 0; s < STAGES; ++s) {
      if (!((issued_mask >> s) & 1u)) continue;
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(full_bar(s), (parity_mask >> s) & 1u)) {
        if (global_ns() - t0 > budget) break;
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    // every MMA this thread issued must have landed before its accumulators
    // are freed: after an abort mid-chain some were never committed to an
    // accumulator barrier, so commit them all to one of their own and wait
    if (lane == 0) {
      umma_commit(drain_bar);
      const uint64_t t0 = global_ns();
      while (!mbar_try_wait(drain_bar, 0)) {
        if (global_ns() - t0 > budget) {
          atomicCAS(status, 0, DEV_TIMEOUT_ACCUM);
          break;
        }
      }
    }
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// The blocked copy as a 4-D tensor {32 columns, 128 rows, column blocks,
// row blocks}; one box is one contiguous 8 KB block.
cudaError_t encode_rows(const __nv_bfloat16 *base, int64_t n, int64_t Dp, CUtensorMap *m) {
  EncodeTiledFn fn = get_encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const int64_t nkb = Dp / BK, nrb = (n + BM - 1) / BM;
  cuuint64_t dims[4] = {(cuuint64_t)BK, (cuuint64_t)BM, (cuuint64_t)nkb, (cuuint64_t)nrb};
  cuuint64_t strides[3] = {(cuuint64_t)BK * 2, (cuuint64_t)BK * BM * 2,
                           (cuuint64_t)nkb * BK * BM * 2};
  cuuint32_t box[4] = {(cuuint32_t)BK, (cuuint32_t)BM, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(base), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t make_tc_tensor_maps(const __nv_bfloat16 *hi, const __nv_bfloat16 *lo, int64_t n,
                                int64_t Dp, void **tmap_hi, void **tmap_lo) {
  CUtensorMap *a = new CUtensorMap, *b = new CUtensorMap;
  cudaError_t e = encode_rows(hi, n, Dp, a);
  if (e == cudaSuccess) e = encode_rows(lo, n, Dp, b);
  if (e != cudaSuccess) {
    delete a;
    delete b;
    return e;
  }
  *tmap_hi = a;
  *tmap_lo = b;
  return cudaSuccess;
}

int64_t tc_grid(int64_t n_tiles) {
  int64_t g = num_sms();
  return g < n_tiles ? g : (n_tiles > 0 ? n_tiles : 1);
}

size_t tc_scratch_doubles(int64_t n_tiles) { return (size_t)tc_grid(n_tiles) * BM * BN; }

void free_tc_tensor_maps(void *a, void *b) {
  delete reinterpret_cast<CUtensorMap *>(a);
  delete reinterpret_cast<CUtensorMap *>(b);
}

cudaError_t launch_gram_tc(const void *tmap_hi, const void *tmap_lo, int64_t n, int64_t Dp,
                           const double *rs, const int32_t *tiles, int64_t n_tiles,
                           int32_t *queue, int32_t *status, double *g64, void *out,
                           int coverage, int ooc, uint64_t budget, int32_t debug,
                           cudaStream_t s) {
  if (n_tiles <= 0) return cudaSuccess;
  static bool attr_done[4] = {false, false, false, false};
  const int v = (coverage ? 1 : 0) + (ooc ? 2 : 0);
  void (*kern)(CUtensorMap, CUtensorMap, int64_t, int64_t, const double *, const int32_t *,
               int64_t, int32_t *, int32_t *, double *, void *, uint64_t, int32_t) =
      v == 0 ? gram_tc_kernel<0, 0> : v == 1 ? gram_tc_kernel<1, 0>
             : v == 2 ? gram_tc_kernel<0, 1> : gram_tc_kernel<1, 1>;
  if (!attr_done[v]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_done[v] = true;
  }
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  int64_t grid = tc_grid(n_tiles);
  kern<<<(int)grid, NUM_THREADS, SMEM_BYTES, s>>>(
      *reinterpret_cast<const CUtensorMap *>(tmap_hi),
      *reinterpret_cast<const CUtensorMap *>(tmap_lo), n, Dp, rs, tiles, n_tiles, queue, status,
      g64, out, budget ? budget : kWaitBudgetNs, debug);
  return cudaGetLastError();
}

}  // namespace ap
