// gram_tc2.cu -- the split-BF16 Gram of the Pearson correlation (normalised
// cross correlation, Sec. V-A) on pairs of SMs: one tcgen05.mma.cta_group::2
// computes a 256 x 256 block of D = Hi_I.Hi_J + Hi_I.Lo_J + Lo_I.Hi_J over
// two CTAs of a cluster, each CTA holding its own 128 rows of the I block and
// half (128 rows) of the J block in shared memory, and its 128 rows of D in
// its own TMEM.  Against one CTA per 128 x 256 tile this halves the J-block
// bytes every SM stages and reads per MMA (32 KB instead of 48 KB a stage),
// the shared-memory traffic that bounds the single-CTA kernel.
//
// Work arrives as units {A row block of CTA 0, of CTA 1, B row block of CTA
// 0, of CTA 1, first row block of the I block, J block (256 items), first and
// end 64-column chunk}: macro pairs (I <= J) of the upper triangle in
// recursive quadrant order (Sec. IV-B), optionally split into column ranges
// that run in waves (all pairs of a wave stream the same columns, which they
// share in L2).  The even CTA of each pair pops units from the atomic queue
// (in-GPU work stealing) and hands them to both CTAs through a ring in
// shared memory, so loading runs ahead across units and the epilogue of one
// unit overlaps the MMAs of the next.
//
// Roles (320 threads per CTA):
//   warp 0     one thread issues the TMA loads of this CTA's operand blocks
//              as soon as the stage is free; both CTAs' loads complete on the
//              even CTA's barrier of the stage; the even CTA's thread also
//              pops units;
//   warp 1     TMEM allocation (both CTAs, collectively); in the even CTA one
//              thread issues the MMAs, re-arms each stage's barrier for the
//              bytes of both CTAs as soon as it has seen the stage full (so
//              that neither CTA waits on the other before loading) and
//              commits the MMAs to the barriers of both CTAs;
//   warps 2-9  epilogue of this CTA's 128 rows: TMEM -> FP32 register sums
//              per 256-column chain (seeded chains, as in the single-CTA
//              kernel), FP64 output through a shared-memory transpose so that
//              the packed upper-triangle stores of a row are contiguous.
// Every wait is bounded by a per-launch budget; a wait that runs out records
// a device error code, stops both CTAs of the pair, drains the copies and
// MMAs in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ap_internal.h"
#include "tc_ptx.cuh"

namespace ap {

namespace {

using namespace tc;

constexpr int BM = 128;                      // rows of the I block per CTA (M = 256 per pair)
constexpr int BN = 256;                      // N of the MMA: one J block
constexpr int BK = kTcKBlock;                // bf16 columns per stage (64 bytes a row)
constexpr int STAGES = 6;
constexpr int OP_BYTES = 128 * BK * 2;       // one 128-row operand block: 8 KB
constexpr int STAGE_BYTES = 4 * OP_BYTES;    // A hi, A lo, B-half hi, B-half lo
constexpr uint32_t PAIR_TX_BYTES = 2 * STAGE_BYTES;   // both CTAs' loads of one stage
constexpr int TMEM_COLS = 2 * BN;            // two 128 x 256 FP32 accumulators per CTA
constexpr int kEpiWarps = 8;
constexpr int NUM_THREADS = 32 * (2 + kEpiWarps);
constexpr int kRing = 4;                     // units handed out ahead
// consumers of a ring slot: the odd CTA's producer, the MMA thread and the
// epilogue warps of both CTAs
constexpr int kUnitConsumers = 2 + 2 * kEpiWarps;
constexpr int kChainStages = 8;              // one accumulation chain = 256 columns of D
constexpr int kHeadStages = 2;               // the first two chains of a unit: 64 columns
constexpr float kSeedBeta = 0.9f;
constexpr int kFlushCols = 16384;
constexpr int kFlushKb = kFlushCols / BK;
constexpr int kUnitChunkStages = kOocChunkCols / BK;
constexpr int kTrStride = 33;                // floats per transposed row (32 + 1 pad)
constexpr int TRANS_BYTES = kEpiWarps * 32 * kTrStride * 4;
constexpr int BAR_BYTES = 512;               // barriers, unit ring, teardown counters
constexpr int SMEM_BYTES = 1024 /*align*/ + STAGES * STAGE_BYTES + TRANS_BYTES + BAR_BYTES;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = 256 (N >> 3 at bit 17), M = 256 over the CTA pair (M >> 4 at bit 24)
constexpr uint32_t IDESC2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ void umma_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC2), "r"(accumulate)
      : "memory");
}

// arrive on the mbarrier at this offset in both CTAs of the pair once the
// MMAs issued so far have completed
__device__ __forceinline__ void umma_commit_both(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"((uint16_t)3)
      : "memory");
}

// the same for this CTA's barrier only
__device__ __forceinline__ void umma_commit_local(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void mbar_complete_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

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

// ATOMIC = 1: the unit's partial Gram is added into FP64 `out` (split-K: several
// column ranges of one block pair); ATOMIC = 0: whole block pairs, out = G rs_i rs_j.
// COVER = 1: no arithmetic, each pair of the unit adds 1 to int32 `out`.
// Registers: each of the SM's four sub-partitions holds 16384 of them and
// ten warps put three warps on two sub-partitions, so 3 x 32 x 168 = 16128
// is the most a thread may take and the CTA still launch.
template <int COVER, int ATOMIC>
__global__ void __maxnreg__(168)
gram_tc2_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                int64_t n, const double *__restrict__ rs, const int32_t *__restrict__ units,
                int32_t n_units, int32_t *queue, int32_t *status, double *__restrict__ g64,
                void *out, uint64_t budget, int32_t debug) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  float *trans = reinterpret_cast<float *>(smem + STAGES * STAGE_BYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES + TRANS_BYTES);
  // bars: full[S] empty[S] tfull[2] tempty[2] ufull[R] uempty[R] drain
  constexpr int B_FULL = 0, B_EMPTY = STAGES, B_TFULL = 2 * STAGES, B_TEMPTY = B_TFULL + 2,
                B_UFULL = B_TEMPTY + 2, B_UEMPTY = B_UFULL + kRing, B_DRAIN = B_UEMPTY + kRing,
                N_BARS = B_DRAIN + 1;
  int32_t *ring = reinterpret_cast<int32_t *>(bars + N_BARS);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ring + kRing);
  volatile int *s_abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  // teardown accounting per stage: phases the MMA thread has seen complete,
  // the phase of this CTA's last load into it (-1: none) and, in the even
  // CTA, the odd CTA's
  int32_t *t_cons = reinterpret_cast<int32_t *>(tmem_slot + 2);
  int32_t *t_load0 = t_cons + STAGES, *t_load1 = t_load0 + STAGES;
  static_assert(N_BARS * 8 + kRing * 4 + 8 + 3 * STAGES * 4 <= BAR_BYTES, "barrier area");

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();        // 0: issues the MMAs, 1: its peer
  const bool leader = rank == 0;
  const uint32_t smem_base = smem_u32(smem);
  auto bar = [&](int k) { return smem_u32(&bars[k]); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(bar(B_FULL + s), 1);
      mbar_init(bar(B_EMPTY + s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(bar(B_TFULL + a), 1);
      mbar_init(bar(B_TEMPTY + a), 2 * kEpiWarps);
    }
    for (int u = 0; u < kRing; ++u) {
      mbar_init(bar(B_UFULL + u), 1);
      mbar_init(bar(B_UEMPTY + u), kUnitConsumers);
    }
    mbar_init(bar(B_DRAIN), 1);
    *s_abort = 0;
    for (int s = 0; s < STAGES; ++s) t_cons[s] = 0, t_load0[s] = -1, t_load1[s] = -1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // the even CTA arms every stage's first phase for the bytes of both CTAs;
    // later phases are armed by the MMA thread when it sees the one before
    if (rank == 0)
      for (int s = 0; s < STAGES; ++s) mbar_expect_tx(bar(B_FULL + s), PAIR_TX_BYTES);
  }
  if (warp == 1) {
    // both CTAs of the pair allocate together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  cluster_sync();                 // the peer's barriers exist before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // the other CTA's copies of a local address
  auto remote = [&](uint32_t local, uint32_t r) { return mapa(local, r); };
  const uint32_t peer = rank ^ 1u;
  // stop both CTAs of the pair: record the code, raise both abort flags
  auto abort_pair = [&](int32_t code) {
    atomicCAS(status, 0, code);
    *s_abort = 1;
    st_cluster_u32(remote(smem_u32((const void *)s_abort), peer), 1u);
  };
  // an arrive on a barrier of the even CTA (local there, remote from the odd one)
  auto arrive_leader = [&](uint32_t local_bar) {
    if (leader) mbar_arrive(local_bar);
    else mbar_arrive_cluster(remote(local_bar, 0));
  };
  auto unit_of = [&](int32_t t, int32_t &rb_a, int32_t &rb_b, int64_t &i0, int64_t &j0,
                     int64_t &kb0, int64_t &nkb) {
    const int32_t *u = units + (size_t)8 * t;
    rb_a = u[rank];
    rb_b = u[2 + rank];
    i0 = (int64_t)(u[4] + (int32_t)rank) * BM;
    j0 = (int64_t)u[5] * BN;
    kb0 = (int64_t)u[6] * kUnitChunkStages;
    nkb = COVER ? 0 : (int64_t)(u[7] - u[6]) * kUnitChunkStages;
  };

  if (warp == 0 && lane == 0) {
    // ---------------- unit hand-out + TMA producer ----------------
    uint32_t us = 0, uph = 0, ps = 0, pph = 0;
    int32_t round = 0;                     // phase of every stage in this pass of the ring
    bool stop = false;
    while (!stop) {
      int32_t t;
      if (leader) {
        if (!mbar_wait(bar(B_UEMPTY + us), uph ^ 1, s_abort, budget)) {
          abort_pair(DEV_TIMEOUT_UNIT);
          break;
        }
        t = atomicAdd(queue, 1);
        if (*s_abort || *reinterpret_cast<volatile int32_t *>(status) != 0) t = n_units;
        if (t > n_units) t = n_units;
        ring[us] = t;
        st_cluster_u32(remote(smem_u32(&ring[us]), 1), (uint32_t)t);
        mbar_arrive(bar(B_UFULL + us));
        mbar_arrive_cluster(remote(bar(B_UFULL + us), 1));
      } else {
        if (!mbar_wait<true>(bar(B_UFULL + us), uph, s_abort, budget)) {
          abort_pair(DEV_TIMEOUT_UNIT);
          break;
        }
        t = ring[us];
        mbar_arrive_cluster(remote(bar(B_UEMPTY + us), 0));
      }
      if (++us == kRing) { us = 0; uph ^= 1; }
      if (t >= n_units) break;
      int32_t rb_a, rb_b;
      int64_t i0, j0, kb0, nkb;
      unit_of(t, rb_a, rb_b, i0, j0, kb0, nkb);
      for (int64_t kb = kb0; kb < kb0 + nkb; ++kb) {
        // the stage is free once the MMAs of its previous phase have landed
        // (and by then the even CTA has armed its next phase)
        if (!mbar_wait(bar(B_EMPTY + ps), pph ^ 1, s_abort, budget)) {
          abort_pair(DEV_TIMEOUT_EMPTY);
          stop = true;
          break;
        }
        const uint32_t sb = smem_base + ps * STAGE_BYTES;
        const int32_t k = (int32_t)kb;
        // debug 1 withholds the even CTA's loads of the first stage of every
        // unit, debug 2 of its sixth (or last), after MMAs of the unit have
        // been issued: the waits for it must run out and report (failure-path
        // testing only)
        const bool withhold = leader && ((debug == 1 && kb == kb0) ||
                                         (debug == 2 && kb == kb0 + (nkb > 5 ? 5 : nkb - 1)));
        if (!withhold) {
          // this CTA's blocks; the loads complete on the even CTA's barrier
          const uint32_t fb = leader ? bar(B_FULL + ps) : remote(bar(B_FULL + ps), 0);
          tma_load_block_pair(sb, &tm_hi, fb, k, rb_a);
          tma_load_block_pair(sb + OP_BYTES, &tm_lo, fb, k, rb_a);
          tma_load_block_pair(sb + 2 * OP_BYTES, &tm_hi, fb, k, rb_b);
          tma_load_block_pair(sb + 3 * OP_BYTES, &tm_lo, fb, k, rb_b);
          t_load0[ps] = round;
        }
        if (++ps == STAGES) { ps = 0; pph ^= 1; ++round; }
      }
    }
    // the odd CTA's load record goes to the even CTA for the teardown
    if (!leader)
      for (int s = 0; s < STAGES; ++s)
        st_cluster_u32(remote(smem_u32(&t_load1[s]), 0), (uint32_t)t_load0[s]);
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (even CTA) ----------------
    uint32_t us = 0, uph = 0, ms = 0, mph = 0, mc = 0;
    int32_t mround = 0;                    // the ring pass of the next stage to wait for
    for (bool ok = true; ok;) {
      if (!mbar_wait(bar(B_UFULL + us), uph, s_abort, budget)) {
        abort_pair(DEV_TIMEOUT_UNIT);
        break;
      }
      const int32_t t = ring[us];
      mbar_arrive(bar(B_UEMPTY + us));
      if (++us == kRing) { us = 0; uph ^= 1; }
      if (t >= n_units) break;
      int32_t rb_a, rb_b;
      int64_t i0, j0, kb0, nkb;
      unit_of(t, rb_a, rb_b, i0, j0, kb0, nkb);
      const int64_t nchains = chain_count(nkb);
      for (int64_t c = 0; c < nchains && ok; ++c, ++mc) {
        const uint32_t a = mc & 1, use = mc >> 1;
        if (!mbar_wait<true>(bar(B_TEMPTY + a), (use & 1) ^ 1, s_abort, budget)) {
          abort_pair(DEV_TIMEOUT_ACCUM);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + a * BN;
        const int64_t stages = chain_stages(c, nkb);
        const uint32_t seeded = c >= 2 ? 1u : 0u;   // later chains start from the epilogue's seed
        for (int s = 0; s < stages; ++s) {
          if (!mbar_wait(bar(B_FULL + ms), mph, s_abort, budget)) {
            abort_pair(DEV_TIMEOUT_FULL);
            ok = false;
            break;
          }
          // arm the stage's next phase now: the loads into it can only start
          // after the MMAs below have landed and released it
          mbar_expect_tx(bar(B_FULL + ms), PAIR_TX_BYTES);
          tc_fence_after();
          const uint32_t sb = smem_base + ms * STAGE_BYTES;
          const uint32_t a_hi = sb, a_lo = sb + OP_BYTES;
          const uint32_t b_hi = sb + 2 * OP_BYTES, b_lo = sb + 3 * OP_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t dah = sw64_desc(a_hi + off), dal = sw64_desc(a_lo + off);
            const uint64_t dbh = sw64_desc(b_hi + off), dbl = sw64_desc(b_lo + off);
            umma_pair(dt, dah, dbh, (seeded | s | kk) != 0 ? 1u : 0u);
            umma_pair(dt, dah, dbl, 1u);
            umma_pair(dt, dal, dbh, 1u);
          }
          umma_commit_both(bar(B_EMPTY + ms));   // both CTAs' stage may be refilled
          if (++ms == STAGES) { ms = 0; mph ^= 1; ++mround; }
        }
        if (!ok) break;
        umma_commit_both(bar(B_TFULL + a));      // both CTAs' accumulators are ready
      }
    }
    // every MMA issued must have landed before TMEM is freed: after an abort
    // mid-chain some were never committed, so commit them all and wait
    umma_commit_local(bar(B_DRAIN));
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar(B_DRAIN), 0)) {
      if (global_ns() - t0 > budget) {
        atomicCAS(status, 0, DEV_TIMEOUT_ACCUM);
        break;
      }
    }
    // phases seen complete per stage: the stages before the next one to wait
    // for have been seen once more in this pass
    for (int s = 0; s < STAGES; ++s) t_cons[s] = mround + (s < (int)ms ? 1 : 0);
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;                // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;         // column half of the 256-wide block
    const int row = q * 32 + lane;
    float *tb = trans + (size_t)(warp - 2) * 32 * kTrStride;
    double *my_g64 = g64 + (size_t)blockIdx.x * (BN * BM);
    uint32_t us = 0, uph = 0, ec = 0;
    for (;;) {
      bool ok = mbar_wait<true>(bar(B_UFULL + us), uph, s_abort, budget);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (lane == 0) abort_pair(DEV_TIMEOUT_UNIT);
        break;
      }
      const int32_t t = ring[us];
      __syncwarp();
      if (lane == 0) arrive_leader(bar(B_UEMPTY + us));
      if (++us == kRing) { us = 0; uph ^= 1; }
      if (t >= n_units) break;
      int32_t rb_a, rb_b;
      int64_t i0, j0, kb0, nkb;
      unit_of(t, rb_a, rb_b, i0, j0, kb0, nkb);
      const int64_t nchains = chain_count(nkb);
      float sum[BN / 2];
#pragma unroll
      for (int c = 0; c < BN / 2; ++c) sum[c] = 0.f;
      bool flushed = false;
      int64_t kb_since = 0;
      for (int64_t c = 0; c < nchains; ++c, ++ec) {
        const uint32_t a = ec & 1, use = ec >> 1;
        ok = mbar_wait(bar(B_TFULL + a), use & 1, s_abort, budget);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (lane == 0) abort_pair(DEV_TIMEOUT_ACCUM);
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + a * BN + h * (BN / 2);
        const int64_t len = chain_stages(c, nkb);
        kb_since += len;
        // The tensor core's accumulate truncates the addends it aligns and
        // rounds toward zero, so a long chain of same-signed products comes
        // out short.  Chain c + 2 in this accumulator starts from -g,
        // g = kSeedBeta x this chain's value scaled to that chain's length,
        // and the register sum takes +g: the accumulator then swings about
        // zero and the errors of its two halves cancel (the single-CTA
        // kernel measures and explains the bias in detail).
        const bool seed = c + 2 < nchains;
        const float ratio =
            seed ? kSeedBeta * (float)chain_stages(c + 2, nkb) / (float)len : 0.f;
#pragma unroll
        for (int m = 0; m < BN / 2 / 16; ++m) {
          uint32_t v[16];
          tmem_ld16(taddr + m * 16, v);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float r = __uint_as_float(v[e]), g = r * ratio;
            sum[m * 16 + e] += r + g;
            v[e] = __float_as_uint(-g);
          }
          if (seed) tmem_st16(taddr + m * 16, v);
        }
        if (seed) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) arrive_leader(bar(B_TEMPTY + a));
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
      if (!ok) break;
      // output: 32 columns at a time through the warp's transpose buffer, so
      // that one warp instruction covers 32 consecutive pairs (i, j..j+31)
      // of one row
      const int64_t j = j0 + h * (BN / 2) + lane;
#pragma unroll
      for (int cb = 0; cb < BN / 2 / 32; ++cb) {
        if (!COVER) {
#pragma unroll
          for (int e = 0; e < 32; ++e) tb[lane * kTrStride + e] = sum[cb * 32 + e];
        }
        __syncwarp();
        const int64_t jc = j + cb * 32;
#pragma unroll 1
        for (int r = 0; r < 32; ++r) {
          const int64_t i = i0 + q * 32 + r;
          if (i < n && jc > i && jc < n) {
            const int64_t p = pair_index(i, jc, n);
            if (COVER) {
              atomicAdd(reinterpret_cast<int32_t *>(out) + p, 1);
            } else {
              double g = (double)tb[r * kTrStride + lane];
              if (flushed) g += my_g64[(size_t)(h * (BN / 2) + cb * 32 + lane) * BM + q * 32 + r];
              if (ATOMIC) atomicAdd(reinterpret_cast<double *>(out) + p, g);
              else reinterpret_cast<double *>(out)[p] = g * rs[i] * rs[jc];
            }
          }
        }
        __syncwarp();
      }
    }
  }

  // ---------------- teardown ----------------
  __syncthreads();
  __syncwarp();
  cluster_sync();                 // both CTAs' counters are in the even CTA
  if (leader && threadIdx.x == 0) {
    // Copies still in flight can only target the phase of each stage that
    // the MMA thread was waiting for (a stage is reloaded only after that
    // phase completes); it is armed for both CTAs' bytes.  Complete the
    // share of a CTA that never loaded it, then wait for the rest to land.
    // After a normal run no phase has outstanding loads and nothing waits.
    const uint64_t t0 = global_ns();
    for (int s = 0; s < STAGES; ++s) {
      const int32_t cur = t_cons[s];
      const bool l0 = t_load0[s] == cur, l1 = t_load1[s] == cur;
      if (!l0 && !l1) continue;
      if (!l0 || !l1) mbar_complete_tx(bar(B_FULL + s), (uint32_t)STAGE_BYTES);
      while (!mbar_try_wait(bar(B_FULL + s), (uint32_t)cur & 1u)) {
        if (global_ns() - t0 > budget) break;
      }
    }
  }
  __syncthreads();
  __syncwarp();
  cluster_sync();                 // no copy or remote access is outstanding past this point
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

using Kern2 = void (*)(CUtensorMap, CUtensorMap, int64_t, const double *, const int32_t *, int32_t,
                       int32_t *, int32_t *, double *, void *, uint64_t, int32_t);

Kern2 pick(int coverage, int atomic) {
  return coverage ? gram_tc2_kernel<1, 0>
                  : (atomic ? gram_tc2_kernel<0, 1> : gram_tc2_kernel<0, 0>);
}

cudaLaunchConfig_t launch_cfg(int pairs, cudaStream_t s, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs, 1, 1);
  cfg.blockDim = dim3(NUM_THREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

std::mutex g_tc2_mutex;
bool g_tc2_attr[3] = {false, false, false};

cudaError_t ensure_attr(int coverage, int atomic) {
  const int v = coverage ? 2 : atomic;
  std::lock_guard<std::mutex> lock(g_tc2_mutex);
  if (g_tc2_attr[v]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(pick(coverage, atomic),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e == cudaSuccess) g_tc2_attr[v] = true;
  return e;
}

}  // namespace

int64_t tc2_pairs() {
  // CTA pairs that fit at once on the current device: two SMs each
  constexpr int kMaxDev = 64;
  static int cached[kMaxDev] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) dev = 0;
  std::lock_guard<std::mutex> lock(g_tc2_mutex);
  if (cached[dev] > 0) return cached[dev];
  int v = 0;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_cfg(1, nullptr, attr);
  if (cudaFuncSetAttribute(gram_tc2_kernel<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           SMEM_BYTES) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&v, gram_tc2_kernel<0, 1>, &cfg) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    v = num_sms() / 2;
  }
  cached[dev] = v;
  return v;
}

cudaError_t launch_gram_tc2(const void *tmap_hi, const void *tmap_lo, int64_t n, const double *rs,
                            const int32_t *units, int64_t n_units, int32_t *queue,
                            int32_t *status, double *g64, void *out, int coverage, int atomic,
                            uint64_t budget, int32_t debug, cudaStream_t s) {
  if (n_units <= 0) return cudaSuccess;
  if (n_units > INT32_MAX / 2) return cudaErrorInvalidValue;
  cudaError_t e = ensure_attr(coverage, atomic);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(queue, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  int64_t pairs = tc2_pairs();
  if (pairs > n_units) pairs = n_units;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_cfg((int)pairs, s, attr);
  return cudaLaunchKernelEx(&cfg, pick(coverage, atomic),
                            *reinterpret_cast<const CUtensorMap *>(tmap_hi),
                            *reinterpret_cast<const CUtensorMap *>(tmap_lo), n, rs, units,
                            (int32_t)n_units, queue, status, g64, out,
                            (uint64_t)(budget ? budget : kWaitBudgetNs), debug);
}

}  // namespace ap
