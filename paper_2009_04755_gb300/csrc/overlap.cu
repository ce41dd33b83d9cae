// overlap.cu -- Gaussian overlap cost between weighted point clouds, the
// cross term of the GMM L2 distance used by the microscopy application
// (Sec. V-C), its adjoint with respect to a rigid 2-D transform, and batched
// gradient ascent for pairwise registration.
//
//   f(i,j) = sum_a sum_b w_a w_b exp(-|x_a - (R x_b + t)|^2 / (2 (s_a^2 + s_b^2)))
//
// Storage (built by cloud_pack): items in planner order, padded to multiples
// of 4 points, s2k = 2 ln2 sigma^2 (stored negated) and lw = log2 w, so each
// term is
//   w_a * 2^(lw_b - d^2 / (s2k_a + s2k_b))
// = one add, one MUFU reciprocal, one FMA and one MUFU ex2 after d^2; the
// FP32 work runs as packed FP32x2 operations on two a-points at a time.
// With a transform the a-points are moved instead of the b-points:
//   |x_a - (R x_b + t)| = |R^T (x_a - t) - x_b|,
// so the inner loop is unchanged, and the adjoint follows from
//   df/dt = 2 ln2 * R sum e r d',   df/dtheta = 2 ln2 * sum e r (x_b d'_y - y_b d'_x)
// with d' = R^T (x_a - t) - x_b and r = 1 / (s2k_a + s2k_b).
//
// The two particle scores of the microscopy application run through the same
// kernel (SCORE 1, 2) on re-scaled copies of the storage (positive s2k):
//   SCORE 1, GMM L2 cross term (s2k = 2 ln2 s^2, lw = log2 w):
//     term = w_a w_b (2 pi s2)^(-d/2) exp(-d^2 / (2 s2)) = C q^d 2^(lw_a + lw_b - d^2 q^2)
//   SCORE 2, Bhattacharyya (s2k = 4 ln2 s^2, lw = log2 w / 2 + (d/2) log2 sigma):
//     term = sqrt(w_a w_b) (2 s_a s_b / s2)^(d/2) exp(-d^2 / (4 s2)) = C q^d 2^(...)
// with q = rsqrt(s2k_a + s2k_b) (one MUFU, as the reciprocal of the overlap)
// and C = (ln2 / pi)^(d/2) or (8 ln2)^(d/2); the L2 distance adds the per-item
// self terms S_i + S_j - 2 C sum in the epilogue.
//
// Schedule: one persistent CTA per SM slot pops tiles (I block, J block) of
// the upper triangle of item blocks from an atomic queue (Sec. IV-B).  The J
// block's points are staged into shared memory with one bulk asynchronous
// copy; the CTA's warps take "row jobs" (a chunk of 32*R points of one item
// of I, held in registers, R per lane) and sweep every item of J with
// broadcast shared-memory reads; per (row job, j) partials are reduced over
// the warp with shuffles, then over the chunks of an item in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "ap_internal.h"

namespace ap {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxRowJobs = kOverlapMaxRowJobs;
constexpr int kMaxBlockItems = kOverlapMaxBlockItems;
constexpr float kTwoLn2 = 1.3862943611198906f;

enum Mode { FWD = 0, FWD_T = 1, GRAD = 2, COVER = 3 };

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsq_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct TileCtx {
  int32_t i_begin, i_end, j_begin, j_end;
  int32_t n_rj;          // row jobs in this tile (partial-sum slots)
  int32_t n_jobs;        // jobs the units sweep: one row job, or two short ones
  int32_t use_smem;      // J block staged in shared memory
  int64_t j_pt0;         // first storage point of the J block
};

struct Params {
  const float4 *pts;
  const float *lw;
  const int64_t *poff;
  const int32_t *cnt;    // real (unpadded) points per stored item
  const int32_t *perm;
  const int32_t *bstart;
  const int32_t *tiles;
  int64_t n_tiles;
  int64_t n_items;
  int32_t *queue;
  int32_t *status;
  int32_t stage_cap;     // points that fit the shared staging buffer
  int32_t max_rj;        // row jobs of the largest block: rows of the partials
  int32_t part_items;    // items of a block: columns of the partials
  int32_t list_mode;     // tiles are listed pairs: tile t's params and outputs
                         // sit at index t (not at the packed pair index)
  // outputs / extra inputs
  float *out;            // FWD: f[P]; COVER: int32 counts[P]
  const float *params;   // [P][3] (theta, tx, ty) or NULL
  const float *grad_out; // [P] or NULL
  float *grad_params;    // [P][3]
  float *f_out;          // [P] or NULL
  float *params_io;      // ascent: params updated in place
  int32_t *flags;        // ascent: skipped steps
  float eta, fmin;
  const double *self;    // SCORE 1: S per original item
  double score_c;        // SCORE 1, 2: the constant C
};

template <int DIM, bool HAS_W, int MODE, int R, int SCORE>
__global__ void __launch_bounds__(kThreads)
overlap_kernel(Params P) {
  constexpr int NV = (MODE == GRAD) ? 4 : 1;     // partial values per (row job, j)
  constexpr int CH = 32 * R;                     // points per chunk
  // 2-D sets (small items) pair their items' short last chunks; the 3-D
  // kernel, at R = 4 with items sorted by size, ran 1% slower doing so
  constexpr bool kMixJobs = DIM == 2;
  extern __shared__ __align__(16) uint8_t smem[];
  float4 *s_pts = reinterpret_cast<float4 *>(smem);
  float *s_lw = reinterpret_cast<float *>(s_pts + P.stage_cap);
  // 3-D: the weight area also holds the log-weights of the paired layout
  float *s_part = (DIM == 3) ? s_lw + P.stage_cap : s_lw;
  int16_t *s_rj_item = reinterpret_cast<int16_t *>(s_part + P.max_rj * P.part_items * NV);
  int16_t *s_rj_chunk = s_rj_item + kMaxRowJobs;
  int16_t *s_rj_first = s_rj_chunk + kMaxRowJobs;            // [kMaxBlockItems + 1]
  int16_t *s_job_a = s_rj_first + kMaxBlockItems + 1;         // [kMaxRowJobs] row job
  int16_t *s_job_b = s_job_a + kMaxRowJobs;                   // [kMaxRowJobs] second, or -1
  int16_t *s_rem_rj = s_job_b + kMaxRowJobs;                  // [kMaxBlockItems] short last
  int16_t *s_rem_n = s_rem_rj + kMaxBlockItems;               // chunks and their points
  uint64_t *s_bar = reinterpret_cast<uint64_t *>(
      (reinterpret_cast<uintptr_t>(s_rem_n + kMaxBlockItems) + 7) & ~uintptr_t(7));
  TileCtx *s_ctx = reinterpret_cast<TileCtx *>(s_bar + 1);
  int *s_tile = reinterpret_cast<int *>(s_ctx + 1);
  int *s_next = s_tile + 1;                      // next (row job, partner) unit

  const int lane = threadIdx.x & 31;
  const uint32_t bar = smem_u32(s_bar);
  uint32_t phase = 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) {
      int t = atomicAdd(P.queue, 1);
      if (*reinterpret_cast<volatile int32_t *>(P.status) != 0) t = (int)P.n_tiles;
      *s_tile = t;
      if (t < P.n_tiles) {
        const int IB = P.tiles[2 * t], JB = P.tiles[2 * t + 1];
        TileCtx c;
        c.i_begin = P.bstart[IB]; c.i_end = P.bstart[IB + 1];
        c.j_begin = P.bstart[JB]; c.j_end = P.bstart[JB + 1];
        // row jobs (chunks of CH points) in item order, each with its own
        // partial-sum slot; off the diagonal, items' last chunks short of
        // CH points are paired into shared jobs (the second item's points
        // on the lanes after the first one's), longest with shortest
        const bool mix = kMixJobs && (MODE != COVER) && IB != JB;
        int nrj = 0, njob = 0, nrem = 0;
        for (int i = c.i_begin; i < c.i_end; ++i) {
          s_rj_first[i - c.i_begin] = (int16_t)nrj;
          const int64_t np = P.cnt[i];
          const int nch = (int)((np + CH - 1) / CH);
          for (int ch = 0; ch < nch && nrj < P.max_rj; ++ch) {
            s_rj_item[nrj] = (int16_t)(i - c.i_begin);
            s_rj_chunk[nrj] = (int16_t)ch;
            const int64_t left = np - (int64_t)ch * CH;
            if (mix && left < CH) {
              // insertion by point count, most first
              int k = nrem++;
              for (; k > 0 && s_rem_n[k - 1] < left; --k) {
                s_rem_rj[k] = s_rem_rj[k - 1];
                s_rem_n[k] = s_rem_n[k - 1];
              }
              s_rem_rj[k] = (int16_t)nrj;
              s_rem_n[k] = (int16_t)left;
            } else {
              s_job_a[njob] = (int16_t)nrj;
              s_job_b[njob++] = -1;
            }
            ++nrj;
          }
        }
        for (int lo = 0, hi = nrem - 1; lo <= hi;) {
          s_job_a[njob] = s_rem_rj[lo];
          if (lo < hi && s_rem_n[lo] + s_rem_n[hi] <= CH) s_job_b[njob++] = s_rem_rj[hi--];
          else s_job_b[njob++] = -1;
          ++lo;
        }
        s_rj_first[c.i_end - c.i_begin] = (int16_t)nrj;
        c.n_rj = nrj;
        c.n_jobs = njob;
        *s_next = 0;
        c.j_pt0 = P.poff[c.j_begin];
        const int64_t jpts = P.poff[c.j_end] - c.j_pt0;
        c.use_smem = (MODE != COVER) && jpts > 0 && jpts <= P.stage_cap;
        if (c.use_smem) {
          // stage the J block: one bulk asynchronous copy per array
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          uint32_t bytes = (uint32_t)(jpts * 16);
          if (DIM == 3 && HAS_W) bytes += (uint32_t)(jpts * 4);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                       "r"(bytes)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                  "r"(smem_u32(s_pts)),
              "l"(P.pts + c.j_pt0), "r"((uint32_t)(jpts * 16)), "r"(bar)
              : "memory");
          if (DIM == 3 && HAS_W)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                    "r"(smem_u32(s_lw)),
                "l"(P.lw + c.j_pt0), "r"((uint32_t)(jpts * 4)), "r"(bar)
                : "memory");
        }
        *s_ctx = c;
      }
    }
    __syncthreads();
    const int t = *s_tile;
    if (t >= P.n_tiles) break;
    const TileCtx c = *s_ctx;
    const int nJ = c.j_end - c.j_begin;
    const bool diag = (P.tiles[2 * t] == P.tiles[2 * t + 1]);

    if (c.use_smem) {
      bool ok = true;
      uint32_t done = 0;
      const uint64_t t0 = global_ns();
      for (uint32_t it = 0;; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) break;
        if ((it & 255u) == 255u && global_ns() - t0 > kWaitBudgetNs) { ok = false; break; }
      }
      phase ^= 1;
      if (!ok && threadIdx.x == 0) atomicCAS(P.status, 0, DEV_TIMEOUT_STAGE);
      if (MODE != COVER) {
        // The staged block in pairs of points: pair q (points 2q, 2q + 1 of
        // an item) becomes {x0, x1, y0, y1} {s0, s1, l0, l1} (2-D) or
        // {x0, x1, y0, y1} {z0, z1, s0, s1} with {l0, l1} in the weight area
        // (3-D), in place, so one packed operation takes two b-points; a
        // point past its item's real count gets log-weight -inf (weight 0),
        // so pairs may run over an odd item's padding.
        float4 *sp4 = reinterpret_cast<float4 *>(s_pts);
        float2 *sl2 = reinterpret_cast<float2 *>(s_lw);
        const int nwarp = blockDim.x >> 5;
        for (int jl = threadIdx.x >> 5; jl < nJ; jl += nwarp) {
          const int j = c.j_begin + jl;
          const int b0 = (int)(P.poff[j] - c.j_pt0), np = (int)(P.poff[j + 1] - P.poff[j]);
          const int cnt = P.cnt[j];
          for (int k = lane; 2 * k < np; k += 32) {
            const int q = (b0 >> 1) + k;
            const float4 u = sp4[2 * q], v = sp4[2 * q + 1];
            const bool r0 = 2 * k < cnt, r1 = 2 * k + 1 < cnt;
            sp4[2 * q] = make_float4(u.x, v.x, u.y, v.y);
            if (DIM == 3) {
              sp4[2 * q + 1] = make_float4(u.z, v.z, u.w, v.w);
              const float2 l = HAS_W ? sl2[q] : make_float2(0.f, 0.f);
              sl2[q] = make_float2(r0 ? l.x : -INFINITY, r1 ? l.y : -INFINITY);
            } else {
              sp4[2 * q + 1] = make_float4(u.z, v.z, r0 ? u.w : -INFINITY, r1 ? v.w : -INFINITY);
            }
          }
        }
        __syncthreads();
      }
    }

    if (MODE != COVER) {
      const float4 *bsrc = c.use_smem ? s_pts : (P.pts + c.j_pt0);
      const float *lsrc = c.use_smem ? s_lw : (P.lw ? P.lw + c.j_pt0 : nullptr);
      // warps take (row job, partner item) units from a shared counter, so
      // every warp of the CTA runs until the tile's work is gone
      for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(s_next, 1);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= c.n_jobs * nJ) break;
        const int k = u / nJ, jl = u - k * nJ;
        const int rj = s_job_a[k], rj2 = kMixJobs ? s_job_b[k] : -1;
        const int il = s_rj_item[rj];
        if (diag && jl <= il) continue;
        const int i = c.i_begin + il;
        const int64_t a_begin = P.poff[i] + (int64_t)s_rj_chunk[rj] * CH;
        const int64_t a_end = P.poff[i] + P.cnt[i];
        // a job of two short chunks: slots [0, nA) hold item i's points,
        // [nA, nA + n2) those of item i2 (bit r of seg2: a-point r is i2's)
        const int nA = (int)(a_end - a_begin < CH ? a_end - a_begin : CH);
        int i2 = i, n2 = 0;
        int64_t a2_begin = 0;
        if (rj2 >= 0) {
          i2 = c.i_begin + s_rj_item[rj2];
          a2_begin = P.poff[i2] + (int64_t)s_rj_chunk[rj2] * CH;
          n2 = (int)(P.poff[i2] + P.cnt[i2] - a2_begin);
        }
        uint32_t seg2 = 0;
        // this lane's a-points, two per float2 (packed FP32x2 arithmetic);
        // coordinates kept negated so d = b - a is one add, s2k is stored
        // negated; padding and out-of-chunk points get weight 0
        constexpr int R2 = R / 2;
        float2 nax[R2], nay[R2], naz[R2], nas[R2], aw2[R2];
#pragma unroll
        for (int p = 0; p < R2; ++p) {
          float v[2][5];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int slot = (2 * p + h) * 32 + lane;
            int64_t a = a_begin + slot;
            bool in = slot < nA;
            if (!in && slot - nA < n2) {
              a = a2_begin + (slot - nA);
              in = true;
              seg2 |= 1u << (2 * p + h);
            }
            if (in) {
              const float4 q = __ldg(P.pts + a);
              v[h][0] = q.x; v[h][1] = q.y;
              if (DIM == 3) { v[h][2] = q.z; v[h][3] = q.w; v[h][4] = HAS_W ? exp2f(__ldg(P.lw + a)) : 1.f; }
              else { v[h][2] = 0.f; v[h][3] = q.z; v[h][4] = exp2f(q.w); }
            } else {
              // outside the item: weight 0, an s2k of the storage's sign
              v[h][0] = 0.f; v[h][1] = 0.f; v[h][2] = 0.f; v[h][3] = SCORE ? 1.f : -1.f;
              v[h][4] = 0.f;
            }
          }
          nax[p] = make_float2(-v[0][0], -v[1][0]);
          nay[p] = make_float2(-v[0][1], -v[1][1]);
          naz[p] = make_float2(-v[0][2], -v[1][2]);
          nas[p] = make_float2(v[0][3], v[1][3]);
          aw2[p] = make_float2(v[0][4], v[1][4]);
        }
        {
          const int j = c.j_begin + jl;
          const int b0 = (int)(P.poff[j] - c.j_pt0), b1 = b0 + P.cnt[j];
          // -a' = R^T (-(x_a - t)) for this pair's transform
          float2 ntx[R2], nty[R2];
          // each pair's transform: (i, j), and (i2, j) for i2's a-points
          float cth[2] = {1.f, 1.f}, sth[2] = {0.f, 0.f}, ttx[2] = {0.f, 0.f}, tty[2] = {0.f, 0.f};
          if (MODE == FWD_T || MODE == GRAD) {
            const float *pp = (MODE == GRAD && P.params_io) ? P.params_io : P.params;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              if (g == 1 && rj2 < 0) break;
              const int oi = P.perm[g ? i2 : i], oj = P.perm[j];
              const int64_t pidx = P.list_mode ? (int64_t)t
                                               : pair_index(oi < oj ? oi : oj, oi < oj ? oj : oi,
                                                            P.n_items);
              if (pp) {
                const float th = pp[3 * pidx];
                ttx[g] = pp[3 * pidx + 1]; tty[g] = pp[3 * pidx + 2];
                sincosf(th, &sth[g], &cth[g]);
              }
            }
          }
#pragma unroll
          for (int p = 0; p < R2; ++p) {
            if (MODE == FWD_T || MODE == GRAD) {
              const bool gx = (seg2 >> (2 * p)) & 1u, gy = (seg2 >> (2 * p + 1)) & 1u;
              const float2 c2 = make_float2(gx ? cth[1] : cth[0], gy ? cth[1] : cth[0]);
              const float2 s2 = make_float2(gx ? sth[1] : sth[0], gy ? sth[1] : sth[0]);
              const float2 ux = __fadd2_rn(nax[p], make_float2(gx ? ttx[1] : ttx[0], gy ? ttx[1] : ttx[0]));
              const float2 uy = __fadd2_rn(nay[p], make_float2(gx ? tty[1] : tty[0], gy ? tty[1] : tty[0]));
              ntx[p] = __ffma2_rn(c2, ux, __fmul2_rn(s2, uy));
              nty[p] = __ffma2_rn(c2, uy, __fmul2_rn(make_float2(-s2.x, -s2.y), ux));
            } else {
              ntx[p] = nax[p]; nty[p] = nay[p];
            }
          }
          const float2 z2 = make_float2(0.f, 0.f);
          float2 accF[R2], cmpF[R2], accX[R2], accY[R2], accT[R2];
#pragma unroll
          for (int p = 0; p < R2; ++p) { accF[p] = z2; cmpF[p] = z2; accX[p] = z2; accY[p] = z2; accT[p] = z2; }
          if (!c.use_smem) {
            // J block read from global memory, one b-point at a time
            for (int bb0 = b0; bb0 < b1; bb0 += 32) {
              const int bb1 = min(bb0 + 32, b1);
              float2 blF[R2], blX[R2], blY[R2], blT[R2];
#pragma unroll
              for (int p = 0; p < R2; ++p) { blF[p] = z2; blX[p] = z2; blY[p] = z2; blT[p] = z2; }
#pragma unroll 4
              for (int b = bb0; b < bb1; ++b) {
                const float4 q = bsrc[b];
                float lwb, s2b;
                if (DIM == 3) { s2b = q.w; lwb = HAS_W ? lsrc[b] : 0.f; }
                else { s2b = q.z; lwb = q.w; }
                const float2 bx2 = make_float2(q.x, q.x), by2 = make_float2(q.y, q.y);
                const float2 bs2 = make_float2(s2b, s2b), lw2 = make_float2(lwb, lwb);
#pragma unroll
                for (int p = 0; p < R2; ++p) {
                  const float2 dx = __fadd2_rn(bx2, ntx[p]);          // b - a'
                  const float2 dy = __fadd2_rn(by2, nty[p]);
                  float2 d2 = __fmul2_rn(dx, dx);
                  d2 = __ffma2_rn(dy, dy, d2);
                  if (DIM == 3) {
                    const float2 dz = __fadd2_rn(make_float2(q.z, q.z), naz[p]);
                    d2 = __ffma2_rn(dz, dz, d2);
                  }
                  const float2 ns = __fadd2_rn(nas[p], bs2);   // -(s2k_a + s2k_b); SCORE: +
                  float2 nr, qd = z2;
                  if (SCORE) {
                    const float2 q = make_float2(rsq_approx(ns.x), rsq_approx(ns.y));
                    nr = __fmul2_rn(q, make_float2(-q.x, -q.y));        // -1 / s2k
                    qd = DIM == 2 ? make_float2(-nr.x, -nr.y)
                                  : __fmul2_rn(q, make_float2(-nr.x, -nr.y));   // q^d
                  } else {
                    nr = make_float2(rcp_approx(ns.x), rcp_approx(ns.y));
                  }
                  const float2 arg = __ffma2_rn(d2, nr, lw2);          // lw_b - d^2 / s2k
                  const float2 e = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
                  blF[p] = SCORE ? __ffma2_rn(e, qd, blF[p]) : __fadd2_rn(blF[p], e);
                  if (MODE == GRAD) {
                    // per a-point sums of -e r, -e r x_b and -e r y_b (e nr = -e r);
                    // the a'-dependent factors are applied once per a-point
                    const float2 ner = __fmul2_rn(e, nr);
                    blX[p] = __fadd2_rn(blX[p], ner);
                    blY[p] = __ffma2_rn(ner, bx2, blY[p]);
                    blT[p] = __ffma2_rn(ner, by2, blT[p]);
                  }
                }
              }
#pragma unroll
              for (int p = 0; p < R2; ++p) {
                // compensated add of the block sum
                const float2 yk = __fadd2_rn(blF[p], make_float2(-cmpF[p].x, -cmpF[p].y));
                const float2 tk = __fadd2_rn(accF[p], yk);
                const float2 dd = __fadd2_rn(tk, make_float2(-accF[p].x, -accF[p].y));
                cmpF[p] = __fadd2_rn(dd, make_float2(-yk.x, -yk.y));
                accF[p] = tk;
                if (MODE == GRAD) {
                  accX[p] = __fadd2_rn(accX[p], blX[p]);
                  accY[p] = __fadd2_rn(accY[p], blY[p]);
                  accT[p] = __fadd2_rn(accT[p], blT[p]);
                }
              }
            }
          } else {
            // J block staged in pairs: each packed operation takes two
            // b-points against one a-point held in both halves, so no
            // b-point is broadcast inside the loop
            const float4 *sp4 = reinterpret_cast<const float4 *>(s_pts);
            const float2 *sl2 = reinterpret_cast<const float2 *>(s_lw);
            float2 pF[R], pC[R], pY[R], pT[R];
#pragma unroll
            for (int r = 0; r < R; ++r) { pF[r] = z2; pC[r] = z2; pY[r] = z2; pT[r] = z2; }
            const int q0 = b0 >> 1, q1 = (b1 + 1) >> 1;
            // RE of the lane's R a-points: a chunk whose real points fit
            // the first half (an item's last chunk) sweeps only that half
            // (the scores' items are large: their last chunks are a small
            // share, and the second copy of the loop costs them registers)
            auto sweep = [&](auto re) {
              constexpr int RE = decltype(re)::value;
              for (int qb = q0; qb < q1; qb += 16) {
                const int qe = min(qb + 16, q1);
                float2 bF[RE];                  // this block's f terms (compensated below)
#pragma unroll
                for (int r = 0; r < RE; ++r) bF[r] = z2;
#pragma unroll 2
                for (int q = qb; q < qe; ++q) {
                  const float4 u = sp4[2 * q], v = sp4[2 * q + 1];
                  const float2 X = make_float2(u.x, u.y), Y = make_float2(u.z, u.w);
                  float2 Z = z2, S, L;
                  if (DIM == 3) { Z = make_float2(v.x, v.y); S = make_float2(v.z, v.w); L = sl2[q]; }
                  else { S = make_float2(v.x, v.y); L = make_float2(v.z, v.w); }
#pragma unroll
                  for (int r = 0; r < RE; ++r) {
                    const int p = r >> 1;
                    const float ax = (r & 1) ? ntx[p].y : ntx[p].x;
                    const float ay = (r & 1) ? nty[p].y : nty[p].x;
                    const float az = (r & 1) ? naz[p].y : naz[p].x;
                    const float as = (r & 1) ? nas[p].y : nas[p].x;
                    const float2 dx = __fadd2_rn(X, make_float2(ax, ax));          // b - a'
                    const float2 dy = __fadd2_rn(Y, make_float2(ay, ay));
                    float2 d2 = __fmul2_rn(dx, dx);
                    d2 = __ffma2_rn(dy, dy, d2);
                    if (DIM == 3) {
                      const float2 dz = __fadd2_rn(Z, make_float2(az, az));
                      d2 = __ffma2_rn(dz, dz, d2);
                    }
                    const float2 ns = __fadd2_rn(make_float2(as, as), S);   // -(s2k_a + s2k_b); SCORE: +
                    float2 nr, qd = z2;
                    if (SCORE) {
                      const float2 qq = make_float2(rsq_approx(ns.x), rsq_approx(ns.y));
                      nr = __fmul2_rn(qq, make_float2(-qq.x, -qq.y));       // -1 / s2k
                      qd = DIM == 2 ? make_float2(-nr.x, -nr.y)
                                    : __fmul2_rn(qq, make_float2(-nr.x, -nr.y));   // q^d
                    } else {
                      nr = make_float2(rcp_approx(ns.x), rcp_approx(ns.y));
                    }
                    const float2 arg = __ffma2_rn(d2, nr, L);              // lw_b - d^2 / s2k
                    const float2 e = make_float2(ex2_approx(arg.x), ex2_approx(arg.y));
                    bF[r] = SCORE ? __ffma2_rn(e, qd, bF[r]) : __fadd2_rn(bF[r], e);
                    if (MODE == GRAD) {
                      // the gradient needs only u = sum -e r d' (d' = b - a'):
                      // df/dt ~ u and df/dtheta ~ nty u_x - ntx u_y, the
                      // b x b terms of sum e r (x_b d'_y - y_b d'_x) cancelling
                      const float2 ner = __fmul2_rn(e, nr);
                      pY[r] = __ffma2_rn(ner, dx, pY[r]);
                      pT[r] = __ffma2_rn(ner, dy, pT[r]);
                    }
                  }
                }
#pragma unroll
                for (int r = 0; r < RE; ++r) {
                  // compensated add of the block sum (each half on its own)
                  const float2 yk = __fadd2_rn(bF[r], make_float2(-pC[r].x, -pC[r].y));
                  const float2 tk = __fadd2_rn(pF[r], yk);
                  const float2 dd = __fadd2_rn(tk, make_float2(-pF[r].x, -pF[r].y));
                  pC[r] = __fadd2_rn(dd, make_float2(-yk.x, -yk.y));
                  pF[r] = tk;
                }
              }
            };
            if constexpr (SCORE == 0) {
              if (nA + n2 <= 16 * R) sweep(std::integral_constant<int, R / 2>());
              else sweep(std::integral_constant<int, R>());
            } else {
              sweep(std::integral_constant<int, R>());
            }
            // each a-point's two halves, back in the form of two a-points per
            // packed value; the gradient's terms as the epilogue below takes
            // them (S x a' + Sx = u, so S = 0 with Sx, Sy = u)
#pragma unroll
            for (int p = 0; p < R2; ++p) {
              accF[p] = make_float2(pF[2 * p].x + pF[2 * p].y, pF[2 * p + 1].x + pF[2 * p + 1].y);
              if (MODE == GRAD) {
                accX[p] = z2;
                accY[p] = make_float2(pY[2 * p].x + pY[2 * p].y, pY[2 * p + 1].x + pY[2 * p + 1].y);
                accT[p] = make_float2(pT[2 * p].x + pT[2 * p].y, pT[2 * p + 1].x + pT[2 * p + 1].y);
              }
            }
          }
          // per a-point terms summed over the warp, into the partial-sum slot
          // of the a-point's item (two slots for a job of two short chunks)
          float v[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
          for (int p = 0; p < R2; ++p) {
            float tF[2] = {aw2[p].x * accF[p].x, aw2[p].y * accF[p].y};
            float tX[2] = {0.f, 0.f}, tY[2] = {0.f, 0.f}, tT[2] = {0.f, 0.f};
            if (MODE == GRAD) {
              // with S = sum -e r, Sx = sum -e r x_b, Sy = sum -e r y_b and
              // -a' = (ntx, nty):  sum e r d'   = (Sx + ntx S, Sy + nty S),
              // sum e r (x_b d'_y - y_b d'_x) = nty Sx - ntx Sy   (the b x b
              // terms cancel)
              const float2 gx = __ffma2_rn(ntx[p], accX[p], accY[p]);
              const float2 gy = __ffma2_rn(nty[p], accX[p], accT[p]);
              const float2 gt = __ffma2_rn(nty[p], accY[p],
                                           __fmul2_rn(make_float2(-ntx[p].x, -ntx[p].y), accT[p]));
              tX[0] = aw2[p].x * gx.x; tX[1] = aw2[p].y * gx.y;
              tY[0] = aw2[p].x * gy.x; tY[1] = aw2[p].y * gy.y;
              tT[0] = aw2[p].x * gt.x; tT[1] = aw2[p].y * gt.y;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const bool second = (seg2 >> (2 * p + h)) & 1u;
              v[0][0] += second ? 0.f : tF[h];
              v[1][0] += second ? tF[h] : 0.f;
              if (MODE == GRAD) {
                v[0][1] += second ? 0.f : tX[h];
                v[1][1] += second ? tX[h] : 0.f;
                v[0][2] += second ? 0.f : tY[h];
                v[1][2] += second ? tY[h] : 0.f;
                v[0][3] += second ? 0.f : tT[h];
                v[1][3] += second ? tT[h] : 0.f;
              }
            }
          }
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            if (g == 1 && rj2 < 0) break;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
              for (int q = 0; q < NV; ++q) v[g][q] += __shfl_xor_sync(0xffffffffu, v[g][q], o);
            }
            if (lane == 0) {
              float *dst = s_part + ((size_t)(g ? rj2 : rj) * P.part_items + jl) * NV;
#pragma unroll
              for (int q = 0; q < NV; ++q) dst[q] = v[g][q];
            }
          }
        }
      }
    }
    __syncthreads();

    // fixed-order reduction over the chunks of each item, then the stores
    const int nI = c.i_end - c.i_begin;
    for (int q = threadIdx.x; q < nI * nJ; q += blockDim.x) {
      const int il = q / nJ, jl = q - il * nJ;
      if (diag && jl <= il) continue;
      const int i = c.i_begin + il, j = c.j_begin + jl;
      const int oi = P.perm[i], oj = P.perm[j];
      const int64_t p =
          P.list_mode ? (int64_t)t : pair_index(oi < oj ? oi : oj, oi < oj ? oj : oi, P.n_items);
      if (MODE == COVER) {
        atomicAdd(reinterpret_cast<int32_t *>(P.out) + p, 1);
        continue;
      }
      double sF = 0.0, sX = 0.0, sY = 0.0, sT = 0.0;
      for (int rj = s_rj_first[il]; rj < s_rj_first[il + 1]; ++rj) {
        const float *src = s_part + ((size_t)rj * P.part_items + jl) * NV;
        sF += (double)src[0];
        if (MODE == GRAD) { sX += (double)src[1]; sY += (double)src[2]; sT += (double)src[3]; }
      }
      if (MODE == FWD || MODE == FWD_T) {
        if (SCORE == 1) P.out[p] = (float)(P.self[oi] + P.self[oj] - 2.0 * P.score_c * sF);
        else if (SCORE == 2) P.out[p] = (float)(P.score_c * sF);
        else P.out[p] = (float)sF;
      } else if (MODE == GRAD) {
        // rotate the translation part back: df/dt = 2 ln2 R sum e r d'
        const float *pp = P.params_io ? P.params_io : P.params;
        float th = 0.f, ttx = 0.f, tty = 0.f;
        if (pp) { th = pp[3 * p]; ttx = pp[3 * p + 1]; tty = pp[3 * p + 2]; }
        float sth, cth;
        sincosf(th, &sth, &cth);
        const float f = (float)sF;
        const float gx = kTwoLn2 * (float)(cth * sX - sth * sY);
        const float gy = kTwoLn2 * (float)(sth * sX + cth * sY);
        const float gt = kTwoLn2 * (float)sT;
        if (P.f_out) P.f_out[p] = f;
        if (P.params_io) {
          // one ascent step on log f
          if (f >= P.fmin) {
            const float s = P.eta / f;
            P.params_io[3 * p] = th + s * gt;
            P.params_io[3 * p + 1] = ttx + s * gx;
            P.params_io[3 * p + 2] = tty + s * gy;
          } else if (P.flags) {
            P.flags[p] = 1;
          }
        } else {
          const float go = P.grad_out ? P.grad_out[p] : 1.f;
          P.grad_params[3 * p] = go * gt;
          P.grad_params[3 * p + 1] = go * gx;
          P.grad_params[3 * p + 2] = go * gy;
        }
      }
    }
    __syncthreads();
  }
}

// Pack one item per CTA into planner order, padded to a multiple of 4 points.
__global__ void cloud_pack_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                  const float *__restrict__ z, const float *__restrict__ sigma,
                                  const float *__restrict__ w, const int64_t *__restrict__ src_off,
                                  const int32_t *__restrict__ perm,
                                  const int64_t *__restrict__ poff, int64_t n, int dim,
                                  float4 *__restrict__ pts, float *__restrict__ lw) {
  const double two_ln2 = 1.3862943611198906;
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    const int64_t o = perm[s];
    const int64_t src0 = src_off[o], cnt = src_off[o + 1] - src_off[o];
    const int64_t dst0 = poff[s], pcnt = poff[s + 1] - poff[s];
    for (int64_t k = threadIdx.x; k < pcnt; k += blockDim.x) {
      float4 p;
      float l;
      if (k < cnt) {
        const int64_t a = src0 + k;
        const double sg = (double)sigma[a];
        const float s2k = (float)(-two_ln2 * sg * sg);   // stored negated
        const float wt = w ? w[a] : 1.f;
        l = (wt > 0.f) ? (float)log2((double)wt) : -INFINITY;
        if (dim == 3) p = make_float4(x[a], y[a], z[a], s2k);
        else p = make_float4(x[a], y[a], s2k, l);
      } else {
        // padding (never visited: loops use the real counts), kept finite
        l = -INFINITY;
        if (dim == 3) p = make_float4(0.f, 0.f, 0.f, -1.f);
        else p = make_float4(0.f, 0.f, -1.f, -INFINITY);
      }
      pts[dst0 + k] = p;
      if (lw) lw[dst0 + k] = l;
    }
  }
}

// Re-scaled storage of a particle score from the overlap's storage
// (s2k = -2 ln2 sigma^2, lw = log2 w): SCORE 1 s2k = +2 ln2 sigma^2 with lw
// unchanged, SCORE 2 s2k = +4 ln2 sigma^2 and lw = lw / 2 + (d/4) log2 sigma^2.
// Padding keeps a positive s2k and lw = -inf.
__global__ void cloud_rescore_kernel(const float4 *__restrict__ pts, const float *__restrict__ lw,
                                     int64_t n_pts, int dim, int score,
                                     float4 *__restrict__ out_pts, float *__restrict__ out_lw) {
  const float ln2x2 = 1.3862943611198906f;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_pts;
       k += (int64_t)gridDim.x * blockDim.x) {
    float4 q = pts[k];
    const float s2k = dim == 3 ? q.w : q.z;          // -2 ln2 sigma^2 (padding: -1)
    float l = dim == 3 ? (lw ? lw[k] : 0.f) : q.w;
    const float t = score == 1 ? -s2k : -2.f * s2k;
    if (score == 2) l = 0.5f * l + 0.25f * (float)dim * __log2f(-s2k / ln2x2);
    if (dim == 3) { q.w = t; if (out_lw) out_lw[k] = l; }
    else { q.z = t; q.w = l; }
    out_pts[k] = q;
  }
}

// S_i = C sum over a, a' in item i of w_a w_a' q^d 2^(-d^2 q^2) (SCORE 1
// storage), one CTA per item, FP32 blocks of 64 terms folded into FP64.
template <int DIM, bool HAS_W>
__global__ void __launch_bounds__(256)
cloud_self_kernel(const float4 *__restrict__ pts, const float *__restrict__ lw,
                  const int64_t *__restrict__ poff, const int32_t *__restrict__ cnt,
                  const int32_t *__restrict__ perm, int64_t n, double c, double *__restrict__ S) {
  __shared__ double red[8];
  for (int64_t it = blockIdx.x; it < n; it += gridDim.x) {
    const int64_t p0 = poff[it];
    const int m = cnt[it];
    double acc = 0.0;
    for (int a = threadIdx.x; a < m; a += blockDim.x) {
      const float4 qa = pts[p0 + a];
      const float sa = DIM == 3 ? qa.w : qa.z;
      const float la = DIM == 3 ? (HAS_W ? lw[p0 + a] : 0.f) : qa.w;
      float part = 0.f;
      for (int b = 0; b < m; ++b) {
        const float4 qb = pts[p0 + b];
        const float dx = qb.x - qa.x, dy = qb.y - qa.y;
        float d2 = fmaf(dx, dx, dy * dy);
        float sb, lb;
        if (DIM == 3) {
          const float dz = qb.z - qa.z;
          d2 = fmaf(dz, dz, d2);
          sb = qb.w;
          lb = HAS_W ? lw[p0 + b] : 0.f;
        } else {
          sb = qb.z;
          lb = qb.w;
        }
        const float q = rsq_approx(sa + sb), r = q * q;
        const float e = ex2_approx(fmaf(-d2, r, la + lb));
        part = fmaf(e, DIM == 2 ? r : r * q, part);
        if ((b & 63) == 63) { acc += (double)part; part = 0.f; }
      }
      acc += (double)part;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
      S[perm[it]] = c * tot;
    }
    __syncthreads();
  }
}

template <int DIM, bool HAS_W, int MODE, int SCORE = 0>
cudaError_t launch_r(const CloudStore &cs, Params &P, int reg_r, cudaStream_t s) {
  constexpr int NV = (MODE == GRAD) ? 4 : 1;
  size_t smem = (size_t)P.stage_cap * 16 + (DIM == 3 ? (size_t)P.stage_cap * 4 : 0) +
                (size_t)P.max_rj * P.part_items * NV * 4 +
                (size_t)(4 * kMaxRowJobs + 3 * kMaxBlockItems + 1) * 2 + 16 + sizeof(TileCtx) + 64;
  void (*kern)(Params) = nullptr;
  switch (reg_r) {
    case 2: kern = overlap_kernel<DIM, HAS_W, MODE, 2, SCORE>; break;
    default: kern = overlap_kernel<DIM, HAS_W, MODE, 4, SCORE>; break;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // listed pairs are tiles of one item against one, a few row jobs each: one
  // warp per CTA and many CTAs per SM keep the warps busy (20 ascent steps on
  // 131K listed pairs: 114 ms at 8 warps per CTA, 89 at 4, 81 at 2, 79 at 1)
  const int threads = cs.list_mode ? kThreads / 8 : kThreads;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms() * per_sm;
  if (grid > P.n_tiles) grid = P.n_tiles;
  e = cudaMemsetAsync(P.queue, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  kern<<<(int)grid, threads, smem, s>>>(P);
  return cudaGetLastError();
}

Params base_params(const CloudStore &cs, int32_t *queue, int32_t *status) {
  Params P{};
  P.pts = cs.d_pts;
  P.lw = cs.d_lw;
  P.poff = cs.d_poff;
  P.cnt = cs.d_cnt;
  P.perm = cs.d_perm;
  P.bstart = cs.d_bstart;
  P.tiles = cs.d_tiles;
  P.n_tiles = cs.n_tiles;
  P.n_items = cs.n;
  P.queue = queue;
  P.status = status;
  P.stage_cap = cs.block_pts;
  P.max_rj = cs.max_rj > 0 ? cs.max_rj : kMaxRowJobs;
  P.part_items = cs.block_items > 0 ? cs.block_items : kMaxBlockItems;
  P.list_mode = cs.list_mode ? 1 : 0;
  return P;
}

}  // namespace

// status word lives right after the queue counter (see api.cu)
static inline int32_t *status_of(int32_t *queue) { return queue + 1; }

cudaError_t launch_overlap(const CloudStore &cs, const float *params, float *out, int coverage,
                           int32_t *queue, cudaStream_t s) {
  if (cs.n_tiles <= 0) return cudaSuccess;
  Params P = base_params(cs, queue, status_of(queue));
  P.out = out;
  P.params = params;
  const bool w3 = (cs.dim == 3) && !cs.unit_weights;
  if (coverage) {
    if (cs.dim == 3) return w3 ? launch_r<3, true, COVER>(cs, P, cs.reg_r, s) : launch_r<3, false, COVER>(cs, P, cs.reg_r, s);
    return launch_r<2, true, COVER>(cs, P, cs.reg_r, s);
  }
  if (params) return launch_r<2, true, FWD_T>(cs, P, cs.reg_r, s);
  if (cs.dim == 3) return w3 ? launch_r<3, true, FWD>(cs, P, cs.reg_r, s) : launch_r<3, false, FWD>(cs, P, cs.reg_r, s);
  return launch_r<2, true, FWD>(cs, P, cs.reg_r, s);
}

cudaError_t launch_score(const CloudStore &cs, int score, const float4 *pts, const float *lw,
                         const double *self, const float *params, float *out, int32_t *queue,
                         cudaStream_t s) {
  if (cs.n_tiles <= 0) return cudaSuccess;
  Params P = base_params(cs, queue, status_of(queue));
  P.pts = pts;
  P.lw = lw;
  P.out = out;
  P.params = params;
  P.self = self;
  P.score_c = score == 1 ? pow(0.6931471805599453 / 3.141592653589793, 0.5 * cs.dim)
                         : pow(8.0 * 0.6931471805599453, 0.5 * cs.dim);
  const bool w3 = (cs.dim == 3) && lw != nullptr;
  if (score == 1) {
    if (params) return launch_r<2, true, FWD_T, 1>(cs, P, cs.reg_r, s);
    if (cs.dim == 3) return w3 ? launch_r<3, true, FWD, 1>(cs, P, cs.reg_r, s)
                               : launch_r<3, false, FWD, 1>(cs, P, cs.reg_r, s);
    return launch_r<2, true, FWD, 1>(cs, P, cs.reg_r, s);
  }
  if (params) return launch_r<2, true, FWD_T, 2>(cs, P, cs.reg_r, s);
  if (cs.dim == 3) return launch_r<3, true, FWD, 2>(cs, P, cs.reg_r, s);
  return launch_r<2, true, FWD, 2>(cs, P, cs.reg_r, s);
}

cudaError_t launch_cloud_rescore(const CloudStore &cs, int score, float4 *pts_out, float *lw_out,
                                 cudaStream_t s) {
  if (cs.total_pts <= 0) return cudaSuccess;
  const int64_t blocks = (cs.total_pts + 255) / 256;
  cloud_rescore_kernel<<<(int)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(
      cs.d_pts, cs.d_lw, cs.total_pts, cs.dim, score, pts_out, lw_out);
  return cudaGetLastError();
}

cudaError_t launch_cloud_self(const CloudStore &cs, const float4 *pts, const float *lw,
                              double *self, cudaStream_t s) {
  if (cs.n <= 0) return cudaSuccess;
  const double c = pow(0.6931471805599453 / 3.141592653589793, 0.5 * cs.dim);
  const int grid = (int)(cs.n < 65535 ? cs.n : 65535);
  if (cs.dim == 3) {
    if (lw) cloud_self_kernel<3, true><<<grid, 256, 0, s>>>(pts, lw, cs.d_poff, cs.d_cnt, cs.d_perm, cs.n, c, self);
    else cloud_self_kernel<3, false><<<grid, 256, 0, s>>>(pts, lw, cs.d_poff, cs.d_cnt, cs.d_perm, cs.n, c, self);
  } else {
    cloud_self_kernel<2, true><<<grid, 256, 0, s>>>(pts, lw, cs.d_poff, cs.d_cnt, cs.d_perm, cs.n, c, self);
  }
  return cudaGetLastError();
}

cudaError_t launch_overlap_grad_q(const CloudStore &cs, int32_t *queue, const float *params,
                                  const float *grad_out, float *grad_params, float *f_out,
                                  float eta, float fmin, float *params_io, int32_t *flags,
                                  cudaStream_t s) {
  if (cs.n_tiles <= 0) return cudaSuccess;
  Params P = base_params(cs, queue, status_of(queue));
  P.params = params;
  P.grad_out = grad_out;
  P.grad_params = grad_params;
  P.f_out = f_out;
  P.params_io = params_io;
  P.flags = flags;
  P.eta = eta;
  P.fmin = fmin;
  return launch_r<2, true, GRAD>(cs, P, cs.reg_r, s);
}

cudaError_t launch_cloud_pack(const float *x, const float *y, const float *z, const float *sigma,
                              const float *w, const int64_t *src_off, const int32_t *perm,
                              const int64_t *poff, int64_t n, int dim, float4 *pts, float *lw,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)(n < 65535 ? n : 65535);
  cloud_pack_kernel<<<grid, 128, 0, s>>>(x, y, z, sigma, w, src_off, perm, poff, n, dim, pts, lw);
  return cudaGetLastError();
}

}  // namespace ap
