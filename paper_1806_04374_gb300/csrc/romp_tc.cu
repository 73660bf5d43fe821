// romp_tc.cu -- rotational OMP with an FP16 tensor-core (tcgen05) scoring pass.
//
// The scores of one greedy step, score(p, m, r) = <S_r d_m, r_p> (OMP of
// Sec. II-C over the augmented dictionary of Fig. "code"), are steps (a) and
// (b) of the method: the per-harmonic contraction G_k = sum_j conj(d) r and
// the angle transform sum_k e^{ik 2 pi r/R} G_k.  Both are linear, so their
// product is one dense contraction of the packed residual with the steered
// dictionary [S_0 D ... S_{R-1} D] (built once per dictionary by the host in
// FP64 and stored in fp16, scaled by kDictScale).  This kernel runs that contraction on the 5th
// generation tensor cores:
//
//   * a CTA owns TILES tiles of 128 patches; a tile's packed residuals are
//     the A operand (fp16, 128 x 112, 128-byte swizzled K-major in shared
//     memory) and every TMEM lane holds one patch;
//   * the steered dictionary streams through a ring of shared-memory stages
//     in chunks of 128 steered atoms, loaded by TMA (one thread issues the
//     loads and the MMAs); each chunk is multiplied into one of two TMEM
//     accumulator buffers per tile while the other buffer is read back;
//   * epilogue (c): every thread reads its patch's scores with tcgen05.ld and
//     keeps the kTcTop (4) largest block maxima of |score| and the largest value it
//     discarded;
//   * per patch, every candidate within 2E of the best (E bounds the fp16
//     error of a score) is re-scored exactly in double-float as
//     <A_c, x> - sum_i a_i <A_c, A_i>, the Gram entries coming from the
//     per-harmonic cross-Gram table; if the window holds more candidates
//     than were kept, the patch is handed to the FP32 path instead;
//   * (e) the Gram row and right-hand side of the winner in double-float,
//     the Cholesky row and solve in FP64, per thread;
//   * (d) the new residual in FP32, scaled by a power of two chosen from the
//     previous norm (rsc_internal.h) and rounded to fp16 into the A tile.
#include <cuda_fp16.h>
#include <math.h>

#include "df.cuh"
#include "rsc_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kTile = 128;
constexpr int kStages = 3;
constexpr int kBlkA = kTile * 128;    // one 64-column block of A (bytes)
constexpr int kBlkB = kTcBN * 128;    // one 64-column block of a B stage (bytes)
constexpr int kStageBytes = 2 * kBlkB;
constexpr uint64_t kWaitNs = 2000000000ull;  // bounded waits: 2 s

struct TcLayout {
  int a_off, b_off, tw_off, bar_off, misc_off, total;
};

__host__ __device__ inline int al(int v, int a) { return (v + a - 1) / a * a; }

template <int TILES>
__host__ __device__ inline TcLayout tc_layout(int H, int R) {
  TcLayout L;
  int off = 0;
  L.a_off = off;
  off += TILES * 2 * kBlkA;
  L.b_off = off;
  off += kStages * kStageBytes;
  L.tw_off = off;
  off = al(off + 4 * H * (R + 1) * 4, 16);
  L.bar_off = off;
  off = al(off + (kStages + 2) * 8, 16);
  L.misc_off = off;
  off += 16;
  L.total = off + 1024;  // slack for the 1024-byte alignment of the base
  return L;
}

// Sink writing packed chunks into row `row` of a 128-byte-swizzled A tile.
struct SmemRow {
  unsigned char *tile;
  int row;
  __device__ void operator()(int cq, uint4 v) const {
    const int blk = cq >> 3, ch = cq & 7;
    *reinterpret_cast<uint4 *>(tile + blk * kBlkA + row * 128 + ((ch ^ (row & 7)) << 4)) = v;
  }
};

__device__ __forceinline__ void record_error(int *err, int code) {
  if (err) atomicCAS(err, 0, code);
}

template <int TILES, int KK>
__global__ void __launch_bounds__(TILES * 128, 1)
    romp_tc_kernel(const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int H = a.H, J = a.J, R = a.R, M = a.M, K = a.K, HJ = H * J;
  const TcLayout Lo = tc_layout<TILES>(H, R);
  unsigned char *sA = smem + Lo.a_off;
  unsigned char *sB = smem + Lo.b_off;
  float *s_tw = reinterpret_cast<float *>(smem + Lo.tw_off);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lo.bar_off);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + Lo.misc_off);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile_id = tid >> 7, row = tid & 127;
  const uint32_t full_bar0 = tc::smem_u32(bars);
  const uint32_t done_bar0 = tc::smem_u32(bars + kStages);
  constexpr uint32_t kCols = TILES * 2 * kTcBN;
  constexpr uint32_t kIdesc = tc::idesc_f16_f32(128, kTcBN);

  // ---- set-up: tables, barriers, TMEM
  for (int i = tid; i < 4 * H * R; i += blockDim.x) {
    const int pk = i / R, r = i - pk * R;
    s_tw[pk * (R + 1) + r] = a.tw[i];
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) tc::mbar_init(full_bar0 + 8 * s, 1);
    for (int b = 0; b < 2; ++b) tc::mbar_init(done_bar0 + 8 * b, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const TwS tw{s_tw, H, R + 1};

  // producer / MMA state, meaningful in thread 0 only
  uint32_t g = 0;              // global chunk counter (MMA order)
  uint32_t tma_next = 0;       // next chunk to load
  uint32_t mma_issued = 0;     // chunks whose MMAs were issued
  uint32_t mma_waited = 0;     // chunks whose completion was observed by thread 0

  auto issue_tma = [&](uint32_t gg) {
    const int s = gg % kStages;
    const int chunk = gg % a.nchunks;
    const uint32_t bar = full_bar0 + 8 * s;
    const uint32_t dst = tc::smem_u32(sB + s * kStageBytes);
    tc::mbar_arrive_expect_tx(bar, kStageBytes);
    tc::tma_load_2d(dst, &tmB, bar, 0, chunk * kTcBN);
    tc::tma_load_2d(dst + kBlkB, &tmB, bar, 64, chunk * kTcBN);
  };
  auto issue_mma = [&](uint32_t gg) -> bool {
    const int s = gg % kStages;
    if (!tc::mbar_wait_bounded(full_bar0 + 8 * s, (gg / kStages) & 1, kWaitNs)) return false;
    tc::fence_after_sync();
    const uint32_t buf = gg & 1;
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB + s * kStageBytes);
#pragma unroll
    for (int tl = 0; tl < TILES; ++tl) {
      const uint32_t d = tmem + (uint32_t)(tl * 2 + buf) * kTcBN;
      for (int ks = 0; ks < a.ksteps; ++ks) {
        const uint32_t off = (ks >> 2) * kBlkA + (ks & 3) * 32;
        const uint32_t boff = (ks >> 2) * kBlkB + (ks & 3) * 32;
        tc::mma_f16(d, tc::smem_desc_sw128(a0 + tl * 2 * kBlkA + off),
                     tc::smem_desc_sw128(b0 + boff), kIdesc, ks > 0 ? 1u : 0u);
      }
    }
    tc::mma_commit(done_bar0 + 8 * buf);
    mma_issued = gg + 1;
    return true;
  };

  if (tid == 0) {
    for (; tma_next < (uint32_t)kStages; ++tma_next) issue_tma(tma_next);
  }

  const int64_t ngroups = (a.P + (int64_t)TILES * kTile - 1) / ((int64_t)TILES * kTile);
  bool aborted = false;
  for (int64_t grp = blockIdx.x; grp < ngroups && !aborted; grp += gridDim.x) {
    const int64_t p = (grp * TILES + tile_id) * kTile + row;
    const bool valid = p < a.P;
    unsigned char *myA = sA + tile_id * 2 * kBlkA;
    const float *xp = a.x + (valid ? p : 0) * (int64_t)(2 * HJ);
    Ls<KK> S;
    int t = 0;
    bool active = valid, redo = false;
    float xnorm = 0.0f, rnorm = 0.0f, dr = 0.0f;
    int escale = 0;  // the A row holds the residual times 2^(kRowLog2 - escale)
    if (valid) {
      df acc = df_make(0.0f);
      for (int e = 0; e < HJ; ++e) {
        float2 v = __ldg(reinterpret_cast<const float2 *>(xp) + e);
        if (e < J) v.y = 0.0f;
        df q = df_add(two_prod(v.x, v.x), two_prod(v.y, v.y));
        acc = df_add(acc, e < J ? q : df_mul_f(q, 2.0f));
      }
      xnorm = sqrtf(fmaxf(acc.hi + acc.lo, 0.0f));
      escale = rsc_row_exponent(xnorm);
      rnorm = sqrtf(write_residual<KK>(SmemRow{myA, row}, ldexpf(1.0f, kRowLog2 - escale), xp,
                                       a.d, J, HJ, a.n, 0, S, tw));
      dr = 2.0f * kU32 * xnorm;
    } else {
      // rows of absent patches: zeros
      for (int cq = 0; cq < kTcKst / 8; ++cq) {
        const int blk = cq >> 3, ch = cq & 7;
        *reinterpret_cast<uint4 *>(myA + blk * kBlkA + row * 128 + ((ch ^ (row & 7)) << 4)) =
            make_uint4(0, 0, 0, 0);
      }
    }
    const float stop_level = 1e-10f * xnorm;

    for (int step = 0; step < K; ++step) {
      tc::fence_proxy_async_smem();
      const int any = __syncthreads_or(active ? 1 : 0);
      if (!any) break;
      // ---- scoring: MMAs chunk by chunk, epilogue keeps the per-patch top-4
      float tv[kTop];
      int ti[kTop];
#pragma unroll
      for (int q = 0; q < kTop; ++q) {
        tv[q] = -INFINITY;
        ti[q] = -1;
      }
      float disc = -INFINITY;
      for (int c = 0; c < a.nchunks; ++c) {
        const uint32_t gg = g + c;
        int fail = 0;
        if (tid == 0) {
          bool ok = true;
          if (c == 0) ok = issue_mma(gg);
          if (ok && c + 1 < a.nchunks) ok = issue_mma(gg + 1);
          if (!ok) fail = 1;
        }
        // completion of chunk gg (every thread observes the barrier)
        bool done = false;
        if (!fail) done = tc::mbar_wait_bounded(done_bar0 + 8 * (gg & 1), (gg >> 1) & 1, kWaitNs);
        if (!done) {
          fail = 1;
          record_error(a.err, RSC_ERR_TIMEOUT);
        }
        tc::fence_after_sync();
        if (tid == 0 && done) {
          mma_waited = gg + 1;
          // stage gg % kStages is free again: prefetch chunk gg + kStages
          issue_tma(tma_next);
          ++tma_next;
        }
        // tcgen05.ld is warp-collective: a warp reads back only if none of its
        // threads saw a failed wait
        if (!__any_sync(0xffffffffu, fail)) {
          const uint32_t col0 = (uint32_t)(tile_id * 2 + (gg & 1)) * kTcBN;
          const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + col0;
          const int nvalid = min(kTcBN, a.MR - c * kTcBN);
#pragma unroll 1
          for (int piece = 0; piece < kTcBN / 32; ++piece) {
            uint32_t v[32];
            tc::tmem_ld32(taddr + piece * 32, v);
            tc::tmem_wait_ld();
            if (active) {
              // rows base .. base+31 of the steered dictionary (angle-major:
              // 32 different atoms).  Common path: the block maximum only;
              // a block whose maximum enters the top-4 also yields its
              // arg-max and second maximum (the latter goes to disc).
              const int base = c * kTcBN + piece * 32;
              const int nv = nvalid - piece * 32;
              float av[32];
#pragma unroll
              for (int u = 0; u < 32; ++u)
                av[u] = (u < nv) ? fabsf(__uint_as_float(v[u])) : -INFINITY;
              float m1 = -INFINITY;
#pragma unroll
              for (int u = 0; u < 32; u += 2) m1 = fmax3(m1, av[u], av[u + 1]);
              if (m1 > tv[kTop - 1]) {
                int us = 0;
                bool found = false;
                float m2 = -INFINITY;
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                  const bool is = !found && (av[u] == m1);
                  us = is ? u : us;
                  found = found || is;
                  m2 = fmaxf(m2, is ? -INFINITY : av[u]);
                }
                topn_insert(tv, ti, disc, m1, base + us);
                disc = fmaxf(disc, m2);
              } else {
                disc = fmaxf(disc, m1);
              }
            }
          }
        }
        tc::fence_before_sync();
        // one CTA-wide decision: a failed wait anywhere ends the kernel
        if (__syncthreads_or(fail)) {
          aborted = true;
          break;
        }
      }
      g += a.nchunks;
      if (aborted) break;

      // ---- per patch: certify, re-score, least squares, residual
      if (active) {
        // accumulator scores are 2^(16 - escale) times the true scores
        const float unscale = ldexpf(1.0f, escale - 16);
#pragma unroll
        for (int q = 0; q < kTop; ++q) tv[q] *= unscale;
        disc *= unscale;
        const float s1 = tv[0];
        // fp16 error of a score (both operands, second order, accumulation,
        // subnormal rounding of dictionary and row entries), times 1.25, plus
        // the FP32 residual's own error
        const float E = 1.25f * (9.765625e-4f + 3.814697265625e-6f + 112.0f * 4.76837158203125e-7f +
                                 11.0f * 1.16415321826934814e-10f) *
                            rnorm +
                        1.25f * 11.0f * ldexpf(1.0f, escale - 33) + 2.0f * dr;
        if (!(s1 + E > stop_level)) {
          active = false;
        } else {
          const float thr = s1 - 2.0f * E;
          if (disc >= thr) {
            redo = true;
            active = false;
          } else {
            // FP32 screen: |f_q - s_q| <= E32 for every candidate, so the
            // exact winner is among those with f_q >= max f - 2 E32
            float asum = 0.0f;
#pragma unroll
            for (int i = 0; i < KK; ++i)
              if (i < t) asum += fabsf(S.ahi[i]);
            const float E32 = 256.0f * kU32 * (xnorm + asum);
            float fs[kTop];
            float fbest = -1.0f;
#pragma unroll
            for (int q = 0; q < kTop; ++q) {
              fs[q] = -1.0f;
              if (ti[q] >= 0 && tv[q] >= thr) {
                const int m = ti[q] % M, r = ti[q] / M;
                fs[q] = fabsf(score32<KK>(a.d + (size_t)m * HJ * 2, xp, a.xgram, M, J, H, R, m, r,
                                          t, S, tw));
                fbest = fmaxf(fbest, fs[q]);
              }
            }
            // exact (double-float) re-score of the survivors:
            // <A_c, x> - sum_i a_i <A_c, A_i>; ties -> smallest m*R + r
            df best = df_make(0.0f), best_ax = df_make(0.0f);
            df bg[KK];
#pragma unroll
            for (int i = 0; i < KK; ++i) bg[i] = df_make(0.0f);
            int bc = -1, bflat = 0;
#pragma unroll
            for (int q = 0; q < kTop; ++q) {
              if (fs[q] >= 0.0f && fs[q] >= fbest - 2.0f * E32) {
                const int m = ti[q] % M, r = ti[q] / M;
                const df ax = score_x(a.d + (size_t)m * HJ * 2, xp, J, H, r, tw);
                df sc = ax;
                df gq[KK];
#pragma unroll
                for (int i = 0; i < KK; ++i) {
                  gq[i] = df_make(0.0f);
                  if (i < t) {
                    gq[i] = gram_entry(a.xgram, M, H, R, m, r, S.m[i], S.r[i], tw);
                    sc = df_sub(sc, df_mul(df{S.ahi[i], S.alo[i]}, gq[i]));
                  }
                }
                const int flat = m * R + r;
                if (bc < 0 || df_abs_gt(sc, best) || (df_abs_eq(sc, best) && flat < bflat)) {
                  best = sc;
                  bc = ti[q];
                  bflat = flat;
                  best_ax = ax;
#pragma unroll
                  for (int i = 0; i < KK; ++i) bg[i] = gq[i];
                }
              }
            }
            if (bc < 0 || !(fabsf(best.hi) > stop_level)) {
              active = false;
            } else {
              const int mb = bc % M, rb = bc / M;
              double gr[KK];
#pragma unroll
              for (int i = 0; i < KK; ++i) gr[i] = (i < t) ? df_to_d(bg[i]) : 0.0;
              const double diag = df_to_d(gram_entry(a.xgram, M, H, R, mb, rb, mb, rb, tw));
              const double rhs = df_to_d(best_ax);
              if (!CholAt<KK, 0>::run(t, S, gr, diag, rhs)) {
                active = false;
              } else {
#pragma unroll
                for (int i = 0; i < KK; ++i)
                  if (i == t) {
                    S.m[i] = mb;
                    S.r[i] = rb;
                  }
                ++t;
                asum = 0.0f;
#pragma unroll
                for (int i = 0; i < KK; ++i)
                  if (i < t) asum += fabsf(S.ahi[i]);
                escale = rsc_row_exponent(rnorm);
                rnorm = sqrtf(write_residual<KK>(SmemRow{myA, row}, ldexpf(1.0f, kRowLog2 - escale),
                                                 xp, a.d, J, HJ, a.n, t, S, tw));
                dr = 2.0f * (t + 6) * kU32 * (xnorm + 1.5f * asum);
              }
            }
          }
        }
        if (redo) {
          const int slot = atomicAdd(a.redo_count, 1);
          a.redo_list[slot] = (int)p;
          if (a.fallbacks) atomicAdd(a.fallbacks, 1ull);
        }
      }
    }

    // ---- outputs of this thread's patch
    if (valid && !redo && !aborted) {
#pragma unroll
      for (int i = 0; i < KK; ++i) {
        if (i < K) {
          const int64_t o = p * K + i;
          if (i < t) {
            a.atom[o] = S.m[i];
            a.angle_idx[o] = S.r[i];
            if (a.angle) a.angle[o] = (float)(6.283185307179586 * S.r[i] / R);
            a.coef[o] = S.a[i];
          } else {
            a.atom[o] = -1;
            a.angle_idx[o] = -1;
            if (a.angle) a.angle[o] = 0.0f;
            a.coef[o] = 0.0;
          }
        }
      }
      if (a.resid_norm2) a.resid_norm2[p] = rnorm * rnorm;
    }
  }

  // ---- drain: every issued TMA load and MMA completes before TMEM is freed
  if (tid == 0) {
    for (uint32_t gg = mma_waited; gg < mma_issued; ++gg)
      tc::mbar_wait_bounded(done_bar0 + 8 * (gg & 1), (gg >> 1) & 1, kWaitNs);
    for (uint32_t gg = mma_issued; gg < tma_next; ++gg)
      tc::mbar_wait_bounded(full_bar0 + 8 * (gg % kStages), (gg / kStages) & 1, kWaitNs);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

template <int TILES, int KK>
int launch_tc_t(const TcArgs &a, const CUtensorMap &tmap, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  int max_optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const TcLayout L = tc_layout<TILES>(a.H, a.R);
  if (L.total > max_optin) return RSC_ERR_UNSUPPORTED;
  auto kern = romp_tc_kernel<TILES, KK>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  const int64_t groups = (a.P + (int64_t)TILES * kTile - 1) / ((int64_t)TILES * kTile);
  const int64_t grid = groups < nsm ? groups : nsm;
  kern<<<(unsigned)grid, TILES * kTile, L.total, stream>>>(tmap, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return RSC_OK;
}

}  // namespace

int rsc_launch_tc(const TcArgs &a, const CUtensorMap &tmap, cudaStream_t stream) {
  if (a.P == 0) return RSC_OK;
  if (a.K <= 3) return launch_tc_t<2, 3>(a, tmap, stream);
  if (a.K <= 5) return launch_tc_t<2, 5>(a, tmap, stream);
  if (a.K <= 8) return launch_tc_t<2, 8>(a, tmap, stream);
  return RSC_ERR_UNSUPPORTED;
}
