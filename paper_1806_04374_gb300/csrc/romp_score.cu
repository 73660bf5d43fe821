// romp_score.cu -- one greedy step's scores on the tensor cores (tcgen05),
// warp-specialised, for the FP16 path of rsc_encode.
//
// score(p, m, r) = <S_r d_m, r_p> for every patch p and every steered atom
// (m, r) is the dense contraction of the packed residuals (fp16, scaled, 112 columns,
// in HBM) with the steered dictionary [S_0 D ... S_{R-1} D] (fp16, scaled, M*R rows,
// angle-major), i.e. steps (a) and (b) of OMP (Sec. II-C) over the augmented
// dictionary of Fig. "code", the two linear maps folded into one.  Per CTA
// (persistent, one per SM) and pair of 128-patch tiles:
//   * warp 8 (one lane) loads the two residual tiles and streams the steered
//     dictionary in 128-row chunks through a 3-stage shared-memory ring with
//     TMA (128-byte swizzle);
//   * warp 9 (one lane) issues tcgen05.mma (M = 128, N = 128, K = 16, fp16 in,
//     f32 out) for both tiles into one of two TMEM accumulator buffers per
//     tile, and tcgen05.commit's the stage, the buffer and the A tiles back;
//   * warps 0-7 (one thread per patch, TMEM lane = patch) read each buffer
//     back with tcgen05.ld and keep the rsc_ntop(L) (4; 8 for long rows)
//     largest block maxima of |score| (block = 32 rows = 32 atoms at one
//     angle) with their rows, plus the
//     largest value left out (disc), then hand the buffer back.  A block whose
//     maximum is more than the patch's window (>= 2 E, from the refine pass)
//     below the running best can neither win nor fall inside the final
//     window, so it is neither kept nor needs its second maximum.
// All hand-offs are mbarriers; every wait is bounded (2 s of globaltimer) and
// a failed wait records RSC_ERR_TIMEOUT, stops the CTA's loops, drains the
// copies and MMAs it issued, and frees its TMEM.
#include "rsc_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kSTile = 128;
constexpr int kSTiles = 2;
constexpr int kSStages = 3;
constexpr int kSBlk = 128 * 128;       // one 64-column block of 128 rows (bytes)
constexpr int kSThreads = 320;         // 8 epilogue warps + TMA warp + MMA warp
constexpr uint64_t kSWaitNs = 2000000000ull;

// Shape of one instantiation: NB 64-column blocks per packed row (2 for rows
// of kTcKst, 4 for kTcKstLong), BR dictionary rows (atoms or atom pairs) per
// chunk, BUFC accumulator columns per TMEM buffer.
template <bool PAIRED, int NB>
struct SShape {
  static constexpr int BR = (PAIRED || NB > 2) ? kTcBP : kTcBN;
  static constexpr int BUFC = PAIRED ? 2 * kTcBP : BR;
  static constexpr uint32_t kCols = kSTiles * 2 * BUFC;  // 512 or 256
  static constexpr int kATile = NB * kSBlk;               // one A tile (bytes)
  static constexpr int kBBlk = BR * 128;                  // one 64-column block of a B stage
  static constexpr int kBStage = NB * kBBlk;
  static constexpr int a_off = 0, b_off = kSTiles * kATile;
  static constexpr int bar_off = b_off + kSStages * kBStage;
  static constexpr int total = bar_off + 256 + 1024;  // barriers + alignment slack
  static constexpr int NT = NB > 2 ? kTcTopLong : kTcTop;  // candidates per patch
};

// barrier slots (8 bytes each)
enum : int {
  kBarAFull = 0,
  kBarAEmpty = 1,
  kBarBFull = 2,                 // + stage
  kBarBEmpty = 2 + kSStages,     // + stage
  kBarAccFull = 2 + 2 * kSStages,      // + buffer
  kBarAccEmpty = 4 + 2 * kSStages,     // + buffer
  kBarCount = 6 + 2 * kSStages,
};

template <bool PAIRED, int NB>
__global__ void __launch_bounds__(kSThreads, 1)
    romp_score_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const ScoreArgs a) {
  using Sh = SShape<PAIRED, NB>;
  constexpr int BR = Sh::BR;
  constexpr uint32_t kBBlk = (uint32_t)Sh::kBBlk;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr Sh Lo{};
  unsigned char *sA = smem + Lo.a_off;
  unsigned char *sB = smem + Lo.b_off;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lo.bar_off);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + kBarCount);
  volatile int *s_abort = reinterpret_cast<volatile int *>(bars + kBarCount) + 1;
  const uint32_t bar0 = tc::smem_u32(bars);
  auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t kCols = Sh::kCols;
  constexpr uint32_t kIdesc = tc::idesc_f16_f32(128, PAIRED ? kTcBP : BR);

  if (tid == 0) {
    tc::mbar_init(bar(kBarAFull), 1);
    tc::mbar_init(bar(kBarAEmpty), 1);
    for (int s = 0; s < kSStages; ++s) {
      tc::mbar_init(bar(kBarBFull + s), 1);
      tc::mbar_init(bar(kBarBEmpty + s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(bar(kBarAccFull + b), 1);
      tc::mbar_init(bar(kBarAccEmpty + b), 8);  // one arrival per epilogue warp
    }
    *s_abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;

  const int64_t npairs = (a.P + kSTiles * kSTile - 1) / (kSTiles * kSTile);
  const int nch = a.nchunks;
  auto fail = [&]() {
    *s_abort = 1;
    if (a.err) atomicCAS(a.err, 0, RSC_ERR_TIMEOUT);
  };

  if (warp == 8) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      uint32_t gB = 0, issuedB = 0, iter = 0, issuedA = 0;
      for (int64_t pair = blockIdx.x; pair < npairs && !*s_abort; pair += gridDim.x, ++iter) {
        if (iter > 0 && !tc::mbar_wait_bounded(bar(kBarAEmpty), (iter - 1) & 1, kSWaitNs)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(bar(kBarAFull), kSTiles * Sh::kATile);
        for (int t = 0; t < kSTiles; ++t) {
          const int y = (int)((pair * kSTiles + t) * kSTile);
          const uint32_t dst = tc::smem_u32(sA + t * Sh::kATile);
#pragma unroll
          for (int j = 0; j < NB; ++j) tc::tma_load_2d(dst + j * kSBlk, &tmA, bar(kBarAFull), 64 * j, y);
        }
        ++issuedA;
        for (int c = 0; c < nch; ++c, ++gB) {
          const int s = gB % kSStages;
          if (gB >= (uint32_t)kSStages &&
              !tc::mbar_wait_bounded(bar(kBarBEmpty + s), ((gB / kSStages) - 1) & 1, kSWaitNs)) {
            fail();
            break;
          }
          const uint32_t dst = tc::smem_u32(sB + s * Sh::kBStage);
          tc::mbar_arrive_expect_tx(bar(kBarBFull + s), Sh::kBStage);
#pragma unroll
          for (int j = 0; j < NB; ++j)
            tc::tma_load_2d(dst + j * kBBlk, &tmB, bar(kBarBFull + s), 64 * j, c * BR);
          ++issuedB;
        }
      }
      // drain: every issued load lands before the CTA exits
      for (uint32_t i = (issuedB > (uint32_t)kSStages ? issuedB - kSStages : 0); i < issuedB; ++i)
        tc::mbar_wait_bounded(bar(kBarBFull + i % kSStages), (i / kSStages) & 1, kSWaitNs);
      if (issuedA) tc::mbar_wait_bounded(bar(kBarAFull), (issuedA - 1) & 1, kSWaitNs);
    }
  } else if (warp == 9) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t g = 0, iter = 0;
      bool any = false;
      for (int64_t pair = blockIdx.x; pair < npairs && !*s_abort; pair += gridDim.x, ++iter) {
        if (!tc::mbar_wait_bounded(bar(kBarAFull), iter & 1, kSWaitNs)) {
          fail();
          break;
        }
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sA);
        bool ok = true;
        for (int c = 0; c < nch; ++c, ++g) {
          const int s = g % kSStages;
          const uint32_t b = g & 1, ub = g >> 1;
          if (!tc::mbar_wait_bounded(bar(kBarBFull + s), (g / kSStages) & 1, kSWaitNs) ||
              (ub > 0 && !tc::mbar_wait_bounded(bar(kBarAccEmpty + b), (ub - 1) & 1, kSWaitNs))) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t b0 = tc::smem_u32(sB + s * Sh::kBStage);
#pragma unroll
          for (int t = 0; t < kSTiles; ++t) {
            const uint32_t d = tmem + (uint32_t)(t * 2 + b) * Sh::BUFC;
            const uint32_t at = a0 + t * Sh::kATile;
            if (PAIRED) {
              // even half (A and B block 0) -> columns 0..63, odd half
              // (block 1) -> columns 64..127 of the buffer
              for (int ks = 0; ks < a.ke; ++ks)
                tc::mma_f16(d, tc::smem_desc_sw128(at + ks * 32), tc::smem_desc_sw128(b0 + ks * 32),
                            kIdesc, ks > 0 ? 1u : 0u);
              for (int ks = 0; ks < a.ko; ++ks)
                tc::mma_f16(d + kTcBP, tc::smem_desc_sw128(at + kSBlk + ks * 32),
                            tc::smem_desc_sw128(b0 + kBBlk + ks * 32), kIdesc, ks > 0 ? 1u : 0u);
            } else {
              for (int ks = 0; ks < a.ksteps; ++ks)
                tc::mma_f16(d, tc::smem_desc_sw128(at + (ks >> 2) * kSBlk + (ks & 3) * 32),
                            tc::smem_desc_sw128(b0 + (ks >> 2) * kBBlk + (ks & 3) * 32), kIdesc,
                            ks > 0 ? 1u : 0u);
            }
          }
          tc::mma_commit(bar(kBarBEmpty + s));
          tc::mma_commit(bar(kBarAccFull + b));
          if (c == nch - 1) tc::mma_commit(bar(kBarAEmpty));
          any = true;
        }
        if (!ok) {
          fail();
          break;
        }
      }
      // drain: the last commit covers every MMA this thread issued
      if (any) tc::mbar_wait_bounded(bar(kBarAccFull + ((g - 1) & 1)), ((g - 1) >> 1) & 1, kSWaitNs);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int tile = warp >> 2, quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    uint32_t g = 0;
    for (int64_t pair = blockIdx.x; pair < npairs; pair += gridDim.x) {
      const int64_t p = (pair * kSTiles + tile) * kSTile + row;
      const bool act = p < a.P && a.status[p] > 0;
      const float win = act ? a.win[p] : 0.0f;
      float tv[Sh::NT];
      int ti[Sh::NT];
#pragma unroll
      for (int q = 0; q < Sh::NT; ++q) {
        tv[q] = -INFINITY;
        ti[q] = -1;
      }
      float disc = -INFINITY;
      bool ok = true;
      for (int c = 0; c < nch; ++c, ++g) {
        const uint32_t b = g & 1, ub = g >> 1;
        const bool done = !*s_abort && tc::mbar_wait_bounded(bar(kBarAccFull + b), ub & 1, kSWaitNs);
        if (!__all_sync(0xffffffffu, done)) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t taddr = tmem + lane_base + (uint32_t)(tile * 2 + b) * Sh::BUFC;
        const int nvalid = min(BR, a.MR - c * BR);
#pragma unroll 1
        for (int piece = 0; piece < BR / 32; ++piece) {
          uint32_t v[32];
          tc::tmem_ld32(taddr + piece * 32, v);
          if (PAIRED) {
            // pair value |E| + |O| = max(|score(r)|, |score(r + R/2)|)
            uint32_t o[32];
            tc::tmem_ld32(taddr + kTcBP + piece * 32, o);
            tc::tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 32; ++u)
              v[u] = __float_as_uint(fabsf(__uint_as_float(v[u])) + fabsf(__uint_as_float(o[u])));
          } else {
            tc::tmem_wait_ld();
          }
          if (act) {
            // keys: |score| with the low 5 mantissa bits replaced by the
            // column within the block; non-negative floats order like their
            // bits, so one max gives the block maximum and its column (the
            // truncation is < 2^-18 relative and covered by the refine's
            // error bound)
            const int base = c * BR + piece * 32;
            const int nv = nvalid - piece * 32;
            float key[32];
#pragma unroll
            for (int u = 0; u < 32; ++u)
              key[u] = __int_as_float((int)((v[u] & 0x7FFFFFE0u) | (uint32_t)u));
            if (nv < 32) {
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (u >= nv) key[u] = -1.0f;
            }
            float m1 = -1.0f;
#pragma unroll
            for (int u = 0; u < 32; u += 2) m1 = fmax3(m1, key[u], key[u + 1]);
            // kept: the block maximum beats the last kept one and is not below
            // the window under the running best (NaN-safe form)
            if (m1 >= 0.0f && m1 > tv[Sh::NT - 1] && !(m1 < tv[0] - win)) {
              const int us = __float_as_int(m1) & 31;
              float m2 = -1.0f;
#pragma unroll
              for (int u = 0; u < 32; ++u) m2 = fmaxf(m2, key[u] < m1 ? key[u] : -1.0f);
              topn_insert(tv, ti, disc, m1, base + us);
              if (m2 >= 0.0f && !(m2 < tv[0] - win)) {
                // the block's second value may lie in the window too: keep it
                // as a candidate and bound the rest by the third value
                float m3 = -1.0f;
#pragma unroll
                for (int u = 0; u < 32; ++u) m3 = fmaxf(m3, key[u] < m2 ? key[u] : -1.0f);
                topn_insert(tv, ti, disc, m2, base + (__float_as_int(m2) & 31));
                disc = fmaxf(disc, m3);
              } else {
                disc = fmaxf(disc, m2);
              }
            } else {
              disc = fmaxf(disc, m1);
            }
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(kBarAccEmpty + b)) : "memory");
      }
      if (!ok) break;
      if (act) {
        int *ci = a.cand_idx + p * Sh::NT;
        float *cv = a.cand_val + p * Sh::NT;
#pragma unroll
        for (int q = 0; q < Sh::NT; q += 4) {
          *reinterpret_cast<int4 *>(ci + q) = make_int4(ti[q], ti[q + 1], ti[q + 2], ti[q + 3]);
          *reinterpret_cast<float4 *>(cv + q) = make_float4(tv[q], tv[q + 1], tv[q + 2], tv[q + 3]);
        }
        a.cand_disc[p] = disc;
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

}  // namespace

namespace {
template <bool PAIRED, int NB>
int launch_score_t(const ScoreArgs &a, const CUtensorMap &tmA, const CUtensorMap &tmB,
                   cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  int max_optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  constexpr int total = SShape<PAIRED, NB>::total;
  if (total > max_optin) return RSC_ERR_UNSUPPORTED;
  auto kern = romp_score_kernel<PAIRED, NB>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, total);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  const int64_t pairs = (a.P + kSTiles * kSTile - 1) / (kSTiles * kSTile);
  const int64_t grid = pairs < nsm ? pairs : nsm;
  kern<<<(unsigned)grid, kSThreads, total, stream>>>(tmA, tmB, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return RSC_OK;
}
}  // namespace

int rsc_launch_score(const ScoreArgs &a, const CUtensorMap &tmA, const CUtensorMap &tmB,
                     cudaStream_t stream) {
  if (a.P == 0) return RSC_OK;
  if (a.L == kTcKst)
    return a.paired ? launch_score_t<true, 2>(a, tmA, tmB, stream)
                    : launch_score_t<false, 2>(a, tmA, tmB, stream);
  if (a.L == kTcKstLong && !a.paired) return launch_score_t<false, 4>(a, tmA, tmB, stream);
  return RSC_ERR_UNSUPPORTED;
}
