// romp_score.cu -- one greedy step's scores on the tensor cores (tcgen05),
// warp-specialised, for the FP16 path of rsc_encode.
//
// score(p, m, r) = <S_r d_m, r_p> for every patch p and every steered atom
// (m, r) is the dense contraction of the packed residuals (fp16, scaled, L
// columns, in HBM) with the steered dictionary [S_0 D ... S_{R-1} D] (fp16,
// scaled, M*R rows, angle-major), i.e. steps (a) and (b) of OMP (Sec. II-C)
// over the augmented dictionary of Fig. "code", the two linear maps folded
// into one.  Per CTA (persistent, one per SM) and 128-patch tile:
//   * warp 8 (one lane) loads the tile's residual rows (A, double-buffered
//     across tiles when they are short) and streams the steered dictionary
//     in chunks of N rows (256 atoms at one angle block, or 128 atom pairs),
//     one 64-column K-block per stage of a shared-memory ring, with TMA
//     (128-byte swizzle);
//   * warp 9 (one lane) issues tcgen05.mma (M = 128, N = 256 or 128, K = 16,
//     fp16 in, f32 out) into one of two TMEM accumulator buffers of 256
//     columns, and tcgen05.commit's each stage, each buffer and the A tile
//     back to their producers.  The time of one MMA hardly depends on N up
//     to 64 on this part (measured: the same launch time at N = 16, 32, 64),
//     so the widest N that two accumulator buffers allow is used;
//   * warps 0-7 read each buffer back with tcgen05.ld: warp w reads TMEM
//     lanes 32 (w mod 4) .. + 31 (one thread per patch) and one column slice
//     (one of kTcSplit, rotated by one per chunk).  Per patch, each warp keeps for every
//     column u of a 32-column block (block = 32 atoms at one angle, or 32 atom
//     pairs) the largest value column u had in any block ("class" u, in
//     registers), and a ring of the blocks whose maximum came within the
//     patch's window (>= 2 E, from the refine pass) of the running best.  At
//     the end of the step every unit within the window of the slice's best
//     lies in a kept block and in a class whose maximum reaches the
//     threshold, so the slice hands over up to kTcTop blocks, the class mask
//     and its best class, plus a bound on what it left out (disc); the refine
//     expands blocks x classes.  Per value that is one add (paired), one max
//     into its class and half a three-input max for its block, with no
//     per-block branch; the slices never synchronise.
// All hand-offs are mbarriers; every wait is bounded (2 s of globaltimer, or
// a shorter limit for the pipeline waits set on the dictionary to test this
// path) and a failed wait records RSC_ERR_TIMEOUT, stops the CTA's loops,
// drains the copies and MMAs it issued (with the 2 s limit), and frees its
// TMEM.
#include "rsc_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kSTile = 128;             // patches per tile (MMA M, TMEM lanes)
constexpr int kSStagesMax = 6;          // barrier slots reserved for the B ring
constexpr int kABlk = kSTile * 128;     // one 64-column block of an A tile (bytes)
constexpr int kSBufC = 256;             // accumulator columns per TMEM buffer
constexpr uint32_t kSCols = 2 * kSBufC; // two buffers: all 512 TMEM columns
constexpr int kSEpi = 4 * kTcSplit;     // epilogue warps: 4 lane quarters x kTcSplit slices
constexpr int kSThreads = 32 * (kSEpi + 2);  // + TMA warp + MMA warp
constexpr uint64_t kSWaitNs = 2000000000ull;  // drain waits (and the default pipeline limit)
constexpr int kRing = 16;               // blocks near the running best kept per step

// Shape of one instantiation: NB 64-column blocks per packed row (2 for rows
// of kTcKst, 4 for kTcKstLong) and STAGES stages of the dictionary ring.
template <bool PAIRED, int NB, int STAGES>
struct SShape {
  static constexpr int N = PAIRED ? kTcSNP : kTcSN;   // B rows per chunk = MMA N
  static constexpr int NKB = NB;                      // K-blocks (ring stages) per chunk
  static constexpr int kATile = NB * kABlk;           // one A tile (bytes)
  static constexpr int kABufs = NB > 2 ? 1 : 2;       // A tiles in flight
  static constexpr int kBStage = N * 128;             // one K-block of a chunk (bytes)
  static constexpr int kStages = STAGES;
  static constexpr int SLICE = N / kTcSplit;          // B rows per epilogue column slice
  static constexpr int PIECES = SLICE / 32;           // 32-column pieces per slice
  static constexpr int a_off = 0, b_off = kABufs * kATile;
  static constexpr int bar_off = b_off + kStages * kBStage;
  static constexpr int total = bar_off + 256 + 1024;  // barriers + alignment slack
  static_assert(kStages <= kSStagesMax, "barrier slots");
  static_assert(PAIRED ? 2 * N == kSBufC : N == kSBufC, "accumulator buffer width");
  static_assert(PIECES >= 1 && SLICE % 32 == 0, "slices of whole 32-column blocks");
};

// barrier slots (8 bytes each)
enum : int {
  kBarAFull = 0,                          // + A buffer
  kBarAEmpty = 2,                         // + A buffer
  kBarBFull = 4,                          // + stage
  kBarBEmpty = 4 + kSStagesMax,           // + stage
  kBarAccFull = 4 + 2 * kSStagesMax,      // + buffer
  kBarAccEmpty = 6 + 2 * kSStagesMax,     // + buffer
  kBarCount = 8 + 2 * kSStagesMax,
};
static_assert(kBarCount * 8 + 8 <= 256, "barrier area");

template <bool PAIRED, int NB, int STAGES>
__global__ void __launch_bounds__(kSThreads, 1)
    romp_score_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const ScoreArgs a) {
  using Sh = SShape<PAIRED, NB, STAGES>;
  constexpr int N = Sh::N, NKB = Sh::NKB, kStages = Sh::kStages, kABufs = Sh::kABufs;
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
  constexpr uint32_t kIdesc = tc::idesc_f16_f32(128, N);

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(bar(kBarAFull + i), 1);
      tc::mbar_init(bar(kBarAEmpty + i), 1);
      tc::mbar_init(bar(kBarAccFull + i), 1);
      tc::mbar_init(bar(kBarAccEmpty + i), kSEpi);  // one arrival per epilogue warp
    }
    for (int s = 0; s < kSStagesMax; ++s) {
      tc::mbar_init(bar(kBarBFull + s), 1);
      tc::mbar_init(bar(kBarBEmpty + s), 1);
    }
    *s_abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kSCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;

  const int64_t ntiles = (a.P + kSTile - 1) / kSTile;
  const int nch = a.nchunks;
  auto fail = [&]() {
    *s_abort = 1;
    if (a.err) atomicCAS(a.err, 0, RSC_ERR_TIMEOUT);
  };

  if (warp == kSEpi) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      uint32_t gs = 0, it = 0;
      uint32_t issuedA[2] = {0u, 0u};
      bool ok = true;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles && !*s_abort; tile += gridDim.x, ++it) {
        const int ab = (int)(it % kABufs);
        const uint32_t ua = it / kABufs;
        if (ua > 0 && !tc::mbar_wait_bounded(bar(kBarAEmpty + ab), (ua - 1) & 1, a.wait_ns)) {
          fail();
          break;
        }
        tc::mbar_arrive_expect_tx(bar(kBarAFull + ab), Sh::kATile);
        const uint32_t dstA = tc::smem_u32(sA + ab * Sh::kATile);
#pragma unroll
        for (int j = 0; j < NB; ++j)
          tc::tma_load_2d(dstA + j * kABlk, &tmA, bar(kBarAFull + ab), 64 * j, (int)(tile * kSTile));
        ++issuedA[ab];
        for (int c = 0; ok && c < nch; ++c) {
          for (int j = 0; j < NKB; ++j, ++gs) {
            const int s = (int)(gs % kStages);
            if (gs >= (uint32_t)kStages &&
                !tc::mbar_wait_bounded(bar(kBarBEmpty + s), ((gs / kStages) - 1) & 1, a.wait_ns)) {
              fail();
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(bar(kBarBFull + s), Sh::kBStage);
            tc::tma_load_2d(tc::smem_u32(sB + s * Sh::kBStage), &tmB, bar(kBarBFull + s), 64 * j, c * N);
          }
        }
      }
      // drain: every issued load lands before the CTA exits
      for (uint32_t i = (gs > (uint32_t)kStages ? gs - kStages : 0); i < gs; ++i)
        tc::mbar_wait_bounded(bar(kBarBFull + i % kStages), (i / kStages) & 1, kSWaitNs);
      for (int ab = 0; ab < kABufs; ++ab)
        if (issuedA[ab]) tc::mbar_wait_bounded(bar(kBarAFull + ab), (issuedA[ab] - 1) & 1, kSWaitNs);
    }
  } else if (warp == kSEpi + 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      uint32_t g = 0, gs = 0, it = 0, last = 0;
      bool any = false, ok = true;
      for (int64_t tile = blockIdx.x; ok && tile < ntiles && !*s_abort; tile += gridDim.x, ++it) {
        const int ab = (int)(it % kABufs);
        const uint32_t ua = it / kABufs;
        if (!tc::mbar_wait_bounded(bar(kBarAFull + ab), ua & 1, a.wait_ns)) {
          fail();
          break;
        }
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sA + ab * Sh::kATile);
        for (int c = 0; c < nch; ++c, ++g) {
          const uint32_t b = g & 1, ub = g >> 1;
          if (ub > 0 && !tc::mbar_wait_bounded(bar(kBarAccEmpty + b), (ub - 1) & 1, a.wait_ns)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t d = tmem + b * kSBufC;
          for (int j = 0; j < NKB; ++j, ++gs) {
            const int s = (int)(gs % kStages);
            if (!tc::mbar_wait_bounded(bar(kBarBFull + s), (gs / kStages) & 1, a.wait_ns)) {
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t b0 = tc::smem_u32(sB + s * Sh::kBStage);
            const uint32_t aj = a0 + j * kABlk;
            if (PAIRED) {
              // block 0: even harmonics -> columns 0..N-1 of the buffer;
              // block 1: odd harmonics -> columns N..2N-1
              const int nk = j == 0 ? a.ke : a.ko;
              for (int ks = 0; ks < nk; ++ks)
                tc::mma_f16(d + (uint32_t)(j * N), tc::smem_desc_sw128(aj + ks * 32),
                            tc::smem_desc_sw128(b0 + ks * 32), kIdesc, ks > 0 ? 1u : 0u);
            } else {
              const int nk = min(4, a.ksteps - 4 * j);
              for (int ks = 0; ks < nk; ++ks)
                tc::mma_f16(d, tc::smem_desc_sw128(aj + ks * 32), tc::smem_desc_sw128(b0 + ks * 32),
                            kIdesc, (j > 0 || ks > 0) ? 1u : 0u);
            }
            tc::mma_commit(bar(kBarBEmpty + s));
            last = gs;
            any = true;
          }
          if (!ok) break;
          tc::mma_commit(bar(kBarAccFull + b));
        }
        if (!ok) {
          fail();
          break;
        }
        tc::mma_commit(bar(kBarAEmpty + ab));
      }
      // drain: every MMA is followed by its stage's commit before this
      // thread waits on anything else, so the last stage commit covers them all
      if (any) tc::mbar_wait_bounded(bar(kBarBEmpty + last % kStages), (last / kStages) & 1, kSWaitNs);
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int quarter = warp & 3, slice = warp >> 2;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    uint32_t g = 0;
    bool ok = true;
    // the patch's status and window are loaded one tile ahead, so that their
    // latency is not paid at the start of every tile
    auto load_sw = [&](int64_t tile, int &st, float &w) {
      const int64_t q = tile * kSTile + row;
      st = 0;
      w = 0.0f;
      if (tile < ntiles && q < a.P) {
        st = a.status[q];
        w = a.win[q];
      }
    };
    int st_next;
    float win_next;
    load_sw(blockIdx.x, st_next, win_next);
    for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      const int64_t p = tile * kSTile + row;
      const bool act = st_next > 0;
      const float win = act ? win_next : 0.0f;
      load_sw(tile + gridDim.x, st_next, win_next);
      // cmax[u]: largest value of column u of any 32-column block this slice
      // saw (a "class": the rows base + u of every block); the ring holds the
      // blocks whose maximum came within `win` of the running best
      float cmax[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) cmax[u] = -1.0f;
      float rbest = -1.0f, lost = -1.0f;
      float rv[kRing];
      int ri[kRing];
      int cnt = 0;
      for (int c = 0; c < nch; ++c, ++g) {
        const uint32_t b = g & 1, ub = g >> 1;
        const bool done = !*s_abort && tc::mbar_wait_bounded(bar(kBarAccFull + b), ub & 1, a.wait_ns);
        if (!__all_sync(0xffffffffu, done)) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        tc::fence_after_sync();
        // this warp's column slice of the buffer, hc = slice + chunk (mod
        // kTcSplit), so the same atom at consecutive angles (consecutive
        // chunks when a chunk is one angle; columns N/2 apart in a paired
        // chunk) lands in different slices: plain rows hc*S .. + S - 1 of the
        // chunk (S = N / kTcSplit); paired: pairs hc*S .. + S - 1, their even
        // parts in columns 0..N-1 and odd parts in N..2N-1
        const int hc = (slice + c) & (kTcSplit - 1);
        const uint32_t taddr = tmem + lane_base + b * kSBufC + (uint32_t)(hc * Sh::SLICE);
        const int nvalid = min(N, a.MR - c * N) - hc * Sh::SLICE;
#pragma unroll 1
        for (int piece = 0; piece < Sh::PIECES; ++piece) {
          const int nv = nvalid - piece * 32;  // valid columns of this block
          // long rows (four blocks per slice): the column maxima of a block
          // are taken after its maximum is known, and skipped when the vote
          // below allows it (measured on the 21 x 21 image sizes: 4.47 ->
          // 4.32 ms per launch; on the short layouts the deferred update
          // costs more than it saves)
          constexpr bool kSkip = NB > 2;
          float hm[2], f[2][16];
#pragma unroll
          for (int sub = 0; sub < 2; ++sub) {
            uint32_t v[16];
            tc::tmem_ld16(taddr + piece * 32 + sub * 16, v);
            if (PAIRED) {
              // pair value |E| + |O| = max(|score(r)|, |score(r + R/2)|)
              uint32_t o[16];
              tc::tmem_ld16(taddr + N + piece * 32 + sub * 16, o);
              tc::tmem_wait_ld();
#pragma unroll
              for (int u = 0; u < 16; ++u)
                f[sub][u] = fabsf(__uint_as_float(v[u])) + fabsf(__uint_as_float(o[u]));
            } else {
              tc::tmem_wait_ld();
#pragma unroll
              for (int u = 0; u < 16; ++u) f[sub][u] = fabsf(__uint_as_float(v[u]));
            }
            if (nv < 32) {
#pragma unroll
              for (int u = 0; u < 16; ++u)
                if (sub * 16 + u >= nv) f[sub][u] = -1.0f;
            }
            // block maximum of the 16 values as a tree of depth 3
            const float *g = f[sub];
            const float t0 = fmax3(g[0], g[1], g[2]), t1 = fmax3(g[3], g[4], g[5]);
            const float t2 = fmax3(g[6], g[7], g[8]), t3 = fmax3(g[9], g[10], g[11]);
            const float t4 = fmax3(g[12], g[13], g[14]);
            hm[sub] = fmax3(fmax3(t0, t1, t2), fmax3(t3, t4, g[15]), -1.0f);
            if constexpr (!kSkip) {
#pragma unroll
              for (int u = 0; u < 16; ++u) cmax[sub * 16 + u] = fmaxf(cmax[sub * 16 + u], g[u]);
            }
          }
          // the block maximum; a block within the window of the running best
          // (NaN-safe form) goes into the ring, and the value it overwrites,
          // if any, is bounded by `lost`
          const float bm = fmaxf(hm[0], hm[1]);
          const bool inwin = !(bm < rbest - win);
          if constexpr (kSkip) {
            // every value of a block below rbest - win is below the final
            // threshold (rbest only grows), so the block can set neither a
            // class bit nor the best class: a warp whose patches all have
            // this block outside their windows skips its column maxima
            if (__any_sync(0xffffffffu, act && inwin)) {
#pragma unroll
              for (int sub = 0; sub < 2; ++sub)
#pragma unroll
                for (int u = 0; u < 16; ++u)
                  cmax[sub * 16 + u] = fmaxf(cmax[sub * 16 + u], f[sub][u]);
            }
          }
          if (inwin) {
            const int sl = cnt & (kRing - 1);
            if (cnt >= kRing) lost = fmaxf(lost, rv[sl]);
            rv[sl] = bm;
            ri[sl] = c * N + hc * Sh::SLICE + piece * 32;
            ++cnt;
          }
          rbest = fmaxf(rbest, bm);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(kBarAccEmpty + b)) : "memory");
      }
      if (!ok) break;
      if (act) {
        // Every unit of this slice with value >= thr = best - win lies in a
        // block of the ring with maximum >= thr and in a class with
        // cmax >= thr: the refine expands (kept blocks) x (class mask).  What
        // is left out is below thr, or a block the list or the ring dropped
        // (their values go to disc).
        const float thr = rbest - win;
        float tv[kTcTop];
        int ti[kTcTop];
#pragma unroll
        for (int q = 0; q < kTcTop; ++q) {
          tv[q] = -INFINITY;
          ti[q] = -1;
        }
        float disc = fmaxf(thr, lost);
        const int nr = min(cnt, kRing);
#pragma unroll 1
        for (int i = 0; i < nr; ++i)
          if (rv[i] >= thr) topn_insert(tv, ti, disc, rv[i], ri[i]);
        uint32_t um = 0;
        int ubest = 0;
        float cb = -1.0f;
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          um |= (cmax[u] >= thr ? 1u : 0u) << u;
          if (cmax[u] > cb) {
            cb = cmax[u];
            ubest = u;
          }
        }
        // this slice's entries [slice * kTcTop, slice * kTcTop + kTcTop) of
        // the patch's kTcCand block slots, its class mask and best class
        int *ci = a.cand_idx + p * kTcCand + slice * kTcTop;
        float *cv = a.cand_val + p * kTcCand + slice * kTcTop;
        *reinterpret_cast<int4 *>(ci) = make_int4(ti[0], ti[1], ti[2], ti[3]);
        *reinterpret_cast<float4 *>(cv) = make_float4(tv[0], tv[1], tv[2], tv[3]);
        a.cand_disc[p * kTcSplit + slice] = disc;
        *reinterpret_cast<uint2 *>(a.cand_mask + p * 2 * kTcSplit + slice * 2) =
            make_uint2(um, (uint32_t)ubest);
      }
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kSCols);
}

}  // namespace

namespace {
template <bool PAIRED, int NB, int STAGES>
int launch_score_t(const ScoreArgs &a, const CUtensorMap &tmA, const CUtensorMap &tmB,
                   cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  int max_optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  constexpr int total = SShape<PAIRED, NB, STAGES>::total;
  if (total > max_optin) return RSC_ERR_UNSUPPORTED;
  auto kern = romp_score_kernel<PAIRED, NB, STAGES>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, total);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  const int64_t tiles = (a.P + kSTile - 1) / kSTile;
  const int64_t grid = tiles < nsm ? tiles : nsm;
  kern<<<(unsigned)grid, kSThreads, total, stream>>>(tmA, tmB, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return RSC_OK;
}
}  // namespace

int rsc_score_stage_options(int L, int paired, int *dflt, int *other) {
  // the instantiated ring depths; the first is the default.  A shallower ring
  // leaves shared memory for refine blocks of other stream groups on the same
  // SM (measured: 2 stages 1.4% faster on 10^6 patches at M = 64, R = 64 in
  // three groups, 3 stages 1.7% faster on the 21 x 21 image sizes in two)
  *dflt = 4;
  *other = L == kTcKst ? 2 : 3;
  (void)paired;
  return RSC_OK;
}

int rsc_launch_score(const ScoreArgs &a, const CUtensorMap &tmA, const CUtensorMap &tmB,
                     cudaStream_t stream) {
  if (a.P == 0) return RSC_OK;
  if (a.L == kTcKst && a.paired)
    return a.stages == 2 ? launch_score_t<true, 2, 2>(a, tmA, tmB, stream)
                         : launch_score_t<true, 2, 4>(a, tmA, tmB, stream);
  if (a.L == kTcKst)
    return a.stages == 2 ? launch_score_t<false, 2, 2>(a, tmA, tmB, stream)
                         : launch_score_t<false, 2, 4>(a, tmA, tmB, stream);
  if (a.L == kTcKstLong && !a.paired)
    return a.stages == 3 ? launch_score_t<false, 4, 3>(a, tmA, tmB, stream)
                         : launch_score_t<false, 4, 4>(a, tmA, tmB, stream);
  return RSC_ERR_UNSUPPORTED;
}
