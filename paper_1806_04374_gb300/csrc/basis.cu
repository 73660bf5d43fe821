// basis.cu -- the discrete steerable basis and the pixel -> coefficient
// projection (Sec. II-D and steps 1-2 of the proposed algorithm, Sec. II-E),
// and coding of whole images.
//
// rsc_basis_create builds, on the host in FP64: the circular N x N patch
// (pixels with rho <= N/2), Gaussian-ring radial profiles b_j(rho) times the
// circular harmonics e^{i k phi} (the synthetic workloads' radial profiles in
// place of the paper's annulus indicators of Eq. (basis-cont)), made
// orthonormal within each harmonic (Loewdin, G^{-1/2} from a Jacobi
// eigendecomposition of the real ring Gram matrix), and the analysis
// operator: the pseudo-inverse of the real synthesis matrix (one-sided
// Jacobi SVD, singular values up to 1e-3 of the largest treated as zero),
// which is the paper's (Phi^* Phi)^{-1} Phi^* whenever Phi^* Phi is
// invertible and its condition number is below 10^3.  The cutoff keeps the
// operator from amplifying pixel noise by more than 10^3 / sigma_max: at
// 21 x 21 pixels with J = 10, kmax = 12 the synthesis matrix has singular
// values down to 4e-8 of the largest, whose directions synthesise almost
// nothing and would otherwise dominate the coefficients.
// Readings: pixel (row, col) at x = col - c, y = c - row, phi = atan2(y, x);
// e^{i k phi} = 0 at the centre pixel for k != 0; ring centres
// r_j = j * spacing (default (N-1)/(2J)), ring width sigma (default 1 px).
//
// project_kernel gathers every stride-1 window of a list of images of
// different sizes (one launch, a prefix sum of patch counts maps a thread to
// its image) and multiplies it by the analysis operator, writing half
// spectra in the layout rsc_encode takes.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "rsc_internal.h"
#include "rsc_trace.h"
#include "tc_ptx.cuh"

#include <cuda_fp16.h>

struct rsc_basis {
  int N, J, kmax, H, npix, n, nout, nout_pad;
  int device;
  int2 *offs;    // device [npix] (dy, dx) of each masked pixel, row-major
  float *Po;     // device [npix][nout_pad]: half-spectrum outputs per pixel
  // tensor-core projection (npix <= 128, nout <= 128; null otherwise): the
  // operator transposed to [NP outputs][KP pixels] fp16, times 2^sb, as a hi
  // part and the lo part of what hi leaves
  uint16_t *Bt;  // device [2][NP][KP]
  int KP, NP, sb;
  // tensor-core projection of larger windows (128 < npix <= 512, n <= 256;
  // null otherwise): [2][256 packed outputs][KPw pixels] fp16, hi then lo,
  // times 2^sbw, streamed by TMA (map tmW: box 64 pixels x 256 outputs)
  uint16_t *Bw;
  int KPw, sbw;
  CUtensorMap tmW;
  int *err;      // device error word of the projection kernels (bounded waits)
  float *Xs;     // device [n][npix]: real synthesis matrix (packed columns), FP32
};

namespace {

// Cyclic Jacobi eigendecomposition of a symmetric n x n matrix (row-major,
// overwritten); V receives the eigenvectors as columns, w the eigenvalues.
void jacobi_eig(std::vector<double> &A, int n, std::vector<double> &V, std::vector<double> &w) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += A[i * n + j] * A[i * n + j];
        if (i != j) off += A[i * n + j] * A[i * n + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

// Pseudo-inverse of the m x n matrix X (column-major: X[c * m + r]) by
// one-sided (Hestenes) Jacobi SVD; returns P (n x m, row-major).
std::vector<double> pinv(std::vector<double> X, int m, int n, double rcond) {
  std::vector<double> V((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;  // column-major too
  for (int sweep = 0; sweep < 80; ++sweep) {
    double worst = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double al = 0.0, be = 0.0, ga = 0.0;
        const double *xp = &X[(size_t)p * m], *xq = &X[(size_t)q * m];
        for (int r = 0; r < m; ++r) {
          al += xp[r] * xp[r];
          be += xq[r] * xq[r];
          ga += xp[r] * xq[r];
        }
        if (al == 0.0 || be == 0.0) continue;
        const double rel = fabs(ga) / sqrt(al * be);
        worst = std::max(worst, rel);
        if (rel < 1e-15) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        double *wp = &X[(size_t)p * m], *wq = &X[(size_t)q * m];
        for (int r = 0; r < m; ++r) {
          const double a = wp[r], b = wq[r];
          wp[r] = c * a - s * b;
          wq[r] = s * a + c * b;
        }
        double *vp = &V[(size_t)p * n], *vq = &V[(size_t)q * n];
        for (int r = 0; r < n; ++r) {
          const double a = vp[r], b = vq[r];
          vp[r] = c * a - s * b;
          vq[r] = s * a + c * b;
        }
      }
    if (worst < 1e-15) break;
  }
  // X V = U S: column i of X is sigma_i u_i
  std::vector<double> sig(n);
  double smax = 0.0;
  for (int i = 0; i < n; ++i) {
    double s2 = 0.0;
    for (int r = 0; r < m; ++r) s2 += X[(size_t)i * m + r] * X[(size_t)i * m + r];
    sig[i] = sqrt(s2);
    smax = std::max(smax, sig[i]);
  }
  std::vector<double> P((size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i) {
    if (!(sig[i] > rcond * smax)) continue;
    const double inv2 = 1.0 / (sig[i] * sig[i]);
    for (int a = 0; a < n; ++a) {
      const double va = V[(size_t)i * n + a] * inv2;
      if (va == 0.0) continue;
      for (int r = 0; r < m; ++r) P[(size_t)a * m + r] += va * X[(size_t)i * m + r];
    }
  }
  return P;
}

struct ImageItem {
  const float *img;
  int h, w;
  int64_t first;  // index of the image's first patch
};

// One pass of project_kernel: outputs oc .. oc + W - 1 of every window of the
// block's tile, the operator's W columns staged in shared memory (npix x W
// floats) and read by all threads as broadcasts; each thread accumulates its
// window's W outputs over the pixels in order (FP32 FMA).
template <int W>
__device__ __forceinline__ void project_pass(float *sP, const float *Po, int npix, int nout_pad,
                                             int oc, const float *base, int w, const int2 *offs,
                                             float *out, int nout, bool vec) {
  __syncthreads();  // the previous pass is done with sP
  for (int i = threadIdx.x; i < npix * (W / 4); i += blockDim.x) {
    const int p = i / (W / 4), c = i - p * (W / 4);
    reinterpret_cast<float4 *>(sP)[i] =
        __ldg(reinterpret_cast<const float4 *>(Po + (size_t)p * nout_pad + oc) + c);
  }
  __syncthreads();
  if (!base) return;
  float acc[W];
#pragma unroll
  for (int u = 0; u < W; ++u) acc[u] = 0.0f;
  // pixels are loaded four at a time ahead of their FMAs (two warps per
  // scheduler do not hide a load's latency otherwise); the sums keep the
  // pixel order
  constexpr int kAhead = 4;
  int p = 0;
  for (; p + kAhead <= npix; p += kAhead) {
    float v[kAhead];
#pragma unroll
    for (int k = 0; k < kAhead; ++k) {
      const int2 o = __ldg(offs + p + k);
      v[k] = __ldg(base + (int64_t)o.x * w + o.y);
    }
#pragma unroll
    for (int k = 0; k < kAhead; ++k) {
      const float4 *row = reinterpret_cast<const float4 *>(sP + (p + k) * W);
#pragma unroll
      for (int u = 0; u < W / 4; ++u) {
        const float4 q = row[u];
        acc[4 * u] = fmaf(q.x, v[k], acc[4 * u]);
        acc[4 * u + 1] = fmaf(q.y, v[k], acc[4 * u + 1]);
        acc[4 * u + 2] = fmaf(q.z, v[k], acc[4 * u + 2]);
        acc[4 * u + 3] = fmaf(q.w, v[k], acc[4 * u + 3]);
      }
    }
  }
  for (; p < npix; ++p) {
    const int2 o = __ldg(offs + p);
    const float v = __ldg(base + (int64_t)o.x * w + o.y);
    const float4 *row = reinterpret_cast<const float4 *>(sP + p * W);
#pragma unroll
    for (int u = 0; u < W / 4; ++u) {
      const float4 q = row[u];
      acc[4 * u] = fmaf(q.x, v, acc[4 * u]);
      acc[4 * u + 1] = fmaf(q.y, v, acc[4 * u + 1]);
      acc[4 * u + 2] = fmaf(q.z, v, acc[4 * u + 2]);
      acc[4 * u + 3] = fmaf(q.w, v, acc[4 * u + 3]);
    }
  }
  if (vec && oc + W <= nout) {
#pragma unroll
    for (int u = 0; u < W; u += 4)
      *reinterpret_cast<float4 *>(out + oc + u) = make_float4(acc[u], acc[u + 1], acc[u + 2], acc[u + 3]);
  } else {
#pragma unroll
    for (int u = 0; u < W; ++u)
      if (oc + u < nout) out[oc + u] = acc[u];
  }
}

// Projection on the CUDA cores (windows of any size): one thread per window,
// 64 outputs per pass (a last pass of 32 when the padded output count asks
// for it), the operator slab in shared memory.
__global__ void __launch_bounds__(128) project_kernel(const ImageItem *items, int n_items,
                                                       int64_t P_total, int N, int npix,
                                                       const int2 *offs, const float *Po, int nout,
                                                       int nout_pad, float *coef) {
  extern __shared__ float sP[];
  const bool vec = (reinterpret_cast<uintptr_t>(coef) & 15) == 0 && (nout & 3) == 0;
  const int64_t ntiles = (P_total + blockDim.x - 1) / blockDim.x;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t g = t * blockDim.x + threadIdx.x;
    const float *base = nullptr;
    int w = 0;
    if (g < P_total) {
      int lo = 0, hi = n_items - 1;  // last item with first <= g
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first <= g) lo = mid; else hi = mid - 1;
      }
      const ImageItem it = items[lo];
      const int64_t local = g - it.first;
      const int nw = it.w - N + 1;
      const int r0 = (int)(local / nw), c0 = (int)(local - (int64_t)r0 * nw);
      base = it.img + (int64_t)r0 * it.w + c0;
      w = it.w;
    }
    float *out = coef + (g < P_total ? g : 0) * nout;
    int oc = 0;
    for (; oc + 64 <= nout_pad && oc < nout; oc += 64)
      project_pass<64>(sP, Po, npix, nout_pad, oc, base, w, offs, out, nout, vec);
    if (oc < nout) project_pass<32>(sP, Po, npix, nout_pad, oc, base, w, offs, out, nout, vec);
  }
}

// Projection on the tensor cores: a tile of 128 windows (one per TMEM lane)
// times the operator, coef = A Po with A the gathered window pixels.  fp16
// keeps 11 bits, so both operands are split, x = hi + lo (hi = fp16(x), lo =
// fp16(x - hi)), and the three products hi*hi + hi*lo + lo*hi are summed in the
// FP32 accumulator: about 2^-21 relative, FP32 accuracy for the coder.  Each
// window's pixels are scaled by a power of two 2^sa with max |x| 2^sa in
// [2^13, 2^14) and the operator by 2^sb, far from fp16's range limits; the
// result is multiplied back by 2^-(sa + sb) (exact).  Two groups of 128
// threads per CTA each own a tile, an A area and 128 TMEM columns; a group
// gathers its windows into 128-byte-swizzled K-major rows, one thread issues
// the 3 x KP/16 MMAs (M = 128, N = NP) and commits them to the group's
// mbarrier (bounded wait), and every thread reads its window's row back with
// tcgen05.ld and writes the half spectrum.
constexpr int kPjThreads = 256;
constexpr int kPjRows = 128;
constexpr int kPjBlkA = kPjRows * 128;  // one 64-pixel block of a 128-window tile
constexpr uint64_t kPjWaitNs = 2000000000ull;

struct PjLayout {
  int b_off, a_off, bar_off, total;
};
__host__ __device__ inline PjLayout pj_layout(int NP) {
  const int bblk = NP * 128;                   // one 64-pixel block of the operator
  const int b_bytes = 2 * 2 * bblk;            // hi, lo; two blocks each
  const int a_bytes = 2 * 2 * 2 * kPjBlkA;     // two groups; hi, lo; two blocks
  return PjLayout{0, b_bytes, b_bytes + a_bytes, b_bytes + a_bytes + 64 + 1024};
}

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kPjRows) : "memory");
}

__global__ void __launch_bounds__(kPjThreads, 1)
    project_tc_kernel(const ImageItem *items, int n_items, int64_t P_total, int N, int npix,
                      const int2 *offs, const uint16_t *Bt, int KP, int NP, int sb, int nout,
                      float *coef, int *err) {
  extern __shared__ unsigned char pj_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(pj_raw) + 1023) & ~uintptr_t(1023));
  const PjLayout Lo = pj_layout(NP);
  const int bblk = NP * 128;
  unsigned char *sB = smem + Lo.b_off;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lo.bar_off);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 2);
  volatile int *s_ok = reinterpret_cast<volatile int *>(bars + 2) + 1;  // [2]
  const int tid = threadIdx.x, warp = tid >> 5, g = tid >> 7, row = tid & 127;
  const int kchunks = KP / 8;  // 16-byte chunks of a row

  // operator hi / lo -> swizzled K-major tiles (row = output, 8 pixels a chunk)
  for (int i = tid; i < 2 * NP * kchunks; i += kPjThreads) {
    const int part = i / (NP * kchunks), rem = i - part * NP * kchunks;
    const int r = rem / kchunks, c = rem - r * kchunks;
    const uint4 v = *reinterpret_cast<const uint4 *>(Bt + ((size_t)part * NP + r) * KP + c * 8);
    *reinterpret_cast<uint4 *>(sB + part * 2 * bblk + (c >> 3) * bblk + r * 128 +
                               (((c & 7) ^ (r & 7)) << 4)) = v;
  }
  if (tid == 0) {
    tc::mbar_init(tc::smem_u32(bars), 1);
    tc::mbar_init(tc::smem_u32(bars + 1), 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), 2 * kPjRows);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const uint32_t bar = tc::smem_u32(bars + g);
  unsigned char *sA = smem + Lo.a_off + g * (2 * 2 * kPjBlkA);  // hi blocks, then lo blocks
  const uint32_t a_hi = tc::smem_u32(sA), a_lo = a_hi + 2 * kPjBlkA;
  const uint32_t b_hi = tc::smem_u32(sB), b_lo = b_hi + 2 * bblk;
  const uint32_t idesc = tc::idesc_f16_f32(kPjRows, NP);
  const uint32_t dcol = tmem + (uint32_t)(g * kPjRows);
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int64_t ntiles = (P_total + kPjRows - 1) / kPjRows;
  uint32_t iter = 0;
  bool alive = true;
  for (int64_t t = (int64_t)blockIdx.x * 2 + g; t < ntiles && alive;
       t += (int64_t)gridDim.x * 2, ++iter) {
    // ---- gather this thread's window, scale, split, write its A rows
    const int64_t p = t * kPjRows + row;
    const float *base = nullptr;
    int w = 0;
    float amax = 0.0f;
    if (p < P_total) {
      int lo = 0, hi = n_items - 1;  // last item with first <= p
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first <= p) lo = mid; else hi = mid - 1;
      }
      const ImageItem it = items[lo];
      const int64_t local = p - it.first;
      const int nw = it.w - N + 1;
      const int r0 = (int)(local / nw), c0 = (int)(local - (int64_t)r0 * nw);
      base = it.img + (int64_t)r0 * it.w + c0;
      w = it.w;
      for (int q = 0; q < npix; ++q) {
        const int2 o = __ldg(offs + q);
        amax = fmaxf(amax, fabsf(__ldg(base + (int64_t)o.x * w + o.y)));
      }
    }
    int ea = 0;
    (void)frexpf(amax, &ea);
    const int sa = 14 - (ea < -100 ? -100 : (ea > 127 ? 127 : ea));  // max |x| 2^sa < 2^14
    const float scale = ldexpf(1.0f, sa);
    for (int c = 0; c < kchunks; ++c) {
      uint32_t hv[4], lv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float x2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = c * 8 + 2 * u + h;
          float x = 0.0f;
          if (base && q < npix) {
            const int2 o = __ldg(offs + q);
            x = __ldg(base + (int64_t)o.x * w + o.y) * scale;
          }
          x2[h] = x;
        }
        const __half2 hh = __floats2half2_rn(x2[0], x2[1]);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn(x2[0] - hf.x, x2[1] - hf.y);
        hv[u] = *reinterpret_cast<const uint32_t *>(&hh);
        lv[u] = *reinterpret_cast<const uint32_t *>(&ll);
      }
      const int off = (c >> 3) * kPjBlkA + row * 128 + (((c & 7) ^ (row & 7)) << 4);
      *reinterpret_cast<uint4 *>(sA + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
      *reinterpret_cast<uint4 *>(sA + 2 * kPjBlkA + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    group_sync(g);
    tc::fence_after_sync();
    // ---- MMAs: hi*hi + hi*lo + lo*hi into the group's accumulator
    if (row == 0) {
      const int ks_n = KP / 16;
      for (int prod = 0; prod < 3; ++prod) {
        const uint32_t aa = prod == 2 ? a_lo : a_hi, bb = prod == 1 ? b_lo : b_hi;
        for (int ks = 0; ks < ks_n; ++ks) {
          const uint32_t ao = (ks >> 2) * kPjBlkA + (ks & 3) * 32;
          const uint32_t bo = (ks >> 2) * bblk + (ks & 3) * 32;
          tc::mma_f16(dcol, tc::smem_desc_sw128(aa + ao), tc::smem_desc_sw128(bb + bo), idesc,
                      (prod | ks) ? 1u : 0u);
        }
      }
      tc::mma_commit(bar);
      const bool done = tc::mbar_wait_bounded(bar, iter & 1, kPjWaitNs);
      if (!done && err) atomicCAS(err, 0, RSC_ERR_TIMEOUT);
      s_ok[g] = done ? 1 : 0;
    }
    group_sync(g);
    tc::fence_after_sync();
    if (!s_ok[g]) {
      alive = false;
      break;
    }
    // ---- read back and write the half spectrum, 32 columns at a time
    const float unscale = ldexpf(1.0f, -(sa + sb));
    float *out = coef + (p < P_total ? p : 0) * nout;
    for (int piece = 0; piece * 32 < NP; ++piece) {
      uint32_t v[32];
      tc::tmem_ld32(dcol + lane_base + piece * 32, v);
      tc::tmem_wait_ld();
      if (p < P_total) {
#pragma unroll
        for (int u = 0; u < 32; u += 4) {
          const int o = piece * 32 + u;
          if (o < nout)
            *reinterpret_cast<float4 *>(out + o) =
                make_float4(__uint_as_float(v[u]) * unscale, __uint_as_float(v[u + 1]) * unscale,
                            __uint_as_float(v[u + 2]) * unscale,
                            __uint_as_float(v[u + 3]) * unscale);
        }
      }
    }
    tc::fence_before_sync();
  }
  // a group whose wait gave up may still have MMAs in flight: wait (bounded)
  // before the accumulator columns are released
  if (!alive && row == 0) tc::mbar_wait_bounded(bar, (iter & 1), kPjWaitNs);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * kPjRows);
}

// Projection of larger windows (kTcKst < npix <= 512 pixels, n <= 256
// packed outputs, e.g. 21 x 21: 349 px -> 250) on the tensor cores.  The
// split operator (hi and lo fp16, [2][256 outputs][KPw pixels], packed output
// order, times 2^sbw) is too large for shared memory, so it streams from L2
// one 64-pixel K-block at a time.  Per CTA and tile of 128 windows:
//   * warps 0-3 (one thread per window) gather each K-block's 64 pixels,
//     scaled by 2^sa and split into hi and lo, into 128-byte-swizzled K-major
//     rows of a 2-stage A ring, then read the accumulator back and write the
//     half spectrum;
//   * warp 4 (one lane) loads the operator's K-block (hi and lo, 64 KB) into
//     a 2-stage B ring with TMA;
//   * warp 5 (one lane) issues hi*hi + hi*lo + lo*hi (3 x 4 MMAs, M = 128,
//     N = 256) per K-block into one 256-column TMEM accumulator.
// The gather warps' TMEM reads of tile t finish before they hand over the
// first A block of tile t + 1 (tcgen05 fences around that mbarrier), so the
// accumulator needs no second handshake.  Every wait is bounded.
constexpr int kPwThreads = 192;
constexpr int kPwBlkA = 128 * 128;     // one part (hi or lo) of an A K-block (bytes)
constexpr int kPwStageA = 2 * kPwBlkA;
constexpr int kPwBlkB = 256 * 128;     // one part of a B K-block: 256 outputs x 64 px
constexpr int kPwStageB = 2 * kPwBlkB;
constexpr int kPwStages = 2;
constexpr int kPwNP = 256;             // MMA N: packed outputs, padded
constexpr int kPwBarOff = kPwStages * (kPwStageA + kPwStageB);
constexpr int kPwSmem = kPwBarOff + 128 + 1024;
enum : int { kPwAFull = 0, kPwAEmpty = 2, kPwBFull = 4, kPwBEmpty = 6, kPwAcc = 8, kPwBars = 9 };

__global__ void __launch_bounds__(kPwThreads, 1)
    project_tcw_kernel(const __grid_constant__ CUtensorMap tmW, const ImageItem *items,
                       int n_items, int64_t P_total, int N, int npix, int nkb, const int2 *offs,
                       int J, int n, int sb, int nout, float *coef, int *err) {
  extern __shared__ unsigned char pw_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(pw_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *sA = smem;
  unsigned char *sB = smem + kPwStages * kPwStageA;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kPwBarOff);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + kPwBars);
  volatile int *s_abort = reinterpret_cast<volatile int *>(bars + kPwBars) + 1;
  const uint32_t bar0 = tc::smem_u32(bars);
  auto bar = [&](int i) { return bar0 + 8u * (uint32_t)i; };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < kPwStages; ++i) {
      tc::mbar_init(bar(kPwAFull + i), 4);  // one arrival per gather warp
      tc::mbar_init(bar(kPwAEmpty + i), 1);
      tc::mbar_init(bar(kPwBFull + i), 1);
      tc::mbar_init(bar(kPwBEmpty + i), 1);
    }
    tc::mbar_init(bar(kPwAcc), 1);
    *s_abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(s_tmem), kPwNP);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const int64_t ntiles = (P_total + 127) / 128;
  auto fail = [&]() {
    *s_abort = 1;
    if (err) atomicCAS(err, 0, RSC_ERR_TIMEOUT);
  };

  if (warp == 4) {
    // ------------------------------------------------------------ TMA (B)
    if (lane == 0) {
      uint32_t gj = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; ok && t < ntiles && !*s_abort; t += gridDim.x) {
        for (int j = 0; j < nkb; ++j, ++gj) {
          const int s = (int)(gj % kPwStages);
          if (gj >= (uint32_t)kPwStages &&
              !tc::mbar_wait_bounded(bar(kPwBEmpty + s), ((gj / kPwStages) - 1) & 1, kPjWaitNs)) {
            fail();
            ok = false;
            break;
          }
          const uint32_t dst = tc::smem_u32(sB + s * kPwStageB);
          tc::mbar_arrive_expect_tx(bar(kPwBFull + s), kPwStageB);
          tc::tma_load_2d(dst, &tmW, bar(kPwBFull + s), 64 * j, 0);
          tc::tma_load_2d(dst + kPwBlkB, &tmW, bar(kPwBFull + s), 64 * j, kPwNP);
        }
      }
      for (uint32_t i = (gj > (uint32_t)kPwStages ? gj - kPwStages : 0); i < gj; ++i)
        tc::mbar_wait_bounded(bar(kPwBFull + i % kPwStages), (i / kPwStages) & 1, kPjWaitNs);
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16_f32(128, kPwNP);
      uint32_t gj = 0, last = 0;
      bool any = false, ok = true;
      for (int64_t t = blockIdx.x; ok && t < ntiles && !*s_abort; t += gridDim.x) {
        for (int j = 0; j < nkb; ++j, ++gj) {
          const int s = (int)(gj % kPwStages);
          const uint32_t par = (gj / kPwStages) & 1;
          if (!tc::mbar_wait_bounded(bar(kPwAFull + s), par, kPjWaitNs) ||
              !tc::mbar_wait_bounded(bar(kPwBFull + s), par, kPjWaitNs)) {
            fail();
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t a_hi = tc::smem_u32(sA + s * kPwStageA), a_lo = a_hi + kPwBlkA;
          const uint32_t b_hi = tc::smem_u32(sB + s * kPwStageB), b_lo = b_hi + kPwBlkB;
          for (int prod = 0; prod < 3; ++prod) {
            const uint32_t aa = prod == 2 ? a_lo : a_hi, bb = prod == 1 ? b_lo : b_hi;
            for (int ks = 0; ks < 4; ++ks)
              tc::mma_f16(tmem, tc::smem_desc_sw128(aa + ks * 32), tc::smem_desc_sw128(bb + ks * 32),
                          idesc, (j | prod | ks) ? 1u : 0u);
          }
          tc::mma_commit(bar(kPwAEmpty + s));
          tc::mma_commit(bar(kPwBEmpty + s));
          last = gj;
          any = true;
          if (j == nkb - 1) tc::mma_commit(bar(kPwAcc));
        }
      }
      // every MMA is followed by its stage's commit: the last one covers all
      if (any)
        tc::mbar_wait_bounded(bar(kPwAEmpty + last % kPwStages), (last / kPwStages) & 1, kPjWaitNs);
    }
  } else if (warp < 4) {
    // ------------------------------------------------ gather and epilogue
    const int row = tid;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t gj = 0, it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++it) {
      const int64_t p = t * 128 + row;
      const float *base = nullptr;
      int w = 0;
      float amax = 0.0f;
      if (p < P_total) {
        int lo = 0, hi = n_items - 1;  // last item with first <= p
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (items[mid].first <= p) lo = mid; else hi = mid - 1;
        }
        const ImageItem itm = items[lo];
        const int64_t local = p - itm.first;
        const int nw = itm.w - N + 1;
        const int r0 = (int)(local / nw), c0 = (int)(local - (int64_t)r0 * nw);
        base = itm.img + (int64_t)r0 * itm.w + c0;
        w = itm.w;
        for (int q = 0; q < npix; ++q) {
          const int2 o = __ldg(offs + q);
          amax = fmaxf(amax, fabsf(__ldg(base + (int64_t)o.x * w + o.y)));
        }
      }
      int ea = 0;
      (void)frexpf(amax, &ea);
      const int sa = 14 - (ea < -100 ? -100 : (ea > 127 ? 127 : ea));  // max |x| 2^sa < 2^14
      const float scale = ldexpf(1.0f, sa);
      for (int j = 0; j < nkb; ++j, ++gj) {
        const int s = (int)(gj % kPwStages);
        const bool done = !*s_abort && (gj < (uint32_t)kPwStages ||
                                        tc::mbar_wait_bounded(bar(kPwAEmpty + s),
                                                              ((gj / kPwStages) - 1) & 1, kPjWaitNs));
        if (!__all_sync(0xffffffffu, done)) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        unsigned char *dst = sA + s * kPwStageA;
        for (int c = 0; c < 8; ++c) {
          uint32_t hv[4], lv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float x2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int q = j * 64 + c * 8 + 2 * u + h;
              float x = 0.0f;
              if (base && q < npix) {
                const int2 o = __ldg(offs + q);
                x = __ldg(base + (int64_t)o.x * w + o.y) * scale;
              }
              x2[h] = x;
            }
            const __half2 hh = __floats2half2_rn(x2[0], x2[1]);
            const float2 hf = __half22float2(hh);
            const __half2 ll = __floats2half2_rn(x2[0] - hf.x, x2[1] - hf.y);
            hv[u] = *reinterpret_cast<const uint32_t *>(&hh);
            lv[u] = *reinterpret_cast<const uint32_t *>(&ll);
          }
          const int off = row * 128 + ((c ^ (row & 7)) << 4);
          *reinterpret_cast<uint4 *>(dst + off) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<uint4 *>(dst + kPwBlkA + off) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar(kPwAFull + s)) : "memory");
      }
      if (!ok) break;
      // ---- read the accumulator back: packed output q -> half spectrum
      // index 2q (q < J: Re of k = 0, whose Im is 0) or J + q
      const bool done = !*s_abort && tc::mbar_wait_bounded(bar(kPwAcc), it & 1, kPjWaitNs);
      if (!__all_sync(0xffffffffu, done)) {
        if (lane == 0) fail();
        break;
      }
      tc::fence_after_sync();
      const float unscale = ldexpf(1.0f, -(sa + sb));
      float *out = coef + (p < P_total ? p : 0) * nout;
      for (int piece = 0; piece * 32 < n; ++piece) {
        uint32_t v[32];
        tc::tmem_ld32(tmem + lane_base + piece * 32, v);
        tc::tmem_wait_ld();
        if (p < P_total) {
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const int q = piece * 32 + u;
            if (q < n) out[q < J ? 2 * q : J + q] = __uint_as_float(v[u]) * unscale;
          }
        }
      }
      if (p < P_total)
        for (int jj = 0; jj < J; ++jj) out[2 * jj + 1] = 0.0f;
      tc::fence_before_sync();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, kPwNP);
}

// Multi-dictionary labelling (the paper's classifier, Sec. III-B): after
// dictionary c has coded every patch, a patch whose squared coding error is
// below the best so far takes label c (strict: ties keep the smaller index).
__global__ void label_update_kernel(int64_t P, int c, const float *__restrict__ rn2,
                                    float *__restrict__ best, int32_t *__restrict__ label) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float v = rn2[p];
    if (c == 0 || v < best[p]) {
      best[p] = v;
      label[p] = c;
    }
  }
}

// One block per coded image: its patches' labels counted in shared memory,
// then written as the image's row of the C-bin histogram.
__global__ void label_hist_kernel(const ImageItem *__restrict__ items, const int *__restrict__ orig,
                                  int N, const int32_t *__restrict__ label, int C,
                                  int32_t *__restrict__ hist) {
  extern __shared__ int counts[];
  for (int c = threadIdx.x; c < C; c += blockDim.x) counts[c] = 0;
  __syncthreads();
  const ImageItem it = items[blockIdx.x];
  const int64_t n = (int64_t)(it.h - N + 1) * (it.w - N + 1);
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) atomicAdd(&counts[label[it.first + q]], 1);
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x)
    hist[(int64_t)orig[blockIdx.x] * C + c] = counts[c];
}

// Reads and clears the basis's device error word (after a synchronisation).
int take_error(const rsc_basis *b) {
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, b->err, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v != 0) e = cudaMemset(b->err, 0, sizeof v);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return v;
}

int launch_project(const rsc_basis *b, const ImageItem *items_dev, int n_items, int64_t P_total,
                   float *coef, cudaStream_t st) {
  if (P_total == 0) return RSC_OK;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (b->Bt && (reinterpret_cast<uintptr_t>(coef) & 15) == 0) {
    const int total = pj_layout(b->NP).total;
    cudaError_t e = cudaFuncSetAttribute(project_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, total);
    if (e != cudaSuccess) return rsc_cuda_fail(e);
    const int64_t tile_pairs = ((P_total + kPjRows - 1) / kPjRows + 1) / 2;
    const unsigned grid = (unsigned)std::min<int64_t>(tile_pairs, (int64_t)nsm);
    project_tc_kernel<<<grid, kPjThreads, total, st>>>(items_dev, n_items, P_total, b->N,
                                                        b->npix, b->offs, b->Bt, b->KP, b->NP,
                                                        b->sb, b->nout, coef, b->err);
    e = cudaGetLastError();
    return e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
  }
  if (b->Bw) {
    cudaError_t e = cudaFuncSetAttribute(project_tcw_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kPwSmem);
    if (e != cudaSuccess) return rsc_cuda_fail(e);
    const int64_t tiles = (P_total + 127) / 128;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, (int64_t)nsm);
    project_tcw_kernel<<<grid, kPwThreads, kPwSmem, st>>>(
        b->tmW, items_dev, n_items, P_total, b->N, b->npix, b->KPw / 64, b->offs, b->J, b->n,
        b->sbw, b->nout, coef, b->err);
    e = cudaGetLastError();
    return e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
  }
  const int64_t blocks = (P_total + 127) / 128;
  const int shm = b->npix * 64 * (int)sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, shm);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  const int per_sm = std::max(1, std::min(4, (220 * 1024) / shm));  // by shared memory, registers
  const unsigned grid = (unsigned)std::min<int64_t>(blocks, (int64_t)nsm * per_sm);
  project_kernel<<<grid, 128, shm, st>>>(items_dev, n_items, P_total, b->N, b->npix, b->offs,
                                         b->Po, b->nout, b->nout_pad, coef);
  e = cudaGetLastError();
  return e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
}

}  // namespace

extern "C" {

int rsc_basis_create(int32_t N, int32_t J, int32_t kmax, double ring_width, double ring_spacing,
                     rsc_basis **out) {
  RscRange nvtx_range("rsc_basis_create");
  if (!out) return RSC_ERR_INVALID;
  *out = nullptr;
  if (N < 1 || J < 1 || kmax < 0) return RSC_ERR_INVALID;
  if (N > 64 || kmax > kMaxKmax || (int64_t)(kmax + 1) * J > kMaxEntries) return RSC_ERR_UNSUPPORTED;
  if (!(ring_width > 0.0)) ring_width = 1.0;
  if (!(ring_spacing > 0.0)) ring_spacing = (N - 1) / (2.0 * J);
  const int H = kmax + 1;
  const double c = (N - 1) / 2.0;
  std::vector<int2> offs;
  std::vector<double> rho, phi;
  for (int r = 0; r < N; ++r)
    for (int col = 0; col < N; ++col) {
      const double x = col - c, y = c - r;
      const double rr = sqrt(x * x + y * y);
      if (rr <= N / 2.0) {
        offs.push_back(make_int2(r, col));
        rho.push_back(rr);
        phi.push_back(atan2(y, x));
      }
    }
  const int npix = (int)offs.size();
  const int n = J + 2 * kmax * J;
  // orthonormalised radial profiles q_jk(pixel), one set for k = 0 and one
  // for k != 0 (the centre pixel is dropped there)
  std::vector<double> prof((size_t)npix * J);
  for (int p = 0; p < npix; ++p)
    for (int j = 0; j < J; ++j) {
      const double d = (rho[p] - ring_spacing * (j + 1)) / ring_width;
      prof[(size_t)p * J + j] = exp(-0.5 * d * d);
    }
  std::vector<double> q[2];
  for (int kk = 0; kk < 2; ++kk) {
    std::vector<double> G((size_t)J * J, 0.0), V, w;
    for (int p = 0; p < npix; ++p) {
      if (kk == 1 && rho[p] == 0.0) continue;
      for (int a = 0; a < J; ++a)
        for (int bb = 0; bb < J; ++bb) G[a * J + bb] += prof[(size_t)p * J + a] * prof[(size_t)p * J + bb];
    }
    jacobi_eig(G, J, V, w);
    for (int i = 0; i < J; ++i)
      if (!(w[i] > 0.0)) return RSC_ERR_INVALID;  // rings not independent on this grid
    std::vector<double> W((size_t)J * J, 0.0);  // G^{-1/2} = V diag(w^-1/2) V^T
    for (int a = 0; a < J; ++a)
      for (int bb = 0; bb < J; ++bb) {
        double s = 0.0;
        for (int i = 0; i < J; ++i) s += V[a * J + i] * V[bb * J + i] / sqrt(w[i]);
        W[a * J + bb] = s;
      }
    q[kk].assign((size_t)npix * J, 0.0);
    for (int p = 0; p < npix; ++p) {
      if (kk == 1 && rho[p] == 0.0) continue;
      for (int j = 0; j < J; ++j) {
        double s = 0.0;
        for (int a = 0; a < J; ++a) s += prof[(size_t)p * J + a] * W[a * J + j];
        q[kk][(size_t)p * J + j] = s;
      }
    }
  }
  // real synthesis matrix X (npix x n, column-major), packed coefficient order
  std::vector<double> X((size_t)n * npix, 0.0);
  for (int j = 0; j < J; ++j)
    for (int p = 0; p < npix; ++p) X[(size_t)j * npix + p] = q[0][(size_t)p * J + j];
  for (int k = 1; k <= kmax; ++k)
    for (int j = 0; j < J; ++j) {
      const int col = J + 2 * ((k - 1) * J + j);
      for (int p = 0; p < npix; ++p) {
        const double qq = q[1][(size_t)p * J + j];
        X[(size_t)col * npix + p] = M_SQRT2 * qq * cos(k * phi[p]);
        X[(size_t)(col + 1) * npix + p] = -M_SQRT2 * qq * sin(k * phi[p]);
      }
    }
  const std::vector<double> Pr = pinv(X, npix, n, 1e-3);  // n x npix
  // outputs: half spectrum [k][j][re, im]; packed k >= 1 slots carry sqrt(2)
  const int nout = 2 * H * J;
  const int nout_pad = (nout + 31) / 32 * 32;
  std::vector<float> Po((size_t)npix * nout_pad, 0.0f);
  for (int p = 0; p < npix; ++p) {
    for (int j = 0; j < J; ++j) Po[(size_t)p * nout_pad + 2 * j] = (float)Pr[(size_t)j * npix + p];
    for (int k = 1; k <= kmax; ++k)
      for (int j = 0; j < J; ++j) {
        const int row = J + 2 * ((k - 1) * J + j);
        const int o = 2 * (k * J + j);
        Po[(size_t)p * nout_pad + o] = (float)(Pr[(size_t)row * npix + p] * M_SQRT1_2);
        Po[(size_t)p * nout_pad + o + 1] = (float)(Pr[(size_t)(row + 1) * npix + p] * M_SQRT1_2);
      }
  }
  // tensor-core operator: [NP outputs][KP pixels], scaled by 2^sb (max entry
  // below 2^14), split into fp16 hi and lo
  const bool tc_ok = npix <= 128 && nout <= 128 && nout % 4 == 0;
  const int KP = (npix + 15) / 16 * 16, NP = (nout + 15) / 16 * 16;
  int sb = 0;
  std::vector<uint16_t> Bt;
  if (tc_ok) {
    std::vector<double> Pd((size_t)NP * KP, 0.0);
    double vmax = 0.0;
    for (int p = 0; p < npix; ++p) {
      for (int j = 0; j < J; ++j) Pd[(size_t)(2 * j) * KP + p] = Pr[(size_t)j * npix + p];
      for (int k = 1; k <= kmax; ++k)
        for (int j = 0; j < J; ++j) {
          const int row = J + 2 * ((k - 1) * J + j), o = 2 * (k * J + j);
          Pd[(size_t)o * KP + p] = Pr[(size_t)row * npix + p] * M_SQRT1_2;
          Pd[(size_t)(o + 1) * KP + p] = Pr[(size_t)(row + 1) * npix + p] * M_SQRT1_2;
        }
    }
    for (double v : Pd) vmax = std::max(vmax, fabs(v));
    int ev = 0;
    (void)frexp(vmax, &ev);
    sb = 14 - ev;
    Bt.assign((size_t)2 * NP * KP, 0);
    for (size_t i = 0; i < Pd.size(); ++i) {
      const double v = ldexp(Pd[i], sb);
      const __half hi = __float2half_rn((float)v);
      const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
      Bt[i] = *reinterpret_cast<const uint16_t *>(&hi);
      Bt[Pd.size() + i] = *reinterpret_cast<const uint16_t *>(&lo);
    }
  }
  // wide operator (packed output order; k >= 1 rows carry 1/sqrt2 like Po)
  const bool tcw_ok = !tc_ok && npix > 128 && npix <= 512 && n <= kPwNP;
  const int KPw = (npix + 63) / 64 * 64;
  int sbw = 0;
  std::vector<uint16_t> Bw;
  if (tcw_ok) {
    std::vector<double> Pd((size_t)kPwNP * KPw, 0.0);
    double vmax = 0.0;
    for (int q = 0; q < n; ++q)
      for (int p = 0; p < npix; ++p)
        Pd[(size_t)q * KPw + p] = Pr[(size_t)q * npix + p] * (q < J ? 1.0 : M_SQRT1_2);
    for (double v : Pd) vmax = std::max(vmax, fabs(v));
    int ev = 0;
    (void)frexp(vmax, &ev);
    sbw = 14 - ev;
    Bw.assign((size_t)2 * kPwNP * KPw, 0);
    for (size_t i = 0; i < Pd.size(); ++i) {
      const double v = ldexp(Pd[i], sbw);
      const __half hi = __float2half_rn((float)v);
      const __half lo = __float2half_rn((float)(v - (double)__half2float(hi)));
      Bw[i] = *reinterpret_cast<const uint16_t *>(&hi);
      Bw[Pd.size() + i] = *reinterpret_cast<const uint16_t *>(&lo);
    }
  }
  rsc_basis *b = new rsc_basis();
  memset(b, 0, sizeof *b);
  b->KPw = KPw;
  b->sbw = sbw;
  b->KP = KP;
  b->NP = NP;
  b->sb = sb;
  b->N = N;
  b->J = J;
  b->kmax = kmax;
  b->H = H;
  b->npix = npix;
  b->n = n;
  b->nout = nout;
  b->nout_pad = nout_pad;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaMalloc(&b->offs, offs.size() * sizeof(int2));
  if (e == cudaSuccess) e = cudaMalloc(&b->Po, Po.size() * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->offs, offs.data(), offs.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->Po, Po.data(), Po.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
  if (e == cudaSuccess && tc_ok) e = cudaMalloc(&b->Bt, Bt.size() * sizeof(uint16_t));
  if (e == cudaSuccess && tc_ok)
    e = cudaMemcpy(b->Bt, Bt.data(), Bt.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  std::vector<float> Xf(X.begin(), X.end());  // [n][npix] (column-major X)
  if (e == cudaSuccess) e = cudaMalloc(&b->Xs, Xf.size() * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->Xs, Xf.data(), Xf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && tcw_ok) e = cudaMalloc(&b->Bw, Bw.size() * sizeof(uint16_t));
  if (e == cudaSuccess && tcw_ok)
    e = cudaMemcpy(b->Bw, Bw.data(), Bw.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  int rc = RSC_OK;
  if (e == cudaSuccess && tcw_ok) rc = rsc_encode_rows_map(&b->tmW, b->Bw, 2 * kPwNP, kPwNP, KPw);
  if (e != cudaSuccess || rc != RSC_OK) {
    cudaFree(b->offs);
    cudaFree(b->Po);
    cudaFree(b->err);
    cudaFree(b->Bt);
    cudaFree(b->Bw);
    cudaFree(b->Xs);
    delete b;
    if (rc != RSC_OK) return rc;
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return RSC_ERR_OOM;
    }
    return rsc_cuda_fail(e);
  }
  *out = b;
  return RSC_OK;
}

int rsc_basis_destroy(rsc_basis *b) {
  if (!b) return RSC_OK;
  cudaFree(b->offs);
  cudaFree(b->Po);
  cudaFree(b->err);
  cudaFree(b->Bt);
  cudaFree(b->Bw);
  cudaFree(b->Xs);
  delete b;
  return RSC_OK;
}

int rsc_basis_info(const rsc_basis *b, int32_t *npix, int32_t *n) {
  if (!b) return RSC_ERR_INVALID;
  if (npix) *npix = b->npix;
  if (n) *n = b->n;
  return RSC_OK;
}

int rsc_project(const rsc_basis *b, const float *image, int32_t h, int32_t w, float *coef,
                void *stream) {
  RscRange nvtx_range("rsc_project");
  if (!b || h < 0 || w < 0) return RSC_ERR_INVALID;
  if (h < b->N || w < b->N) return RSC_OK;  // no complete window
  if (!image || !coef) return RSC_ERR_INVALID;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != b->device) return RSC_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ImageItem it{image, h, w, 0};
  ImageItem *d_it = nullptr;
  e = rsc_scratch_alloc(reinterpret_cast<void **>(&d_it), sizeof(ImageItem), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_it, &it, sizeof it, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  const int64_t P = (int64_t)(h - b->N + 1) * (w - b->N + 1);
  int rc = launch_project(b, d_it, 1, P, coef, st);
  rsc_scratch_free(d_it, st);
  // the host copy of `it` must outlive the async copy
  e = cudaStreamSynchronize(st);
  if (rc == RSC_OK && e != cudaSuccess) rc = rsc_cuda_fail(e);
  if (rc == RSC_OK) rc = take_error(b);
  return rc;
}

int rsc_encode_images(const rsc_dict *dict, const rsc_basis *b, const float *const *images,
                      const int32_t *h, const int32_t *w, int32_t n_images, int32_t K,
                      int32_t prec, int32_t *atom, int32_t *angle_idx, float *angle,
                      double *coef, float *resid_norm2, void *stream) {
  RscRange nvtx_range("rsc_encode_images");
  if (!dict || !b || n_images < 0 || (n_images > 0 && (!images || !h || !w)))
    return RSC_ERR_INVALID;
  if (b->J != dict->J || b->kmax != dict->kmax) return RSC_ERR_INVALID;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != b->device || dev != dict->device) return RSC_ERR_INVALID;
  std::vector<ImageItem> items;
  int64_t P = 0;
  for (int i = 0; i < n_images; ++i) {
    if (h[i] < 0 || w[i] < 0) return RSC_ERR_INVALID;
    if (h[i] < b->N || w[i] < b->N) continue;
    if (!images[i]) return RSC_ERR_INVALID;
    items.push_back(ImageItem{images[i], h[i], w[i], P});
    P += (int64_t)(h[i] - b->N + 1) * (w[i] - b->N + 1);
  }
  if (P == 0) return RSC_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t bI = (items.size() * sizeof(ImageItem) + 255) & ~(size_t)255;
  unsigned char *scratch = nullptr;
  e = rsc_scratch_alloc(reinterpret_cast<void **>(&scratch), bI + (size_t)P * b->nout * 4, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  ImageItem *d_items = reinterpret_cast<ImageItem *>(scratch);
  float *xc = reinterpret_cast<float *>(scratch + bI);
  int rc = RSC_OK;
  e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(ImageItem),
                      cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = rsc_cuda_fail(e);
  if (rc == RSC_OK) rc = launch_project(b, d_items, (int)items.size(), P, xc, st);
  if (rc == RSC_OK)
    rc = rsc_encode(dict, xc, P, K, prec, atom, angle_idx, angle, coef, resid_norm2, stream);
  rsc_scratch_free(scratch, st);
  // the host work list must outlive its async copy
  e = cudaStreamSynchronize(st);
  if (rc == RSC_OK && e != cudaSuccess) rc = rsc_cuda_fail(e);
  if (rc == RSC_OK) rc = take_error(b);
  return rc;
}

int rsc_classify_images(const rsc_dict *const *dicts, int32_t C, const rsc_basis *b,
                        const float *const *images, const int32_t *h, const int32_t *w,
                        int32_t n_images, int32_t K, int32_t prec, int32_t *labels,
                        int32_t *hist, void *stream) {
  RscRange nvtx_range("rsc_classify_images");
  if (!dicts || C < 1 || C > 4096 || !b || n_images < 0 || !hist ||
      (n_images > 0 && (!images || !h || !w)) || K < 1 || K > kMaxK)
    return RSC_ERR_INVALID;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != b->device) return RSC_ERR_INVALID;
  for (int c = 0; c < C; ++c)
    if (!dicts[c] || dicts[c]->J != b->J || dicts[c]->kmax != b->kmax || dicts[c]->device != dev)
      return RSC_ERR_INVALID;
  std::vector<ImageItem> items;
  std::vector<int> orig;
  int64_t P = 0;
  for (int i = 0; i < n_images; ++i) {
    if (h[i] < 0 || w[i] < 0) return RSC_ERR_INVALID;
    if (h[i] < b->N || w[i] < b->N) continue;
    if (!images[i]) return RSC_ERR_INVALID;
    items.push_back(ImageItem{images[i], h[i], w[i], P});
    orig.push_back(i);
    P += (int64_t)(h[i] - b->N + 1) * (w[i] - b->N + 1);
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(hist, 0, (size_t)n_images * C * sizeof(int32_t), st);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (P == 0) return RSC_OK;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t bI = al(items.size() * sizeof(ImageItem)), bO = al(orig.size() * sizeof(int));
  const size_t bX = al((size_t)P * b->nout * 4), bA = al((size_t)P * K * 4),
               bC = al((size_t)P * K * 8), bP = al((size_t)P * 4);
  unsigned char *scratch = nullptr;
  e = rsc_scratch_alloc(reinterpret_cast<void **>(&scratch), bI + bO + bX + 2 * bA + bC + 3 * bP, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  unsigned char *q = scratch;
  auto take = [&](size_t n) {
    unsigned char *r = q;
    q += n;
    return r;
  };
  ImageItem *d_items = reinterpret_cast<ImageItem *>(take(bI));
  int *d_orig = reinterpret_cast<int *>(take(bO));
  float *xc = reinterpret_cast<float *>(take(bX));
  int32_t *s_atom = reinterpret_cast<int32_t *>(take(bA));
  int32_t *s_ang = reinterpret_cast<int32_t *>(take(bA));
  double *s_coef = reinterpret_cast<double *>(take(bC));
  float *s_rn2 = reinterpret_cast<float *>(take(bP));
  float *s_best = reinterpret_cast<float *>(take(bP));
  int32_t *s_label = reinterpret_cast<int32_t *>(take(bP));
  int32_t *lab = labels ? labels : s_label;
  int rc = RSC_OK;
  e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(ImageItem),
                      cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_orig, orig.data(), orig.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = rsc_cuda_fail(e);
  if (rc == RSC_OK) rc = launch_project(b, d_items, (int)items.size(), P, xc, st);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<int64_t>((P + 255) / 256, (int64_t)nsm * 8);
  for (int c = 0; c < C && rc == RSC_OK; ++c) {
    rc = rsc_encode(dicts[c], xc, P, K, prec, s_atom, s_ang, nullptr, s_coef, s_rn2, stream);
    if (rc == RSC_OK) {
      label_update_kernel<<<grid, 256, 0, st>>>(P, c, s_rn2, s_best, lab);
      e = cudaGetLastError();
      if (e != cudaSuccess) rc = rsc_cuda_fail(e);
    }
  }
  if (rc == RSC_OK) {
    label_hist_kernel<<<(unsigned)items.size(), 256, (size_t)C * sizeof(int), st>>>(
        d_items, d_orig, b->N, lab, C, hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) rc = rsc_cuda_fail(e);
  }
  rsc_scratch_free(scratch, st);
  // the host work lists must outlive their async copies
  e = cudaStreamSynchronize(st);
  if (rc == RSC_OK && e != cudaSuccess) rc = rsc_cuda_fail(e);
  if (rc == RSC_OK) rc = take_error(b);
  return rc;
}

}  // extern "C"

int rsc_images_scratch_bytes(const rsc_basis *b, int64_t P, int32_t n_images, uint64_t *bytes) {
  if (!b || !bytes || P < 0 || n_images < 0) return RSC_ERR_INVALID;
  // as rsc_encode_images takes it: the work list (256-byte aligned), then the
  // projected windows
  const uint64_t bI = ((uint64_t)n_images * sizeof(ImageItem) + 255) & ~(uint64_t)255;
  *bytes = P > 0 ? bI + (uint64_t)P * b->nout * 4 : 0;
  return RSC_OK;
}

int rsc_basis_internals(const rsc_basis *b, rsc_basis_view *v) {
  if (!b || !v) return RSC_ERR_INVALID;
  *v = rsc_basis_view{b->device, b->npix, b->n, b->J, b->nout, b->Xs};
  return RSC_OK;
}
