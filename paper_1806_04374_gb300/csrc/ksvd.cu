// ksvd.cu -- the rotational K-SVD dictionary update (inner loop of the
// R-K-SVD pseudocode, Fig. "code", Sec. II-C) on the GPU.
//
// For atom m, every patch whose code uses m at angle r0 contributes the
// column y = S_{-r0}(x_p - D_aug b_p), b_p being the patch's code with the
// (m, r0) entry removed -- equivalently y = S_{-r0} e_p + a_{i0} d_m with the
// full coding residual e_p = x_p - sum_i a_i S_{r_i} d_{m_i}.  The new atom is
// the first left singular vector of [y ...], i.e. the leading eigenvector of
// C_m = sum y y^T.  Every atom is updated from the same (old) dictionary and
// the same codes.  Readings: a repeated atom uses its occurrence with the
// largest |weight| (ties: earliest); an unused atom is reset to the
// unit-normalised patch with the largest coding error (successive patches in
// descending error for several, ties: smaller index); the eigenvector's
// largest-magnitude packed entry is made positive.
//
// Kernels: per patch (count samples per atom, fill the per-atom sample lists,
// packed FP32 residuals and coding errors); per atom kCovSplit CTAs
// accumulating C_m over slices of its samples (4 x 4 register tiles, FP32
// partial sums over 32 samples folded into FP64, FP64 atomics) and one CTA
// running an FP64 power iteration from the old atom; one CTA for the resets.  All
// vectors are packed reals (k = 0 real parts, sqrt(2) Re/Im of k >= 1).
#include <math.h>

#include <algorithm>

#include "rsc_internal.h"

namespace {

constexpr int kCovThreads = 256;
constexpr int kCovBatch = 32;
constexpr int kEigThreads = 256;
constexpr int kMaxPacked = 2 * kMaxEntries;

struct KsvdArgs {
  const float *x;
  int64_t P;
  int K, M, J, H, R, n, ldE;
  const float *d;   // [M][H][J][2]
  const float *tw;  // [4][H][R]
  const int32_t *atom;
  const int32_t *angle;
  const double *coef;
  float *E;         // [P][ldE] packed residuals
  float *err;       // [P]
  int *count;       // [M]
  int *offset;      // [M + 1]
  int *cursor;      // [M]
  int2 *samples;    // [sum count] (patch, occurrence)
  double *C;        // [M][n][n]
  float *new_coef;  // [M][H][J][2]
  int32_t *n_used;  // [M] or null
  // the patches of largest coding error (descending, ties: smaller index),
  // unit-normalised, for the reset of unused atoms
  int ntop;         // entries of the list
  int top_needed;   // 1: list only as long as the atoms with count 0 need (one rank)
  float *top_err;   // [ntop]
  int64_t *top_idx; // [ntop] patch index (-1: none)
  float *top_vec;   // [ntop][H][J][2]
};

constexpr int kTopMax = 64;  // patches kept for the resets (unused atoms beyond: unchanged)

// Occurrence i of patch p is the one that represents its atom (largest
// |weight| among the occurrences of that atom, ties: earliest).
__device__ __forceinline__ bool chosen(const KsvdArgs &a, int64_t p, int i) {
  const int m = a.atom[p * a.K + i];
  if (m < 0) return false;
  const double w = fabs(a.coef[p * a.K + i]);
  for (int q = 0; q < a.K; ++q) {
    if (q == i || a.atom[p * a.K + q] != m) continue;
    const double v = fabs(a.coef[p * a.K + q]);
    if (v > w || (v == w && q < i)) return false;
  }
  return true;
}

__global__ void ksvd_count_kernel(const KsvdArgs a) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.P;
       p += (int64_t)gridDim.x * blockDim.x)
    for (int i = 0; i < a.K; ++i)
      if (chosen(a, p, i)) atomicAdd(&a.count[a.atom[p * a.K + i]], 1);
}

__global__ void ksvd_scan_kernel(const KsvdArgs a) {
  if (threadIdx.x == 0) {
    int s = 0;
    for (int m = 0; m < a.M; ++m) {
      a.offset[m] = s;
      a.cursor[m] = s;
      s += a.count[m];
      if (a.n_used) a.n_used[m] = a.count[m];
    }
    a.offset[a.M] = s;
  }
}

// Fills the sample lists and writes each patch's packed FP32 residual.
__global__ void ksvd_fill_kernel(const KsvdArgs a) {
  const int J = a.J, H = a.H, HJ = H * J, R = a.R;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.P;
       p += (int64_t)gridDim.x * blockDim.x) {
    for (int i = 0; i < a.K; ++i)
      if (chosen(a, p, i)) {
        const int slot = atomicAdd(&a.cursor[a.atom[p * a.K + i]], 1);
        a.samples[slot] = make_int2((int)p, i);
      }
    const float2 *xp = reinterpret_cast<const float2 *>(a.x + p * (int64_t)(2 * HJ));
    float *ep = a.E + p * (int64_t)a.ldE;
    float n2 = 0.0f;
    for (int e = 0; e < HJ; ++e) {
      const int k = e / J;
      float2 v = xp[e];
      float re = v.x, im = k ? v.y : 0.0f;
      for (int i = 0; i < a.K; ++i) {
        const int m = a.atom[p * a.K + i];
        if (m < 0) continue;
        const int r = a.angle[p * a.K + i];
        const float c = a.tw[(0 * H + k) * R + r], s = a.tw[(2 * H + k) * R + r];
        const float2 dv = reinterpret_cast<const float2 *>(a.d)[(size_t)m * HJ + e];
        const float dim = k ? dv.y : 0.0f;
        const float w = (float)a.coef[p * a.K + i];
        re = fmaf(-w, fmaf(c, dv.x, s * dim), re);
        im = fmaf(-w, fmaf(c, dim, -s * dv.x), im);
      }
      if (k == 0) {
        ep[e] = re;
        n2 = fmaf(re, re, n2);
      } else {
        const int q = 2 * e - J;
        ep[q] = 1.41421356237309515f * re;
        ep[q + 1] = 1.41421356237309515f * im;
        n2 = fmaf(2.0f * re, re, fmaf(2.0f * im, im, n2));
      }
    }
    a.err[p] = n2;
  }
}

// C_m = sum over the atom's samples of y y^T.  The samples of atom m are
// split over kCovSplit CTAs; each thread owns 4 x 4 tiles of the upper
// triangle (two float4 reads of a sample row feed 16 FMAs), sums 32 samples
// in FP32, folds them into FP64, and adds its tiles to C with FP64 atomics
// (C starts at zero).
constexpr int kCovSplit = 8;

__global__ void __launch_bounds__(kCovThreads) ksvd_cov_kernel(const KsvdArgs a) {
  extern __shared__ __align__(16) float ysm[];  // kCovBatch rows of ldy floats
  const int m = blockIdx.x / kCovSplit, part = blockIdx.x - m * kCovSplit;
  const int n = a.n, J = a.J, H = a.H, HJ = H * J, R = a.R;
  const int nb4 = (n + 3) / 4, ldy = 4 * nb4 + 4;  // +4: rows start in different banks
  auto ys = [&](int s, int q) -> float & { return ysm[s * ldy + q]; };
  const int beg0 = a.offset[m], cnt = a.offset[m + 1] - beg0;
  const int per = (cnt + kCovSplit - 1) / kCovSplit;
  const int beg = beg0 + part * per, end = min(beg0 + cnt, beg + per);
  if (beg >= end) return;
  double *Cm = a.C + (size_t)m * n * n;
  const int ntiles = nb4 * (nb4 + 1) / 2;
  for (int t = threadIdx.x; t - threadIdx.x < ntiles; t += kCovThreads) {
    // tile (bi, bj), bi <= bj, of the upper triangle (row bi starts at
    // bi*nb4 - bi(bi-1)/2)
    int bi = -1, bj = -1;
    if (t < ntiles) {
      int lo = 0, hi = nb4 - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mid * nb4 - mid * (mid - 1) / 2 <= t) lo = mid; else hi = mid - 1;
      }
      bi = lo;
      bj = bi + (t - (bi * nb4 - bi * (bi - 1) / 2));
    }
    double acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0.0;
    for (int b0 = beg; b0 < end; b0 += kCovBatch) {
      const int nb = min(kCovBatch, end - b0);
      __syncthreads();
      // build y for the batch: y = S_{-r0} e_p + a_{i0} d_m (packed; zero pad)
      for (int w = threadIdx.x; w < nb * ldy; w += blockDim.x) ysm[w] = 0.0f;
      __syncthreads();
      for (int w = threadIdx.x; w < nb * HJ; w += blockDim.x) {
        const int s = w / HJ, e = w - s * HJ;
        const int2 smp = a.samples[b0 + s];
        const int64_t p = smp.x;
        const int i0 = smp.y;
        const int r0 = a.angle[p * a.K + i0];
        // the code entry of (m, r0): every occurrence of that pair (Fig.
        // "code" zeroes the whole entry b_{r0}[m])
        double wsum = 0.0;
        for (int i = 0; i < a.K; ++i)
          if (a.atom[p * a.K + i] == m && a.angle[p * a.K + i] == r0) wsum += a.coef[p * a.K + i];
        const float w0 = (float)wsum;
        const int k = e / J;
        const float *ep = a.E + p * (int64_t)a.ldE;
        const float2 dv = reinterpret_cast<const float2 *>(a.d)[(size_t)m * HJ + e];
        if (k == 0) {
          ys(s, e) = ep[e] + w0 * dv.x;
        } else {
          const int q = 2 * e - J;
          const float re = ep[q], im = ep[q + 1];
          // S_{-theta}: harmonic k times exp(+i k theta)
          const float c = a.tw[(0 * H + k) * R + r0], sn = a.tw[(2 * H + k) * R + r0];
          ys(s, q) = fmaf(re, c, -im * sn) + 1.41421356237309515f * w0 * dv.x;
          ys(s, q + 1) = fmaf(re, sn, im * c) + 1.41421356237309515f * w0 * dv.y;
        }
      }
      __syncthreads();
      if (bi >= 0) {
        float part16[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) part16[u] = 0.0f;
        for (int s = 0; s < nb; ++s) {
          const float4 yi = *reinterpret_cast<const float4 *>(&ysm[s * ldy + 4 * bi]);
          const float4 yj = *reinterpret_cast<const float4 *>(&ysm[s * ldy + 4 * bj]);
          const float vi[4] = {yi.x, yi.y, yi.z, yi.w}, vj[4] = {yj.x, yj.y, yj.z, yj.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) part16[u * 4 + v] = fmaf(vi[u], vj[v], part16[u * 4 + v]);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] += (double)part16[u];
      }
    }
    if (bi >= 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int i = 4 * bi + u, j = 4 * bj + v;
          if (i < n && j < n && i <= j) {
            atomicAdd(Cm + (size_t)i * n + j, acc[u * 4 + v]);
            if (i != j) atomicAdd(Cm + (size_t)j * n + i, acc[u * 4 + v]);
          }
        }
    }
  }
}

__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// Leading eigenvector of C_m by FP64 power iteration from the old atom.
__global__ void __launch_bounds__(kEigThreads) ksvd_eig_kernel(const KsvdArgs a, int max_iter) {
  extern __shared__ __align__(16) double es[];
  const int m = blockIdx.x;
  const int n = a.n, J = a.J, H = a.H, HJ = H * J;
  if (a.count[m] == 0) {  // unused: the old atom, unless the reset replaces it
    for (int i = threadIdx.x; i < 2 * HJ; i += blockDim.x)
      a.new_coef[(size_t)m * HJ * 2 + i] = a.d[(size_t)m * HJ * 2 + i];
    return;
  }
  double *Cs = es;                 // n * n
  double *u = Cs + n * n;          // n
  double *v = u + n;               // n
  double *red = v + n;             // 32
  const double *Cm = a.C + (size_t)m * n * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) Cs[i] = Cm[i];
  // start: the old atom, packed
  for (int e = threadIdx.x; e < HJ; e += blockDim.x) {
    const int k = e / J;
    const float2 dv = reinterpret_cast<const float2 *>(a.d)[(size_t)m * HJ + e];
    if (k == 0) {
      u[e] = dv.x;
    } else {
      u[2 * e - J] = 1.4142135623730951 * dv.x;
      u[2 * e - J + 1] = 1.4142135623730951 * dv.y;
    }
  }
  __syncthreads();
  double lam_old = 0.0;
  for (int it = 0; it < max_iter; ++it) {
    double loc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s = fma(Cs[i * n + j], u[j], s);
      v[i] = s;
      loc = fma(s, s, loc);
    }
    const double nv2 = block_sum(loc, red);
    double dot = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) dot = fma(v[i], u[i], dot);
    const double lam = block_sum(dot, red);  // Rayleigh quotient (u unit)
    const double inv = nv2 > 0.0 ? 1.0 / sqrt(nv2) : 0.0;
    double dif = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double nu = v[i] * inv;
      dif = fma(nu - u[i], nu - u[i], dif);
      u[i] = nu;
    }
    const double d2 = block_sum(dif, red);
    if (nv2 == 0.0) break;
    if (it > 0 && d2 < 1e-26 && fabs(lam - lam_old) <= 1e-15 * fabs(lam)) break;
    lam_old = lam;
  }
  __syncthreads();
  // sign: the largest-magnitude entry positive (first index on ties)
  if (threadIdx.x == 0) {
    int arg = 0;
    for (int i = 1; i < n; ++i)
      if (fabs(u[i]) > fabs(u[arg])) arg = i;
    red[0] = u[arg] < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  const double sg = red[0];
  float *out = a.new_coef + (size_t)m * HJ * 2;
  for (int e = threadIdx.x; e < HJ; e += blockDim.x) {
    const int k = e / J;
    if (k == 0) {
      out[2 * e] = (float)(sg * u[e]);
      out[2 * e + 1] = 0.0f;
    } else {
      out[2 * e] = (float)(sg * u[2 * e - J] * 0.7071067811865476);
      out[2 * e + 1] = (float)(sg * u[2 * e - J + 1] * 0.7071067811865476);
    }
  }
}

// The a.ntop patches of largest coding error, in descending error (ties:
// smaller index), each unit-normalised (one CTA of 1024 threads).
__global__ void ksvd_top_kernel(const KsvdArgs a) {
  __shared__ float bv[1024];
  __shared__ long long bi[1024];
  __shared__ float prev_e;
  __shared__ long long prev_i;
  __shared__ double nrm;
  const int J = a.J, HJ = a.H * J;
  __shared__ int ntop;
  if (threadIdx.x == 0) {
    prev_e = INFINITY;
    prev_i = -1;
    int n = a.ntop;
    if (a.top_needed) {  // the counts are final: as many entries as unused atoms
      int unused = 0;
      for (int m = 0; m < a.M; ++m) unused += a.count[m] == 0;
      n = min(n, unused);
      for (int t = n; t < a.ntop; ++t) a.top_idx[t] = -1;
    }
    ntop = n;
  }
  __syncthreads();
  for (int t = 0; t < ntop; ++t) {
    // the t-th entry is the largest (error, then smaller index) below the
    // previous one in that order
    const float pe = prev_e;
    const long long pi = prev_i;
    float best = -1.0f;
    long long bp = -1;
    for (int64_t p = threadIdx.x; p < a.P; p += blockDim.x) {
      const float e = a.err[p];
      if (!(e < pe || (e == pe && p > pi))) continue;
      if (e > best) {
        best = e;
        bp = p;
      }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = bp;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        const float o = bv[threadIdx.x + s];
        const long long oi = bi[threadIdx.x + s];
        if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi >= 0 &&
                                    (bi[threadIdx.x] < 0 || oi < bi[threadIdx.x]))) {
          bv[threadIdx.x] = o;
          bi[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    const long long p = bi[0];
    __syncthreads();
    if (threadIdx.x == 0) {
      if (p >= 0) {
        prev_e = bv[0];
        prev_i = p;
      }
      a.top_idx[t] = p;
      a.top_err[t] = p >= 0 ? bv[0] : -1.0f;
      double s2 = 0.0;
      if (p >= 0) {
        const float *xp = a.x + p * (int64_t)(2 * HJ);
        for (int e = 0; e < HJ; ++e) {
          const double re = xp[2 * e], im = e < J ? 0.0 : xp[2 * e + 1];
          s2 += (e < J ? 1.0 : 2.0) * (re * re + im * im);
        }
      }
      nrm = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    }
    __syncthreads();
    float *out = a.top_vec + (size_t)t * HJ * 2;
    const float *xp = a.x + (p >= 0 ? p : 0) * (int64_t)(2 * HJ);
    for (int e = threadIdx.x; e < HJ; e += blockDim.x) {
      out[2 * e] = p >= 0 ? (float)(xp[2 * e] * nrm) : 0.0f;
      out[2 * e + 1] = (p >= 0 && e >= J) ? (float)(xp[2 * e + 1] * nrm) : 0.0f;
    }
    __syncthreads();
  }
}

// Unused atoms (count 0), in atom order, take the successive entries of the
// top list; atoms beyond the list (or beyond its valid entries) keep the
// eigen-kernel's output, which is the old atom for an atom with no samples.
__global__ void ksvd_reset_kernel(const KsvdArgs a) {
  const int HJ = a.H * a.J;
  int t = 0;
  for (int m = 0; m < a.M; ++m) {
    if (a.count[m] != 0) continue;
    if (t >= a.ntop || a.top_idx[t] < 0) break;
    const float *v = a.top_vec + (size_t)t * HJ * 2;
    float *out = a.new_coef + (size_t)m * HJ * 2;
    for (int i = threadIdx.x; i < 2 * HJ; i += blockDim.x) out[i] = v[i];
    ++t;
  }
}

}  // namespace

namespace {

// Checks shared by the entry points; fills the sizes of `a`.
int ksvd_setup(const rsc_dict *dict, int64_t P, int K, KsvdArgs &a) {
  if (!dict || P < 1 || K < 1 || K > kMaxK) return RSC_ERR_INVALID;
  if (P >= ((int64_t)1 << 31)) return RSC_ERR_UNSUPPORTED;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != dict->device) return RSC_ERR_INVALID;
  a = KsvdArgs{};
  a.P = P;
  a.K = K;
  a.M = dict->M;
  a.J = dict->J;
  a.H = dict->H;
  a.R = dict->R;
  a.n = dict->J + 2 * dict->kmax * dict->J;
  if (a.n > kMaxPacked) return RSC_ERR_UNSUPPORTED;
  a.ldE = (a.n + 3) & ~3;
  a.d = dict->d;
  a.tw = dict->tw;
  return RSC_OK;
}

// Accumulation: sample lists, residuals, C (zeroed here) and counts, and the
// top list of a.ntop patches; the per-patch scratch comes from one
// stream-ordered allocation freed on `st`.
int ksvd_accumulate(KsvdArgs &a, cudaStream_t st) {
  const int64_t P = a.P;
  const int M = a.M, n = a.n;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t bE = al((size_t)P * a.ldE * 4), bErr = al((size_t)P * 4), bCur = al((size_t)M * 4),
               bOff = al((size_t)(M + 1) * 4), bSmp = al((size_t)P * a.K * 8);
  unsigned char *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), bE + bErr + bCur + bOff + bSmp,
                                  st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  unsigned char *q = scratch;
  a.E = reinterpret_cast<float *>(q);
  q += bE;
  a.err = reinterpret_cast<float *>(q);
  q += bErr;
  a.cursor = reinterpret_cast<int *>(q);
  q += bCur;
  a.offset = reinterpret_cast<int *>(q);
  q += bOff;
  a.samples = reinterpret_cast<int2 *>(q);
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)std::min<int64_t>((P + 255) / 256, (int64_t)nsm * 8);
  e = cudaMemsetAsync(a.count, 0, (size_t)M * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.C, 0, (size_t)M * n * n * 8, st);
  if (e == cudaSuccess) {
    ksvd_count_kernel<<<grid, 256, 0, st>>>(a);
    ksvd_scan_kernel<<<1, 32, 0, st>>>(a);
    ksvd_fill_kernel<<<grid, 256, 0, st>>>(a);
    const size_t cov_smem = (size_t)kCovBatch * (4 * ((n + 3) / 4) + 4) * 4;
    e = cudaFuncSetAttribute(ksvd_cov_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cov_smem);
    if (e == cudaSuccess) ksvd_cov_kernel<<<M * kCovSplit, kCovThreads, cov_smem, st>>>(a);
    if (e == cudaSuccess && a.ntop > 0) ksvd_top_kernel<<<1, 1024, 0, st>>>(a);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  int rc = e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
  const cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (rc == RSC_OK && e2 != cudaSuccess) rc = rsc_cuda_fail(e2);
  return rc;
}

// New atoms from C, the counts and the top list.
int ksvd_finish(KsvdArgs &a, cudaStream_t st) {
  const int n = a.n;
  const size_t eig_smem = ((size_t)n * n + 2 * n + 32) * 8;
  cudaError_t e = cudaFuncSetAttribute(ksvd_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)eig_smem);
  if (e == cudaSuccess) {
    ksvd_eig_kernel<<<a.M, kEigThreads, eig_smem, st>>>(a, 5000);
    ksvd_reset_kernel<<<1, 256, 0, st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && a.n_used)
    e = cudaMemcpyAsync(a.n_used, a.count, (size_t)a.M * 4, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
}

}  // namespace

extern "C" int rsc_ksvd_update(const rsc_dict *dict, const float *x, int64_t P, int32_t K,
                               const int32_t *atom, const int32_t *angle_idx, const double *coef,
                               float *new_coef, int32_t *n_used, void *stream) {
  if (!x || !atom || !angle_idx || !coef || !new_coef) return RSC_ERR_INVALID;
  KsvdArgs a;
  int rc = ksvd_setup(dict, P, K, a);
  if (rc != RSC_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int M = a.M, n = a.n, HJ = a.H * a.J;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t bC = al((size_t)M * n * n * 8), bCnt = al((size_t)M * 4),
               bTe = al(kTopMax * 4), bTi = al(kTopMax * 8), bTv = al((size_t)kTopMax * HJ * 8);
  unsigned char *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&scratch), bC + bCnt + bTe + bTi + bTv,
                                  st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  unsigned char *q = scratch;
  a.C = reinterpret_cast<double *>(q);
  q += bC;
  a.count = reinterpret_cast<int *>(q);
  q += bCnt;
  a.top_err = reinterpret_cast<float *>(q);
  q += bTe;
  a.top_idx = reinterpret_cast<int64_t *>(q);
  q += bTi;
  a.top_vec = reinterpret_cast<float *>(q);
  a.ntop = kTopMax;
  a.top_needed = 1;
  a.x = x;
  a.atom = atom;
  a.angle = angle_idx;
  a.coef = coef;
  a.new_coef = new_coef;
  a.n_used = n_used;
  rc = ksvd_accumulate(a, st);
  if (rc == RSC_OK) rc = ksvd_finish(a, st);
  e = cudaFreeAsync(scratch, st);
  if (rc == RSC_OK && e != cudaSuccess) rc = rsc_cuda_fail(e);
  return rc;
}

extern "C" int rsc_ksvd_accumulate(const rsc_dict *dict, const float *x, int64_t P, int32_t K,
                                   const int32_t *atom, const int32_t *angle_idx,
                                   const double *coef, double *C, int32_t *count, float *top_err,
                                   int64_t *top_idx, float *top_vec, int32_t ntop, void *stream) {
  if (!x || !atom || !angle_idx || !coef || !C || !count) return RSC_ERR_INVALID;
  if (ntop < 0 || ntop > kTopMax || (ntop > 0 && (!top_err || !top_idx || !top_vec)))
    return RSC_ERR_INVALID;
  KsvdArgs a;
  int rc = ksvd_setup(dict, P, K, a);
  if (rc != RSC_OK) return rc;
  a.x = x;
  a.atom = atom;
  a.angle = angle_idx;
  a.coef = coef;
  a.C = C;
  a.count = count;
  a.ntop = ntop;
  a.top_err = top_err;
  a.top_idx = top_idx;
  a.top_vec = top_vec;
  return ksvd_accumulate(a, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int rsc_ksvd_finish(const rsc_dict *dict, const double *C, const int32_t *count,
                               const int64_t *top_idx, const float *top_vec, int32_t ntop,
                               float *new_coef, int32_t *n_used, void *stream) {
  if (!dict || !C || !count || !new_coef) return RSC_ERR_INVALID;
  if (ntop < 0 || ntop > kTopMax || (ntop > 0 && (!top_idx || !top_vec))) return RSC_ERR_INVALID;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != dict->device) return RSC_ERR_INVALID;
  KsvdArgs a{};
  a.M = dict->M;
  a.J = dict->J;
  a.H = dict->H;
  a.R = dict->R;
  a.n = dict->J + 2 * dict->kmax * dict->J;
  if (a.n > kMaxPacked) return RSC_ERR_UNSUPPORTED;
  a.d = dict->d;
  a.tw = dict->tw;
  a.C = const_cast<double *>(C);
  a.count = const_cast<int *>(count);
  a.ntop = ntop;
  a.top_idx = const_cast<int64_t *>(top_idx);
  a.top_vec = const_cast<float *>(top_vec);
  a.new_coef = new_coef;
  a.n_used = n_used;
  return ksvd_finish(a, reinterpret_cast<cudaStream_t>(stream));
}
