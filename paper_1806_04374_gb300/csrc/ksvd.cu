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
// Kernels: per chunk of patches (count samples per atom; then the per-atom
// sample lists in patch order and the packed residuals in double-float); per
// atom kCovSplit CTAs accumulating partial sums of C_m over slices of its
// samples (4 x 4 register tiles; the columns y in double-float, each product
// y_i y_j as an exact FP32 product plus its cross terms, summed Dot2-style
// over 32 samples and folded into FP64), then the kCovSplit partials added in
// a fixed order, so that the update is FP64-grade and the same on every run;
// one CTA per atom running an FP64 power iteration from the old atom; one CTA
// for the resets.  All vectors are packed reals (k = 0 real parts, sqrt(2)
// Re/Im of k >= 1).
#include <math.h>

#include <algorithm>

#include "df.cuh"
#include "rsc_internal.h"
#include "rsc_trace.h"

namespace {

constexpr int kCovThreads = 384;  // one 4 x 4 tile each: all 351 tiles of n = 102 in one round
constexpr int kFillChunk = 256;   // patches per chunk of the sample lists
constexpr int kMaxAtomsKsvd = 12288;  // per-atom cursors of a chunk in shared memory
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
  float *E;         // [2][P][ldE] packed residuals, double-float (hi plane, lo plane)
  float *err;       // [P]
  int *count;       // [M]
  int *offset;      // [M + 1]
  int *chunk_cnt;   // [nchunk][M] samples of each atom in each chunk of patches
  int *chunk_base;  // [nchunk][M] first slot of each atom's samples of each chunk
  int nchunk;
  int2 *samples;    // [sum count] (patch, occurrence), patch order within an atom
  double *C;        // [M][n][n]
  double *Cpart;    // [kCovSplit][M][n][n] partial sums (every entry written)
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

// Samples of each atom in each chunk of kFillChunk patches (shared-memory
// histogram; integer counts do not depend on the order of the additions).
__global__ void ksvd_chunk_count_kernel(const KsvdArgs a) {
  extern __shared__ int hist[];  // [M]
  for (int m = threadIdx.x; m < a.M; m += blockDim.x) hist[m] = 0;
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * kFillChunk;
  const int64_t p1 = min(a.P, p0 + kFillChunk);
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x)
    for (int i = 0; i < a.K; ++i)
      if (chosen(a, p, i)) atomicAdd(&hist[a.atom[p * a.K + i]], 1);
  __syncthreads();
  for (int m = threadIdx.x; m < a.M; m += blockDim.x)
    a.chunk_cnt[(size_t)blockIdx.x * a.M + m] = hist[m];
}

// Per atom: its count, its first slot (offset, atoms in order) and the first
// slot of its samples from each chunk (chunks in order).  One CTA.
__global__ void ksvd_chunk_scan_kernel(const KsvdArgs a) {
  for (int m = threadIdx.x; m < a.M; m += blockDim.x) {
    int t = 0;
    for (int c = 0; c < a.nchunk; ++c) t += a.chunk_cnt[(size_t)c * a.M + m];
    a.count[m] = t;
    if (a.n_used) a.n_used[m] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int m = 0; m < a.M; ++m) {
      a.offset[m] = s;
      s += a.count[m];
    }
    a.offset[a.M] = s;
  }
  __syncthreads();
  for (int m = threadIdx.x; m < a.M; m += blockDim.x) {
    int b = a.offset[m];
    for (int c = 0; c < a.nchunk; ++c) {
      a.chunk_base[(size_t)c * a.M + m] = b;
      b += a.chunk_cnt[(size_t)c * a.M + m];
    }
  }
}

// Per chunk: the packed residuals e_p = x_p - sum_i a_i S_{r_i} d_{m_i} of
// its patches in double-float (one thread per patch; the weights are FP64,
// the steering factors double-float) with their coding errors, and the
// chunk's sample slots in patch order (one thread walks the chunk, so every
// atom's list is in patch order on every run).
__global__ void ksvd_fill_kernel(const KsvdArgs a) {
  // [M] next slot of each atom in this chunk, then [kFillChunk][K] the atom
  // of each chosen occurrence (-1: not chosen), filled in parallel
  extern __shared__ int cur[];
  int *occ = cur + a.M;
  const int J = a.J, H = a.H, HJ = H * J, R = a.R;
  const int64_t p0 = (int64_t)blockIdx.x * kFillChunk;
  const int64_t p1 = min(a.P, p0 + kFillChunk);
  for (int m = threadIdx.x; m < a.M; m += blockDim.x)
    cur[m] = a.chunk_base[(size_t)blockIdx.x * a.M + m];
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x)
    for (int i = 0; i < a.K; ++i)
      occ[(p - p0) * a.K + i] = chosen(a, p, i) ? a.atom[p * a.K + i] : -1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int n = (int)(p1 - p0) * a.K;
    for (int w = 0; w < n; ++w) {
      const int m = occ[w];
      if (m >= 0) a.samples[cur[m]++] = make_int2((int)(p0 + w / a.K), w % a.K);
    }
  }
  const df sqrt2 = df_from_d(1.4142135623730951);
  const size_t plane = (size_t)a.P * a.ldE;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const float2 *xp = reinterpret_cast<const float2 *>(a.x + p * (int64_t)(2 * HJ));
    float *eh = a.E + p * (int64_t)a.ldE;
    float *el = eh + plane;
    double n2 = 0.0;
    for (int e = 0; e < HJ; ++e) {
      const int k = e / J;
      const float2 v = xp[e];
      df re = df_make(v.x), im = df_make(k ? v.y : 0.0f);
      for (int i = 0; i < a.K; ++i) {
        const int m = a.atom[p * a.K + i];
        if (m < 0) continue;
        const int r = a.angle[p * a.K + i];
        const df c = {a.tw[(0 * H + k) * R + r], a.tw[(1 * H + k) * R + r]};
        const df sn = {a.tw[(2 * H + k) * R + r], a.tw[(3 * H + k) * R + r]};
        const float2 dv = reinterpret_cast<const float2 *>(a.d)[(size_t)m * HJ + e];
        const float dim = k ? dv.y : 0.0f;
        const df w = df_from_d(a.coef[p * a.K + i]);
        // S_r d: harmonic k times exp(-i k theta_r)
        const df sre = df_add(df_mul_f(c, dv.x), df_mul_f(sn, dim));
        const df sim = df_sub(df_mul_f(c, dim), df_mul_f(sn, dv.x));
        re = df_sub(re, df_mul(w, sre));
        im = df_sub(im, df_mul(w, sim));
      }
      if (k == 0) {
        eh[e] = re.hi;
        el[e] = re.lo;
        const double r0 = df_to_d(re);
        n2 = fma(r0, r0, n2);
      } else {
        const int q = 2 * e - J;
        const df pr = df_mul(re, sqrt2), pi = df_mul(im, sqrt2);
        eh[q] = pr.hi;
        el[q] = pr.lo;
        eh[q + 1] = pi.hi;
        el[q + 1] = pi.lo;
        const double r0 = df_to_d(pr), i0 = df_to_d(pi);
        n2 = fma(r0, r0, fma(i0, i0, n2));
      }
    }
    a.err[p] = (float)n2;
  }
}

// C_m = sum over the atom's samples of y y^T, y = S_{-r0} e_p + a_{i0} d_m.
// The samples of atom m are split over kCovSplit CTAs (slices in list order);
// each thread owns 4 x 4 tiles of the upper triangle.  The columns y of a
// batch of kCovBatch samples are built in double-float in shared memory; a
// product y_i y_j is the exact product of the hi parts (TwoProd) plus the
// cross terms hi_i lo_j + lo_i hi_j, and the batch's products are summed
// Dot2-style (TwoSum of the hi parts, the errors and lo parts summed apart),
// then added to FP64 accumulators.  Each CTA writes its partial sums to its
// own slice of Cpart (every entry, zero when it has no samples); a second
// kernel adds the kCovSplit slices in order.
constexpr int kCovSplit = 8;

__global__ void __launch_bounds__(kCovThreads) ksvd_cov_kernel(const KsvdArgs a) {
  extern __shared__ __align__(16) float ysm[];  // 2 x kCovBatch rows of ldy floats
  __shared__ int s_p[kCovBatch], s_r0[kCovBatch];
  __shared__ df s_w[kCovBatch];
  const int m = blockIdx.x / kCovSplit, part = blockIdx.x - m * kCovSplit;
  const int n = a.n, J = a.J, H = a.H, HJ = H * J, R = a.R;
  const int nb4 = (n + 3) / 4, ldy = 4 * nb4 + 4;  // +4: rows start in different banks
  float *yhi = ysm, *ylo = ysm + kCovBatch * ldy;
  const int beg0 = a.offset[m], cnt = a.offset[m + 1] - beg0;
  const int per = (cnt + kCovSplit - 1) / kCovSplit;
  const int beg = beg0 + part * per, end = min(beg0 + cnt, beg + per);
  double *Cm = a.Cpart + ((size_t)part * a.M + m) * n * n;
  const size_t plane = (size_t)a.P * a.ldE;
  const df sqrt2 = df_from_d(1.4142135623730951);
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
      for (int w = threadIdx.x; w < nb * ldy; w += blockDim.x) {
        yhi[w] = 0.0f;
        ylo[w] = 0.0f;
      }
      if (threadIdx.x < nb) {
        const int2 smp = a.samples[b0 + threadIdx.x];
        const int64_t p = smp.x;
        const int r0 = a.angle[p * a.K + smp.y];
        // the code entry of (m, r0): every occurrence of that pair (Fig.
        // "code" zeroes the whole entry b_{r0}[m])
        double wsum = 0.0;
        for (int i = 0; i < a.K; ++i)
          if (a.atom[p * a.K + i] == m && a.angle[p * a.K + i] == r0) wsum += a.coef[p * a.K + i];
        s_p[threadIdx.x] = smp.x;
        s_r0[threadIdx.x] = r0;
        s_w[threadIdx.x] = df_from_d(wsum);
      }
      __syncthreads();
      for (int w = threadIdx.x; w < nb * HJ; w += blockDim.x) {
        const int s = w / HJ, e = w - s * HJ;
        const int64_t p = s_p[s];
        const int r0 = s_r0[s];
        const df w0 = s_w[s];
        const int k = e / J;
        const float *eh = a.E + p * (int64_t)a.ldE, *el = eh + plane;
        const float2 dv = reinterpret_cast<const float2 *>(a.d)[(size_t)m * HJ + e];
        if (k == 0) {
          const df y = df_add(df{eh[e], el[e]}, df_mul_f(w0, dv.x));
          yhi[s * ldy + e] = y.hi;
          ylo[s * ldy + e] = y.lo;
        } else {
          const int q = 2 * e - J;
          const df re = {eh[q], el[q]}, im = {eh[q + 1], el[q + 1]};
          // S_{-theta}: harmonic k times exp(+i k theta)
          const df c = {a.tw[(0 * H + k) * R + r0], a.tw[(1 * H + k) * R + r0]};
          const df sn = {a.tw[(2 * H + k) * R + r0], a.tw[(3 * H + k) * R + r0]};
          const df w2 = df_mul(w0, sqrt2);
          const df yr = df_add(df_sub(df_mul(re, c), df_mul(im, sn)), df_mul_f(w2, dv.x));
          const df yi = df_add(df_add(df_mul(re, sn), df_mul(im, c)), df_mul_f(w2, dv.y));
          yhi[s * ldy + q] = yr.hi;
          ylo[s * ldy + q] = yr.lo;
          yhi[s * ldy + q + 1] = yi.hi;
          ylo[s * ldy + q + 1] = yi.lo;
        }
      }
      __syncthreads();
      if (bi >= 0) {
        float sh[16], sl[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) sh[u] = sl[u] = 0.0f;
        for (int s = 0; s < nb; ++s) {
          const float4 hi4 = *reinterpret_cast<const float4 *>(&yhi[s * ldy + 4 * bi]);
          const float4 hj4 = *reinterpret_cast<const float4 *>(&yhi[s * ldy + 4 * bj]);
          const float4 li4 = *reinterpret_cast<const float4 *>(&ylo[s * ldy + 4 * bi]);
          const float4 lj4 = *reinterpret_cast<const float4 *>(&ylo[s * ldy + 4 * bj]);
          const float hi[4] = {hi4.x, hi4.y, hi4.z, hi4.w}, hj[4] = {hj4.x, hj4.y, hj4.z, hj4.w};
          const float li[4] = {li4.x, li4.y, li4.z, li4.w}, lj[4] = {lj4.x, lj4.y, lj4.z, lj4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const df pp = two_prod(hi[u], hj[v]);
              const float cross = __fmaf_rn(hi[u], lj[v], __fmaf_rn(li[u], hj[v], pp.lo));
              const df ts = two_sum(sh[u * 4 + v], pp.hi);
              sh[u * 4 + v] = ts.hi;
              sl[u * 4 + v] = __fadd_rn(sl[u * 4 + v], __fadd_rn(ts.lo, cross));
            }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] += (double)sh[u] + (double)sl[u];
      }
    }
    if (bi >= 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int i = 4 * bi + u, j = 4 * bj + v;
          if (i < n && j < n && i <= j) Cm[(size_t)i * n + j] = acc[u * 4 + v];
        }
    }
  }
}

// C_m[i][j] = sum over the kCovSplit partial sums in slice order (upper
// triangle), mirrored to the lower triangle.
__global__ void ksvd_cov_sum_kernel(const KsvdArgs a) {
  const int n = a.n;
  const size_t nn = (size_t)n * n, per_part = (size_t)a.M * nn;
  for (size_t w = (size_t)blockIdx.x * blockDim.x + threadIdx.x; w < per_part;
       w += (size_t)gridDim.x * blockDim.x) {
    const size_t m = w / nn, ij = w - m * nn;
    const int i = (int)(ij / n), j = (int)(ij - (size_t)i * n);
    if (i > j) continue;
    double s = 0.0;
    for (int part = 0; part < kCovSplit; ++part) s += a.Cpart[part * per_part + w];
    a.C[w] = s;
    if (i != j) a.C[m * nn + (size_t)j * n + i] = s;
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
  if (a.n > kMaxPacked || a.M > kMaxAtomsKsvd) return RSC_ERR_UNSUPPORTED;
  a.ldE = (a.n + 3) & ~3;
  a.d = dict->d;
  a.tw = dict->tw;
  return RSC_OK;
}

// Accumulation: sample lists, residuals, C (written here) and counts, and the
// top list of a.ntop patches; the per-patch scratch comes from one
// stream-ordered allocation freed on `st`.
int ksvd_accumulate(KsvdArgs &a, cudaStream_t st) {
  const int64_t P = a.P;
  const int M = a.M, n = a.n;
  a.nchunk = (int)((P + kFillChunk - 1) / kFillChunk);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t bE = al((size_t)2 * P * a.ldE * 4), bErr = al((size_t)P * 4),
               bOff = al((size_t)(M + 1) * 4), bCh = al((size_t)a.nchunk * M * 4),
               bSmp = al((size_t)P * a.K * 8), bCp = al((size_t)kCovSplit * M * n * n * 8);
  unsigned char *scratch = nullptr;
  cudaError_t e = rsc_scratch_alloc(reinterpret_cast<void **>(&scratch),
                                  bE + bErr + bOff + 2 * bCh + bSmp + bCp, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  unsigned char *q = scratch;
  auto take = [&](size_t b) {
    unsigned char *r = q;
    q += b;
    return r;
  };
  a.E = reinterpret_cast<float *>(take(bE));
  a.err = reinterpret_cast<float *>(take(bErr));
  a.offset = reinterpret_cast<int *>(take(bOff));
  a.chunk_cnt = reinterpret_cast<int *>(take(bCh));
  a.chunk_base = reinterpret_cast<int *>(take(bCh));
  a.samples = reinterpret_cast<int2 *>(take(bSmp));
  a.Cpart = reinterpret_cast<double *>(take(bCp));
  const size_t hist_smem = (size_t)M * 4;
  const size_t cov_smem = (size_t)2 * kCovBatch * (4 * ((n + 3) / 4) + 4) * 4;
  e = cudaFuncSetAttribute(ksvd_cov_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)cov_smem);
  if (e == cudaSuccess) {
    ksvd_chunk_count_kernel<<<a.nchunk, 256, hist_smem, st>>>(a);
    ksvd_chunk_scan_kernel<<<1, 1024, 0, st>>>(a);
    ksvd_fill_kernel<<<a.nchunk, kFillChunk, hist_smem + (size_t)kFillChunk * a.K * 4, st>>>(a);
    ksvd_cov_kernel<<<M * kCovSplit, kCovThreads, cov_smem, st>>>(a);
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t work = (size_t)M * n * n;
    const unsigned gsum = (unsigned)std::min<size_t>((work + 255) / 256, (size_t)nsm * 8);
    ksvd_cov_sum_kernel<<<gsum, 256, 0, st>>>(a);
    if (a.ntop > 0) ksvd_top_kernel<<<1, 1024, 0, st>>>(a);
    e = cudaGetLastError();
  }
  int rc = e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
  const cudaError_t e2 = rsc_scratch_free(scratch, st);
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
  RscRange nvtx_range("rsc_ksvd_update");
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
  cudaError_t e = rsc_scratch_alloc(reinterpret_cast<void **>(&scratch), bC + bCnt + bTe + bTi + bTv,
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
  e = rsc_scratch_free(scratch, st);
  if (rc == RSC_OK && e != cudaSuccess) rc = rsc_cuda_fail(e);
  return rc;
}

extern "C" int rsc_ksvd_accumulate(const rsc_dict *dict, const float *x, int64_t P, int32_t K,
                                   const int32_t *atom, const int32_t *angle_idx,
                                   const double *coef, double *C, int32_t *count, float *top_err,
                                   int64_t *top_idx, float *top_vec, int32_t ntop, void *stream) {
  RscRange nvtx_range("rsc_ksvd_accumulate");
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
  RscRange nvtx_range("rsc_ksvd_finish");
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
