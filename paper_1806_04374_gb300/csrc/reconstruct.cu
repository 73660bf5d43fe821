// reconstruct.cu -- the way back from codes to patches: step 4 of the
// proposed algorithm (Sec. II-E: the learned dictionary returns to the patch
// domain as D = Phi D_hat) and the reconstruction of coded patches.
//
// rsc_reconstruct: x_hat_p = sum_i a_i S_{r_i} d_{m_i} for each patch's code
//   (steering of Eq. (Sr): harmonic k of an atom times exp(-i k 2 pi r / R)),
//   one thread per (patch, entry), accumulated in FP64 from the dictionary's
//   FP32 atoms and its double-float steering factors.
// rsc_synthesize: pixels = Phi x_hat over the circular patch, one thread per
//   (patch, pixel), with the basis's real synthesis matrix (FP32, [n][npix],
//   columns in the packed order: Re of k = 0, then sqrt2 Re and sqrt2 Im).
#include "rsc_internal.h"
#include "rsc_trace.h"

namespace {

__global__ void reconstruct_kernel(const float *__restrict__ d, const float *__restrict__ tw,
                                   int H, int J, int R, int64_t P, int K,
                                   const int32_t *__restrict__ atom,
                                   const int32_t *__restrict__ angle_idx,
                                   const double *__restrict__ coef, float *__restrict__ out) {
  const int HJ = H * J;
  const int64_t total = P * HJ;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / HJ;
    const int e = (int)(idx - p * HJ), k = e / J;
    double re = 0.0, im = 0.0;
    for (int i = 0; i < K; ++i) {
      const int m = atom[p * K + i];
      if (m < 0) continue;
      const int r = angle_idx[p * K + i];
      const double a = coef[p * K + i];
      const float2 dv = reinterpret_cast<const float2 *>(d)[(int64_t)m * HJ + e];
      const double dr = dv.x, di = k ? (double)dv.y : 0.0;
      // steering factor exp(-i k theta_r) from the hi + lo parts of the table
      const double c = (double)tw[(0 * H + k) * R + r] + (double)tw[(1 * H + k) * R + r];
      const double s = (double)tw[(2 * H + k) * R + r] + (double)tw[(3 * H + k) * R + r];
      re += a * (dr * c + di * s);
      im += a * (di * c - dr * s);
    }
    reinterpret_cast<float2 *>(out)[idx] = make_float2((float)re, k ? (float)im : 0.0f);
  }
}

__global__ void synthesize_kernel(const float *__restrict__ X, int n, int npix, int J, int64_t P,
                                  const float *__restrict__ coef, int nout,
                                  float *__restrict__ pix) {
  const int64_t total = P * npix;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / npix;
    const int q = (int)(idx - p * npix);
    const float *c = coef + p * nout;
    float acc = 0.0f;
    // packed coefficient of column col: Re c[k=0][col] for col < J, else
    // sqrt2 times half-spectrum entry J + col (Re or Im of c[j][k >= 1])
    for (int col = 0; col < J; ++col) acc = fmaf(X[(int64_t)col * npix + q], c[2 * col], acc);
    for (int col = J; col < n; ++col)
      acc = fmaf(X[(int64_t)col * npix + q], 1.41421356237309515f * c[J + col], acc);
    pix[idx] = acc;
  }
}

unsigned grid_for(int64_t total, int device) {
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  const int64_t blocks = (total + 255) / 256, cap = (int64_t)nsm * 16;
  return (unsigned)(blocks < cap ? blocks : cap);
}

}  // namespace

extern "C" int rsc_reconstruct(const rsc_dict *dict, int64_t P, int32_t K, const int32_t *atom,
                               const int32_t *angle_idx, const double *coef, float *out,
                               void *stream) {
  RscRange nvtx_range("rsc_reconstruct");
  if (!dict || P < 0 || K < 1 || K > kMaxK) return RSC_ERR_INVALID;
  if (P == 0) return RSC_OK;
  if (!atom || !angle_idx || !coef || !out) return RSC_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(out) & 7) || (reinterpret_cast<uintptr_t>(coef) & 7) ||
      (reinterpret_cast<uintptr_t>(atom) & 3) || (reinterpret_cast<uintptr_t>(angle_idx) & 3))
    return RSC_ERR_INVALID;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != dict->device) return RSC_ERR_INVALID;
  const int64_t total = P * dict->H * dict->J;
  reconstruct_kernel<<<grid_for(total, dev), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      dict->d, dict->tw, dict->H, dict->J, dict->R, P, K, atom, angle_idx, coef, out);
  e = cudaGetLastError();
  return e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
}

extern "C" int rsc_synthesize(const rsc_basis *basis, const float *coef, int64_t P, float *pixels,
                              void *stream) {
  RscRange nvtx_range("rsc_synthesize");
  if (!basis || P < 0) return RSC_ERR_INVALID;
  if (P == 0) return RSC_OK;
  if (!coef || !pixels) return RSC_ERR_INVALID;
  rsc_basis_view v;
  int rc = rsc_basis_internals(basis, &v);
  if (rc != RSC_OK) return rc;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != v.device) return RSC_ERR_INVALID;
  const int64_t total = P * v.npix;
  synthesize_kernel<<<grid_for(total, dev), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      v.X, v.n, v.npix, v.J, P, coef, v.nout, pixels);
  e = cudaGetLastError();
  return e == cudaSuccess ? RSC_OK : rsc_cuda_fail(e);
}
