// rsc_noalloc.cu -- rsc_encode_noalloc: the FP16 tensor-core coding path
// without any device allocation.
//
// rsc_encode's FP16 path needs one scratch buffer per call: the list of
// patches the tensor-core kernel hands to the FP32 kernel, plus its counter.
// It takes that buffer from the library's stream-ordered memory pool.
// Some callers cannot allocate while they code: a serving process that
// reserves all of its device memory up front and forbids allocation in its
// steady state, code running under another framework's memory pool, or a
// caller that must not risk an allocation failure (or an allocator
// synchronisation) in the middle of a latency-bound request.  This entry
// point keeps that list in a fixed file-scope device array instead.
#include <mutex>

#include "rsc_internal.h"
#include "rsc_trace.h"

namespace {

// Largest P one call accepts; the array holds the hand-off counter (padded to
// 16 bytes) and one slot per patch: (2^20 + 4) int32 = 4 MiB, held by every
// GPU that loads the library until the process exits.
constexpr int64_t kNoAllocMaxPatches = (int64_t)1 << 20;
static __device__ __align__(256) int g_handoff_scratch[kNoAllocMaxPatches + 4];

constexpr int kMaxDevices = 64;
int *g_scratch_ptr[kMaxDevices] = {};  // device address of g_handoff_scratch, per device
std::mutex g_scratch_mu;

// Per-device set-up: the host-side name g_handoff_scratch is only a stand-in,
// so the device address comes from cudaGetSymbolAddress with the device
// current.  Done on the first call on each device.
int scratch_for_current_device(int **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return RSC_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_handoff_scratch);
    if (e != cudaSuccess) return rsc_cuda_fail(e);
    g_scratch_ptr[dev] = static_cast<int *>(p);
  }
  *out = g_scratch_ptr[dev];
  return RSC_OK;
}

}  // namespace

extern "C" int rsc_encode_noalloc(const rsc_dict *dict, const float *x, int64_t P, int32_t K,
                                  int32_t *atom, int32_t *angle_idx, float *angle, double *coef,
                                  float *resid_norm2, void *stream) {
  RscRange nvtx_range("rsc_encode_noalloc");
  if (!dict || P < 0 || K < 1 || K > kMaxK) return RSC_ERR_INVALID;
  if (P > kNoAllocMaxPatches) return RSC_ERR_UNSUPPORTED;
  if (P == 0) return RSC_OK;
  if (!x || !atom || !angle_idx || !coef) return RSC_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(x) & 15u) || (reinterpret_cast<uintptr_t>(coef) & 7u) ||
      (reinterpret_cast<uintptr_t>(atom) & 3u) || (reinterpret_cast<uintptr_t>(angle_idx) & 3u) ||
      (angle && (reinterpret_cast<uintptr_t>(angle) & 3u)) ||
      (resid_norm2 && (reinterpret_cast<uintptr_t>(resid_norm2) & 3u)))
    return RSC_ERR_INVALID;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  if (dev != dict->device) return RSC_ERR_INVALID;
  if (!dict->steered_f16 || dict->row_len != kTcKst || K > kTcMaxK) return RSC_ERR_UNSUPPORTED;
  int *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != RSC_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the counter starts at zero
  e = cudaMemsetAsync(scratch, 0, sizeof(int), st);
  if (e != cudaSuccess) return rsc_cuda_fail(e);

  TcArgs ta;
  ta.x = x;
  ta.P = P;
  ta.K = K;
  ta.M = dict->M;
  ta.J = dict->J;
  ta.kmax = dict->kmax;
  ta.R = dict->R;
  ta.H = dict->H;
  ta.n = dict->n;
  ta.ksteps = (dict->n + 15) / 16;
  ta.MR = dict->M * dict->R;
  ta.nchunks = (ta.MR + kTcBN - 1) / kTcBN;
  ta.d = dict->d;
  ta.tw = dict->tw;
  ta.xgram = dict->xgram;
  ta.atom = atom;
  ta.angle_idx = angle_idx;
  ta.angle = angle;
  ta.coef = coef;
  ta.resid_norm2 = resid_norm2;
  ta.err = dict->err;
  ta.redo_count = scratch;
  ta.redo_list = scratch + 4;
  ta.fallbacks = dict->fallbacks;
  rc = rsc_launch_tc(ta, dict->tmap_b, st);
  if (rc != RSC_OK) return rc;

  RompArgs a;
  a.x = x;
  a.P = P;
  a.K = K;
  a.M = dict->M;
  a.J = dict->J;
  a.kmax = dict->kmax;
  a.R = dict->R;
  a.H = dict->H;
  a.d = dict->d;
  a.dT = dict->dT;
  a.tw = dict->tw;
  a.atom = atom;
  a.angle_idx = angle_idx;
  a.angle = angle;
  a.coef = coef;
  a.resid_norm2 = resid_norm2;
  a.err = dict->err;
  a.fallbacks = nullptr;
  a.redo_count = scratch;
  a.redo_list = scratch + 4;
  return rsc_launch_f32(a, st);
}
