// rsc_capi.cu -- host side of the librsc C ABI (declared in include/rsc.h):
// argument checks, dictionary set-up (the once-per-dictionary tables of the
// steering matrix of Eq. (Sr)) and dispatch of the coding kernels.
#include <dlfcn.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_fp16.h>

#include <mutex>
#include <string>
#include <vector>

#include "rsc_internal.h"
#include "rsc_trace.h"

namespace {

thread_local char g_cuda_msg[256] = "no error";

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <class T>
bool aligned_as(const void *p) {
  return (reinterpret_cast<uintptr_t>(p) % alignof(T)) == 0;
}

struct TimedPair {
  int phase;
  cudaEvent_t a, b;
};
typedef std::vector<TimedPair> TimingLog;

void clear_timing(rsc_dict *d) {
  TimingLog *log = static_cast<TimingLog *>(d->timing_state);
  if (!log) return;
  for (auto &p : *log) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  log->clear();
}

// Records the start event of a timed launch; returns its slot or -1.
int timing_begin(const rsc_dict *dc, int phase, cudaStream_t st) {
  rsc_dict *d = const_cast<rsc_dict *>(dc);
  if (!d->timing) return -1;
  TimingLog *log = static_cast<TimingLog *>(d->timing_state);
  if (!log) {
    log = new TimingLog();
    d->timing_state = log;
  }
  TimedPair p{phase, nullptr, nullptr};
  if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  cudaEventRecord(p.a, st);
  log->push_back(p);
  return (int)log->size() - 1;
}

void timing_end(const rsc_dict *d, int slot, cudaStream_t st) {
  if (slot < 0) return;
  TimingLog *log = static_cast<TimingLog *>(d->timing_state);
  cudaEventRecord((*log)[slot].b, st);
}

// Device buffers of rsc_encode_host: two chunks (double-buffered on two
// streams), grown when a call needs more, kept with the dictionary so that
// calls allocate and free nothing (cudaFree would also synchronise the device).
struct HostStage {
  std::mutex mu;  // one rsc_encode_host at a time per dictionary
  int64_t chunk = 0;
  int K = 0, vec = 0, nbuf = 0;
  cudaStream_t s[2] = {nullptr, nullptr};
  struct Buf {
    float *x = nullptr;
    int32_t *atom = nullptr, *ang = nullptr;
    float *angf = nullptr, *rn2 = nullptr;
    double *coef = nullptr;
  } b[2];
  void release() {
    for (int i = 0; i < 2; ++i) {
      if (s[i]) cudaStreamSynchronize(s[i]);
      cudaFree(b[i].x);
      cudaFree(b[i].atom);
      cudaFree(b[i].ang);
      cudaFree(b[i].angf);
      cudaFree(b[i].coef);
      cudaFree(b[i].rn2);
      b[i] = Buf{};
    }
    chunk = 0;
    K = 0;
    nbuf = 0;
  }
  ~HostStage() {
    release();
    for (int i = 0; i < 2; ++i)
      if (s[i]) cudaStreamDestroy(s[i]);
  }
  // `nb` buffers (1 or 2) for chunks of `n` patches of K steps and `v` floats each.
  cudaError_t reserve(int64_t n, int k, int v, int nb) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
      if (!s[i]) e = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking);
    if (e != cudaSuccess || (n <= chunk && k <= K && v == vec && nb <= nbuf)) return e;
    release();
    nbuf = nb;
    for (int i = 0; i < nb && e == cudaSuccess; ++i) {
      Buf &B = b[i];
      e = cudaMalloc(&B.x, (size_t)n * v * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&B.atom, (size_t)n * k * sizeof(int32_t));
      if (e == cudaSuccess) e = cudaMalloc(&B.ang, (size_t)n * k * sizeof(int32_t));
      if (e == cudaSuccess) e = cudaMalloc(&B.angf, (size_t)n * k * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&B.coef, (size_t)n * k * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&B.rn2, (size_t)n * sizeof(float));
    }
    if (e != cudaSuccess) {
      release();
      return e;
    }
    chunk = n;
    K = k;
    vec = v;
    return cudaSuccess;
  }
};
std::mutex g_stage_mu;  // creation of a dictionary's HostStage

void free_dict(rsc_dict *d) {
  if (!d) return;
  delete static_cast<HostStage *>(d->host_stage);
  clear_timing(d);
  delete static_cast<TimingLog *>(d->timing_state);
  cudaFree(d->d);
  cudaFree(d->dT);
  cudaFree(d->tw);
  cudaFree(d->err);
  cudaFree(d->fallbacks);
  cudaFree(d->steered_f16);
  cudaFree(d->paired_f16);
  cudaFree(d->xgram);
  cudaFree(d->anorm);
  delete d;
}


typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// TMA map of a row-major fp16 matrix [rows][kTcKst]: box 64 columns x
// box_rows rows, 128-byte swizzle, zero fill outside (columns kTcKst..127,
// rows >= rows).
int encode_rows_map(CUtensorMap *map, void *base, size_t rows, int box_rows, int row_len) {
  static EncodeTiledFn fn = nullptr;
  static cudaError_t fn_err = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    fn_err = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                              cudaEnableDefault, &q);
    if (fn_err == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = (EncodeTiledFn)f;
  });
  if (!fn) return rsc_cuda_fail(fn_err != cudaSuccess ? fn_err : cudaErrorNotSupported);
  const cuuint64_t gdim[2] = {(cuuint64_t)row_len, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)row_len * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult cr = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, gdim, gstride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) {
    snprintf(g_cuda_msg, sizeof g_cuda_msg, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
    return RSC_ERR_CUDA;
  }
  return RSC_OK;
}

// Packed steered rows (rsc_slot_code layout): entry q of row r*M + m,
// r < nR, is slot q of kDictScale S_r d_m in fp16, computed in FP64 from the
// atoms; the angle k r 2 pi / R is reduced exactly (k r mod R).
__global__ void steered_rows_kernel(const float *__restrict__ d, int M, int J, int kmax, int R,
                                    int nR, int L, int paired, uint16_t *out) {
  const int HJ = (kmax + 1) * J;
  const int64_t total = (int64_t)nR * M * L;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % L);
    const int64_t row = idx / L;
    const int m = (int)(row % M), r = (int)(row / M);
    const int code = rsc_slot_code(q, J, kmax, paired != 0);
    uint16_t bits = 0;
    if (code >= 0) {
      const int e = code >> 8, k = (code >> 1) & 127, c = code & 1;
      const double th = 2.0 * M_PI * (double)(int)(((int64_t)k * r) % R) / (double)R;
      const double co = cos(th), si = sin(th);
      const double dre = d[((size_t)m * HJ + e) * 2];
      const double dim = k ? (double)d[((size_t)m * HJ + e) * 2 + 1] : 0.0;
      const double re = co * dre + si * dim, im = co * dim - si * dre;  // e^{-ik theta} d
      const double v = (k == 0 ? re : M_SQRT2 * (c ? im : re)) * (double)kDictScale;
      const __half hv = __double2half(v);
      bits = *reinterpret_cast<const uint16_t *>(&hv);
    }
    out[idx] = bits;
  }
}

// Cross-Gram table H_k(a, b) = sum_j conj(d_a[j,k]) d_b[j,k] in FP64, stored
// as double-float (re hi, re lo, im hi, im lo) at [(a M + b) H + k].
__global__ void xgram_kernel(const float *__restrict__ d, int M, int J, int H,
                             float4 *__restrict__ X) {
  const int HJ = H * J;
  const int64_t total = (int64_t)M * M * H;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % H);
    const int64_t ab = idx / H;
    const int mb = (int)(ab % M), ma = (int)(ab / M);
    double re = 0.0, im = 0.0;
    for (int j = 0; j < J; ++j) {
      const double ar = d[((size_t)ma * HJ + k * J + j) * 2];
      const double ai = k ? (double)d[((size_t)ma * HJ + k * J + j) * 2 + 1] : 0.0;
      const double br = d[((size_t)mb * HJ + k * J + j) * 2];
      const double bi = k ? (double)d[((size_t)mb * HJ + k * J + j) * 2 + 1] : 0.0;
      re += ar * br + ai * bi;
      im += ar * bi - ai * br;
    }
    const float rh = (float)re, ih = (float)im;
    X[idx] = make_float4(rh, (float)(re - (double)rh), ih, (float)(im - (double)ih));
  }
}

// ||d_m||^2 in FP64, stored as double-float.
__global__ void anorm_kernel(const float *__restrict__ d, int M, int J, int H,
                             float2 *__restrict__ NA) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int HJ = H * J;
  double n2 = 0.0;
  for (int k = 0; k < H; ++k)
    for (int j = 0; j < J; ++j) {
      const double re = d[((size_t)m * HJ + k * J + j) * 2];
      const double im = k ? (double)d[((size_t)m * HJ + k * J + j) * 2 + 1] : 0.0;
      n2 += (k ? 2.0 : 1.0) * (re * re + im * im);
    }
  const float hi = (float)n2;
  NA[m] = make_float2(hi, (float)(n2 - (double)hi));
}

// Tables of the tensor-core path: the packed steered dictionary (fp16 of
// kDictScale times the entries, row r*M + m = S_r d_m, angle-major so that 32 consecutive rows hold different
// atoms; the packed layout described in rsc_internal.h), the
// per-harmonic cross-Gram table H_k(a, b) in double-float and the TMA map.
// Returns RSC_OK also when the sizes are outside the path (tables left null).
int build_tc_tables(rsc_dict *d, cudaStream_t st) {
  const int M = d->M, J = d->J, H = d->H, R = d->R;
  const int n = J + 2 * d->kmax * J;
  d->n = n;
  const size_t rows = (size_t)M * R;
  const int L = n <= kTcKst ? kTcKst : kTcKstLong;
  d->row_len = L;
  if (n > kTcMaxN || rows * L * 2 > ((size_t)1 << 30) ||
      (size_t)M * M * H * 16 > ((size_t)1 << 28))
    return RSC_OK;
  const bool paired = L == kTcKst && rsc_paired_ok(J, d->kmax, R);
  if (paired) {
    int ne, no;
    rsc_paired_counts(J, d->kmax, &ne, &no);
    d->ke = (ne + 15) / 16;
    d->ko = (no + 15) / 16;
  }
  cudaError_t e = cudaMalloc(&d->steered_f16, rows * L * 2);
  if (e == cudaSuccess && paired) e = cudaMalloc(&d->paired_f16, rows / 2 * kTcKst * 2);
  if (e == cudaSuccess) e = cudaMalloc(&d->xgram, (size_t)M * M * H * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&d->anorm, (size_t)M * sizeof(float2));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  // the tables are built on the device from the uploaded atoms (FP64 arithmetic)
  const int T = 256;
  const int64_t nb = (int64_t)rows * L, np = paired ? (int64_t)rows / 2 * kTcKst : 0;
  steered_rows_kernel<<<(unsigned)((nb + T - 1) / T), T, 0, st>>>(
      d->d, M, J, d->kmax, R, R, L, 0, static_cast<uint16_t *>(d->steered_f16));
  if (paired)
    steered_rows_kernel<<<(unsigned)((np + T - 1) / T), T, 0, st>>>(
        d->d, M, J, d->kmax, R, R / 2, kTcKst, 1, static_cast<uint16_t *>(d->paired_f16));
  const int64_t nx = (int64_t)M * M * H;
  xgram_kernel<<<(unsigned)((nx + T - 1) / T), T, 0, st>>>(d->d, M, J, H, d->xgram);
  anorm_kernel<<<(M + T - 1) / T, T, 0, st>>>(d->d, M, J, H, d->anorm);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rsc_cuda_fail(e);

  int rc = encode_rows_map(&d->tmap_b, d->steered_f16, rows, kTcBN, L);
  if (rc == RSC_OK) rc = encode_rows_map(&d->tmap_bs, d->steered_f16, rows, kTcSN, L);
  if (rc == RSC_OK && paired)
    rc = encode_rows_map(&d->tmap_bp, d->paired_f16, rows / 2, kTcSNP, kTcKst);
  return rc;
}

int check_device(const rsc_dict *d) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return dev == d->device ? RSC_OK : RSC_ERR_INVALID;
}

// The FP16 path splits its patches into at most `groups` (tuning, <=
// kMaxGroups) groups of at least `group_min` patches, one stream each.
constexpr int kMaxGroups = 4;
constexpr int kDefaultGroups = 2;
constexpr int64_t kGroupMin = 65536;
constexpr int kDefaultRefineBlocks = 32;

// ---------------------------------------------------------------- tuning
struct TuneEntry {
  int n, M, R, K;
  rsc_tuning t;
};

bool tuning_in_range(const rsc_tuning &t) {
  return t.groups >= 0 && t.groups <= kMaxGroups && t.group_min >= 0 &&
         t.refine_blocks_per_sm >= 0 && t.refine_blocks_per_sm <= 64 &&
         (t.score_stages == 0 || (t.score_stages >= 2 && t.score_stages <= 6));
}

// Reads a table of "n M R K groups group_min refine_blocks_per_sm
// score_stages" lines ('#' starts a comment); false when unreadable.
bool read_tuning_table(const char *path, std::vector<TuneEntry> &out) {
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    char *hash = strchr(line, '#');
    if (hash) *hash = 0;
    TuneEntry e{};
    int v[8];
    if (sscanf(line, "%d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6],
               &v[7]) != 8)
      continue;
    e.n = v[0];
    e.M = v[1];
    e.R = v[2];
    e.K = v[3];
    e.t = rsc_tuning{v[4], v[5], v[6], v[7], 1};
    if (tuning_in_range(e.t)) out.push_back(e);
  }
  fclose(f);
  return true;
}

std::once_flag g_table_once;
std::vector<TuneEntry> g_table;

// The process-wide table: RSC_TUNING_TABLE, else rsc_tuning.txt beside this
// library (found with dladdr); absent or unreadable means no entries.
void load_default_table() {
  std::string path;
  const char *env = getenv("RSC_TUNING_TABLE");
  if (env && *env) {
    path = env;
  } else {
    Dl_info info;
    if (dladdr(reinterpret_cast<void *>(&rsc_version), &info) && info.dli_fname) {
      path = info.dli_fname;
      const size_t slash = path.rfind('/');
      path = (slash == std::string::npos ? std::string(".") : path.substr(0, slash)) +
             "/rsc_tuning.txt";
    }
  }
  if (!path.empty()) read_tuning_table(path.c_str(), g_table);
}

// A ring depth the dictionary's layout has, or 0.
int valid_stages(const rsc_dict *d, int st) {
  if (!d->steered_f16 || st == 0) return 0;
  int a = 0, b = 0;
  rsc_score_stage_options(d->row_len, d->paired_f16 != nullptr, &a, &b);
  return (st == a || st == b) ? st : 0;
}

// Field by field: the override, the table entry for K, the default.
rsc_tuning effective_tuning(const rsc_dict *d, int K) {
  const rsc_tuning &ov = d->tune_override;
  const rsc_tuning tb = (K >= 1 && K <= kMaxK) ? d->tune_table[K] : rsc_tuning{};
  rsc_tuning r{};
  int src = 0;
  auto pick = [&](int32_t o, int32_t t, int32_t dflt) {
    if (o > 0) {
      src = 2;
      return o;
    }
    if (t > 0) {
      if (src < 1) src = 1;
      return t;
    }
    return dflt;
  };
  r.groups = pick(ov.groups, tb.groups, kDefaultGroups);
  r.group_min = pick(ov.group_min, tb.group_min, (int32_t)kGroupMin);
  r.refine_blocks_per_sm = pick(ov.refine_blocks_per_sm, tb.refine_blocks_per_sm,
                                kDefaultRefineBlocks);
  int dflt_st = 0, other = 0;
  if (d->steered_f16) rsc_score_stage_options(d->row_len, d->paired_f16 != nullptr, &dflt_st, &other);
  r.score_stages = pick(valid_stages(d, ov.score_stages), valid_stages(d, tb.score_stages), dflt_st);
  r.source = src;
  return r;
}

// Splits P patches of the FP16 path into G groups (one stream each); returns G
// and fills Pg[] and the scratch bytes of each group.
int f16_groups(const rsc_dict *dict, int64_t P, int K, int64_t Pg[], size_t bytes[]);

// Scratch of the FP16 path for P patches and K steps (256-byte aligned parts).
size_t f16_scratch_bytes(int64_t P, int K, int L) {
  int nD = 0, nF = 0, nI = 0;
  rsc_state_layout(K, &nD, &nF, &nI);
  auto al256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return al256((size_t)P * L * 2) + 2 * al256((size_t)P * kTcCand * 4) +
         al256((size_t)P * kTcSplit * 4) + al256((size_t)P * kTcSplit * 8) +
         2 * al256((size_t)P * 4) + al256((size_t)nD * P * 8) + al256((size_t)nF * P * 4) +
         al256((size_t)nI * P * 4) + 2 * al256((size_t)(P + 4) * 4);
}

int f16_groups(const rsc_dict *dict, int64_t P, int K, int64_t Pg[], size_t bytes[]) {
  const rsc_tuning tu = effective_tuning(dict, K);
  int G = (int)(P / (tu.group_min > 0 ? tu.group_min : kGroupMin));
  const int gmax = tu.groups < 1 ? 1 : (tu.groups > kMaxGroups ? kMaxGroups : tu.groups);
  G = G < 1 ? 1 : (G > gmax ? gmax : G);
  if (dict->timing == 2) G = 1;  // timing of each kernel alone
  int64_t done = 0;
  for (int g = 0, left = G; g < G; ++g, --left) {
    Pg[g] = left == 1 ? P - done : (((P - done) / left + 255) & ~(int64_t)255);
    bytes[g] = f16_scratch_bytes(Pg[g], K, dict->row_len);
    done += Pg[g];
  }
  return G;
}

// Enqueues the FP16 path for the patches of `a` on `st`: init, K x (scoring,
// refine), then the FP32 hand-off of the patches the path gives back, with the
// scratch (f16_scratch_bytes) at `scratch`.
int encode_f16_group(const rsc_dict *dict, const RompArgs &base, unsigned char *scratch,
                     cudaStream_t st) {
  const int64_t P = base.P;
  const int K = base.K;
  if (P == 0) return RSC_OK;
  int nD = 0, nF = 0, nI = 0;
  const int cap = rsc_state_layout(K, &nD, &nF, &nI);
  auto al256 = [](size_t v) { return (v + 255) & ~(size_t)255; };
  unsigned char *q = scratch;
  auto take = [&](size_t b) {
    unsigned char *r = q;
    q += al256(b);
    return r;
  };
  RefineArgs ra;
  ra.x = base.x;
  ra.P = P;
  ra.K = K;
  ra.M = dict->M;
  ra.J = dict->J;
  ra.kmax = dict->kmax;
  ra.R = dict->R;
  ra.H = dict->H;
  ra.n = dict->n;
  ra.d = dict->d;
  ra.tw = dict->tw;
  ra.xgram = dict->xgram;
  ra.anorm = dict->anorm;
  ra.L = dict->row_len;
  ra.A = take((size_t)P * ra.L * 2);
  ra.cand_idx = reinterpret_cast<int *>(take((size_t)P * kTcCand * 4));
  ra.cand_val = reinterpret_cast<float *>(take((size_t)P * kTcCand * 4));
  ra.cand_disc = reinterpret_cast<float *>(take((size_t)P * kTcSplit * 4));
  ra.cand_mask = reinterpret_cast<unsigned *>(take((size_t)P * kTcSplit * 8));
  ra.status = reinterpret_cast<int *>(take((size_t)P * 4));
  ra.win = reinterpret_cast<float *>(take((size_t)P * 4));
  ra.sD = reinterpret_cast<double *>(take((size_t)nD * P * 8));
  ra.sF = reinterpret_cast<float *>(take((size_t)nF * P * 4));
  ra.sI = reinterpret_cast<int *>(take((size_t)nI * P * 4));
  int *redo = reinterpret_cast<int *>(take((size_t)(P + 4) * 4));
  ra.redo_count = redo;
  ra.redo_list = redo + 4;
  int *slow = reinterpret_cast<int *>(take((size_t)(P + 4) * 4));
  ra.slow_count = slow;
  ra.slow_list = slow + 4;
  ra.paired = dict->paired_f16 != nullptr ? 1 : 0;
  ra.atom = base.atom;
  ra.angle_idx = base.angle_idx;
  ra.angle = base.angle;
  ra.coef = base.coef;
  ra.resid_norm2 = base.resid_norm2;
  ra.fallbacks = dict->fallbacks;
  ScoreArgs sa;
  sa.P = P;
  sa.ksteps = (dict->n + 15) / 16;
  sa.L = ra.L;
  sa.paired = ra.paired;
  sa.ke = dict->ke;
  sa.ko = dict->ko;
  sa.MR = sa.paired ? dict->M * (dict->R / 2) : dict->M * dict->R;
  // B rows per chunk: kTcSN atoms (plain) or kTcSNP atom pairs (paired)
  const int br = sa.paired ? kTcSNP : kTcSN;
  sa.nchunks = (sa.MR + br - 1) / br;
  sa.status = ra.status;
  sa.cand_idx = const_cast<int *>(ra.cand_idx);
  sa.cand_val = const_cast<float *>(ra.cand_val);
  sa.cand_disc = const_cast<float *>(ra.cand_disc);
  sa.cand_mask = const_cast<unsigned *>(ra.cand_mask);
  sa.win = ra.win;
  sa.err = dict->err;
  sa.wait_ns = dict->wait_ns ? dict->wait_ns : 2000000000ull;
  const rsc_tuning tu = effective_tuning(dict, K);
  sa.stages = tu.score_stages;
  ra.blocks_per_sm = tu.refine_blocks_per_sm;
  CUtensorMap tmA;
  int rc = encode_rows_map(&tmA, ra.A, (size_t)P, kTcBN, ra.L);
  if (rc == RSC_OK) {
    const cudaError_t e = cudaMemsetAsync(redo, 0, sizeof(int), st);
    if (e != cudaSuccess) rc = rsc_cuda_fail(e);
  }
  if (rc == RSC_OK) {
    const int slot = timing_begin(dict, 2, st);
    rc = rsc_launch_refine(ra, true, st);
    timing_end(dict, slot, st);
  }
  for (int step = 0; step < K && rc == RSC_OK; ++step) {
    int slot = timing_begin(dict, 0, st);
    rc = rsc_launch_score(sa, tmA, sa.paired ? dict->tmap_bp : dict->tmap_bs, st);
    timing_end(dict, slot, st);
    if (rc != RSC_OK) break;
    slot = timing_begin(dict, 2, st);
    rc = rsc_launch_refine(ra, false, st);
    timing_end(dict, slot, st);
  }
  if (rc == RSC_OK) {
    RompArgs a = base;
    a.redo_count = ra.redo_count;
    a.redo_list = ra.redo_list;
    a.resume_sI = ra.sI;
    a.resume_P = P;
    a.resume_cap = cap;
    a.fallbacks = nullptr;
    const int slot = timing_begin(dict, 1, st);
    rc = rsc_launch_f32(a, st);
    timing_end(dict, slot, st);
  }
  return rc;
}

}  // namespace

int rsc_encode_rows_map(CUtensorMap *map, void *base, size_t rows, int box_rows, int row_len) {
  return encode_rows_map(map, base, rows, box_rows, row_len);
}

int rsc_cuda_fail(cudaError_t e) {
  snprintf(g_cuda_msg, sizeof g_cuda_msg, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return RSC_ERR_CUDA;
}

// The scratch pools.  The device's default pool has a release threshold of
// 0: it gives freed memory back at every synchronisation, and the next call's
// allocation maps it again (measured at 10^6 patches: 1.5 ms of a 10.9 ms
// call, and a host-to-device copy on another stream did not overlap it).  The
// library's own pool keeps what it has handed out; other users of the
// default pool are not affected.
namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
}  // namespace

cudaError_t rsc_scratch_alloc(void **p, size_t bytes, cudaStream_t st) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&g_pool[dev], &props);
      if (e != cudaSuccess) {
        g_pool[dev] = nullptr;
        return e;
      }
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

cudaError_t rsc_scratch_free(void *p, cudaStream_t st) { return cudaFreeAsync(p, st); }

void rsc_scratch_trim() {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  for (int i = 0; i < kMaxPoolDevices; ++i)
    if (g_pool[i]) cudaMemPoolTrimTo(g_pool[i], 0);
}

extern "C" {

const char *rsc_last_cuda_error(void) { return g_cuda_msg; }

int rsc_version(void) { return (1 << 16) | 0; }

const char *rsc_status_string(int s) {
  switch (s) {
    case RSC_OK: return "ok";
    case RSC_ERR_INVALID: return "invalid argument";
    case RSC_ERR_OOM: return "out of memory";
    case RSC_ERR_CUDA: return "CUDA error";
    case RSC_ERR_TIMEOUT: return "device-side wait timed out";
    case RSC_ERR_UNSUPPORTED: return "unsupported size or option";
    default: return "unknown status";
  }
}

int rsc_dict_create(const float *coef, rsc_dims dims, void *stream, rsc_dict **out) {
  RscRange nvtx_range("rsc_dict_create");
  if (!out) return RSC_ERR_INVALID;
  *out = nullptr;
  if (!coef || !aligned16(coef)) return RSC_ERR_INVALID;
  if (dims.M < 1 || dims.J < 1 || dims.kmax < 0 || dims.R < 1) return RSC_ERR_INVALID;
  const int H = dims.kmax + 1;
  if (dims.kmax > kMaxKmax || dims.R > kMaxR || (int64_t)H * dims.J > kMaxEntries)
    return RSC_ERR_UNSUPPORTED;
  if ((int64_t)dims.M * dims.R >= (int64_t)1 << 30) return RSC_ERR_UNSUPPORTED;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int M = dims.M, J = dims.J, R = dims.R, HJ = H * J;
  const size_t nd = (size_t)M * HJ * 2;

  std::vector<float> h(nd);
  cudaError_t e = cudaMemcpyAsync(h.data(), coef, nd * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rsc_cuda_fail(e);

  // Im of k = 0 is ignored: store it as 0.  Atoms must have unit norm.
  for (int m = 0; m < M; ++m) {
    double n2 = 0.0;
    for (int k = 0; k < H; ++k)
      for (int j = 0; j < J; ++j) {
        float *c = &h[((size_t)m * HJ + k * J + j) * 2];
        if (k == 0) c[1] = 0.0f;
        if (!isfinite(c[0]) || !isfinite(c[1])) return RSC_ERR_INVALID;
        double w = k ? 2.0 : 1.0;
        n2 += w * ((double)c[0] * c[0] + (double)c[1] * c[1]);
      }
    if (fabs(n2 - 1.0) > 1e-4) return RSC_ERR_INVALID;
  }
  std::vector<float> hT((size_t)2 * HJ * M);
  for (int m = 0; m < M; ++m)
    for (int q = 0; q < HJ; ++q) {
      hT[(size_t)q * M + m] = h[((size_t)m * HJ + q) * 2];
      hT[(size_t)(HJ + q) * M + m] = h[((size_t)m * HJ + q) * 2 + 1];
    }
  // steering factors exp(-i k 2 pi r / R) of Eq. (Sr) as cos/sin in
  // double-float (hi + lo) from FP64, argument reduced exactly: k r mod R
  std::vector<float> tw((size_t)4 * H * R);
  for (int k = 0; k < H; ++k)
    for (int r = 0; r < R; ++r) {
      const double th = 2.0 * M_PI * (double)(((int64_t)k * r) % R) / (double)R;
      const double c = cos(th), s = sin(th);
      const float ch = (float)c, sh = (float)s;
      tw[(size_t)(0 * H + k) * R + r] = ch;
      tw[(size_t)(1 * H + k) * R + r] = (float)(c - (double)ch);
      tw[(size_t)(2 * H + k) * R + r] = sh;
      tw[(size_t)(3 * H + k) * R + r] = (float)(s - (double)sh);
    }

  rsc_dict *d = new rsc_dict();
  memset(d, 0, sizeof *d);
  d->M = M;
  d->J = J;
  d->kmax = dims.kmax;
  d->R = R;
  d->H = H;
  e = cudaGetDevice(&d->device);
  if (e == cudaSuccess) e = cudaMalloc(&d->d, nd * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d->dT, hT.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d->tw, tw.size() * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d->fallbacks, sizeof(unsigned long long));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    free_dict(d);
    return RSC_ERR_OOM;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d->d, h.data(), nd * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d->dT, hT.data(), hT.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d->tw, tw.data(), tw.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d->fallbacks, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_dict(d);
    return rsc_cuda_fail(e);
  }
  const int rc = build_tc_tables(d, st);
  if (rc != RSC_OK) {
    free_dict(d);
    return rc;
  }
  // the measured tunings of this (n, M, R), per K
  std::call_once(g_table_once, load_default_table);
  for (const TuneEntry &te : g_table)
    if (te.n == d->n && te.M == M && te.R == R && te.K >= 1 && te.K <= kMaxK)
      d->tune_table[te.K] = te.t;
  *out = d;
  return RSC_OK;
}

int rsc_dict_destroy(rsc_dict *dict) {
  free_dict(dict);
  // scratch the pool keeps beyond what calls in flight hold goes back
  rsc_scratch_trim();
  return RSC_OK;
}

int rsc_dict_dims(const rsc_dict *dict, rsc_dims *dims) {
  if (!dict || !dims) return RSC_ERR_INVALID;
  dims->M = dict->M;
  dims->J = dict->J;
  dims->kmax = dict->kmax;
  dims->R = dict->R;
  return RSC_OK;
}

namespace {

// Host buffers of rsc_encode_host for one call of encode_impl: the patches
// and the outputs, laid out as rsc_encode's device arguments.
struct HostIO {
  const float *x;
  int32_t *atom, *angle_idx;
  float *angle;
  double *coef;
  float *resid_norm2;
};

RompArgs base_args(const rsc_dict *dict, const float *x, int64_t P, int32_t K, int32_t *atom,
                   int32_t *angle_idx, float *angle, double *coef, float *resid_norm2) {
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
  a.fallbacks = dict->fallbacks;
  return a;
}

// Copies of patches [off, off + n) of a call with host buffers: the patches
// in (to the device slice at ad.x), or the outputs out (from ad's slices).
cudaError_t copy_in(const HostIO &h, const RompArgs &ad, int64_t off, int64_t n, int64_t vec,
                    cudaStream_t st) {
  return cudaMemcpyAsync(const_cast<float *>(ad.x), h.x + off * vec, (size_t)(n * vec) * sizeof(float),
                         cudaMemcpyHostToDevice, st);
}

cudaError_t copy_out(const HostIO &h, const RompArgs &ad, int64_t off, int64_t n, int K,
                     cudaStream_t st) {
  const size_t nk = (size_t)(n * K);
  cudaError_t e = cudaMemcpyAsync(h.atom + off * K, ad.atom, nk * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.angle_idx + off * K, ad.angle_idx, nk * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && h.angle)
    e = cudaMemcpyAsync(h.angle + off * K, ad.angle, nk * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.coef + off * K, ad.coef, nk * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && h.resid_norm2)
    e = cudaMemcpyAsync(h.resid_norm2 + off, ad.resid_norm2, (size_t)n * sizeof(float),
                        cudaMemcpyDeviceToHost, st);
  return e;
}

// The coder on `st` (arguments validated).  With host buffers `h`, a's
// pointers are device staging buffers: each stream group copies its own
// patches in before its first kernel and its outputs out after its last, so
// that one group's copies overlap another group's kernels.
int encode_impl(const rsc_dict *dict, const RompArgs &a, int32_t prec, cudaStream_t st,
                const HostIO *h) {
  const int64_t P = a.P, vec = (int64_t)dict->H * dict->J * 2;
  const int K = a.K;
  int rc = RSC_OK;
  cudaError_t e = cudaSuccess;
  if (prec == RSC_FP32 || prec == RSC_FP32_PRUNE) {
    if (h && (e = copy_in(*h, a, 0, P, vec, st)) != cudaSuccess) return rsc_cuda_fail(e);
    RompArgs af = a;
    af.prune = prec == RSC_FP32_PRUNE;
    const int slot = timing_begin(dict, 0, st);
    rc = rsc_launch_f32(af, st);
    timing_end(dict, slot, st);
    if (rc == RSC_OK && h && (e = copy_out(*h, a, 0, P, K, st)) != cudaSuccess)
      rc = rsc_cuda_fail(e);
    return rc;
  }

  // FP16 tensor-core path, split per greedy step into a scoring kernel and a
  // per-patch refine kernel; patches it hands back are coded by the FP32 path
  if (!dict->steered_f16 || K > kTcMaxK || P >= ((int64_t)1 << 31)) return RSC_ERR_UNSUPPORTED;
  // Independent groups of patches on their own streams: the scoring pass of
  // one group (tensor and ALU pipes, one CTA per SM) runs beside the refine
  // pass of another (latency-bound), so each hides part of the other.
  int64_t Pg[kMaxGroups] = {};
  size_t bytes[kMaxGroups] = {}, total = 0;
  const int G = f16_groups(dict, P, K, Pg, bytes);
  for (int g = 0; g < G; ++g) total += bytes[g];
  // a scratch budget set on the dictionary stands in for the allocator's
  // refusal (testing the error path without exhausting device memory)
  if (dict->scratch_limit && total > dict->scratch_limit) return RSC_ERR_OOM;
  unsigned char *scratch = nullptr;
  e = rsc_scratch_alloc(reinterpret_cast<void **>(&scratch), total, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  cudaStream_t sg[kMaxGroups] = {};
  cudaEvent_t fork = nullptr, join[kMaxGroups] = {}, cin[kMaxGroups] = {};
  sg[0] = st;
  if (G > 1) {
    e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(fork, st);
    for (int g = 1; g < G && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&sg[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[g], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(sg[g], fork, 0);
    }
    // with host buffers the groups' copies in go one after the other, so
    // that group 0 starts once its own patches are in rather than once all
    // groups' copies, sharing the link, are done
    for (int g = 0; h && g + 1 < G && e == cudaSuccess; ++g)
      e = cudaEventCreateWithFlags(&cin[g], cudaEventDisableTiming);
    if (e != cudaSuccess) rc = rsc_cuda_fail(e);
  }
  int64_t off = 0;
  size_t soff = 0;
  static const char *const kGroupRange[kMaxGroups] = {"rsc_encode group 0", "rsc_encode group 1",
                                                      "rsc_encode group 2", "rsc_encode group 3"};
  for (int g = 0; g < G && rc == RSC_OK; ++g) {
    RscRange nvtx_group(kGroupRange[g]);
    RompArgs ag = a;
    ag.x = a.x + off * vec;
    ag.P = Pg[g];
    ag.atom = a.atom + off * K;
    ag.angle_idx = a.angle_idx + off * K;
    ag.angle = a.angle ? a.angle + off * K : nullptr;
    ag.coef = a.coef + off * K;
    ag.resid_norm2 = a.resid_norm2 ? a.resid_norm2 + off : nullptr;
    if (h) {
      if (g > 0 && cin[g - 1]) e = cudaStreamWaitEvent(sg[g], cin[g - 1], 0);
      if (e == cudaSuccess) e = copy_in(*h, ag, off, Pg[g], vec, sg[g]);
      if (e == cudaSuccess && cin[g]) e = cudaEventRecord(cin[g], sg[g]);
      if (e != cudaSuccess) rc = rsc_cuda_fail(e);
    }
    if (rc == RSC_OK) rc = encode_f16_group(dict, ag, scratch + soff, sg[g]);
    if (rc == RSC_OK && h && (e = copy_out(*h, ag, off, Pg[g], K, sg[g])) != cudaSuccess)
      rc = rsc_cuda_fail(e);
    off += Pg[g];
    soff += bytes[g];
  }
  // join every side stream (also after a failed launch, so that the scratch
  // is released after all work that uses it)
  for (int g = 1; g < G; ++g) {
    if (!sg[g] || !join[g]) continue;
    e = cudaEventRecord(join[g], sg[g]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, join[g], 0);
    if (rc == RSC_OK && e != cudaSuccess) rc = rsc_cuda_fail(e);
  }
  if (fork) cudaEventDestroy(fork);
  for (int g = 0; g < G; ++g)
    if (cin[g]) cudaEventDestroy(cin[g]);
  for (int g = 1; g < G; ++g) {
    if (join[g]) cudaEventDestroy(join[g]);
    if (sg[g]) cudaStreamDestroy(sg[g]);
  }
  e = rsc_scratch_free(scratch, st);
  if (rc == RSC_OK && e != cudaSuccess) rc = rsc_cuda_fail(e);
  return rc;
}

}  // namespace

int rsc_encode(const rsc_dict *dict, const float *x, int64_t P, int32_t K, int32_t prec,
               int32_t *atom, int32_t *angle_idx, float *angle, double *coef, float *resid_norm2,
               void *stream) {
  RscRange nvtx_range("rsc_encode");
  if (!dict || P < 0 || K < 1 || K > kMaxK) return RSC_ERR_INVALID;
  if (prec != RSC_FP32 && prec != RSC_FP32_PRUNE && prec != RSC_F16_RESCORE) return RSC_ERR_INVALID;
  if (P == 0) return RSC_OK;
  if (!x || !atom || !angle_idx || !coef) return RSC_ERR_INVALID;
  if (!aligned16(x) || !aligned_as<int32_t>(atom) || !aligned_as<int32_t>(angle_idx) ||
      !aligned_as<double>(coef) || (angle && !aligned_as<float>(angle)) ||
      (resid_norm2 && !aligned_as<float>(resid_norm2)))
    return RSC_ERR_INVALID;
  const int rc = check_device(dict);
  if (rc != RSC_OK) return rc;
  const RompArgs a = base_args(dict, x, P, K, atom, angle_idx, angle, coef, resid_norm2);
  return encode_impl(dict, a, prec, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

int rsc_workspace_bytes(const rsc_dict *dict, const rsc_basis *basis, int64_t P, int32_t n_images,
                        int32_t K, int32_t prec, uint64_t *bytes) {
  if (!dict || !bytes || P < 0 || n_images < 0 || K < 1 || K > kMaxK) return RSC_ERR_INVALID;
  if (prec != RSC_FP32 && prec != RSC_FP32_PRUNE && prec != RSC_F16_RESCORE) return RSC_ERR_INVALID;
  uint64_t total = 0;
  if (P > 0 && prec == RSC_F16_RESCORE) {
    int64_t Pg[kMaxGroups] = {};
    size_t b[kMaxGroups] = {};
    const int G = f16_groups(dict, P, K, Pg, b);
    for (int g = 0; g < G; ++g) total += b[g];
  }
  if (basis && P > 0) {
    uint64_t img = 0;
    const int rc = rsc_images_scratch_bytes(basis, P, n_images, &img);
    if (rc != RSC_OK) return rc;
    total += img;
  }
  *bytes = total;
  return RSC_OK;
}

int rsc_encode_host(const rsc_dict *dict, const float *x, int64_t P, int32_t K, int32_t prec,
                    int32_t *atom, int32_t *angle_idx, float *angle, double *coef,
                    float *resid_norm2) {
  RscRange nvtx_range("rsc_encode_host");
  if (!dict || P < 0 || K < 1 || K > kMaxK) return RSC_ERR_INVALID;
  if (prec != RSC_FP32 && prec != RSC_FP32_PRUNE && prec != RSC_F16_RESCORE) return RSC_ERR_INVALID;
  if (P == 0) return RSC_OK;
  if (!x || !atom || !angle_idx || !coef) return RSC_ERR_INVALID;
  int rc = check_device(dict);
  if (rc != RSC_OK) return rc;
  const int64_t vec = (int64_t)dict->H * dict->J * 2;
  // chunks of up to 2^20 patches, two in flight when there are more; within
  // a chunk the stream groups overlap their copies with each other's kernels
  const int64_t cap = (int64_t)1 << 20;
  const int64_t chunk = P < cap ? P : cap;
  const int nb = P > chunk ? 2 : 1;
  HostStage *hs = nullptr;
  {
    std::lock_guard<std::mutex> g(g_stage_mu);
    if (!dict->host_stage) dict->host_stage = new HostStage();
    hs = static_cast<HostStage *>(dict->host_stage);
  }
  std::lock_guard<std::mutex> lock(hs->mu);
  cudaError_t e = hs->reserve(chunk, K, (int)vec, nb);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return RSC_ERR_OOM;
  }
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  rc = RSC_OK;
  for (int64_t lo = 0, ci = 0; rc == RSC_OK && lo < P; lo += chunk, ++ci) {
    const int64_t n = (P - lo) < chunk ? (P - lo) : chunk;
    HostStage::Buf &B = hs->b[ci % nb];
    const RompArgs a = base_args(dict, B.x, n, K, B.atom, B.ang, angle ? B.angf : nullptr, B.coef,
                                 resid_norm2 ? B.rn2 : nullptr);
    const HostIO h{x + lo * vec, atom + lo * K, angle_idx + lo * K, angle ? angle + lo * K : nullptr,
                   coef + lo * K, resid_norm2 ? resid_norm2 + lo : nullptr};
    rc = encode_impl(dict, a, prec, hs->s[ci % nb], &h);
  }
  for (int i = 0; i < 2; ++i) {
    const cudaError_t se = cudaStreamSynchronize(hs->s[i]);
    if (se != cudaSuccess && rc == RSC_OK) rc = rsc_cuda_fail(se);
  }
  return rc;
}

int rsc_dict_check(const rsc_dict *dict, void *stream) {
  if (!dict) return RSC_ERR_INVALID;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  int v = 0;
  e = cudaMemcpy(&v, dict->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(dict->err, 0, sizeof(int));
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  return v;
}

int rsc_dict_set_tuning(rsc_dict *dict, const rsc_tuning *t) {
  if (!dict) return RSC_ERR_INVALID;
  if (!t) {
    dict->tune_override = rsc_tuning{};
    return RSC_OK;
  }
  rsc_tuning v = *t;
  v.source = 0;
  if (!tuning_in_range(v) || (v.score_stages != 0 && !valid_stages(dict, v.score_stages)))
    return RSC_ERR_INVALID;
  dict->tune_override = v;
  return RSC_OK;
}

int rsc_dict_tuning(const rsc_dict *dict, int32_t K, rsc_tuning *out) {
  if (!dict || !out || K < 1 || K > kMaxK) return RSC_ERR_INVALID;
  *out = effective_tuning(dict, K);
  return RSC_OK;
}

int rsc_tuning_table_lookup(const char *path, int32_t n, int32_t M, int32_t R, int32_t K,
                            rsc_tuning *out) {
  if (!path || !out) return RSC_ERR_INVALID;
  std::vector<TuneEntry> tab;
  if (!read_tuning_table(path, tab)) return RSC_ERR_INVALID;
  *out = rsc_tuning{};
  for (const TuneEntry &e : tab)
    if (e.n == n && e.M == M && e.R == R && e.K == K) *out = e.t;
  return RSC_OK;
}

int rsc_dict_set_limits(rsc_dict *dict, uint64_t pipeline_wait_ns, uint64_t scratch_limit) {
  if (!dict) return RSC_ERR_INVALID;
  dict->wait_ns = pipeline_wait_ns;
  dict->scratch_limit = scratch_limit;
  return RSC_OK;
}

int rsc_dict_set_timing(rsc_dict *dict, int enable) {
  if (!dict) return RSC_ERR_INVALID;
  dict->timing = enable == 2 ? 2 : (enable ? 1 : 0);
  return RSC_OK;
}

int rsc_dict_timing(rsc_dict *dict, double ms[3], int64_t launches[3]) {
  if (!dict || !ms || !launches) return RSC_ERR_INVALID;
  for (int i = 0; i < 3; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  TimingLog *log = static_cast<TimingLog *>(dict->timing_state);
  int rc = RSC_OK;
  if (log) {
    for (auto &p : *log) {
      cudaError_t e = cudaEventSynchronize(p.b);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.a, p.b);
      if (e != cudaSuccess) {
        rc = rsc_cuda_fail(e);
        break;
      }
      ms[p.phase] += t;
      launches[p.phase] += 1;
    }
    clear_timing(dict);
  }
  return rc;
}

int rsc_dict_fallback_count(const rsc_dict *dict, int64_t *count) {
  if (!dict || !count) return RSC_ERR_INVALID;
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpy(&v, dict->fallbacks, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(dict->fallbacks, 0, sizeof v);
  if (e != cudaSuccess) return rsc_cuda_fail(e);
  *count = (int64_t)v;
  return RSC_OK;
}

}  // extern "C"
