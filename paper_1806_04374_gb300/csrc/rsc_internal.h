// rsc_internal.h -- state shared by the host side of librsc and its kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "rsc.h"

// Stop rules of the coder (the paper is silent on them; both are readings):
// a patch stops when max |score| <= kStopRel * ||x|| or when the new pivot^2
// of the Cholesky factor is <= kPivotRel times its Gram diagonal entry.
constexpr double kStopRel = 1e-10;
constexpr double kPivotRel = 1e-12;
constexpr int kMaxK = 16;       // greedy steps per patch
constexpr int kMaxKmax = 16;    // highest harmonic
constexpr int kMaxR = 128;      // angles
constexpr int kMaxEntries = 512;  // (kmax+1)*J complex entries per vector

struct rsc_dict {
  int M, J, kmax, R, H;  // H = kmax + 1
  int device;
  float *d;      // [M][H][J][2]  atoms as given
  float *dT;     // [2][H*J][M]   re plane, im plane: lane-per-atom reads
  float *tw;     // [4][H][R]     cos hi, cos lo, sin hi, sin lo of 2 pi k r / R
  int *err;      // device error word (first error code recorded)
  unsigned long long *fallbacks;  // device counter of exact re-scans
  // tensor-core path: steered dictionary and cross-Gram table (null when the
  // sizes are outside what the path handles)
  void *steered_f16;     // [R*M][row_len] fp16 of kDictScale x packed S_r d_m (row r*M + m)
  int row_len;           // packed row length of the tensor-core operands: kTcKst or kTcKstLong
  // paired layout (even R): rows r*M + m for r < R/2, slots split by the
  // parity of k (rsc_slot_code); null when the sizes do not allow it
  void *paired_f16;
  int ke, ko;            // paired: MMA K-steps (16 slots) of the even / odd halves
  float4 *xgram;         // [M][M][H] double-float complex H_k(a,b) = sum_j conj(d_a) d_b
  float2 *anorm;         // [M] ||d_m||^2 in double-float
  int n;                 // packed real length J (2 kmax + 1)
  // per-phase timing (diagnostic): event pairs recorded around launches
  int timing;
  void *timing_state;    // owned std::vector of recorded pairs, see rsc_capi.cu
  CUtensorMap tmap_b;    // TMA map of steered_f16, box 64 x kTcBN (fused kernel)
  CUtensorMap tmap_bs;   // TMA map of steered_f16, box 64 x kTcSN (scoring pass)
  CUtensorMap tmap_bp;   // TMA map of paired_f16, box 64 x kTcSNP (scoring pass)
  // device buffers and streams of rsc_encode_host (rsc_capi.cu), made on its
  // first call and kept until rsc_dict_destroy
  mutable void *host_stage;
  // diagnostic limits (rsc_dict_set_limits; 0 = default): the wait limit of
  // the FP16 scoring kernel's pipeline waits (ns) and a budget for the FP16
  // path's per-call scratch (bytes)
  uint64_t wait_ns;
  uint64_t scratch_limit;
  // tuning (rsc_tuning): the overrides set by rsc_dict_set_tuning, and the
  // table entries of this dictionary's (n, M, R) read at creation, per K
  rsc_tuning tune_override;
  rsc_tuning tune_table[kMaxK + 1];
};

// Packed real coordinates of a half spectrum, shared by the tensor-core
// operands: slot q < J is Re c[j=q, k=0]; slot J + 2 ((k-1) J + j) + c holds
// sqrt(2) Re (c = 0) or sqrt(2) Im (c = 1) of c[j, k], k >= 1.  The Euclidean
// dot product of two packed vectors is the coefficient inner product.
constexpr int kTcKst = 112;  // stored row length of the steered dictionary (fp16)
constexpr int kTcKstLong = 256;  // row length for packed lengths 113..256 (plain layout only)
constexpr int kTcOdd = 64;   // first slot of the odd harmonics in the paired layout
constexpr int kTcMaxN = 256; // packed lengths the tensor-core path handles
constexpr int kTcBN = 128;   // steered atoms per MMA (N) and per TMA box
constexpr int kTcMaxK = 8;   // greedy steps the tensor-core path handles

constexpr int kTcSN = 256;   // steered atoms per chunk (MMA N) of the scoring pass
constexpr int kTcSNP = 128;  // steered-atom pairs per chunk (MMA N), paired layout

// Slot layouts of a packed row (kTcKst fp16 slots) of the tensor-core path;
// returns (e << 8) | (k << 1) | c for slot q holding Re (c = 0) or Im (c = 1)
// of entry e = k J + j (weight sqrt(2) for k >= 1), or -1 for a zero slot.
// Plain: the order described above, zeros from slot n.  Paired: the even
// harmonics (k = 0, then k = 2, 4, ... in (Re, Im) pairs) from slot 0 and
// the odd harmonics (k = 1, 3, ...) from slot kTcOdd.  Steering by half a
// turn multiplies harmonic k by (-1)^k (Eq. (Sr)), so with E and O the even
// and odd parts of <S_r d, x>, <S_{r + R/2} d, x> = E - O and
// max(|E + O|, |E - O|) = |E| + |O|: one contraction scores both angles.
__host__ __device__ inline int rsc_paired_counts(int J, int kmax, int *ne, int *no) {
  *ne = J + 2 * J * (kmax / 2);
  *no = 2 * J * ((kmax + 1) / 2);
  return 0;
}
__host__ __device__ inline bool rsc_paired_ok(int J, int kmax, int R) {
  int ne, no;
  rsc_paired_counts(J, kmax, &ne, &no);
  return R >= 2 && (R % 2) == 0 && kmax >= 1 && ne <= kTcOdd && no <= kTcKst - kTcOdd;
}
__host__ __device__ inline int rsc_slot_code(int q, int J, int kmax, bool paired) {
  if (!paired) {
    const int n = J + 2 * kmax * J;
    if (q < J) return q << 8;
    if (q >= n) return -1;
    const int qq = q - J, e = J + (qq >> 1);
    return (e << 8) | ((e / J) << 1) | (qq & 1);
  }
  int ne, no;
  rsc_paired_counts(J, kmax, &ne, &no);
  if (q < J) return q << 8;
  int qq, k0;
  if (q < ne) {
    qq = q - J;
    k0 = 2;
  } else if (q >= kTcOdd && q < kTcOdd + no) {
    qq = q - kTcOdd;
    k0 = 1;
  } else {
    return -1;
  }
  const int idx = qq >> 1, k = k0 + 2 * (idx / J), e = k * J + idx % J;
  return (e << 8) | (k << 1) | (qq & 1);
}

// fp16 operand scaling of the tensor-core path.  The steered dictionary holds
// kDictScale * entries (unit atoms: |entries| <= 256); a residual row is
// stored times 2^(kRowLog2 - e), e = rsc_row_exponent(bound) for a bound >= the
// row's norm, so its entries are below 2^kRowLog2 and far from fp16's
// subnormal range.  A score read from the accumulator is therefore
// 2^(16 - e) times the true score; both scales are powers of two (exact).
constexpr float kDictScale = 256.0f;
constexpr int kRowLog2 = 8;
__host__ __device__ inline int rsc_row_exponent(float bound) {
  int e = 0;
  (void)frexpf(bound, &e);  // bound = f 2^e, f in [0.5, 1); 0 for bound = 0
  return e < -100 ? -100 : (e > 126 ? 126 : e);
}

struct TcArgs {
  const float *x;
  int64_t P;
  int K;
  int M, J, kmax, R, H, n, ksteps, MR, nchunks;
  const float *d;
  const float *tw;
  const float4 *xgram;
  int32_t *atom;
  int32_t *angle_idx;
  float *angle;
  double *coef;
  float *resid_norm2;
  int *err;
  int *redo_list;
  int *redo_count;
  unsigned long long *fallbacks;
};

// FP16 tensor-core scoring path fused with the per-patch steps in one
// persistent kernel (romp_tc.cu; used by rsc_encode_noalloc); patches whose
// candidates overflow are appended to redo_list for the FP32 path.
int rsc_launch_tc(const TcArgs &a, const CUtensorMap &tmap, cudaStream_t stream);

// TMA map of a row-major fp16 matrix [rows][row_len] (row_len * 2 bytes a
// multiple of 16): box 64 columns x box_rows rows, 128-byte swizzle, zero fill
// outside the matrix.
int rsc_encode_rows_map(CUtensorMap *map, void *base, size_t rows, int box_rows, int row_len);

// What other translation units need of a basis handle (basis.cu owns it).
struct rsc_basis_view {
  int device, npix, n, J, nout;
  const float *X;  // device [n][npix]: real synthesis matrix, packed column order
};
int rsc_basis_internals(const rsc_basis *basis, rsc_basis_view *view);
// Scratch bytes rsc_encode_images takes for its work list and projected
// windows (basis.cu).
int rsc_images_scratch_bytes(const rsc_basis *basis, int64_t P, int32_t n_images, uint64_t *bytes);

// Candidates kept per patch and greedy step by the tensor-core scoring:
// kTcTop per list (the fused kernel: block maxima; the split scoring pass:
// blocks of 32 rows within the window, one list per slice of the accumulator
// columns, kTcSplit slices, kTcCand in all, expanded by a class mask, see
// ScoreArgs).
constexpr int kTcTop = 4;
constexpr int kTcSplit = 2;
constexpr int kTcCand = kTcSplit * kTcTop;

// One scoring pass of the split FP16 path (romp_score.cu): packed fp16
// residual rows (TMA map tmA: [P][kTcKst]) times the steered dictionary
// (tmB) -> per patch and slice (kTcSplit per chunk of rows): up to kTcTop
// blocks of 32 rows (first row b, multiple of 32; rows b + u, u < 32) whose
// maximum |score| lies within the window of the slice's best, their maxima,
// the mask of the columns u whose largest value over all blocks of the slice
// lies within it, the column of the slice's best value, and a bound on every
// value left out.  Every row within the window is b + u for a kept b and a
// masked u of the same slice.
struct ScoreArgs {
  int64_t P;
  int ksteps, MR, nchunks;
  // paired layout (rsc_slot_code): B rows are steered-atom pairs (r < R/2),
  // MR counts pairs, and the MMAs run ke / ko K-steps on the even / odd halves
  int paired, ke, ko;
  int L;  // packed row length (kTcKst or kTcKstLong; the latter plain only)
  const int *status;  // > 0: patch still being coded
  int *cand_idx;      // [P][kTcCand] first rows of the kept blocks (-1: none)
  float *cand_val;    // [P][kTcCand] their maxima (accumulator units)
  float *cand_disc;   // [P][kTcSplit] bound on the values each slice left out
  unsigned *cand_mask;  // [P][2 kTcSplit] per slice: column mask, column of its best
  // [P] per-patch certification window in accumulator units (written by the
  // refine pass with the row): a block maximum more than `win` below the
  // running best can neither win nor reach the window, so it is not kept
  const float *win;
  int *err;
  // limit of the pipeline waits (ns); the waits that drain issued copies and
  // MMAs before the CTA exits keep their own limit
  uint64_t wait_ns;
  int stages;  // dictionary-ring stages (one of rsc_score_stage_options; else the default)
};
int rsc_launch_score(const ScoreArgs &a, const CUtensorMap &tmA, const CUtensorMap &tmB,
                     cudaStream_t stream);
// The two ring depths instantiated for a row length and layout (the first
// is the default).
int rsc_score_stage_options(int L, int paired, int *dflt, int *other);

// Per-patch steps of the split FP16 path (romp_refine.cu): init (packed x,
// state) or one refine (certify, re-score, Cholesky, residual).
struct RefineArgs {
  const float *x;
  int64_t P;
  int K, M, J, kmax, R, H, n;
  const float *d;
  const float *tw;       // [4][H][R]
  const float4 *xgram;
  const float2 *anorm;   // [M] ||d_m||^2 in double-float
  unsigned char *A;      // [P][L] fp16 packed residual rows, scaled (see below)
  int L;                 // packed row length (kTcKst or kTcKstLong)
  const int *cand_idx;
  const float *cand_val;
  const float *cand_disc;
  const unsigned *cand_mask;  // see ScoreArgs
  float *win;            // [P] window of the next scoring pass (see ScoreArgs)
  int paired;            // rows and candidates in the paired layout (rsc_slot_code)
  int *status;           // 1 active, 0 done, -1 handed to the FP32 path
  double *sD;            // state, structure of arrays
  float *sF;
  int *sI;
  int32_t *atom;
  int32_t *angle_idx;
  float *angle;
  double *coef;
  float *resid_norm2;
  int *redo_list;
  int *redo_count;
  // [P] + counter: patches whose window holds more than one unit, finished by
  // the refine's second pass (see romp_refine.cu)
  int *slow_list;
  int *slow_count;
  unsigned long long *fallbacks;
  int blocks_per_sm;  // grid cap of the init/refine launches per SM (0: 32)
};
int rsc_launch_refine(const RefineArgs &a, bool init, cudaStream_t stream);
// Number of double / float / int state arrays for K steps; returns the
// compile-time capacity used (K rounded up to 3, 5 or 8).
int rsc_state_layout(int K, int *nD, int *nF, int *nI);

struct RompArgs {
  const float *x;
  int64_t P;
  int K;
  int M, J, kmax, R, H;
  const float *d;
  const float *dT;
  const float *tw;
  int32_t *atom;
  int32_t *angle_idx;
  float *angle;
  double *coef;
  float *resid_norm2;
  int *err;
  unsigned long long *fallbacks;
  // when set, code only patches redo_list[0 .. *redo_count) (device memory)
  const int *redo_list = nullptr;
  const int *redo_count = nullptr;
  // when set, patch p resumes from the steps the FP16 path already certified:
  // t0 = sI[2 cap * sP + p] steps with atoms sI[i * sP + p] and angles
  // sI[(cap + i) * sP + p], i < t0 (the refine kernel's state layout)
  const int *resume_sI = nullptr;
  int64_t resume_P = 0;
  int resume_cap = 0;
  // the exact |G| bound pruning of the angle transform (RSC_FP32_PRUNE)
  int prune = 0;
};

// FP32 CUDA-core scoring path (romp_f32.cu).
int rsc_launch_f32(const RompArgs &a, cudaStream_t stream);

// Records a CUDA error text for rsc_last_cuda_error and returns RSC_ERR_CUDA.
int rsc_cuda_fail(cudaError_t e);

// Per-call device scratch of the coders and the K-SVD update: stream-ordered
// allocations from a memory pool per device that the library owns and that
// keeps its memory between calls (rsc_capi.cu).  rsc_scratch_trim gives the
// unused part back (rsc_dict_destroy calls it).
cudaError_t rsc_scratch_alloc(void **p, size_t bytes, cudaStream_t st);
cudaError_t rsc_scratch_free(void *p, cudaStream_t st);
void rsc_scratch_trim();
