// rsc_internal.h -- state shared by the host side of librsc and its kernels.
#pragma once

#include <cuda_runtime.h>
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
  // tensor-core path (bf16 steered dictionary), built lazily
  void *steered_bf16;    // [M*R][Kpad] bf16, row (m*R + r) = packed S_r d_m
  int kpad;              // padded contraction depth (multiple of 16)
};

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
};

// FP32 CUDA-core scoring path (romp_f32.cu).
int rsc_launch_f32(const RompArgs &a, cudaStream_t stream);

// Records a CUDA error text for rsc_last_cuda_error and returns RSC_ERR_CUDA.
int rsc_cuda_fail(cudaError_t e);
