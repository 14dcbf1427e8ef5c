// Low-rank form work space (see lowrank.cu).
#pragma once

#include <cuda_runtime.h>

#include "tc_gemm.cuh"

namespace mrstat {

constexpr int kMaxRank = 32;

// Constants of the factorised phase-encode DFT (ny = 32 N1, N1 <= 8), passed to the
// kernels by value so that they are constant-bank operands of the multiply-adds:
// c[k-1][i-1] = cos(2 pi k i / N1) and s[k-1][i-1] = sin(2 pi k i / N1) for
// 0 < k, i < N1 / 2 (the N1-point DFT), wm[k] = exp(-2 pi i k / (2 N1)) for k < N1 (the
// radix-2 step to 2 N1 points).
struct DftSmall {
  float c[4][4], s[4][4];
  float2 wm[8];
};

struct LowRank {
  int R = 0;
  int k1 = 0, k23 = 0, k4 = 0;     // padded K of the operands (2 nx, 2 ny, 2 nkx)
  float* U = nullptr;              // [ntr][R] time basis
  float* Ug = nullptr;             // [ntr][R] rows of U in ky order (the order of kytr)
  float* UgT = nullptr;            // [R][ntr] the same, transposed
  float* UgS = nullptr;            // [R][ky_count_max][ny]: the i-th TR of ky at [r][i][ky], else 0
  float* UgQ = nullptr;            // the same for ky_count_max <= 8 in planes of slots: float4 [R][ny] of
                                   // slots 0-3, then slot 4 as float [R][ny] (5 slots) or slots 4-7 as float4
  int* kyof = nullptr;             // [ntr] ky of each TR in that order
  int gram_rows_max = 0;           // most TRs of any 32 consecutive ky values
  int ky_count_max = 0;            // most TRs of any single ky value
  int smem_optin = 0;              // opt-in shared memory per block
  float* Mky = nullptr;            // [ny][R][R] per-ky Gram of U rows
  int* kyptr = nullptr;            // [ny + 1] TR lists per ky residue
  int* kytr = nullptr;             // [ntr]
  float* coef = nullptr;           // [3][R][nv]: c, dc/dlnT1, dc/dlnT2 (masked)
  float* coef2 = nullptr;          // [3][R][nv]: trial point of the surrogate Gauss-Newton phase
  float* gpart = nullptr;          // [ceil(R/8)][4][nv]: per-chunk partial sums of J^H J v
  float* coefT = nullptr;          // [3 R][nx][ny]: coef in image-column order (column kernel)
  const float* coefT_src = nullptr;  // the coef buffer coefT was made from
  bool coefT_dirty = true;         // coef changed in place since
  void *a1_hi = nullptr, *a1_lo = nullptr;    // [R ny][k1]   readout-DFT input rows
  void *a23_hi = nullptr, *a23_lo = nullptr;  // [R nkx][k23] phase-encode DFT input rows
  void *a4_hi = nullptr, *a4_lo = nullptr;    // [R ny][k4]   readout adjoint input rows
  void *by_hi = nullptr, *by_lo = nullptr;    // [2 ny][k23] phase-encode DFT (K-major)
  void *bya_hi = nullptr, *bya_lo = nullptr;  // [2 ny][k23] its adjoint
  float* X1 = nullptr;             // [R ny][2 nkx]
  float* H = nullptr;              // [R nkx][2 ny]
  float* Y3 = nullptr;             // [R nkx][2 ny]
  float* P = nullptr;              // [R ny][2 nx]
  TcOperand op_a1, op_a23, op_a4, op_by, op_bya;
  bool active = false;             // the plan's current linearisation is this low-rank one
  bool full_readout = false;       // nkx == nx: J^H J v skips the readout DFT pair
  bool fft_y = false;              // ... and ny = 32 N1 (N1 <= 8): the factorised phase-encode DFT applies
  DftSmall dft_small;              // constants of the factorised phase-encode DFT
  bool column_path = false;        // fft_y and the column kernel's shared memory fits
  int sms = 1;                     // SM count (grid of the Gram kernel)
};

}  // namespace mrstat
