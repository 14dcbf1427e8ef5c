// Internal declarations shared by the translation units of libmrstat.so.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mrstat.h"

namespace mrstat {

// Number of channels of the cached time courses: m_y, dm_y/dlnT1, dm_y/dlnT2.
constexpr int kChannels = 3;
// Blocks of the first stage of the float64 reductions.
constexpr int kRedBlocks = 608;

struct Plan {
  int nx = 0, ny = 0, nkx = 0, ntr = 0;
  int ntr_pad = 0;   // ntr rounded up to a multiple of 4
  int nq = 0;        // ntr_pad / 4 TR quads
  int nv = 0;
  int form = 0;
  int device = 0;
  double tr_ms = 0, te_ms = 0;
  int inversion = 0, alternate = 0;

  // per-TR tables (device)
  float2* cs = nullptr;     // [ntr_pad] (cos phi_n, sin phi_n), phi_n the signed flip
  float* phi = nullptr;     // [ntr_pad] signed flip (radians)
  int* kyi = nullptr;       // [ntr_pad] ky mod ny in [0, ny)
  float2* roots = nullptr;  // [ny] exp(-2 pi i k / ny)
  float2* ft = nullptr;     // [nx][nkx] exp(-2 pi i kx ix / nx)
  float2* fh = nullptr;     // [nkx][nx] exp(+2 pi i kx ix / nx)

  // cached linearisation
  float4* D = nullptr;      // [3][nq][nv] four consecutive TRs per float4
  float2* rho = nullptr;    // [nv] rho * mask
  float* maskf = nullptr;   // [nv] 1 inside the mask, 0 outside
  bool linearized = false;

  // scratch
  float4* dfwd = nullptr;   // [nq][nv] m_y only, for mrstat_forward
  float2* cf = nullptr;     // [3][nv] per-voxel complex coefficients of the y-contraction
  float2* A = nullptr;      // [ntr][nx] y-contracted image rows
  float2* wt = nullptr;     // [ntr_pad][nx] x-adjoint of a k-space vector (rows >= ntr zero)
  double* red = nullptr;    // [kRedBlocks] reduction partials
  float* cg_r = nullptr;    // [4][nv]
  float* cg_p = nullptr;    // [4][nv]
  float* cg_q = nullptr;    // [4][nv]
  float2* cg_jv = nullptr;  // [ntr][nkx]
  double* cg_s = nullptr;   // CG scalars, 4 per iteration
  int* cg_frozen = nullptr; // CG stop flag
  int cg_s_cap = 0;         // iterations the scalar buffer holds

  int64_t bytes = 0;
  int64_t d_bytes = 0;

  // tracing
  int64_t launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool prof_on = false;
  uint32_t prof_mask = 0;
  struct Mark {
    int kid;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
  size_t pool_used = 0;
};

// error reporting (thread-local message)
void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// ---- launchers (each returns the launch's cudaError_t) ----
// bloch.cu
cudaError_t launch_bloch(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                         float4* D, int nch, cudaStream_t st);
// encode.cu
cudaError_t launch_prep_forward(const Plan& p, const float* alpha, const uint8_t* mask, cudaStream_t st);
cudaError_t launch_prep_linearize(const Plan& p, const float* alpha, const uint8_t* mask, cudaStream_t st);
cudaError_t launch_prep_jvp(const Plan& p, const float* v, cudaStream_t st);
cudaError_t launch_ycontract(const Plan& p, const float4* D, int nch, cudaStream_t st);
cudaError_t launch_jhw_dot(const Plan& p, float* g, cudaStream_t st);
cudaError_t launch_timecourse(const Plan& p, int channel, float* out, cudaStream_t st);
// dft.cu
cudaError_t launch_cgemm(const float2* A, const float2* B, float2* C, int M, int N, int K, cudaStream_t st);
// reduce.cu
cudaError_t launch_dot(const float* a, const float* b, int64_t n, double* partials, double* out,
                       cudaStream_t st);
cudaError_t launch_cg_init(const float* rhs, float* x, float* r, float* p, int64_t n, cudaStream_t st);
cudaError_t launch_cg_update_xr(float* x, float* r, const float* p, const float* q, int64_t n,
                                const double* rr, const double* pq, int* frozen, cudaStream_t st);
cudaError_t launch_cg_update_p(float* p, const float* r, int64_t n, const double* rr_old,
                               const double* rr_new, const int* frozen, cudaStream_t st);

}  // namespace mrstat
