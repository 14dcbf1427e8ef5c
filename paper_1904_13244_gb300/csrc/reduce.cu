// K5: float64-accumulated inner products and the vector updates of the inner CG
// solve (Algorithm 6; Eq. 4 solved by CG).
//
// Reductions are deterministic and single-pass: every block writes its partial sum,
// and the last block to finish (a release fence plus an atomic ticket) adds the
// partials in block order and resets the ticket for the next launch.  A thread forms
// the products of its few elements (grid-stride, a handful per thread) in float32;
// everything from the warp level up is added in float64.  GB300 runs float64 at a small
// fraction of the float32 rate, and converting every element to float64 kept the FP64
// pipe busy for most of these kernels' time.  CG scalars
// never leave the device: each update kernel reads the float64 inner products it
// needs, forms alpha or beta once per block (GB300's float64 rate makes a per-thread
// division visible) and the x/r update also produces the partial sums of r.r.
#include "internal.cuh"
#include "reduce.cuh"

namespace mrstat {
namespace {

using namespace red;

constexpr int kT = 256;

__global__ void __launch_bounds__(kT)
dot_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n, double* part,
           unsigned* ticket, double* __restrict__ out) {
  __shared__ double ws[kT / 32];
  float sf = 0.f;
#pragma unroll 4
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    sf = fmaf(a[i], b[i], sf);
  const double s = block_sum<kT>((double)sf, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  finish_reduction<kT>(part, ticket, out, ws);
}

__global__ void cg_init_kernel(const float* __restrict__ rhs, float* __restrict__ x,
                               float* __restrict__ r, float* __restrict__ p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float b = rhs[i];
    x[i] = 0.f;
    r[i] = b;
    p[i] = b;
  }
}

// x += alpha p, r -= alpha q with alpha = rr / pq (0 once frozen: pq <= 0 or rr == 0),
// then rr_new = r.r.  When alpha is 0 the vectors are left alone and rr_new = rr.
__global__ void __launch_bounds__(kT)
cg_update_xr_kernel(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                    const float* __restrict__ q, int64_t n, const double* __restrict__ rr,
                    const double* __restrict__ pq, int* __restrict__ frozen, double* part,
                    unsigned* ticket, double* __restrict__ rr_new) {
  __shared__ double ws[kT / 32];
  __shared__ float s_alpha;
  __shared__ int s_apply;
  if (threadIdx.x == 0) {
    const double rrv = *rr, pqv = *pq;
    const bool ok = !*frozen && pqv > 0.0 && rrv > 0.0;
    s_alpha = ok ? (float)(rrv / pqv) : 0.f;
    s_apply = ok;
    if (!ok && blockIdx.x == 0) *frozen = 1;
  }
  __syncthreads();
  const float al = s_alpha;
  float sf = 0.f;
#pragma unroll 4
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    float ri = r[i];
    if (s_apply) {
      x[i] = fmaf(al, p[i], x[i]);
      ri = fmaf(-al, q[i], ri);
      r[i] = ri;
    }
    sf = fmaf(ri, ri, sf);
  }
  const double s = block_sum<kT>((double)sf, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  finish_reduction<kT>(part, ticket, rr_new, ws);
}

__global__ void __launch_bounds__(kT)
cg_update_p_kernel(float* __restrict__ p, const float* __restrict__ r, int64_t n,
                   const double* __restrict__ rr_old, const double* __restrict__ rr_new,
                   const int* __restrict__ frozen) {
  __shared__ float s_beta;
  __shared__ int s_apply;
  if (threadIdx.x == 0) {
    s_apply = !*frozen;
    s_beta = s_apply ? (float)(*rr_new / *rr_old) : 0.f;
  }
  __syncthreads();
  if (!s_apply) return;
  const float beta = s_beta;
#pragma unroll 4
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    p[i] = fmaf(beta, p[i], r[i]);
}

// About four elements per thread: fewer blocks to schedule and fewer partials for the
// last block to add than one element per thread, with the loads unrolled by four.
int grid_for(int64_t n) {
  int64_t b = (n + 4 * kT - 1) / (4 * kT);
  if (b > kRedBlocks) b = kRedBlocks;
  return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_dot(const float* a, const float* b, int64_t n, double* partials, unsigned* ticket,
                       double* out, cudaStream_t st) {
  dot_kernel<<<grid_for(n), kT, 0, st>>>(a, b, n, partials, ticket, out);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const float* rhs, float* x, float* r, float* p, int64_t n, cudaStream_t st) {
  cg_init_kernel<<<grid_for(n), kT, 0, st>>>(rhs, x, r, p, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_xr(float* x, float* r, const float* p, const float* q, int64_t n,
                                const double* rr, const double* pq, int* frozen, double* partials,
                                unsigned* ticket, double* rr_new, cudaStream_t st) {
  cg_update_xr_kernel<<<grid_for(n), kT, 0, st>>>(x, r, p, q, n, rr, pq, frozen, partials, ticket, rr_new);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_p(float* p, const float* r, int64_t n, const double* rr_old,
                               const double* rr_new, const int* frozen, cudaStream_t st) {
  cg_update_p_kernel<<<grid_for(n), kT, 0, st>>>(p, r, n, rr_old, rr_new, frozen);
  return cudaGetLastError();
}

}  // namespace mrstat
