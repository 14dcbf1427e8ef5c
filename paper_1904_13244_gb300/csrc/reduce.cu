// K5: float64-accumulated inner products and the vector updates of the inner CG
// solve (Algorithm 6; Eq. 4 solved by CG).  Reductions are deterministic: a fixed
// grid of partial sums (warp shuffles, then shared memory), then one block that sums
// the partials in a fixed order.  CG scalars never leave the device: each update
// kernel reads the float64 inner products it needs and forms alpha or beta itself.
#include "internal.cuh"

namespace mrstat {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int THREADS>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[THREADS / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  v = (threadIdx.x < THREADS / 32) ? ws[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;  // valid in thread 0
}

__global__ void __launch_bounds__(256)
dot_partial_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                   double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma((double)a[i], (double)b[i], s);
  s = block_sum<256>(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256)
dot_final_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += 256) s += part[i];
  s = block_sum<256>(s);
  if (threadIdx.x == 0) *out = s;
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

// alpha = rr / pq, or 0 once the iteration is frozen (pq <= 0 or rr == 0)
__device__ __forceinline__ double cg_alpha(double rr, double pq, int frozen) {
  return (frozen || !(pq > 0.0) || !(rr > 0.0)) ? 0.0 : rr / pq;
}

__global__ void cg_update_xr_kernel(float* __restrict__ x, float* __restrict__ r,
                                    const float* __restrict__ p, const float* __restrict__ q,
                                    int64_t n, const double* __restrict__ rr,
                                    const double* __restrict__ pq, int* __restrict__ frozen) {
  const int fz = *frozen;
  const double al = cg_alpha(*rr, *pq, fz);
  if (blockIdx.x == 0 && threadIdx.x == 0 && al == 0.0) *frozen = 1;
  if (al == 0.0) return;
  const float a = (float)al;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fmaf(a, p[i], x[i]);
    r[i] = fmaf(-a, q[i], r[i]);
  }
}

__global__ void cg_update_p_kernel(float* __restrict__ p, const float* __restrict__ r, int64_t n,
                                   const double* __restrict__ rr_old,
                                   const double* __restrict__ rr_new, const int* __restrict__ frozen) {
  if (*frozen) return;
  const float beta = (float)(*rr_new / *rr_old);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fmaf(beta, p[i], r[i]);
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 2 * kRedBlocks ? (b > 0 ? b : 1) : 2 * kRedBlocks);
}

}  // namespace

cudaError_t launch_dot(const float* a, const float* b, int64_t n, double* partials, double* out,
                       cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > kRedBlocks) blocks = kRedBlocks;
  if (blocks < 1) blocks = 1;
  dot_partial_kernel<<<(int)blocks, 256, 0, st>>>(a, b, n, partials);
  dot_final_kernel<<<1, 256, 0, st>>>(partials, (int)blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const float* rhs, float* x, float* r, float* p, int64_t n, cudaStream_t st) {
  cg_init_kernel<<<grid_for(n), 256, 0, st>>>(rhs, x, r, p, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_xr(float* x, float* r, const float* p, const float* q, int64_t n,
                                const double* rr, const double* pq, int* frozen, cudaStream_t st) {
  cg_update_xr_kernel<<<grid_for(n), 256, 0, st>>>(x, r, p, q, n, rr, pq, frozen);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_p(float* p, const float* r, int64_t n, const double* rr_old,
                               const double* rr_new, const int* frozen, cudaStream_t st) {
  cg_update_p_kernel<<<grid_for(n), 256, 0, st>>>(p, r, n, rr_old, rr_new, frozen);
  return cudaGetLastError();
}

}  // namespace mrstat
