// K5: float64-accumulated inner products and the vector updates of the inner CG
// solve (Algorithm 6; Eq. 4 solved by CG).
//
// Reductions are deterministic and single-pass: every block writes its partial sum,
// and the last block to finish (a release fence plus an atomic ticket) adds the
// partials in block order and resets the ticket for the next launch.  A thread forms
// the products of its few elements (about one float4) in float32;
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

// Vector layout of these kernels: elements [0, 4 n4) as float4 (n4 = n / 4 when every
// pointer is 16-byte aligned, else 0), the rest [4 n4, n) element by element.  A thread
// handles about one float4; the loads of its first float4 are issued before the kernel
// reads its float64 scalars, so the two latencies overlap.
__device__ __forceinline__ float4 ld4(const float* p, int64_t i) { return reinterpret_cast<const float4*>(p)[i]; }
__device__ __forceinline__ void st4(float* p, int64_t i, float4 v) { reinterpret_cast<float4*>(p)[i] = v; }
__device__ __forceinline__ float dot4(float4 a, float4 b, float s) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
}
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {  // a x + y
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

__global__ void __launch_bounds__(kT)
dot_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n, int64_t n4, double* part,
           unsigned* ticket, double* __restrict__ out, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  __shared__ double ws[kT / 32];
  const int64_t t0 = blockIdx.x * (int64_t)kT + threadIdx.x, stride = (int64_t)gridDim.x * kT;
  float sf = 0.f;
  for (int64_t i = t0; i < n4; i += stride) sf = dot4(ld4(a, i), ld4(b, i), sf);
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) sf = fmaf(a[i], b[i], sf);
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
// then rr_new = r.r.  When alpha is 0 the vectors are left alone and rr_new = rr.  Lane 0
// of each warp forms alpha in float64 (once per warp: GB300's float64 rate makes a
// per-thread division visible).  Block 0 marks the solve frozen; a block that reads the
// flag after that reaches the same decision, since the flag is only set when it holds.
__global__ void __launch_bounds__(kT)
cg_update_xr_kernel(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
                    const float* __restrict__ q, int64_t n, int64_t n4, const double* __restrict__ rr,
                    const double* __restrict__ pq, int* __restrict__ frozen, double* part,
                    unsigned* ticket, double* __restrict__ rr_new) {
  __shared__ double ws[kT / 32];
  const int64_t t0 = blockIdx.x * (int64_t)kT + threadIdx.x, stride = (int64_t)gridDim.x * kT;
  float4 xv, rv, pv, qv;
  if (t0 < n4) {
    xv = ld4(x, t0);
    rv = ld4(r, t0);
    pv = ld4(p, t0);
    qv = ld4(q, t0);
  }
  float al = 0.f;
  int apply = 0;
  if ((threadIdx.x & 31) == 0) {
    const double rrv = *rr, pqv = *pq;
    apply = !*frozen && pqv > 0.0 && rrv > 0.0;
    al = apply ? (float)(rrv / pqv) : 0.f;
    if (!apply && blockIdx.x == 0 && threadIdx.x == 0) *frozen = 1;
  }
  al = __shfl_sync(0xffffffffu, al, 0);
  apply = __shfl_sync(0xffffffffu, apply, 0);
  float sf = 0.f;
  for (int64_t i = t0; i < n4; i += stride) {
    if (i != t0) {
      xv = ld4(x, i);
      rv = ld4(r, i);
      pv = ld4(p, i);
      qv = ld4(q, i);
    }
    if (apply) {
      st4(x, i, axpy4(al, pv, xv));
      rv = axpy4(-al, qv, rv);
      st4(r, i, rv);
    }
    sf = dot4(rv, rv, sf);
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
    float ri = r[i];
    if (apply) {
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

// p = r + beta p with beta = rr_new / rr_old (left alone once frozen)
__global__ void __launch_bounds__(kT)
cg_update_p_kernel(float* __restrict__ p, const float* __restrict__ r, int64_t n, int64_t n4,
                   const double* __restrict__ rr_old, const double* __restrict__ rr_new,
                   const int* __restrict__ frozen) {
  const int64_t t0 = blockIdx.x * (int64_t)kT + threadIdx.x, stride = (int64_t)gridDim.x * kT;
  float4 pv, rv;
  if (t0 < n4) {
    pv = ld4(p, t0);
    rv = ld4(r, t0);
  }
  float beta = 0.f;
  int apply = 0;
  if ((threadIdx.x & 31) == 0) {
    apply = !*frozen;
    beta = apply ? (float)(*rr_new / *rr_old) : 0.f;
  }
  beta = __shfl_sync(0xffffffffu, beta, 0);
  apply = __shfl_sync(0xffffffffu, apply, 0);
  if (!apply) return;
  for (int64_t i = t0; i < n4; i += stride) {
    if (i != t0) {
      pv = ld4(p, i);
      rv = ld4(r, i);
    }
    st4(p, i, axpy4(beta, pv, rv));
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) p[i] = fmaf(beta, p[i], r[i]);
}

// About one float4 per thread, at most kRedBlocks blocks (one float64 partial each).
int grid_for(int64_t n) {
  int64_t b = (n + 4 * kT - 1) / (4 * kT);
  if (b > kRedBlocks) b = kRedBlocks;
  return (int)(b > 0 ? b : 1);
}

bool aligned16(const void* a) { return (reinterpret_cast<uintptr_t>(a) & 15u) == 0; }

}  // namespace

cudaError_t launch_dot(const float* a, const float* b, int64_t n, double* partials, unsigned* ticket,
                       double* out, cudaStream_t st, const int* gate) {
  const int64_t n4 = aligned16(a) && aligned16(b) ? n / 4 : 0;
  dot_kernel<<<grid_for(n), kT, 0, st>>>(a, b, n, n4, partials, ticket, out, gate);
  return cudaGetLastError();
}

cudaError_t launch_cg_init(const float* rhs, float* x, float* r, float* p, int64_t n, cudaStream_t st) {
  cg_init_kernel<<<grid_for(n), kT, 0, st>>>(rhs, x, r, p, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_xr(float* x, float* r, const float* p, const float* q, int64_t n,
                                const double* rr, const double* pq, int* frozen, double* partials,
                                unsigned* ticket, double* rr_new, cudaStream_t st) {
  const int64_t n4 = aligned16(x) && aligned16(r) && aligned16(p) && aligned16(q) ? n / 4 : 0;
  cg_update_xr_kernel<<<grid_for(n), kT, 0, st>>>(x, r, p, q, n, n4, rr, pq, frozen, partials, ticket, rr_new);
  return cudaGetLastError();
}

cudaError_t launch_cg_update_p(float* p, const float* r, int64_t n, const double* rr_old,
                               const double* rr_new, const int* frozen, cudaStream_t st) {
  const int64_t n4 = aligned16(p) && aligned16(r) ? n / 4 : 0;
  cg_update_p_kernel<<<grid_for(n), kT, 0, st>>>(p, r, n, n4, rr_old, rr_new, frozen);
  return cudaGetLastError();
}

}  // namespace mrstat
