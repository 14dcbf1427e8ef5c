// K5: float64-accumulated inner products and the vector update of the inner CG solve
// (Algorithm 6; Eq. 4 solved by CG).
//
// Reductions are deterministic and single-pass: every block writes its partial sum,
// and the last block to finish (a release fence plus an atomic ticket) adds the
// partials in block order and resets the ticket for the next launch.  A thread forms
// the products of its few elements (about one float4) in float32;
// everything from the warp level up is added in float64.  GB300 runs float64 at a small
// fraction of the float32 rate, and converting every element to float64 kept the FP64
// pipe busy for most of these kernels' time.  CG scalars
// never leave the device: the update kernel reads the float64 inner products it needs and
// forms alpha and beta once per warp.
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

__global__ void cg_init_kernel(const float* __restrict__ rhs, float* __restrict__ x, float* __restrict__ r,
                               float* __restrict__ p, float* __restrict__ q, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = 0.f;
    r[i] = rhs[i];
    p[i] = 0.f;
    q[i] = 0.f;
  }
}

// One CG iteration in the Chronopoulos-Gear form on B x = b, after the product w = B r
// that also left delta = <r, w> and gamma = <r, r> in sk[0] and sk[1]:
//   beta = gamma / gamma_prev (0 in the first iteration),
//   pq = delta - beta gamma / alpha_prev (= <p, B p> of the new p; delta at first),
//   alpha = gamma / pq,
//   p = r + beta p,  q = w + beta q (= B p),  x += alpha p,  r -= alpha q.
// In exact arithmetic these are the iterates of textbook CG; the product is applied to r,
// so the inner products come with it and one vector pass remains.  An iteration with
// pq <= 0 or gamma == 0 freezes x, r, p and q for the rest (block 0 marks the solve
// frozen with the iteration index + 1; a block that reads the flag after that reaches the
// same decision).  Lane 0 of
// each warp forms the scalars in float64 (GB300's float64 rate makes a per-thread
// division visible); block 0 keeps alpha for the next iteration in sk[2].
__global__ void __launch_bounds__(kT)
cg_cg_step_kernel(float* __restrict__ x, float* __restrict__ r, float* __restrict__ p, float* __restrict__ q,
                  const float* __restrict__ w, int64_t n, int64_t n4, double* __restrict__ sk,
                  const double* __restrict__ sp, int* __restrict__ frozen, int it) {
  pdl_trigger();
  pdl_wait();  // w and the inner products come from the product launch
  const int64_t t0 = blockIdx.x * (int64_t)kT + threadIdx.x, stride = (int64_t)gridDim.x * kT;
  float4 xv, rv, pv, qv, wv;
  if (t0 < n4) {
    xv = ld4(x, t0);
    rv = ld4(r, t0);
    pv = ld4(p, t0);
    qv = ld4(q, t0);
    wv = ld4(w, t0);
  }
  float al = 0.f, be = 0.f;
  int apply = 0;
  if ((threadIdx.x & 31) == 0) {
    const double delta = sk[0], gamma = sk[1];
    double beta = 0.0, pq = delta;
    if (sp != nullptr) {
      beta = gamma / sp[1];
      pq = delta - beta * gamma / sp[2];
    }
    const int fz = *frozen;
    apply = !fz && pq > 0.0 && gamma > 0.0;
    if (apply) {
      al = (float)(gamma / pq);
      be = (float)beta;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (apply) sk[2] = gamma / pq;
      else if (!fz) *frozen = it + 1;
    }
  }
  al = __shfl_sync(0xffffffffu, al, 0);
  be = __shfl_sync(0xffffffffu, be, 0);
  apply = __shfl_sync(0xffffffffu, apply, 0);
  if (!apply) return;
  for (int64_t i = t0; i < n4; i += stride) {
    if (i != t0) {
      xv = ld4(x, i);
      rv = ld4(r, i);
      pv = ld4(p, i);
      qv = ld4(q, i);
      wv = ld4(w, i);
    }
    pv = axpy4(be, pv, rv);
    qv = axpy4(be, qv, wv);
    st4(p, i, pv);
    st4(q, i, qv);
    st4(x, i, axpy4(al, pv, xv));
    st4(r, i, axpy4(-al, qv, rv));
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
    const float pi = fmaf(be, p[i], r[i]), qi = fmaf(be, q[i], w[i]);
    p[i] = pi;
    q[i] = qi;
    x[i] = fmaf(al, pi, x[i]);
    r[i] = fmaf(-al, qi, r[i]);
  }
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

cudaError_t launch_cg_init(const float* rhs, float* x, float* r, float* p, float* q, int64_t n, cudaStream_t st) {
  cg_init_kernel<<<grid_for(n), kT, 0, st>>>(rhs, x, r, p, q, n);
  return cudaGetLastError();
}

cudaError_t launch_cg_cg_step(float* x, float* r, float* p, float* q, const float* w, int64_t n, double* sk,
                              const double* sp, int* frozen, int it, cudaStream_t st) {
  const int64_t n4 = aligned16(x) && aligned16(r) && aligned16(p) && aligned16(q) && aligned16(w) ? n / 4 : 0;
  return launch_pdl(cg_cg_step_kernel, dim3(grid_for(n)), dim3(kT), 0, st, x, r, p, q, w, n, n4, sk, sp, frozen,
                    it);
}

}  // namespace mrstat
