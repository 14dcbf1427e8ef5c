// Deterministic single-pass reductions shared by the vector kernels: float64 warp and
// block sums, and the last-block finish (release fence plus an atomic ticket; the last
// block adds the per-block partials in block order and resets the ticket).
#pragma once

#include <cuda_runtime.h>

namespace mrstat {
namespace red {

// Programmatic dependent launch (sm_90+): a kernel launched with the programmatic
// stream-serialization attribute may start while its predecessor runs; pdl_wait() returns
// once the predecessor has completed and its memory is visible (at once when there was
// no early start), and pdl_trigger() lets this kernel's own successor start early.
// Everything a kernel reads from earlier launches must come after its pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; the result is valid in thread 0.  Uses `ws` (>= THREADS/32 doubles).
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* ws) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  v = (threadIdx.x < THREADS / 32) ? ws[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

// Called by every thread after thread 0 of each block stored its partial in part[blockIdx.x].
// The last block sums all partials in order into *out.
template <int THREADS>
__device__ __forceinline__ void finish_reduction(double* part, unsigned* ticket, double* out, double* ws) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += THREADS) s += ((volatile double*)part)[i];
  s = block_sum<THREADS>(s, ws);
  if (threadIdx.x == 0) {
    *out = s;
    *ticket = 0u;
  }
}

// Two sums at once: after thread 0 of each block stored its partials in part[blockIdx.x]
// and part[gridDim.x + blockIdx.x], the last block adds each in block order into out0,
// out1.  Uses `ws` (>= THREADS/32 doubles).
template <int THREADS>
__device__ __forceinline__ void finish_reduction2(double* part, unsigned* ticket, double* out0, double* out1,
                                                  double* ws) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += THREADS) {
    s0 += ((volatile double*)part)[i];
    s1 += ((volatile double*)part)[gridDim.x + i];
  }
  s0 = block_sum<THREADS>(s0, ws);
  s1 = block_sum<THREADS>(s1, ws);
  if (threadIdx.x == 0) {
    *out0 = s0;
    *out1 = s1;
    *ticket = 0u;
  }
}

}  // namespace red
}  // namespace mrstat
