// Allocation-free inner product: mrstat_dot_static.
//
// Callers that cannot call cudaMalloc (code that runs while another framework owns the
// device allocator, inside a memory-pool budget that must not grow, or in a process that
// forbids allocation after start-up) still need a scratch buffer for the block partial
// sums of a reduction.  Here that scratch is a file-scope __device__ array of a fixed
// size, so the entry point allocates nothing: no cudaMalloc, cudaFree or allocating
// library call.  Its address on a device is looked up once per device with
// cudaGetSymbolAddress, by the first call made with that device current.
//
// The kernel is its own copy of the float64-accumulated reduction of the CG inner
// products (one float32 partial per thread over kItems elements, float64 from the warp
// level up, deterministic last-block sum in block order); the existing mrstat_dot path
// is unchanged.
#include <mutex>

#include "internal.cuh"

namespace mrstat {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                                   // elements per thread
constexpr int kMaxPartials = 4096;                           // blocks, one partial each
constexpr int64_t kMaxN = (int64_t)kMaxPartials * kThreads * kItems;  // 16,777,216
constexpr int kMaxDevices = 64;

// [0, kMaxPartials): block partials; then the last-block ticket.  Shared by every call
// on this device; each call clears the ticket first.
static __device__ __align__(256) double g_dot_scratch[kMaxPartials + 32];

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum_d(double v, double* ws) {
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) ws[w] = v;
  __syncthreads();
  v = (threadIdx.x < kThreads / 32) ? ws[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum_d(v);
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kThreads)
dot_static_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t n, double* scratch,
                  double* __restrict__ out) {
  __shared__ double ws[kThreads / 32];
  __shared__ bool last;
  double* part = scratch;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch + kMaxPartials);
  const int64_t base = (int64_t)blockIdx.x * kThreads * kItems + threadIdx.x;
  float sf = 0.f;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int64_t i = base + (int64_t)k * kThreads;
    if (i < n) sf = fmaf(a[i], b[i], sf);
  }
  const double s = block_sum_d((double)sf, ws);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) t += ((volatile double*)part)[i];
  t = block_sum_d(t, ws);
  if (threadIdx.x == 0) {
    *out = t;
    *ticket = 0u;
  }
}

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_dot_scratch on the current device (looked up once per device).
int scratch_for_current_device(double** ptr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "mrstat_dot_static: no current device");
  if (dev < 0 || dev >= kMaxDevices) return fail(MRSTAT_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "mrstat_dot_static: cudaGetSymbolAddress of the scratch array");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *ptr = g_scratch_ptr[dev];
  return MRSTAT_OK;
}

}  // namespace
}  // namespace mrstat

using namespace mrstat;

extern "C" int mrstat_dot_static(const float* a, const float* b, int64_t n, double* out, void* stream) {
  if (out == nullptr || n < 0 || (n > 0 && (a == nullptr || b == nullptr)))
    return fail(MRSTAT_ERR_INVALID_ARG, "bad argument to mrstat_dot_static");
  if (n > kMaxN)
    return fail(MRSTAT_ERR_INVALID_ARG,
                "mrstat_dot_static: n = %lld exceeds the static scratch limit of %lld elements (use mrstat_dot)",
                (long long)n, (long long)kMaxN);
  double* scratch = nullptr;
  const int s = scratch_for_current_device(&scratch);
  if (s != MRSTAT_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch + kMaxPartials, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return cuda_fail(e, "mrstat_dot_static: ticket reset");
  const int64_t per_block = (int64_t)kThreads * kItems;
  const int blocks = n == 0 ? 1 : (int)((n + per_block - 1) / per_block);
  dot_static_kernel<<<blocks, kThreads, 0, st>>>(a, b, n, scratch, out);
  e = cudaGetLastError();
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "mrstat_dot_static launch");
}
