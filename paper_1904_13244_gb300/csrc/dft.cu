// K3 (plain FP32 form): the readout-direction DFT of the y-contracted rows and its
// adjoint, as a dense complex matrix product on the CUDA cores.
//   forward:  s[n][k]  = sum_ix A[n][ix] Ft[ix][k],  Ft[ix][k] = exp(-2 pi i kx(k) ix / nx)
//   adjoint:  Wt[n][ix] = sum_k w[n][k] Fh[k][ix],    Fh = conj(Ft)^T
// Complex row-major operands; C[M][N] = A[M][K] B[K][N].  32x32 output tile per block,
// 256 threads with 2x2 outputs each, K staged through shared memory in chunks of 16.
#include "internal.cuh"

namespace mrstat {
namespace {

constexpr int TM = 32, TN = 32, TK = 16;

__global__ void __launch_bounds__(256)
cgemm_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
             int M, int N, int K) {
  __shared__ float2 As[TK][TM + 1];
  __shared__ float2 Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float cr[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, ci[2][2] = {{0.f, 0.f}, {0.f, 0.f}};

  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = tid; e < TM * TK; e += 256) {
      const int mm = e / TK, kk = e - mm * TK;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[(size_t)m * K + k] : make_float2(0.f, 0.f);
    }
    for (int e = tid; e < TK * TN; e += 256) {
      const int kk = e / TN, nn = e - kk * TN;
      const int k = k0 + kk, n = n0 + nn;
      Bs[kk][nn] = (k < K && n < N) ? B[(size_t)k * N + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const float2 a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
      const float2 b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      const float2 a[2] = {a0, a1}, b[2] = {b0, b1};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          cr[i][j] = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, cr[i][j]));
          ci[i][j] = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, ci[i][j]));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + 2 * ty + i, n = n0 + 2 * tx + j;
      if (m < M && n < N) C[(size_t)m * N + n] = make_float2(cr[i][j], ci[i][j]);
    }
}

}  // namespace

cudaError_t launch_cgemm(const float2* A, const float2* B, float2* C, int M, int N, int K,
                         cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  cgemm_kernel<<<grid, 256, 0, st>>>(A, B, C, M, N, K);
  return cudaGetLastError();
}

}  // namespace mrstat
