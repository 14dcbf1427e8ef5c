// K3 (plain FP32 form): the readout-direction DFT of the y-contracted rows and its
// adjoint, as a dense complex matrix product on the CUDA cores.
//   forward:  s[n][k]  = sum_ix A[n][ix] Ft[ix][k],  Ft[ix][k] = exp(-2 pi i kx(k) ix / nx)
//   adjoint:  Wt[n][ix] = sum_k w[n][k] Fh[k][ix],    Fh = conj(Ft)^T
// Complex row-major operands; C[M][N] = A[M][K] B[K][N].  A 32 x 64 output tile per
// block of 128 threads, 4 x 4 complex outputs per thread held in registers; K runs in
// chunks of 16 staged through shared memory, with the next chunk loaded into registers
// while the current one is consumed.
#include "internal.cuh"

namespace mrstat {
namespace {

constexpr int BM = 32, BN = 64, BK = 16, NT = 128;

__global__ void __launch_bounds__(NT)
cgemm_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
             int M, int N, int K, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  __shared__ __align__(16) float2 As[BK][BM];
  __shared__ __align__(16) float2 Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // 16 column groups x 8 row groups
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  // global -> register staging: A chunk is BM x BK = 512 elements (4 per thread),
  // B chunk is BK x BN = 1024 elements (8 per thread)
  float2 ra[4], rb[8];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * NT;
      const int mm = e >> 4, kk = e & 15;
      const int m = m0 + mm, k = k0 + kk;
      ra[u] = (m < M && k < K) ? A[(size_t)m * K + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * NT;
      const int kk = e >> 6, nn = e & 63;
      const int k = k0 + kk, n = n0 + nn;
      rb[u] = (k < K && n < N) ? B[(size_t)k * N + n] : make_float2(0.f, 0.f);
    }
  };
  auto store_chunk = [&]() {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * NT;
      As[e & 15][e >> 4] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * NT;
      Bs[e >> 6][e & 63] = rb[u];
    }
  };

  float cr[4][4], ci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) cr[i][j] = ci[i][j] = 0.f;

  load_chunk(0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();
    store_chunk();
    __syncthreads();
    if (k0 + BK < K) load_chunk(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[4], b[4];
      const float4* ap = reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4* bp = reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      float4 t0 = ap[0], t1 = ap[1];
      a[0] = make_float2(t0.x, t0.y); a[1] = make_float2(t0.z, t0.w);
      a[2] = make_float2(t1.x, t1.y); a[3] = make_float2(t1.z, t1.w);
      t0 = bp[0]; t1 = bp[1];
      b[0] = make_float2(t0.x, t0.y); b[1] = make_float2(t0.z, t0.w);
      b[2] = make_float2(t1.x, t1.y); b[3] = make_float2(t1.z, t1.w);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          cr[i][j] = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, cr[i][j]));
          ci[i][j] = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, ci[i][j]));
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n < N) C[(size_t)m * N + n] = make_float2(cr[i][j], ci[i][j]);
    }
  }
}

}  // namespace

cudaError_t launch_cgemm(const float2* A, const float2* B, float2* C, int M, int N, int K,
                         const int* gate, cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  cgemm_kernel<<<grid, NT, 0, st>>>(A, B, C, M, N, K, gate);
  return cudaGetLastError();
}

}  // namespace mrstat
