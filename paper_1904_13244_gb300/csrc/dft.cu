// K3 (plain FP32 form): the readout-direction DFT of the y-contracted rows and its
// adjoint, as a dense complex matrix product on the CUDA cores.
//   forward:  s[n][k]  = sum_ix A[n][ix] Ft[ix][k],  Ft[ix][k] = exp(-2 pi i kx(k) ix / nx)
//   adjoint:  Wt[n][ix] = sum_k w[n][k] Fh[k][ix],    Fh = conj(Ft)^T
// Complex row-major operands; C[M][N] = A[M][K] B[K][N].  A 32 x 64 output tile per
// block of 512 threads: four groups of 128 threads each take a quarter of K (split-K
// inside the block, so an SM holds 16 warps although the grid is only ~one block per
// SM for the 1120 x 224 x 224 DFT), 4 x 4 complex outputs per thread held in registers.
// K runs in chunks of 16 staged through shared memory, the next chunk prefetched into
// registers while the current one is consumed; the four partial tiles are added
// through shared memory at the end.
#include "internal.cuh"

namespace mrstat {
namespace {

constexpr int BM = 32, BN = 64, BK = 16, NT = 128, KSPLIT = 4;
constexpr int BMP = BM + 2;  // padded row of the A tile (keeps float4 alignment, fewer bank conflicts)

__global__ void __launch_bounds__(NT * KSPLIT, 1)
cgemm_kernel(const float2* __restrict__ A, const float2* __restrict__ B, float2* __restrict__ C,
             int M, int N, int K, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  // dynamic shared memory: staging tiles of the four groups, reused for the reduction
  extern __shared__ float4 smem_f4[];
  float2* smem = reinterpret_cast<float2*>(smem_f4);
  const int grp = threadIdx.x / NT;
  const int tid = threadIdx.x - grp * NT;
  float2 (*As)[BMP] = reinterpret_cast<float2 (*)[BMP]>(smem + (size_t)grp * BK * BMP);
  float2 (*Bs)[BN] = reinterpret_cast<float2 (*)[BN]>(smem + (size_t)KSPLIT * BK * BMP + (size_t)grp * BK * BN);
  const int tx = tid & 15, ty = tid >> 4;  // 16 column groups x 8 row groups
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // this group's share of K, in whole chunks
  const int nchunks = (K + BK - 1) / BK;
  const int ca = (nchunks * grp) / KSPLIT, ce = (nchunks * (grp + 1)) / KSPLIT;
  const int kbeg = ca * BK, kend = min(K, ce * BK);

  // global -> register staging: A chunk is BM x BK = 512 elements (4 per thread),
  // B chunk is BK x BN = 1024 elements (8 per thread)
  float2 ra[4], rb[8];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + u * NT;
      const int mm = e >> 4, kk = e & 15;
      const int m = m0 + mm, k = k0 + kk;
      ra[u] = (m < M && k < kend) ? A[(size_t)m * K + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = tid + u * NT;
      const int kk = e >> 6, nn = e & 63;
      const int k = k0 + kk, n = n0 + nn;
      rb[u] = (k < kend && n < N) ? B[(size_t)k * N + n] : make_float2(0.f, 0.f);
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

  // every group runs the same number of barrier rounds (empty rounds contribute zeros)
  const int rounds = (nchunks + KSPLIT - 1) / KSPLIT;
  if (kbeg < kend) load_chunk(kbeg);
  for (int rd = 0; rd < rounds; ++rd) {
    const int k0 = kbeg + rd * BK;
    const bool live = k0 < kend;
    __syncthreads();
    if (live) store_chunk();
    __syncthreads();
    if (!live) continue;
    if (k0 + BK < kend) load_chunk(k0 + BK);
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
  // add the KSPLIT partial tiles: groups 1..3 park theirs in shared memory (reusing the
  // staging buffers), group 0 adds and stores
  __syncthreads();
  float2* red = smem;  // (KSPLIT - 1) partial tiles of BM x BN
  if (grp > 0) {
    float2* dst = red + (size_t)(grp - 1) * BM * BN;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) dst[(ty * 4 + i) * BN + tx * 4 + j] = make_float2(cr[i][j], ci[i][j]);
  }
  __syncthreads();
  if (grp != 0) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      float sr = cr[i][j], si = ci[i][j];
#pragma unroll
      for (int g = 0; g < KSPLIT - 1; ++g) {
        const float2 v = red[(size_t)g * BM * BN + (ty * 4 + i) * BN + tx * 4 + j];
        sr += v.x;
        si += v.y;
      }
      if (m < M && n < N) C[(size_t)m * N + n] = make_float2(sr, si);
    }
  }
}

constexpr size_t kSmemFloat2 =
    (KSPLIT * BK * (BMP + BN) > (KSPLIT - 1) * BM * BN) ? KSPLIT * BK * (BMP + BN) : (KSPLIT - 1) * BM * BN;

}  // namespace

cudaError_t launch_cgemm(const float2* A, const float2* B, float2* C, int M, int N, int K,
                         const int* gate, cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
  const size_t sm = kSmemFloat2 * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(cgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cgemm_kernel<<<grid, NT * KSPLIT, sm, st>>>(A, B, C, M, N, K, gate);
  return cudaGetLastError();
}

}  // namespace mrstat
