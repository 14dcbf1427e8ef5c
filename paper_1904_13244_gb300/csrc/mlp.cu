// Learned surrogate of the compressed Bloch model (K8): an MLP 3 -> H -> H -> H -> R
// from (ln T1, ln T2, B1) to the coefficients of the echo time course in the plan's
// time basis, with its derivatives in ln T1 and ln T2 by forward-mode tangents.
//
// Network (tanh hidden layers, linear output, per-coefficient output scale):
//     u = ((ln T1 - mu1)/s1, (ln T2 - mu2)/s2, (B1 - mu3)/s3)
//     a_l = tanh(W_l a_{l-1} + b_l),   c = scale * (W_4 a_3 + b_4)
// A tanh layer maps a tangent t to (1 - a^2) (W t); the tangents of u along ln T1 and
// ln T2 are (1/s1, 0, 0) and (0, 1/s2, 0).  So a batch of B samples runs as M = 3B rows
// (values, ln T1 tangents, ln T2 tangents) through every layer: one BF16 tcgen05 GEMM
// per layer shared by the value and both tangent streams, float32 accumulation,
// then one element-wise kernel for the activation and the tangent scaling.
//
// Training minimises the Sobolev loss
//     L = 1/B sum_b sum_r [(c - c*)^2 + lam ((dc1 - dc1*)^2 + (dc2 - dc2*)^2)] / scale_r^2
// with a hand-written backward pass: through s_k = (1 - a^2) z_k the value
// pre-activation receives (g_a - 2 a sum_k g_sk z_k)(1 - a^2) and each tangent
// pre-activation g_sk (1 - a^2); weight gradients are GEMMs of the gradient rows with
// the layer inputs over all 3B rows, input gradients GEMMs with the transposed weights.
// Adam keeps float32 master weights and refreshes the BF16 copies (row-major and
// transposed) used by the GEMMs.
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include <cuda_bf16.h>

#include "internal.cuh"
#include "mlp.cuh"
#include "tc_prims.cuh"

namespace mrstat {
namespace {

constexpr int kLayers = 4;

inline int pad8(int k) { return (k + 7) / 8 * 8; }

__global__ void mlp_input_kernel(const float* __restrict__ lnT, const float* __restrict__ b1, int B, float mu1,
                                 float s1, float mu2, float s2, float mu3, float s3, __nv_bfloat16* __restrict__ X0,
                                 __nv_bfloat16* __restrict__ X0T, int ldt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float bb = b1 != nullptr ? b1[b] : 1.f;
  const float u[3] = {(lnT[b] - mu1) / s1, (lnT[B + b] - mu2) / s2, (bb - mu3) / s3};
  const float t1[3] = {1.f / s1, 0.f, 0.f}, t2[3] = {0.f, 1.f / s2, 0.f};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float v0 = k < 3 ? u[k] : 0.f, v1 = k < 3 ? t1[k] : 0.f, v2 = k < 3 ? t2[k] : 0.f;
    X0[(size_t)b * 8 + k] = __float2bfloat16_rn(v0);
    X0[(size_t)(B + b) * 8 + k] = __float2bfloat16_rn(v1);
    X0[(size_t)(2 * B + b) * 8 + k] = __float2bfloat16_rn(v2);
    if (X0T != nullptr && k < 3) {
      X0T[(size_t)k * ldt + b] = __float2bfloat16_rn(v0);
      X0T[(size_t)k * ldt + B + b] = __float2bfloat16_rn(v1);
      X0T[(size_t)k * ldt + 2 * B + b] = __float2bfloat16_rn(v2);
    }
  }
}

// hidden layer: value rows a = tanh(z + bias), tangent rows (1 - a^2) z_k
__global__ void mlp_act_kernel(const float* __restrict__ Z, const float* __restrict__ bias, int B, int H,
                               __nv_bfloat16* __restrict__ X, int ldx, __nv_bfloat16* __restrict__ XT, int ldt) {
  const int64_t total = (int64_t)B * H;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / H), n = (int)(e - (int64_t)b * H);
    const float a = tanhf(Z[(size_t)b * H + n] + bias[n]);
    const float d = 1.f - a * a;
    const float s1 = d * Z[(size_t)(B + b) * H + n];
    const float s2 = d * Z[(size_t)(2 * B + b) * H + n];
    X[(size_t)b * ldx + n] = __float2bfloat16_rn(a);
    X[(size_t)(B + b) * ldx + n] = __float2bfloat16_rn(s1);
    X[(size_t)(2 * B + b) * ldx + n] = __float2bfloat16_rn(s2);
    if (XT != nullptr) {
      XT[(size_t)n * ldt + b] = __float2bfloat16_rn(a);
      XT[(size_t)n * ldt + B + b] = __float2bfloat16_rn(s1);
      XT[(size_t)n * ldt + 2 * B + b] = __float2bfloat16_rn(s2);
    }
  }
}

// output layer: predictions (c, dc1, dc2) [3][R][B] and, with targets, the loss and its
// gradient with respect to the output pre-activations
__global__ void mlp_output_kernel(const float* __restrict__ Z, const float* __restrict__ bias,
                                  const float* __restrict__ scale, int B, int R, float lam,
                                  const float* __restrict__ target, float* __restrict__ pred,
                                  __nv_bfloat16* __restrict__ GZ, int ldg, __nv_bfloat16* __restrict__ GZT, int ldt,
                                  double* __restrict__ loss) {
  const int64_t total = (int64_t)B * R;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / R), r = (int)(e - (int64_t)b * R);
    const float sc = scale[r];
    const float y0 = Z[(size_t)b * R + r] + bias[r];
    const float y1 = Z[(size_t)(B + b) * R + r];
    const float y2 = Z[(size_t)(2 * B + b) * R + r];
    if (pred != nullptr) {
      pred[(size_t)r * B + b] = sc * y0;
      pred[(size_t)(R + r) * B + b] = sc * y1;
      pred[(size_t)(2 * R + r) * B + b] = sc * y2;
    }
    if (target != nullptr) {
      const float r0 = y0 - target[(size_t)r * B + b] / sc;
      const float r1 = y1 - target[(size_t)(R + r) * B + b] / sc;
      const float r2 = y2 - target[(size_t)(2 * R + r) * B + b] / sc;
      acc += (double)r0 * r0 + (double)lam * ((double)r1 * r1 + (double)r2 * r2);
      const float inv = 2.f / (float)B;
      const float g0 = inv * r0, g1 = inv * lam * r1, g2 = inv * lam * r2;
      GZ[(size_t)b * ldg + r] = __float2bfloat16_rn(g0);
      GZ[(size_t)(B + b) * ldg + r] = __float2bfloat16_rn(g1);
      GZ[(size_t)(2 * B + b) * ldg + r] = __float2bfloat16_rn(g2);
      GZT[(size_t)r * ldt + b] = __float2bfloat16_rn(g0);
      GZT[(size_t)r * ldt + B + b] = __float2bfloat16_rn(g1);
      GZT[(size_t)r * ldt + 2 * B + b] = __float2bfloat16_rn(g2);
    }
  }
  if (target != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(loss, acc / (double)B);
  }
}

// backward through a tanh layer: GX [3B][H] = dL/d(layer output) -> GZ (and transposed), db
__global__ void mlp_backact_kernel(const float* __restrict__ GX, const float* __restrict__ Z,
                                   const float* __restrict__ bias, int B, int H, __nv_bfloat16* __restrict__ GZ,
                                   int ldg, __nv_bfloat16* __restrict__ GZT, int ldt, float* __restrict__ db) {
  const int64_t total = (int64_t)B * H;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / H), n = (int)(e - (int64_t)b * H);
    const float a = tanhf(Z[(size_t)b * H + n] + bias[n]);
    const float d = 1.f - a * a;
    const float z1 = Z[(size_t)(B + b) * H + n], z2 = Z[(size_t)(2 * B + b) * H + n];
    const float ga = GX[(size_t)b * H + n], g1 = GX[(size_t)(B + b) * H + n], g2 = GX[(size_t)(2 * B + b) * H + n];
    const float gz1 = g1 * d, gz2 = g2 * d;
    const float gz = (ga - 2.f * a * (g1 * z1 + g2 * z2)) * d;
    GZ[(size_t)b * ldg + n] = __float2bfloat16_rn(gz);
    GZ[(size_t)(B + b) * ldg + n] = __float2bfloat16_rn(gz1);
    GZ[(size_t)(2 * B + b) * ldg + n] = __float2bfloat16_rn(gz2);
    GZT[(size_t)n * ldt + b] = __float2bfloat16_rn(gz);
    GZT[(size_t)n * ldt + B + b] = __float2bfloat16_rn(gz1);
    GZT[(size_t)n * ldt + 2 * B + b] = __float2bfloat16_rn(gz2);
    atomicAdd(db + n, gz);
  }
}

// output-layer bias gradient: sum over the value rows of the output gradient
__global__ void mlp_out_bias_grad_kernel(const float* __restrict__ Z, const float* __restrict__ bias,
                                         const float* __restrict__ scale, const float* __restrict__ target, int B,
                                         int R, float* __restrict__ db) {
  const int r = blockIdx.x;
  float acc = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x)
    acc += 2.f / (float)B * (Z[(size_t)b * R + r] + bias[r] - target[(size_t)r * B + b] / scale[r]);
  __shared__ float ws[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    db[r] = s;
  }
}

// Adam on one layer (weights [out][in] then bias [out]) and refresh of its BF16 copies
__global__ void mlp_adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, int out, int in, float lr, float b1, float b2, float eps,
                                float c1, float c2, __nv_bfloat16* __restrict__ W, int ldw,
                                __nv_bfloat16* __restrict__ WT, int ldwt) {
  const int total = out * in + out;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float w = theta[e] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    theta[e] = w;
    if (e < out * in) {
      const int o = e / in, i = e - o * in;
      W[(size_t)o * ldw + i] = __float2bfloat16_rn(w);
      WT[(size_t)i * ldwt + o] = __float2bfloat16_rn(w);
    }
  }
}

// BF16 copies of one layer's weights from the float32 master (after set_params)
__global__ void mlp_cast_kernel(const float* __restrict__ theta, int out, int in, __nv_bfloat16* __restrict__ W,
                                int ldw, __nv_bfloat16* __restrict__ WT, int ldwt) {
  const int total = out * in;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int o = e / in, i = e - o * in;
    const __nv_bfloat16 w = __float2bfloat16_rn(theta[e]);
    W[(size_t)o * ldw + i] = w;
    WT[(size_t)i * ldwt + o] = w;
  }
}

// ---------------------------------------------------------------------------
// Fused inference layer.  Per K chunk TMA brings the three 128-row tiles of the layer
// input (value rows b, ln T1 tangent rows B + b, ln T2 tangent rows 2B + b) and one weight
// tile; one thread issues three tcgen05.mma per K step into three TMEM accumulators, so
// the epilogue sees z, z1, z2 of the same (sample, feature) and applies the layer there:
//   hidden: a = tanh(z + bias), s_k = (1 - a^2) z_k, written as the next layer's BF16 input;
//   output: pred[k][r][b] = scale_r (z_k + [k = 0] bias_r), coalesced along the samples.
// The pre-activations never reach global memory.  The hidden-layer tanh is the hardware
// tanh.approx.f32 (relative error about 2^-11, below the BF16 rounding of the values it
// produces).
//
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Persistent kernel: one CTA per SM walks the (128-row tile, 64-column tile) pairs, n
// fastest, so the CTAs working on one row tile at a time share its three input tiles
// through L2.  Warp 0 issues the TMA loads (three input
// tiles and the weight tile per 64-wide K chunk) into a ring of stages, warp 1 issues the
// three MMAs per K step into one of two TMEM accumulator sets (3 x 64 columns each), and
// sixteen epilogue warps (four per TMEM lane quarter, one 16-column chunk each: enough
// warps to hide the latency of the per-element work) run the epilogue of tile i while the
// MMAs of tile i + 1 proceed: bias and tanh, the tangent scaling 1 - a^2, BF16, 32-byte stores
// straight to the next layer's input rows (or, for the last layer, the scaled outputs).
// Every wait is bounded; a CTA that gives up sets err and drains its copies in flight.
// ---------------------------------------------------------------------------
// Layer 0 (three inputs: ln T1, ln T2, B1) on the CUDA cores, straight from the
// parameters: the same BF16-rounded inputs and weights and float32 sums as a tensor-core
// layer, then the hidden-layer epilogue, written as layer 1's BF16 input rows (value,
// ln T1 tangent, ln T2 tangent).  Thread per (sample, 8 features): consecutive threads
// take consecutive feature groups of one sample, so the 16-byte stores of a warp fill
// whole rows; the block's copy of the weights and biases sits in shared memory as
// [input][feature within group][group], which the lanes of a warp read without bank
// conflicts.  N <= 256 features (groups <= 32), N a multiple of 8.
constexpr int kFirstMaxGroups = 32;
__global__ void __launch_bounds__(256)
mlp_first_layer_kernel(const float* __restrict__ lnT, const float* __restrict__ b1, int B, float mu1, float s1,
                       float mu2, float s2, float mu3, float s3, const __nv_bfloat16* __restrict__ W0, int ldw,
                       const float* __restrict__ bias, int N, __nv_bfloat16* __restrict__ xn, int ldn) {
  __shared__ float ws[4][8][kFirstMaxGroups];
  const int groups = N / 8;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const int g = n >> 3, j = n & 7;
    ws[0][j][g] = __bfloat162float(W0[(size_t)n * ldw]);
    ws[1][j][g] = __bfloat162float(W0[(size_t)n * ldw + 1]);
    ws[2][j][g] = __bfloat162float(W0[(size_t)n * ldw + 2]);
    ws[3][j][g] = bias[n];
  }
  __syncthreads();
  const float d1 = __bfloat162float(__float2bfloat16_rn(1.f / s1));
  const float d2 = __bfloat162float(__float2bfloat16_rn(1.f / s2));
  const int total = B * groups;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int b = e / groups, g = e - b * groups;
    const float bb = b1 != nullptr ? b1[b] : 1.f;
    const float u0 = __bfloat162float(__float2bfloat16_rn((lnT[b] - mu1) / s1));
    const float u1 = __bfloat162float(__float2bfloat16_rn((lnT[B + b] - mu2) / s2));
    const float u2 = __bfloat162float(__float2bfloat16_rn((bb - mu3) / s3));
    __align__(16) __nv_bfloat16 o0[8], o1[8], o2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float w0 = ws[0][j][g], w1 = ws[1][j][g], w2 = ws[2][j][g];
      const float z = fmaf(w2, u2, fmaf(w1, u1, w0 * u0));
      const float a = tanh_fast(z + ws[3][j][g]);
      const float dd = 1.f - a * a;
      o0[j] = __float2bfloat16_rn(a);
      o1[j] = __float2bfloat16_rn(dd * (w0 * d1));
      o2[j] = __float2bfloat16_rn(dd * (w1 * d2));
    }
    const size_t row = (size_t)b * ldn + 8 * g, plane = (size_t)B * ldn;
    *reinterpret_cast<uint4*>(xn + row) = *reinterpret_cast<const uint4*>(o0);
    *reinterpret_cast<uint4*>(xn + plane + row) = *reinterpret_cast<const uint4*>(o1);
    *reinterpret_cast<uint4*>(xn + 2 * plane + row) = *reinterpret_cast<const uint4*>(o2);
  }
}

constexpr int kPerStages = 3;
struct PerShape {
  static constexpr int BN = 64;
  static constexpr uint32_t kA = tc::BM * tc::BK * 2;  // one 128-row input tile
  static constexpr uint32_t kB = BN * tc::BK * 2;      // one 64-row weight tile
  static constexpr uint32_t kStage = 3 * kA + kB;
  static constexpr uint32_t kTmemCols = 512;           // 2 sets x 3 streams x 64 columns
  static constexpr size_t kSmem = (size_t)kPerStages * kStage + 1024 + 256;
};

constexpr int kPerEpiWarps = 16;  // four per TMEM lane quarter, one 16-column chunk each
constexpr int kPerThreads = 64 + 32 * kPerEpiWarps;

template <bool LAST>
__global__ void __launch_bounds__(kPerThreads, 1)
mlp_layer_persistent_kernel(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tw, int B,
                            int N, int K, const float* __restrict__ bias, __nv_bfloat16* __restrict__ xn, int ldn,
                            const float* __restrict__ scale, float* __restrict__ pred, int* __restrict__ err) {
  using namespace tc;
  using PS = PerShape;
  constexpr int BN = PS::BN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kPerStages * PS::kStage);
  uint64_t* empty = full + kPerStages;
  uint64_t* accf = empty + kPerStages;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (N + BN - 1) / BN;
  const int tiles = ((B + BM - 1) / BM) * n_tiles;
  const int nk = (K + BK - 1) / BK;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPerStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], kPerEpiWarps);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc<PS::kTmemCols>(tmem_slot);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool go = true;
      for (int t = blockIdx.x; t < tiles && go; t += gridDim.x) {
        const int b0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
        for (int c = 0; c < nk; ++c, ++g) {
          const int s = g % kPerStages;
          const uint32_t use = (uint32_t)(g / kPerStages);
          if (g >= kPerStages && !mbar_wait(&empty[s], (use - 1) & 1u, abort_flag)) {
            go = false;
            break;
          }
          uint8_t* st = smem + s * PS::kStage;
          mbar_expect_tx(&full[s], PS::kStage);
          tma_load_2d(&tx, &full[s], st, c * BK, b0);
          tma_load_2d(&tx, &full[s], st + PS::kA, c * BK, B + b0);
          tma_load_2d(&tx, &full[s], st + 2 * PS::kA, c * BK, 2 * B + b0);
          tma_load_2d(&tw, &full[s], st + 3 * PS::kA, c * BK, n0);
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc(BM, BN);
      int g = 0, i = 0;
      bool go = true;
      for (int t = blockIdx.x; t < tiles && go; t += gridDim.x, ++i) {
        const int acc = i & 1;
        if (i >= 2 && !mbar_wait(&acce[acc], (uint32_t)((i >> 1) - 1) & 1u, abort_flag)) break;
        fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * 3 * BN);
        for (int c = 0; c < nk; ++c, ++g) {
          const int s = g % kPerStages;
          if (!mbar_wait(&full[s], (uint32_t)(g / kPerStages) & 1u, abort_flag)) {
            go = false;
            break;
          }
          fence_after();
          const uint8_t* st = smem + s * PS::kStage;
          const uint64_t d0 = sdesc_sw128(st), d1 = sdesc_sw128(st + PS::kA), d2 = sdesc_sw128(st + 2 * PS::kA);
          const uint64_t dw = sdesc_sw128(st + 3 * PS::kA);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t off = 2ull * k;
            const uint32_t accum = (c > 0 || k > 0) ? 1u : 0u;
            mma_bf16(d, d0 + off, dw + off, idesc, accum);
            mma_bf16(d + BN, d1 + off, dw + off, idesc, accum);
            mma_bf16(d + 2 * BN, d2 + off, dw + off, idesc, accum);
          }
          mma_commit(&empty[s]);
        }
        if (go) mma_commit(&accf[acc]);
      }
    }
  } else {
    const int q = warp & 3;              // TMEM lane quarter of this warp
    const int cb = ((warp - 2) >> 2) * 16;  // its 16-column chunk of the tile
    int i = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
      const int acc = i & 1;
      if (!mbar_wait(&accf[acc], (uint32_t)(i >> 1) & 1u, abort_flag)) break;
      __syncwarp();
      fence_after();
      const int b0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
      const int b = b0 + q * 32 + lane;  // this lane's row (sample)
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 3 * BN);
      float v0[16], v1[16], v2[16];
      tmem_ld16(trow + (uint32_t)cb, v0);
      tmem_ld16(trow + (uint32_t)(BN + cb), v1);
      tmem_ld16(trow + (uint32_t)(2 * BN + cb), v2);
      // this warp's part of the accumulator set is in registers: hand it back
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[acc]);
      if (b >= B) continue;
      if (LAST) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int r = n0 + cb + j;
          if (r < N) {
            const float sc = scale[r];
            pred[(size_t)r * B + b] = sc * (v0[j] + bias[r]);
            pred[(size_t)(N + r) * B + b] = sc * v1[j];
            pred[(size_t)(2 * N + r) * B + b] = sc * v2[j];
          }
        }
      } else {
        __align__(16) __nv_bfloat16 o[3][16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + cb + j;
          const float a = tanh_fast(v0[j] + (n < N ? bias[n] : 0.f));
          const float dd = 1.f - a * a;
          o[0][j] = __float2bfloat16_rn(a);
          o[1][j] = __float2bfloat16_rn(dd * v1[j]);
          o[2][j] = __float2bfloat16_rn(dd * v2[j]);
        }
        const int col = n0 + cb;
        if (col + 16 <= ldn) {  // 32 bytes per stream (ldn and col are multiples of 8 elements)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            uint4* dst = reinterpret_cast<uint4*>(xn + ((size_t)k * B + b) * ldn + col);
            dst[0] = reinterpret_cast<const uint4*>(o[k])[0];
            dst[1] = reinterpret_cast<const uint4*>(o[k])[1];
          }
        } else {
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (col + j < ldn) xn[((size_t)k * B + b) * ldn + col + j] = o[k][j];
        }
      }
    }
  }

  __syncwarp();
  if (threadIdx.x == 0 && *abort_flag) {
    atomicExch(err, 1);
    // let the copies this thread issued land before the CTA's shared memory goes away
    for (int g = issued > kPerStages ? issued - kPerStages : 0; g < issued; ++g) {
      int spins = 0;
      while (!mbar_try_wait(&full[g % kPerStages], (uint32_t)(g / kPerStages) & 1u) && ++spins < (1 << 16)) {
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc<PS::kTmemCols>(tmem);
}

int blocks_for(int64_t n, int t = 256) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

}  // namespace

// ---------------------------------------------------------------------------
Mlp::~Mlp() {
  release_batch();
  free_weights();
  if (dev_err) cudaFree(dev_err);
}

void Mlp::free_weights() {
  void* ptrs[] = {theta, adam_m, adam_v, grad, scale_dev};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int l = 0; l < 4; ++l) {
    if (Wb[l]) cudaFree(Wb[l]);
    if (WTb[l]) cudaFree(WTb[l]);
    Wb[l] = WTb[l] = nullptr;
  }
  theta = adam_m = adam_v = grad = scale_dev = nullptr;
}

void Mlp::release_batch() {
  for (int l = 0; l < 4; ++l) {
    void* ptrs[] = {X[l], XT[l], Z[l], GZ[l], GZT[l]};
    for (void* q : ptrs)
      if (q) cudaFree(q);
    X[l] = XT[l] = GZ[l] = GZT[l] = nullptr;
    Z[l] = nullptr;
  }
  if (GX) cudaFree(GX);
  if (loss_dev) cudaFree(loss_dev);
  GX = nullptr;
  loss_dev = nullptr;
  cap = 0;
  maps_b = -1;
}

int Mlp::setup(int h, int r, uint64_t seed) {
  H = h;
  R = r;
  const int dims[5] = {3, H, H, H, R};
  np = 0;
  for (int l = 0; l < 4; ++l) {
    in[l] = dims[l];
    out[l] = dims[l + 1];
    off[l] = np;
    np += (int64_t)out[l] * in[l] + out[l];
  }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t q) {
    if (e == cudaSuccess) e = q;
  };
  chk(cudaMalloc(&theta, np * sizeof(float)));
  chk(cudaMalloc(&adam_m, np * sizeof(float)));
  chk(cudaMalloc(&adam_v, np * sizeof(float)));
  chk(cudaMalloc(&grad, np * sizeof(float)));
  chk(cudaMalloc(&scale_dev, R * sizeof(float)));
  chk(cudaMalloc(&dev_err, sizeof(int)));
  if (e == cudaSuccess) chk(cudaMemset(dev_err, 0, sizeof(int)));
  for (int l = 0; l < 4; ++l) {
    chk(cudaMalloc(&Wb[l], (size_t)out[l] * pad8(in[l]) * 2));
    chk(cudaMalloc(&WTb[l], (size_t)in[l] * pad8(out[l]) * 2));
    if (e == cudaSuccess) {
      chk(cudaMemset(Wb[l], 0, (size_t)out[l] * pad8(in[l]) * 2));
      chk(cudaMemset(WTb[l], 0, (size_t)in[l] * pad8(out[l]) * 2));
      chk(make_split_operand(&opW[l], Wb[l], Wb[l], out[l], in[l], pad8(in[l]), false));
      chk(make_bf16_tmap(&wmap64[l], Wb[l], out[l], in[l], pad8(in[l]), PerShape::BN));
      chk(make_split_operand(&opWT[l], WTb[l], WTb[l], in[l], out[l], pad8(out[l]), false));
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "surrogate allocation");
  // Glorot-uniform weights, zero biases, unit output scale
  std::vector<float> th(np, 0.f), sc(R, 1.f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < 4; ++l) {
    const float lim = std::sqrt(6.f / (float)(in[l] + out[l]));
    std::uniform_real_distribution<float> U(-lim, lim);
    for (int64_t k = 0; k < (int64_t)out[l] * in[l]; ++k) th[off[l] + k] = U(rng);
  }
  chk(cudaMemcpy(scale_dev, sc.data(), R * sizeof(float), cudaMemcpyHostToDevice));
  scale_host = sc;
  chk(cudaMemset(adam_m, 0, np * sizeof(float)));
  chk(cudaMemset(adam_v, 0, np * sizeof(float)));
  if (e != cudaSuccess) return cuda_fail(e, "surrogate init");
  return set_params(th.data(), nullptr);
}

int Mlp::set_params(const float* host, cudaStream_t st) {
  cudaError_t e = cudaMemcpy(theta, host, np * sizeof(float), cudaMemcpyHostToDevice);
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    mlp_cast_kernel<<<blocks_for((int64_t)out[l] * in[l]), 256, 0, st>>>(theta + off[l], out[l], in[l], Wb[l],
                                                                        pad8(in[l]), WTb[l], pad8(out[l]));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  step = 0;
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "surrogate parameters");
}

// (re)allocates the activation buffers for up to B samples and encodes the tensor maps
int Mlp::ensure_batch(int B, bool train) {
  if (B > cap || (train && !have_train_buffers)) {
    release_batch();
    const int Mc = 3 * B, Mp = pad8(Mc);
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t q) {
      if (e == cudaSuccess) e = q;
    };
    for (int l = 0; l < 4; ++l) {
      chk(cudaMalloc(&X[l], (size_t)Mc * pad8(in[l]) * 2));
      if (train) {
        chk(cudaMalloc(&Z[l], (size_t)Mc * out[l] * sizeof(float)));
        chk(cudaMalloc(&XT[l], (size_t)in[l] * Mp * 2));
        chk(cudaMalloc(&GZ[l], (size_t)Mc * pad8(out[l]) * 2));
        chk(cudaMalloc(&GZT[l], (size_t)out[l] * Mp * 2));
      }
    }
    if (train) chk(cudaMalloc(&GX, (size_t)Mc * H * sizeof(float)));
    chk(cudaMalloc(&loss_dev, sizeof(double)));
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
      chk(cudaMemset(X[l], 0, (size_t)Mc * pad8(in[l]) * 2));
      if (train) {
        chk(cudaMemset(XT[l], 0, (size_t)in[l] * Mp * 2));
        chk(cudaMemset(GZ[l], 0, (size_t)Mc * pad8(out[l]) * 2));
        chk(cudaMemset(GZT[l], 0, (size_t)out[l] * Mp * 2));
      }
    }
    if (e != cudaSuccess) {
      release_batch();
      return cuda_fail(e, "surrogate batch buffers");
    }
    cap = B;
    have_train_buffers = train;
  }
  if (maps_b != B || maps_train != train) {
    const int Mc = 3 * B, Mp = pad8(3 * cap);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
      e = make_split_operand(&opX[l], X[l], X[l], Mc, in[l], pad8(in[l]), true);
      if (e == cudaSuccess && train) e = make_split_operand(&opXT[l], XT[l], XT[l], in[l], Mc, Mp, false);
      if (e == cudaSuccess && train) e = make_split_operand(&opGZ[l], GZ[l], GZ[l], Mc, out[l], pad8(out[l]), true);
      if (e == cudaSuccess && train) e = make_split_operand(&opGZT[l], GZT[l], GZT[l], out[l], Mc, Mp, true);
    }
    if (e != cudaSuccess) return cuda_fail(e, "surrogate tensor maps");
    maps_b = B;
    maps_train = train;
  }
  return MRSTAT_OK;
}

int Mlp::forward(const float* lnT, const float* b1, int B, bool train, cudaStream_t st) {
  const int Mc = 3 * B;
  const int ldt = pad8(3 * cap);
  mlp_input_kernel<<<blocks_for(B), 256, 0, st>>>(lnT, b1, B, norm[0], norm[1], norm[2], norm[3], norm[4], norm[5],
                                                  X[0], train ? XT[0] : nullptr, ldt);
  cudaError_t e = cudaGetLastError();
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    e = launch_tc_gemm(opX[l], opW[l], Z[l], Mc, out[l], in[l], out[l], 1, nullptr, dev_err, st);
    if (e != cudaSuccess || l == 3) break;
    mlp_act_kernel<<<blocks_for((int64_t)B * out[l]), 256, 0, st>>>(Z[l], theta + off[l] + (int64_t)out[l] * in[l],
                                                                    B, out[l], X[l + 1], pad8(in[l + 1]),
                                                                    train ? XT[l + 1] : nullptr, ldt);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "surrogate forward");
}

int Mlp::backward(const float* target, int B, cudaStream_t st) {
  const int Mc = 3 * B;
  const int ldt = pad8(3 * cap);
  cudaError_t e = cudaMemsetAsync(grad, 0, np * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss_dev, 0, sizeof(double), st);
  // output layer
  const float* b4 = theta + off[3] + (int64_t)out[3] * in[3];
  if (e == cudaSuccess) {
    mlp_output_kernel<<<blocks_for((int64_t)B * R), 256, 0, st>>>(Z[3], b4, scale_dev, B, R, lam, target, nullptr,
                                                                  GZ[3], pad8(out[3]), GZT[3], ldt, loss_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    mlp_out_bias_grad_kernel<<<R, 256, 0, st>>>(Z[3], b4, scale_dev, target, B, R,
                                                grad + off[3] + (int64_t)out[3] * in[3]);
    e = cudaGetLastError();
  }
  for (int l = 3; l >= 0 && e == cudaSuccess; --l) {
    // dW_l = GZ_l^T X_l over all 3B rows
    e = launch_tc_gemm(opGZT[l], opXT[l], grad + off[l], out[l], in[l], Mc, in[l], 1, nullptr, dev_err, st);
    if (e != cudaSuccess || l == 0) break;
    // dL/dX_l = GZ_l W_l, then back through layer l-1's tanh
    e = launch_tc_gemm(opGZ[l], opWT[l], GX, Mc, in[l], out[l], in[l], 1, nullptr, dev_err, st);
    if (e != cudaSuccess) break;
    const int lp = l - 1;
    mlp_backact_kernel<<<blocks_for((int64_t)B * out[lp]), 256, 0, st>>>(
        GX, Z[lp], theta + off[lp] + (int64_t)out[lp] * in[lp], B, out[lp], GZ[lp], pad8(out[lp]), GZT[lp], ldt,
        grad + off[lp] + (int64_t)out[lp] * in[lp]);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "surrogate backward");
}

int Mlp::adam(float lr, cudaStream_t st) {
  ++step;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
    mlp_adam_kernel<<<blocks_for((int64_t)out[l] * in[l] + out[l]), 256, 0, st>>>(
        theta + off[l], adam_m + off[l], adam_v + off[l], grad + off[l], out[l], in[l], lr, b1, b2, eps, c1, c2, Wb[l],
        pad8(in[l]), WTb[l], pad8(out[l]));
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "surrogate Adam step");
}


template <bool LAST>
static cudaError_t launch_persistent(const TcOperand& x, const CUtensorMap& w64, int B, int N, int K,
                                     const float* bias, __nv_bfloat16* xn, int ldn, const float* scale, float* pred,
                                     int* err, cudaStream_t st) {
  const size_t sm = PerShape::kSmem;
  cudaError_t e = cudaFuncSetAttribute(mlp_layer_persistent_kernel<LAST>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tiles = ((B + tc::BM - 1) / tc::BM) * ((N + PerShape::BN - 1) / PerShape::BN);
  const int grid = std::max(1, std::min(tiles, sms));
  mlp_layer_persistent_kernel<LAST><<<grid, kPerThreads, sm, st>>>(x.hi, w64, B, N, K, bias, xn, ldn, scale, pred, err);
  return cudaGetLastError();
}

// Inference: layer 0 on the CUDA cores, then one persistent fused tensor-core kernel per
// layer (no pre-activation buffers).
int Mlp::infer_fused(const float* lnT, const float* b1, int B, float* pred, cudaStream_t st) {
  {
    const int groups = out[0] / 8;  // hidden width 64, 128 or 256
    mlp_first_layer_kernel<<<blocks_for((int64_t)B * groups), 256, 0, st>>>(
        lnT, b1, B, norm[0], norm[1], norm[2], norm[3], norm[4], norm[5], Wb[0], pad8(in[0]),
        theta + off[0] + (int64_t)out[0] * in[0], out[0], X[1], pad8(in[1]));
  }
  cudaError_t e = cudaGetLastError();
  for (int l = 1; l < 4 && e == cudaSuccess; ++l) {
    const float* bias = theta + off[l] + (int64_t)out[l] * in[l];
    const bool last = l == 3;
    __nv_bfloat16* xn = last ? nullptr : X[l + 1];
    const int ldn = last ? 0 : pad8(in[l + 1]);
    e = last ? launch_persistent<true>(opX[l], wmap64[l], B, out[l], in[l], bias, xn, ldn, scale_dev, pred, dev_err, st)
             : launch_persistent<false>(opX[l], wmap64[l], B, out[l], in[l], bias, xn, ldn, scale_dev, pred, dev_err,
                                        st);
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "surrogate inference");
}

int mlp_infer(Mlp* m, const float* lnT, const float* b1, int n, float* coef, cudaStream_t st) {
  int s = m->ensure_batch(n, false);
  if (s == MRSTAT_OK) s = m->infer_fused(lnT, b1, n, coef, st);
  return s;
}

}  // namespace mrstat

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
using namespace mrstat;

struct mrstat_mlp : public Mlp {};

extern "C" {

int mrstat_mlp_create(const mrstat_mlp_config* cfg, mrstat_mlp** out) {
  if (out == nullptr || cfg == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL config or out");
  *out = nullptr;
  if ((cfg->hidden != 64 && cfg->hidden != 128 && cfg->hidden != 256) || cfg->rank < 1 || cfg->rank > kMaxRank)
    return fail(MRSTAT_ERR_INVALID_ARG, "hidden %d (64, 128 or 256) or rank %d (1..32) not supported", cfg->hidden,
                cfg->rank);
  for (int k = 1; k < 6; k += 2)
    if (!(cfg->norm[k] > 0)) return fail(MRSTAT_ERR_INVALID_ARG, "normalisation scales must be positive");
  mrstat_mlp* m = new mrstat_mlp();
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return fail(MRSTAT_ERR_CUDA, "no CUDA device");
  }
  for (int k = 0; k < 6; ++k) m->norm[k] = cfg->norm[k];
  m->lam = cfg->sobolev_weight;
  const int s = m->setup(cfg->hidden, cfg->rank, cfg->seed);
  if (s != MRSTAT_OK) {
    delete m;
    return s;
  }
  *out = m;
  return MRSTAT_OK;
}

int mrstat_mlp_destroy(mrstat_mlp* m) {
  if (m == nullptr) return MRSTAT_OK;
  DeviceGuard g(m->device);
  cudaDeviceSynchronize();
  delete m;
  return MRSTAT_OK;
}

int64_t mrstat_mlp_num_params(const mrstat_mlp* m) { return m ? m->np : 0; }

int mrstat_mlp_set_output_scale(mrstat_mlp* m, const float* scale) {
  if (m == nullptr || scale == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL argument");
  for (int r = 0; r < m->R; ++r)
    if (!(scale[r] > 0)) return fail(MRSTAT_ERR_INVALID_ARG, "output scales must be positive");
  DeviceGuard g(m->device);
  m->scale_host.assign(scale, scale + m->R);
  cudaError_t e = cudaMemcpy(m->scale_dev, scale, m->R * sizeof(float), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "output scale");
}

int mrstat_mlp_get_params(mrstat_mlp* m, float* host) {
  if (m == nullptr || host == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(m->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host, m->theta, m->np * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "get parameters");
}

int mrstat_mlp_set_params(mrstat_mlp* m, const float* host) {
  if (m == nullptr || host == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(m->device);
  cudaDeviceSynchronize();
  return m->set_params(host, nullptr);
}

int mrstat_mlp_infer(mrstat_mlp* m, const float* lnT, const float* b1, int32_t n, float* coef, void* stream) {
  MRSTAT_ABI_RANGE();
  if (m == nullptr || lnT == nullptr || coef == nullptr || n < 1)
    return fail(MRSTAT_ERR_INVALID_ARG, "bad argument to mrstat_mlp_infer");
  DeviceGuard g(m->device);
  return mlp_infer(m, lnT, b1, n, coef, reinterpret_cast<cudaStream_t>(stream));
}

int mrstat_mlp_train_step(mrstat_mlp* m, const float* lnT, const float* b1, const float* target, int32_t B, float lr,
                          double* loss_out, void* stream) {
  MRSTAT_ABI_RANGE();
  if (m == nullptr || lnT == nullptr || target == nullptr || B < 1 || !(lr >= 0))
    return fail(MRSTAT_ERR_INVALID_ARG, "bad argument to mrstat_mlp_train_step");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int s = m->ensure_batch(B, true);
  if (s == MRSTAT_OK) s = m->forward(lnT, b1, B, true, st);
  if (s == MRSTAT_OK) s = m->backward(target, B, st);
  if (s == MRSTAT_OK && lr > 0) s = m->adam(lr, st);
  if (s == MRSTAT_OK && loss_out != nullptr) {
    cudaError_t e = cudaMemcpyAsync(loss_out, m->loss_dev, sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) s = cuda_fail(e, "loss copy");
  }
  return s;
}

int mrstat_mlp_loss_grad(mrstat_mlp* m, const float* lnT, const float* b1, const float* target, int32_t B,
                         double* loss_host, float* grad, void* stream) {
  MRSTAT_ABI_RANGE();
  if (m == nullptr || lnT == nullptr || target == nullptr || B < 1)
    return fail(MRSTAT_ERR_INVALID_ARG, "bad argument to mrstat_mlp_loss_grad");
  DeviceGuard g(m->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int s = m->ensure_batch(B, true);
  if (s == MRSTAT_OK) s = m->forward(lnT, b1, B, true, st);
  if (s == MRSTAT_OK) s = m->backward(target, B, st);
  if (s != MRSTAT_OK) return s;
  cudaError_t e = cudaSuccess;
  if (grad) e = cudaMemcpyAsync(grad, m->grad, m->np * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, m->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, m->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "surrogate gradient");
  if (herr) {
    cudaMemset(m->dev_err, 0, sizeof(int));
    return fail(MRSTAT_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on its pipeline barriers");
  }
  return MRSTAT_OK;
}

}  // extern "C"
