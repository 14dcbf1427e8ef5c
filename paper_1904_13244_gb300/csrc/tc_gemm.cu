// Tensor-core GEMM for sm_103a: C[M][N] (float32) = sum_p A_p[M][K] B_p[N][K]^T with
// BF16 operands, float32 accumulation in tensor memory.
//
// Used for the split-BF16 form of the readout DFT: an FP32 operand x is carried as
// x_hi + x_lo with x_hi = bf16(x) and x_lo = bf16(x - x_hi), and the product keeps
// the three leading terms A_hi B_hi + A_hi B_lo + A_lo B_hi (about 16 significant
// bits per operand; the dropped A_lo B_lo term is ~2^-18 relative).
//
// Structure (one 128 x BN output tile per CTA, 128 threads):
//   warp 0 lane 0   TMA producer: 128B-swizzled K-major tiles of 64 K elements into
//                   a STAGES-deep shared-memory ring (mbarrier expect-tx per stage);
//   warp 1 lane 0   MMA issuer: tcgen05.mma.kind::f16 M=128 N=BN K=16, accumulating
//                   in TMEM; tcgen05.commit frees each stage and finally signals done;
//   warps 0..3      epilogue: tcgen05.ld 32 lanes x 16 columns per warp, float32 stores.
// Every mbarrier wait is bounded; on timeout the CTA records an error code, skips the
// rest of its work, releases its tensor memory and returns.
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstring>

#include "internal.cuh"
#include "tc_gemm.cuh"
#include "tc_prims.cuh"

namespace mrstat {
namespace {

using namespace tc;

template <int BN, int STAGES>
struct TileShape {
  static constexpr uint32_t kA = BM * BK * 2;            // bytes of one A tile
  static constexpr uint32_t kB = BN * BK * 2;            // bytes of one B tile
  static constexpr uint32_t kStage = 2 * kA + 2 * kB;    // hi and lo of both
  static constexpr uint32_t kTmemCols = BN < 32 ? 32 : BN;
  static constexpr size_t kSmem = (size_t)STAGES * kStage + 1024 /* align */ + 256 /* barriers */;
  static_assert((size_t)STAGES * kStage >= (size_t)4 * 32 * (BN + 1) * 4, "epilogue staging fits the ring");
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(128, 2)
tc_gemm_kernel(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
               const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
               float* __restrict__ C, int M, int N, int K, int ldc, int nprod, const int* __restrict__ gate,
               int* __restrict__ err) {
  using TS = TileShape<BN, STAGES>;
  static_assert(BN == 64 || BN == 128, "N tiles of 64 or 128 columns");
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * TS::kStage);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc<TS::kTmemCols>(tmem_slot);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // chunks whose loads the producer issued
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    for (int c = 0; c < nk; ++c) {
      const int s = c % STAGES;
      const uint32_t use = (uint32_t)(c / STAGES);
      if (c >= STAGES && !mbar_wait(&empty[s], (use - 1) & 1u, abort_flag)) break;
      uint8_t* a_hi = smem + s * TS::kStage;
      uint8_t* a_lo = a_hi + TS::kA;
      uint8_t* b_hi = a_lo + TS::kA;
      uint8_t* b_lo = b_hi + TS::kB;
      mbar_expect_tx(&full[s], nprod == 3 ? TS::kStage : TS::kA + TS::kB);
      tma_load_2d(&ta_hi, &full[s], a_hi, c * BK, m0);
      tma_load_2d(&tb_hi, &full[s], b_hi, c * BK, n0);
      if (nprod == 3) {
        tma_load_2d(&ta_lo, &full[s], a_lo, c * BK, m0);
        tma_load_2d(&tb_lo, &full[s], b_lo, c * BK, n0);
      }
      issued = c + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t idesc = make_idesc(BM, BN);
    for (int c = 0; c < nk; ++c) {
      const int s = c % STAGES;
      if (!mbar_wait(&full[s], (uint32_t)(c / STAGES) & 1u, abort_flag)) break;
      fence_after();
      const uint8_t* a_hi = smem + s * TS::kStage;
      const uint8_t* a_lo = a_hi + TS::kA;
      const uint8_t* b_hi = a_lo + TS::kA;
      const uint8_t* b_lo = b_hi + TS::kB;
      const uint64_t dah = sdesc_sw128(a_hi), dal = sdesc_sw128(a_lo);
      const uint64_t dbh = sdesc_sw128(b_hi), dbl = sdesc_sw128(b_lo);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        const uint64_t off = 2ull * k;  // 16 BF16 = 32 B along K, in 16-byte units
        mma_bf16(tmem, dah + off, dbh + off, idesc, (c > 0 || k > 0) ? 1u : 0u);
        if (nprod == 3) {
          mma_bf16(tmem, dah + off, dbl + off, idesc, 1u);
          mma_bf16(tmem, dal + off, dbh + off, idesc, 1u);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }

  // ---------------- epilogue ----------------
  // the other lanes of the producer and MMA warps wait here, not in the spin below, so
  // that they do not compete with their role lane for the warp's issue slots
  __syncwarp();
  const bool ok = mbar_wait(done, 0, abort_flag) && *abort_flag == 0;
  __syncwarp();
  fence_after();
  if (ok) {
    // Every MMA has completed, so the pipeline's shared memory is free: each warp stages
    // its 32 accumulator rows there (row stride BN + 1 floats: conflict-free both ways)
    // and then writes whole row segments, 32 consecutive columns per store.
    float* stage = reinterpret_cast<float*>(smem) + warp * 32 * (BN + 1);
#pragma unroll
    for (int cb = 0; cb < BN; cb += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) stage[lane * (BN + 1) + cb + j] = v[j];
    }
    __syncwarp();
    const int rows = min(32, M - (m0 + warp * 32));
    for (int r = 0; r < rows; ++r) {
      float* crow = C + (size_t)(m0 + warp * 32 + r) * ldc;
#pragma unroll
      for (int c = lane; c < BN; c += 32)
        if (n0 + c < N) crow[n0 + c] = stage[r * (BN + 1) + c];
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
    // let the copies this thread issued land before the CTA's shared memory goes away
    for (int c = issued > STAGES ? issued - STAGES : 0; c < issued; ++c) {
      int spins = 0;
      while (!mbar_try_wait(&full[c % STAGES], (uint32_t)(c / STAGES) & 1u) && ++spins < (1 << 16)) {
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc<TS::kTmemCols>(tmem);
}

// ---------------------------------------------------------------------------
// Persistent form (one CTA per SM walks tiles blockIdx.x, + gridDim.x, ...; N tiles of an
// M tile are consecutive, so CTAs running together share the A rows in L2):
//   warp 0 lane 0  TMA producer, one ring of STAGES chunks across all of its tiles (the
//                  ring never drains between tiles);
//   warp 1 lane 0  MMA issuer into one of two TMEM accumulators (tile i uses i mod 2);
//   warps 2..5     epilogue: wait for an accumulator, read it with tcgen05.ld (warp w
//                  reads TMEM lanes 32 (w mod 4) ..), hand it back to the MMA warp, and
//                  write the tile through a per-warp 32 x 33 float staging block, one
//                  128-byte row piece per store.
// The epilogue of tile i overlaps the loads and MMAs of tile i + 1.
// ---------------------------------------------------------------------------
template <int BN, int STAGES>
struct PersistentShape {
  static constexpr uint32_t kA = BM * BK * 2;
  static constexpr uint32_t kB = BN * BK * 2;
  static constexpr uint32_t kStage = 2 * kA + 2 * kB;
  static constexpr uint32_t kTmemCols = 2 * BN;  // two accumulators (128 or 256: powers of 2)
  static constexpr uint32_t kOut = 4 * 32 * 33 * 4;
  static constexpr size_t kSmem = (size_t)STAGES * kStage + kOut + 1024 + 256;
};

template <int BN, int STAGES>
__global__ void __launch_bounds__(192, 1)
tc_gemm_persistent_kernel(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
                          const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                          float* __restrict__ C, int M, int N, int K, int ldc, int nprod,
                          const int* __restrict__ gate, int* __restrict__ err) {
  using PS = PersistentShape<BN, STAGES>;
  static_assert(BN == 64 || BN == 128, "N tiles of 64 or 128 columns");
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* outst = reinterpret_cast<float*>(smem + STAGES * PS::kStage);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * PS::kStage + PS::kOut);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;
  uint64_t* acce = accf + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (N + BN - 1) / BN;
  const int tiles = ((M + BM - 1) / BM) * n_tiles;
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accf[a], 1);
      mbar_init(&acce[a], 4);  // one arrival per epilogue warp
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
        const int m0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
        for (int c = 0; c < nk; ++c, ++g) {
          const int s = g % STAGES;
          const uint32_t use = (uint32_t)(g / STAGES);
          if (g >= STAGES && !mbar_wait(&empty[s], (use - 1) & 1u, abort_flag)) {
            go = false;
            break;
          }
          uint8_t* a_hi = smem + s * PS::kStage;
          uint8_t* a_lo = a_hi + PS::kA;
          uint8_t* b_hi = a_lo + PS::kA;
          uint8_t* b_lo = b_hi + PS::kB;
          mbar_expect_tx(&full[s], nprod == 3 ? PS::kStage : PS::kA + PS::kB);
          tma_load_2d(&ta_hi, &full[s], a_hi, c * BK, m0);
          tma_load_2d(&tb_hi, &full[s], b_hi, c * BK, n0);
          if (nprod == 3) {
            tma_load_2d(&ta_lo, &full[s], a_lo, c * BK, m0);
            tma_load_2d(&tb_lo, &full[s], b_lo, c * BK, n0);
          }
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
        const uint32_t d = tmem + (uint32_t)(acc * BN);
        for (int c = 0; c < nk; ++c, ++g) {
          const int s = g % STAGES;
          if (!mbar_wait(&full[s], (uint32_t)(g / STAGES) & 1u, abort_flag)) {
            go = false;
            break;
          }
          fence_after();
          const uint8_t* a_hi = smem + s * PS::kStage;
          const uint8_t* a_lo = a_hi + PS::kA;
          const uint8_t* b_hi = a_lo + PS::kA;
          const uint8_t* b_lo = b_hi + PS::kB;
          const uint64_t dah = sdesc_sw128(a_hi), dal = sdesc_sw128(a_lo);
          const uint64_t dbh = sdesc_sw128(b_hi), dbl = sdesc_sw128(b_lo);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t off = 2ull * k;
            mma_bf16(d, dah + off, dbh + off, idesc, (c > 0 || k > 0) ? 1u : 0u);
            if (nprod == 3) {
              mma_bf16(d, dah + off, dbl + off, idesc, 1u);
              mma_bf16(d, dal + off, dbh + off, idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        if (go) mma_commit(&accf[acc]);
      }
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    float* stg = outst + (warp - 2) * 32 * 33;
    int i = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
      const int acc = i & 1;
      if (!mbar_wait(&accf[acc], (uint32_t)(i >> 1) & 1u, abort_flag)) break;
      __syncwarp();
      fence_after();
      const int m0 = (t / n_tiles) * BM, n0 = (t % n_tiles) * BN;
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN);
#pragma unroll 1
      for (int cb = 0; cb < BN; cb += 32) {
        float v[32];
        tmem_ld16(taddr + (uint32_t)cb, *reinterpret_cast<float(*)[16]>(v));
        tmem_ld16(taddr + (uint32_t)(cb + 16), *reinterpret_cast<float(*)[16]>(v + 16));
        if (cb + 32 >= BN) {
          // the whole accumulator is in registers: hand it back to the MMA warp
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce[acc]);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
        __syncwarp();
        const int col = n0 + cb + lane;
        for (int r = 0; r < 32; ++r) {
          const int row = m0 + q * 32 + r;
          if (row < M && col < N) C[(size_t)row * ldc + col] = stg[r * 33 + lane];
        }
        __syncwarp();
      }
    }
  }

  __syncwarp();
  if (threadIdx.x == 0 && *abort_flag) {
    atomicExch(err, 1);
    // let the copies this thread issued land before the CTA's shared memory goes away
    for (int g = issued > STAGES ? issued - STAGES : 0; g < issued; ++g) {
      int spins = 0;
      while (!mbar_try_wait(&full[g % STAGES], (uint32_t)(g / STAGES) & 1u) && ++spins < (1 << 16)) {
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc<PS::kTmemCols>(tmem);
}

// x (float, rows x cols, row stride ld_src) -> hi, lo (bf16, rows x ldk, zero padded)
__global__ void split_bf16_kernel(const float* __restrict__ x, int rows, int cols, int ld_src,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldk,
                                  const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int64_t total = (int64_t)rows * ldk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldk;
    const int c = (int)(e - r * ldk);
    const float v = c < cols ? x[r * ld_src + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}


}  // namespace

// A K-major BF16 matrix [rows][ldk] (ldk a multiple of 8 elements = 16 bytes), K valid
// columns; box = 64 K elements x box_rows rows, 128-byte swizzle, zero fill out of bounds.
cudaError_t make_bf16_tmap(CUtensorMap* map, const void* base, int rows, int k, int ldk, int box_rows) {
  EncodeFn fn = encode_fn();
  if (fn == nullptr) return cudaErrorNotSupported;
  if ((ldk % 8) != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0) return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

int tc_gemm_tile_n(int n) { return n <= 64 ? 64 : 128; }

cudaError_t make_split_operand(TcOperand* op, const void* hi, const void* lo, int rows, int k, int ldk,
                               bool is_a) {
  op->rows = rows;
  op->k = k;
  op->ldk = ldk;
  op->box = is_a ? BM : tc_gemm_tile_n(rows);
  cudaError_t e = make_bf16_tmap(&op->hi, hi, rows, k, ldk, op->box);
  if (e == cudaSuccess) e = make_bf16_tmap(&op->lo, lo, rows, k, ldk, op->box);
  return e;
}

size_t tc_gemm_smem_bytes() { return TileShape<64, 4>::kSmem; }

// Which of the two schedules launch_tc_gemm uses (persistent by default).
static bool g_tc_persistent = true;
void tc_gemm_set_persistent(bool on) { g_tc_persistent = on; }

template <int BN, int STAGES>
static cudaError_t launch_tile(const TcOperand& a, const TcOperand& b, float* C, int M, int N, int K, int ldc,
                               int nprod, const int* gate, int* err, cudaStream_t st) {
  const size_t sm = TileShape<BN, STAGES>::kSmem;
  // the attribute is per device; setting it on every launch is cheap
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  tc_gemm_kernel<BN, STAGES><<<grid, 128, sm, st>>>(a.hi, a.lo, b.hi, b.lo, C, M, N, K, ldc, nprod, gate, err);
  return cudaGetLastError();
}

// The N tile is the B operand's TMA box (chosen from its row count when it was made).
// Rings: 64-wide tiles with short K loops (<= 8 chunks of 64) use 2 stages so that two
// CTAs share an SM and one CTA's epilogue overlaps the other's loads, longer ones 4;
// 128-wide tiles use 3 stages (about 190 KB of shared memory, one CTA per SM).
template <int BN, int STAGES>
static cudaError_t launch_persistent(const TcOperand& a, const TcOperand& b, float* C, int M, int N, int K,
                                     int ldc, int nprod, const int* gate, int* err, cudaStream_t st) {
  const size_t sm = PersistentShape<BN, STAGES>::kSmem;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_persistent_kernel<BN, STAGES>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  const int grid = std::max(1, std::min(tiles, sms));
  tc_gemm_persistent_kernel<BN, STAGES><<<grid, 192, sm, st>>>(a.hi, a.lo, b.hi, b.lo, C, M, N, K, ldc, nprod,
                                                               gate, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcOperand& a, const TcOperand& b, float* C, int M, int N, int K, int ldc,
                           int nprod, const int* gate, int* err, cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  if (a.box != BM) return cudaErrorInvalidValue;
  if (g_tc_persistent) {
    if (b.box == 128) return launch_persistent<128, 3>(a, b, C, M, N, K, ldc, nprod, gate, err, st);
    if (b.box == 64) return launch_persistent<64, 4>(a, b, C, M, N, K, ldc, nprod, gate, err, st);
    return cudaErrorInvalidValue;
  }
  switch (b.box) {
    case 64:
      if ((K + BK - 1) / BK <= 8) return launch_tile<64, 2>(a, b, C, M, N, K, ldc, nprod, gate, err, st);
      return launch_tile<64, 4>(a, b, C, M, N, K, ldc, nprod, gate, err, st);
    case 128: return launch_tile<128, 3>(a, b, C, M, N, K, ldc, nprod, gate, err, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_split_bf16(const float* x, int rows, int cols, int ld_src, void* hi, void* lo, int ldk,
                              const int* gate, cudaStream_t st) {
  const int64_t total = (int64_t)rows * ldk;
  if (total == 0) return cudaSuccess;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  split_bf16_kernel<<<blocks, 256, 0, st>>>(x, rows, cols, ld_src, reinterpret_cast<__nv_bfloat16*>(hi),
                                            reinterpret_cast<__nv_bfloat16*>(lo), ldk, gate);
  return cudaGetLastError();
}

// host-side round-to-nearest-even float -> bf16 bits, and back
uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

float host_bf16_to_float(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

}  // namespace mrstat
