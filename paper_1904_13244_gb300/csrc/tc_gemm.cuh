// Tensor-core GEMM (tcgen05, TMA) helpers: see tc_gemm.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace mrstat {

// A split-BF16 operand: K-major hi and lo matrices [rows][ldk] with TMA descriptors.
struct TcOperand {
  CUtensorMap hi;
  CUtensorMap lo;
  int rows = 0, k = 0, ldk = 0;
  int box = 0;  // rows per TMA box: 128 for an A operand, the GEMM's N tile for a B operand
};

// N tile for a GEMM with N columns (a B operand with N rows): 64 up to 64 columns, else 128.
int tc_gemm_tile_n(int n);

cudaError_t make_bf16_tmap(CUtensorMap* map, const void* base, int rows, int k, int ldk, int box_rows);
cudaError_t make_split_operand(TcOperand* op, const void* hi, const void* lo, int rows, int k, int ldk,
                               bool is_a);
// C[M][N] (row stride ldc floats) = sum over nprod in {1, 3} split products of A [M][K] B [N][K]^T
cudaError_t launch_tc_gemm(const TcOperand& a, const TcOperand& b, float* C, int M, int N, int K, int ldc,
                           int nprod, const int* gate, int* err, cudaStream_t st);
// float matrix -> zero-padded bf16 hi/lo pair
cudaError_t launch_split_bf16(const float* x, int rows, int cols, int ld_src, void* hi, void* lo, int ldk,
                              const int* gate, cudaStream_t st);
size_t tc_gemm_smem_bytes();
// Persistent schedule (default) or one CTA per output tile.
void tc_gemm_set_persistent(bool on);
uint16_t host_bf16(float f);
float host_bf16_to_float(uint16_t b);

}  // namespace mrstat
