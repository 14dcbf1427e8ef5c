// Learned surrogate (see mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "tc_gemm.cuh"

namespace mrstat {

struct Mlp {
  int H = 0, R = 0;
  int in[4] = {0, 0, 0, 0}, out[4] = {0, 0, 0, 0};
  int64_t off[4] = {0, 0, 0, 0};
  int64_t np = 0;
  float norm[6] = {0, 1, 0, 1, 1, 1};
  float lam = 1.f;
  int step = 0;
  int device = 0;
  float *theta = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr, *scale_dev = nullptr;
  std::vector<float> scale_host;
  __nv_bfloat16* Wb[4] = {nullptr, nullptr, nullptr, nullptr};   // bf16 [out][pad8(in)]
  __nv_bfloat16* WTb[4] = {nullptr, nullptr, nullptr, nullptr};  // bf16 [in][pad8(out)]
  TcOperand opW[4], opWT[4];
  CUtensorMap wmap64[4];  // the weights with 64-row boxes (the persistent inference layers)
  // batch buffers (M = 3 B rows: values, ln T1 tangents, ln T2 tangents)
  int cap = 0, maps_b = -1;
  bool maps_train = false, have_train_buffers = false;
  __nv_bfloat16* X[4] = {nullptr, nullptr, nullptr, nullptr};    // bf16 [M][pad8(in)] layer inputs
  __nv_bfloat16* XT[4] = {nullptr, nullptr, nullptr, nullptr};   // bf16 [in][pad8(3 cap)]
  float* Z[4] = {nullptr, nullptr, nullptr, nullptr};   // [M][out] pre-activations (no bias; training)
  __nv_bfloat16* GZ[4] = {nullptr, nullptr, nullptr, nullptr};   // bf16 [M][pad8(out)]
  __nv_bfloat16* GZT[4] = {nullptr, nullptr, nullptr, nullptr};  // bf16 [out][pad8(3 cap)]
  float* GX = nullptr;                                  // [M][H]
  double* loss_dev = nullptr;
  TcOperand opX[4], opXT[4], opGZ[4], opGZT[4];
  int* dev_err = nullptr;

  ~Mlp();
  int setup(int h, int r, uint64_t seed);
  int set_params(const float* host, cudaStream_t st);
  int ensure_batch(int B, bool train);
  int forward(const float* lnT, const float* b1, int B, bool train, cudaStream_t st);
  int backward(const float* target, int B, cudaStream_t st);
  int adam(float lr, cudaStream_t st);
  int infer_fused(const float* lnT, const float* b1, int B, float* pred, cudaStream_t st);
  void release_batch();
  void free_weights();
};

// Coefficients [3][R][n] of n samples (lnT [2][n], b1 [n] or NULL) on stream st.
int mlp_infer(Mlp* m, const float* lnT, const float* b1, int n, float* coef, cudaStream_t st);

}  // namespace mrstat
