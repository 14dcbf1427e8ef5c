// C entry points of the low-rank form and the time-basis computation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace mrstat {
namespace {

// Cyclic Jacobi eigen-decomposition of a small symmetric matrix (row-major n x n, in
// place): on return a holds the eigenvalues on its diagonal and v the eigenvectors in
// its columns.
void jacobi_eigen(std::vector<double>& a, std::vector<double>& v, int n) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    if (off <= 1e-30 * (diag + 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double theta = 0.5 * (aqq - app) / apq;
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// Modified Gram-Schmidt on the b columns of the row-major m x b matrix q (twice).
void orthonormalize(std::vector<double>& q, int m, int b) {
  for (int pass = 0; pass < 2; ++pass)
    for (int j = 0; j < b; ++j) {
      for (int k = 0; k < j; ++k) {
        double d = 0.0;
        for (int i = 0; i < m; ++i) d += q[(size_t)i * b + j] * q[(size_t)i * b + k];
        for (int i = 0; i < m; ++i) q[(size_t)i * b + j] -= d * q[(size_t)i * b + k];
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += q[(size_t)i * b + j] * q[(size_t)i * b + j];
      nrm = std::sqrt(nrm);
      const double inv = nrm > 0 ? 1.0 / nrm : 0.0;
      for (int i = 0; i < m; ++i) q[(size_t)i * b + j] *= inv;
    }
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace
}  // namespace mrstat

using namespace mrstat;

extern "C" {

int mrstat_lowrank_set_basis(mrstat_plan* plan_, const float* U, int32_t rank, void* stream) {
  MRSTAT_ABI_RANGE();
  Plan* p = reinterpret_cast<Plan*>(plan_);
  if (p == nullptr || U == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan or basis");
  if (p->npar != 4) return fail(MRSTAT_ERR_UNSUPPORTED, "the low-rank form does not estimate B1");
  if (p->slice_iso > 0) return fail(MRSTAT_ERR_UNSUPPORTED, "the low-rank forms use the hard-pulse model");
  DeviceGuard g(p->device);
  return lowrank_setup(p, U, rank, as_stream(stream));
}

int mrstat_lowrank_linearize(mrstat_plan* plan_, const float* alpha, const float* b1, const uint8_t* mask,
                             const float* coef, void* stream) {
  MRSTAT_ABI_RANGE();
  Plan* p = reinterpret_cast<Plan*>(plan_);
  if (p == nullptr || alpha == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan or alpha");
  if (p->slice_iso > 0) return fail(MRSTAT_ERR_UNSUPPORTED, "the low-rank forms use the hard-pulse model");
  if (p->lr == nullptr) return fail(MRSTAT_ERR_NOT_LINEARIZED, "no time basis: call mrstat_lowrank_set_basis");
  DeviceGuard g(p->device);
  cudaStream_t st = as_stream(stream);
  LowRank& L = *p->lr;
  p->linearized = false;
  L.active = false;
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = launch_prep_linearize(*p, alpha, mask, p->rho, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prep_linearize launch");
  if (coef == nullptr) {
    Span sp(p, MRSTAT_K_BLOCH, st);
    e = lowrank_project(*p, L, alpha, b1, mask, L.coef, st);
  } else {
    e = cudaMemcpyAsync(L.coef, coef, (size_t)3 * L.R * p->nv * sizeof(float), cudaMemcpyDeviceToDevice, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "low-rank coefficients");
  L.coefT_dirty = true;
  L.active = true;
  p->linearized = true;
  return MRSTAT_OK;
}

int mrstat_lowrank_coefficients(mrstat_plan* plan_, float* coef, void* stream) {
  MRSTAT_ABI_RANGE();
  Plan* p = reinterpret_cast<Plan*>(plan_);
  if (p == nullptr || coef == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan or coef");
  if (p->lr == nullptr || !p->lr->active)
    return fail(MRSTAT_ERR_NOT_LINEARIZED, "no low-rank linearisation");
  DeviceGuard g(p->device);
  cudaError_t e = cudaMemcpyAsync(coef, p->lr->coef, (size_t)3 * p->lr->R * p->nv * sizeof(float),
                                  cudaMemcpyDeviceToDevice, as_stream(stream));
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "coefficient copy");
}

int mrstat_lowrank_project_samples(mrstat_plan* plan_, const float* params, const float* b1, int32_t ns,
                                   float* coef, void* stream) {
  MRSTAT_ABI_RANGE();
  Plan* p = reinterpret_cast<Plan*>(plan_);
  if (p == nullptr || params == nullptr || coef == nullptr || ns < 1)
    return fail(MRSTAT_ERR_INVALID_ARG, "bad argument to mrstat_lowrank_project_samples");
  if (p->slice_iso > 0) return fail(MRSTAT_ERR_UNSUPPORTED, "the low-rank forms use the hard-pulse model");
  if (p->lr == nullptr) return fail(MRSTAT_ERR_NOT_LINEARIZED, "no time basis: call mrstat_lowrank_set_basis");
  DeviceGuard g(p->device);
  Plan q;  // the plan's sequence tables with ns voxels
  q.nv = ns;
  q.ntr = p->ntr;
  q.cs = p->cs;
  q.phi = p->phi;
  q.te_ms = p->te_ms;
  q.tr_ms = p->tr_ms;
  q.inversion = p->inversion;
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_BLOCH, as_stream(stream));
    e = lowrank_project(q, *p->lr, params, b1, nullptr, coef, as_stream(stream));
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "sample projection");
}

int mrstat_lowrank_rank(const mrstat_plan* plan_) {
  const Plan* p = reinterpret_cast<const Plan*>(plan_);
  return (p && p->lr) ? p->lr->R : 0;
}

int mrstat_lowrank_basis(mrstat_plan* plan_, const float* train, const float* train_b1, int32_t ns,
                         int32_t rank, float* U_out, double* sv_out, void* stream) {
  MRSTAT_ABI_RANGE();
  Plan* p = reinterpret_cast<Plan*>(plan_);
  if (p == nullptr || train == nullptr || U_out == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, training set or output");
  if (ns < 1 || rank < 1 || rank > kMaxRank || rank > p->ntr)
    return fail(MRSTAT_ERR_INVALID_ARG, "bad training size %d or rank %d", ns, rank);
  if (p->slice_iso > 0) return fail(MRSTAT_ERR_UNSUPPORTED, "the low-rank forms use the hard-pulse model");

  DeviceGuard g(p->device);
  cudaStream_t st = as_stream(stream);
  const int ntr = p->ntr, nq = p->nq;
  const int K = 3 * ns;
  const int b = std::min(ntr, rank + 8);
  float4* D = nullptr;
  float2 *Y = nullptr, *Yt = nullptr, *Qc = nullptr, *Zc = nullptr, *Wc = nullptr;
  cudaError_t e = cudaMalloc(&D, (size_t)3 * nq * ns * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&Y, (size_t)ntr * K * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&Yt, (size_t)ntr * K * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&Qc, (size_t)ntr * b * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&Zc, (size_t)K * b * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&Wc, (size_t)ntr * b * sizeof(float2));
  // 1. training time courses and their tangents
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_BLOCH, st);
    e = launch_bloch_n(*p, train, train_b1, D, ns, st);
  }
  // 2. Y = [m_y | dm_y/dlnT1 | dm_y/dlnT2] as rows n (and its transpose), float32 in
  //    complex storage so that the complex GEMM kernel applies
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = lowrank_train_matrix(D, ns, nq, ntr, Y, Yt, st);
  }
  // 3. subspace iteration Q <- orth(Y (Y^T Q)): float32 products on the device (no Gram
  //    matrix, which would square the singular-value ratios), float64 Gram-Schmidt here
  std::vector<double> Q((size_t)ntr * b);
  {
    uint64_t x = 0x9E3779B97F4A7C15ull;
    for (auto& q : Q) {
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      q = (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
  }
  orthonormalize(Q, ntr, b);
  std::vector<float2> Qh((size_t)ntr * b), Wh((size_t)ntr * b), Zh((size_t)K * b);
  auto step = [&](bool want_z) -> cudaError_t {
    for (size_t i = 0; i < Q.size(); ++i) Qh[i] = make_float2((float)Q[i], 0.f);
    cudaError_t r = cudaMemcpyAsync(Qc, Qh.data(), Qh.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
    if (r == cudaSuccess) r = launch_cgemm(Yt, Qc, Zc, K, b, ntr, nullptr, st);   // Z = Y^T Q
    if (want_z) {
      if (r == cudaSuccess) r = cudaMemcpyAsync(Zh.data(), Zc, Zh.size() * sizeof(float2), cudaMemcpyDeviceToHost, st);
    } else {
      if (r == cudaSuccess) r = launch_cgemm(Y, Zc, Wc, ntr, b, K, nullptr, st);  // W = Y Z
      if (r == cudaSuccess) r = cudaMemcpyAsync(Wh.data(), Wc, Wh.size() * sizeof(float2), cudaMemcpyDeviceToHost, st);
    }
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    return r;
  };
  for (int it = 0; it < 40 && e == cudaSuccess; ++it) {
    e = step(false);
    for (size_t i = 0; i < Q.size(); ++i) Q[i] = Wh[i].x;
    orthonormalize(Q, ntr, b);
  }
  // 4. Rayleigh-Ritz: T = Z^T Z with Z = Y^T Q; U = Q V (leading `rank` eigenvectors)
  std::vector<float> Uf((size_t)ntr * rank);
  std::vector<double> sv(rank);
  if (e == cudaSuccess) e = step(true);
  if (e == cudaSuccess) {
    std::vector<double> T((size_t)b * b, 0.0), V;
    for (int i = 0; i < b; ++i)
      for (int j = i; j < b; ++j) {
        double s2 = 0.0;
        for (int k = 0; k < K; ++k) s2 += (double)Zh[(size_t)k * b + i].x * (double)Zh[(size_t)k * b + j].x;
        T[(size_t)i * b + j] = T[(size_t)j * b + i] = s2;
      }
    jacobi_eigen(T, V, b);
    std::vector<int> order(b);
    for (int i = 0; i < b; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return T[(size_t)x * b + x] > T[(size_t)y * b + y]; });
    std::vector<double> Ud((size_t)ntr * rank, 0.0);
    for (int r = 0; r < rank; ++r) {
      const int c = order[r];
      sv[r] = std::sqrt(std::max(T[(size_t)c * b + c], 0.0));
      for (int n = 0; n < ntr; ++n) {
        double s2 = 0.0;
        for (int k = 0; k < b; ++k) s2 += Q[(size_t)n * b + k] * V[(size_t)k * b + c];
        Ud[(size_t)n * rank + r] = s2;
      }
    }
    orthonormalize(Ud, ntr, rank);
    // sign convention: the largest-magnitude entry of every basis vector is positive
    for (int r = 0; r < rank; ++r) {
      double best = 0.0;
      for (int n = 0; n < ntr; ++n)
        if (std::fabs(Ud[(size_t)n * rank + r]) > std::fabs(best)) best = Ud[(size_t)n * rank + r];
      const double sg = best < 0 ? -1.0 : 1.0;
      for (int n = 0; n < ntr; ++n) Uf[(size_t)n * rank + r] = (float)(sg * Ud[(size_t)n * rank + r]);
    }
    e = cudaMemcpy(U_out, Uf.data(), Uf.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (sv_out) std::memcpy(sv_out, sv.data(), sizeof(double) * rank);
  }
  void* ptrs[] = {D, Y, Yt, Qc, Zc, Wc};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "time basis");
}

}  // extern "C"
