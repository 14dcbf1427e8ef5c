// K2 (phase-encode contraction of J.v and s) and K4 (phase-encode adjoint fused with
// the per-voxel tangent inner products of Re(J^H w)).
//
// The encoding phase of voxel (iy, ix) in TR n at readout kx separates as
// exp(-2 pi i kx ix/nx) * exp(-2 pi i ky(n) iy/ny) (Theory, Eqs. 1-2), so the signal
// sum over voxels is a contraction over iy per TR (here) followed by a dense
// x-DFT over ix (dft.cu):
//     A[n][ix] = sum_iy Ey[n][iy] Q[n][iy][ix],   Ey[n][iy] = exp(-2 pi i ky(n) iy / ny),
// where Q[n][j] = i * (c0_j y0[n][j] + c1_j y1[n][j] + c2_j y2[n][j]) combines the
// cached real time courses y_c (m = i m_y) with per-voxel complex coefficients
// (forward: c0 = rho; J.v: c0 = v_re + i v_im, c1 = rho v_lnT1, c2 = rho v_lnT2).
// The phase factor is looked up exactly: Ey = roots[(kyi(n) * iy) mod ny] with
// roots[k] = exp(-2 pi i k / ny), so no trigonometric function runs per element.
//
// The adjoint of the same chain (Algorithm 4): with Wt[n][ix] = sum_kx conj(F[kx][ix])
// w[n][kx] (dft.cu), voxel j gets Z_c = sum_n y_c[n][j] conj(Ey[n][iy]) Wt[n][ix] and
// g = (Im(conj(rho) Z_1), Im(conj(rho) Z_2), Im(Z_0), -Re(Z_0)) * mask, i.e. the real
// parts of the inner products of d(rho m)/d alpha_k with the back-projected residual.
#include "internal.cuh"

namespace mrstat {
namespace {

// ---------------------------------------------------------------------------
// per-voxel coefficient preparation
// ---------------------------------------------------------------------------
__global__ void prep_forward_kernel(const float* __restrict__ alpha, const uint8_t* __restrict__ mask,
                                    int nv, float2* __restrict__ cf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const float m = (mask == nullptr || mask[j]) ? 1.f : 0.f;
  cf[j] = make_float2(alpha[2 * nv + j] * m, alpha[3 * nv + j] * m);
}

__global__ void prep_linearize_kernel(const float* __restrict__ alpha, const uint8_t* __restrict__ mask,
                                      int nv, float2* __restrict__ rho, float* __restrict__ maskf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const float m = (mask == nullptr || mask[j]) ? 1.f : 0.f;
  rho[j] = make_float2(alpha[2 * nv + j] * m, alpha[3 * nv + j] * m);
  maskf[j] = m;
}

__global__ void prep_rho_kernel(const float2* __restrict__ rho, int nv, float2* __restrict__ cf) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nv) cf[j] = rho[j];
}

__global__ void prep_jvp_kernel(const float* __restrict__ v, const float2* __restrict__ rho,
                                const float* __restrict__ maskf, int nv, int nch, float2* __restrict__ cf,
                                const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const float2 r = rho[j];  // already zero outside the mask
  const float m = maskf[j];
  const float v0 = v[j], v1 = v[nv + j];
  cf[j] = make_float2(v[2 * nv + j] * m, v[3 * nv + j] * m);
  cf[nv + j] = make_float2(r.x * v0, r.y * v0);
  cf[2 * nv + j] = make_float2(r.x * v1, r.y * v1);
  if (nch > 3) {
    const float v4 = v[4 * (size_t)nv + j];
    cf[3 * (size_t)nv + j] = make_float2(r.x * v4, r.y * v4);
  }
}

__device__ __forceinline__ int mod_small(int a, int n, float inv_n) {
  // a in [0, 2^24), n <= 4096: float quotient estimate, then exact correction
  int q = __float2int_rz(__int2float_rn(a) * inv_n);
  int r = a - q * n;
  r += (r < 0) ? n : 0;
  r -= (r >= n) ? n : 0;
  return r;
}

__device__ __forceinline__ float f4get(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------
// K2: A[n][ix] = sum_iy Ey[n][iy] * i * sum_c cf_c[j] y_c[n][j]
// block (32, 8): lanes over 32 columns, warps over row groups iy = ty, ty + 8, ...
// grid (ceil(nx / 32), ceil(nq / QB)); each block covers QB TR quads.
// ---------------------------------------------------------------------------
template <int NCH, int QB>
__global__ void __launch_bounds__(256)
ycontract_kernel(const float4* __restrict__ D, const float2* __restrict__ cf,
                 const int* __restrict__ kyi, const float2* __restrict__ roots, int nx, int ny,
                 int nv, int nq, int ntr, float inv_ny, float2* __restrict__ A,
                 const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ float2 smem[];
  constexpr int T = 4 * QB;  // TRs per block
  float2* ey = smem;         // [T][ny]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int q0 = blockIdx.y * QB;
  const int ix = blockIdx.x * 32 + tx;

  for (int e = tid; e < T * ny; e += 256) {
    const int t = e / ny, iy = e - t * ny;
    const int n = 4 * q0 + t;
    float2 val = make_float2(0.f, 0.f);
    if (n < 4 * nq) val = roots[mod_small(__ldg(kyi + n) * iy, ny, inv_ny)];
    ey[e] = val;
  }
  __syncthreads();

  float ar[T], ai[T];
#pragma unroll
  for (int t = 0; t < T; ++t) ar[t] = ai[t] = 0.f;

  if (ix < nx) {
    const size_t cstride = (size_t)nq * nv;
#pragma unroll 2
    for (int iy = ty; iy < ny; iy += 8) {
      const int j = iy * nx + ix;
      const float2 c0 = __ldg(cf + j);
      float2 c1 = make_float2(0.f, 0.f), c2 = c1, c3 = c1;
      if (NCH > 1) {
        c1 = __ldg(cf + nv + j);
        c2 = __ldg(cf + 2 * nv + j);
      }
      if (NCH > 3) c3 = __ldg(cf + 3 * (size_t)nv + j);
#pragma unroll
      for (int qb = 0; qb < QB; ++qb) {
        const int q = q0 + qb;
        if (q >= nq) break;
        const float4 y0 = __ldg(D + (size_t)q * nv + j);
        float4 y1 = make_float4(0.f, 0.f, 0.f, 0.f), y2 = y1, y3 = y1;
        if (NCH > 1) {
          y1 = __ldg(D + cstride + (size_t)q * nv + j);
          y2 = __ldg(D + 2 * cstride + (size_t)q * nv + j);
        }
        if (NCH > 3) y3 = __ldg(D + 3 * cstride + (size_t)q * nv + j);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float a0 = f4get(y0, k);
          float pr = c0.x * a0, pi = c0.y * a0;
          if (NCH > 1) {
            const float a1 = f4get(y1, k), a2 = f4get(y2, k);
            pr = fmaf(c1.x, a1, fmaf(c2.x, a2, pr));
            pi = fmaf(c1.y, a1, fmaf(c2.y, a2, pi));
          }
          if (NCH > 3) {
            const float a3 = f4get(y3, k);
            pr = fmaf(c3.x, a3, pr);
            pi = fmaf(c3.y, a3, pi);
          }
          // Q = i P = (-pi, pr); acc += E * Q
          const float2 e = ey[(qb * 4 + k) * ny + iy];
          ar[qb * 4 + k] = fmaf(-e.x, pi, fmaf(-e.y, pr, ar[qb * 4 + k]));
          ai[qb * 4 + k] = fmaf(e.x, pr, fmaf(-e.y, pi, ai[qb * 4 + k]));
        }
      }
    }
  }
  __syncthreads();  // ey no longer needed: reuse shared memory for the reduction over ty
  float2* red = smem;  // [8][T][32]
#pragma unroll
  for (int t = 0; t < T; ++t) red[(ty * T + t) * 32 + tx] = make_float2(ar[t], ai[t]);
  __syncthreads();
  for (int e = tid; e < T * 32; e += 256) {
    const int t = e / 32, x = e - t * 32;
    const int n = 4 * q0 + t;
    const int col = blockIdx.x * 32 + x;
    if (n < ntr && col < nx) {
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const float2 v = red[(w * T + t) * 32 + x];
        sr += v.x;
        si += v.y;
      }
      A[(size_t)n * nx + col] = make_float2(sr, si);
    }
  }
}

// ---------------------------------------------------------------------------
// K4: g = Re(J^H w) from Wt.  block (32, 8): lanes over 32 consecutive voxels, warps
// over 8 segments of the TR quads; partial sums reduced through shared memory.
// ---------------------------------------------------------------------------
template <int NCH>
__global__ void __launch_bounds__(256)
jhw_dot_kernel(const float4* __restrict__ D, const float2* __restrict__ wt,
               const int* __restrict__ kyi, const float2* __restrict__ roots_g,
               const float2* __restrict__ rho, const float* __restrict__ maskf, int nx, int ny,
               int nv, int nq, float inv_ny, float scale, float* __restrict__ g, const int* __restrict__ gate) {
  constexpr int NZ = 2 * NCH;  // real and imaginary part per channel
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ float2 smem[];
  float2* roots = smem;                                  // [ny]
  float* red = reinterpret_cast<float*>(smem + ny);      // [8][NZ][32]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  for (int e = tid; e < ny; e += 256) roots[e] = roots_g[e];
  __syncthreads();

  const int j = blockIdx.x * 32 + tx;
  float z[NZ];
#pragma unroll
  for (int c = 0; c < NZ; ++c) z[c] = 0.f;
  if (j < nv) {
    const int iy = j / nx, ix = j - iy * nx;
    const int qa = (int)(((long long)nq * ty) / 8), qe = (int)(((long long)nq * (ty + 1)) / 8);
    const size_t cstride = (size_t)nq * nv;
    for (int q = qa; q < qe; ++q) {
      float4 y[NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) y[c] = __ldg(D + c * cstride + (size_t)q * nv + j);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int n = 4 * q + k;
        const float2 e = roots[mod_small(__ldg(kyi + n) * iy, ny, inv_ny)];
        const float2 w = __ldg(wt + (size_t)n * nx + ix);
        // u = conj(Ey) * Wt
        const float ur = fmaf(e.x, w.x, e.y * w.y);
        const float ui = fmaf(e.x, w.y, -e.y * w.x);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const float a = f4get(y[c], k);
          z[2 * c] = fmaf(a, ur, z[2 * c]);
          z[2 * c + 1] = fmaf(a, ui, z[2 * c + 1]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NZ; ++c) red[(ty * NZ + c) * 32 + tx] = z[c];
  __syncthreads();
  if (ty == 0 && j < nv) {
    float s[NZ];
#pragma unroll
    for (int c = 0; c < NZ; ++c) {
      float a = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) a += red[(w * NZ + c) * 32 + tx];
      s[c] = a * scale;
    }
    const float2 r = rho[j];
    const float m = maskf[j];
    g[j] = (r.x * s[3] - r.y * s[2]) * m;           // Im(conj(rho) Z1)
    g[nv + j] = (r.x * s[5] - r.y * s[4]) * m;      // Im(conj(rho) Z2)
    g[2 * nv + j] = s[1] * m;                       // Im(Z0)
    g[3 * nv + j] = -s[0] * m;                      // -Re(Z0)
    if (NCH > 3) g[4 * (size_t)nv + j] = (r.x * s[7] - r.y * s[6]) * m;  // Im(conj(rho) Z3): B1
  }
}

__global__ void timecourse_kernel(const float4* __restrict__ D, int nv, int nq, int ntr, int channel,
                                  float* __restrict__ out) {
  const size_t total = (size_t)ntr * nv;
  const float* src = reinterpret_cast<const float*>(D + (size_t)channel * nq * nv);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t n = e / nv, j = e - n * nv;
    out[e] = src[((n >> 2) * nv + j) * 4 + (n & 3)];
  }
}

constexpr int kQB = 2;

}  // namespace

cudaError_t launch_prep_forward(const Plan& p, const float* alpha, const uint8_t* mask, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  prep_forward_kernel<<<(p.nv + 255) / 256, 256, 0, st>>>(alpha, mask, p.nv, p.cf);
  return cudaGetLastError();
}

cudaError_t launch_prep_linearize(const Plan& p, const float* alpha, const uint8_t* mask, float2* rho,
                                  cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  prep_linearize_kernel<<<(p.nv + 255) / 256, 256, 0, st>>>(alpha, mask, p.nv, rho, p.maskf);
  return cudaGetLastError();
}

cudaError_t launch_prep_rho(const Plan& p, const float2* rho, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  prep_rho_kernel<<<(p.nv + 255) / 256, 256, 0, st>>>(rho, p.nv, p.cf);
  return cudaGetLastError();
}

cudaError_t launch_prep_jvp(const Plan& p, const float* v, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  prep_jvp_kernel<<<(p.nv + 255) / 256, 256, 0, st>>>(v, p.rho, p.maskf, p.nv, p.nch, p.cf, p.gate);
  return cudaGetLastError();
}

cudaError_t launch_ycontract(const Plan& p, const float4* D, int nch, cudaStream_t st) {
  dim3 block(32, 8);
  dim3 grid((p.nx + 31) / 32, (p.nq + kQB - 1) / kQB);
  const int T = 4 * kQB;
  size_t sm = sizeof(float2) * (size_t)((T * p.ny > 8 * T * 32) ? T * p.ny : 8 * T * 32);
  const float inv_ny = 1.0f / (float)p.ny;
  if (nch == 1) {
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(ycontract_kernel<1, kQB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ycontract_kernel<1, kQB><<<grid, block, sm, st>>>(D, p.cf, p.kyi, p.roots, p.nx, p.ny, p.nv,
                                                      p.nq, p.ntr, inv_ny, p.A, p.gate);
  } else if (nch == 4) {
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(ycontract_kernel<4, kQB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ycontract_kernel<4, kQB><<<grid, block, sm, st>>>(D, p.cf, p.kyi, p.roots, p.nx, p.ny, p.nv, p.nq, p.ntr,
                                                      inv_ny, p.A, p.gate);
  } else {
    if (sm > 48 * 1024)
      cudaFuncSetAttribute(ycontract_kernel<kChannels, kQB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
    ycontract_kernel<kChannels, kQB><<<grid, block, sm, st>>>(D, p.cf, p.kyi, p.roots, p.nx, p.ny,
                                                              p.nv, p.nq, p.ntr, inv_ny, p.A, p.gate);
  }
  return cudaGetLastError();
}

template <int NCH>
static cudaError_t launch_jhw_dot_t(const Plan& p, float* g, cudaStream_t st, const float2* wt, float scale) {
  dim3 block(32, 8);
  dim3 grid((p.nv + 31) / 32);
  size_t sm = sizeof(float2) * p.ny + sizeof(float) * 8 * 2 * NCH * 32;
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(jhw_dot_kernel<NCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  jhw_dot_kernel<NCH><<<grid, block, sm, st>>>(p.D, wt != nullptr ? wt : p.wt, p.kyi, p.roots, p.rho, p.maskf,
                                               p.nx, p.ny, p.nv, p.nq, 1.0f / (float)p.ny, scale, g, p.gate);
  return cudaGetLastError();
}

cudaError_t launch_jhw_dot(const Plan& p, float* g, cudaStream_t st, const float2* wt, float scale) {
  if (p.nv == 0) return cudaSuccess;
  return p.nch == 4 ? launch_jhw_dot_t<4>(p, g, st, wt, scale) : launch_jhw_dot_t<kChannels>(p, g, st, wt, scale);
}

cudaError_t launch_timecourse(const Plan& p, int channel, float* out, cudaStream_t st) {
  const size_t total = (size_t)p.ntr * p.nv;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  timecourse_kernel<<<blocks, 256, 0, st>>>(p.D, p.nv, p.nq, p.ntr, channel, out);
  return cudaGetLastError();
}

}  // namespace mrstat
