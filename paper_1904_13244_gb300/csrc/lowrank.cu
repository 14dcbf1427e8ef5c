// Low-rank (compressed) form of the signal model and its Jacobian products.
//
// Every echo time course is represented in a real time basis U [ntr][R]:
//     m_j[n] ~ i sum_r U[n][r] c_r,j   (and the same for dm/dlnT1, dm/dlnT2),
// the SVD compression the paper's comparison pipeline applies to its dictionary
// (Methods, "Numerical Brain Simulation"), applied here to the model itself.  Because
// U does not depend on the voxel, the encoding sum of Eqs. 1-2 turns into R images
// and R two-dimensional DFTs:
//     J.v:  s[n][kx] = sum_r U[n][r] H_r[ky(n)][kx],   H_r = DFT2(h_r),
//           h_r,j = i (rho_j (v0 dc1_r,j + v1 dc2_r,j) + (v2 + i v3) c_r,j) * mask_j,
//     J^H w: g_k,j = Re sum_r conj(dh_r,j / dv_k) P_r,j,   P_r = DFT2^H(G_r),
//           G_r[ky][kx] = sum_{n : ky(n) = ky} U[n][r] w[n][kx],
// and for J^H J v the per-ky Gram matrices M_ky = sum_{n : ky(n) = ky} U[n]^T U[n]
// give G_r = sum_r' M_ky[r][r'] H_r' without ever expanding to the TR axis.
// Each DFT2 is two GEMMs (readout x, then phase encode y) on the tcgen05 tensor cores in
// split-BF16 with float32 accumulation (tc_gemm.cu); between them a transpose kernel
// writes the next GEMM's K-major BF16 hi/lo operand directly.
//
// The coefficients c, dc1, dc2 come either from the exact Bloch recursion projected onto
// U on the fly (lr_project_kernel: no time course is ever stored) or from a caller (the
// learned surrogate).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "lowrank.cuh"
#include "reduce.cuh"
#include "steihaug.cuh"

namespace mrstat {
namespace {

__device__ __forceinline__ void put_split(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t idx, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[idx] = h;
  lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// ---------------------------------------------------------------------------
// exact linearisation projected onto U: Bloch recursion with tangents (as bloch.cu),
// accumulating c_r += U[n][r] m_y, dc1_r += U[n][r] dm_y/dlnT1, dc2_r += U[n][r] dm_y/dlnT2
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(128)
lr_project_kernel(const float* __restrict__ alpha, const float* __restrict__ b1,
                  const uint8_t* __restrict__ mask, const float2* __restrict__ cs, const float* __restrict__ phi,
                  const float* __restrict__ U, int nv, int ntr, float te, float tb, float m0z,
                  float* __restrict__ coef) {
  constexpr int CH = 64;  // TRs of U staged per chunk
  __shared__ __align__(16) float us[CH * R];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = j < nv;
  const bool on = valid && (mask == nullptr || mask[j] != 0);
  // a block whose voxels all lie outside the mask has only zeros to write
  if (!__syncthreads_or(on)) {
    if (valid)
      for (int r = 0; r < 3 * R; ++r) coef[(size_t)r * nv + j] = 0.f;
    return;
  }
  float t1 = 1000.f, t2 = 100.f, bj = 1.f;
  if (valid) {
    t1 = expf(alpha[j]);
    t2 = expf(alpha[nv + j]);
    if (b1 != nullptr) bj = b1[j];
  }
  const float ra1 = te / t1, ra2 = te / t2, rb1 = tb / t1, rb2 = tb / t2;
  const float x1a = expm1f(-ra1), x2a = expm1f(-ra2), x1b = expm1f(-rb1), x2b = expm1f(-rb2);
  const float d1a = ra1 * (1.f + x1a), d2a = ra2 * (1.f + x2a), d1b = rb1 * (1.f + x1b), d2b = rb2 * (1.f + x2b);
  float my = 0.f, mz = m0z, ay = 0.f, az = 0.f, by = 0.f, bz = 0.f;
  float c0[R], c1[R], c2[R];
#pragma unroll
  for (int r = 0; r < R; ++r) c0[r] = c1[r] = c2[r] = 0.f;

  for (int n0 = 0; n0 < ntr; n0 += CH) {
    const int cnt = min(CH, ntr - n0);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt * R; e += blockDim.x) us[e] = U[(size_t)n0 * R + e];
    __syncthreads();
    for (int t = 0; t < cnt; ++t) {
      const int n = n0 + t;
      float c, s;
      if (b1 != nullptr) {
        sincosf(__ldg(phi + n) * bj, &s, &c);
      } else {
        const float2 v = __ldg(cs + n);
        c = v.x;
        s = v.y;
      }
      float ty = c * my + s * mz;
      mz = c * mz - s * my;
      my = ty;
      ty = c * ay + s * az;
      az = c * az - s * ay;
      ay = ty;
      ty = c * by + s * bz;
      bz = c * bz - s * by;
      by = ty;
      float zm1 = mz - 1.f;
      ay = fmaf(x2a, ay, ay);
      az = fmaf(x1a, az, fmaf(d1a, zm1, az));
      by = fmaf(x2a, by, fmaf(d2a, my, by));
      bz = fmaf(x1a, bz, bz);
      my = fmaf(x2a, my, my);
      mz = fmaf(x1a, zm1, mz);
      const float4* u4 = reinterpret_cast<const float4*>(us + t * R);
#pragma unroll
      for (int r4 = 0; r4 < R / 4; ++r4) {
        const float4 u = u4[r4];
        c0[4 * r4 + 0] = fmaf(u.x, my, c0[4 * r4 + 0]);
        c0[4 * r4 + 1] = fmaf(u.y, my, c0[4 * r4 + 1]);
        c0[4 * r4 + 2] = fmaf(u.z, my, c0[4 * r4 + 2]);
        c0[4 * r4 + 3] = fmaf(u.w, my, c0[4 * r4 + 3]);
        c1[4 * r4 + 0] = fmaf(u.x, ay, c1[4 * r4 + 0]);
        c1[4 * r4 + 1] = fmaf(u.y, ay, c1[4 * r4 + 1]);
        c1[4 * r4 + 2] = fmaf(u.z, ay, c1[4 * r4 + 2]);
        c1[4 * r4 + 3] = fmaf(u.w, ay, c1[4 * r4 + 3]);
        c2[4 * r4 + 0] = fmaf(u.x, by, c2[4 * r4 + 0]);
        c2[4 * r4 + 1] = fmaf(u.y, by, c2[4 * r4 + 1]);
        c2[4 * r4 + 2] = fmaf(u.z, by, c2[4 * r4 + 2]);
        c2[4 * r4 + 3] = fmaf(u.w, by, c2[4 * r4 + 3]);
      }
      zm1 = mz - 1.f;
      ay = fmaf(x2b, ay, ay);
      az = fmaf(x1b, az, fmaf(d1b, zm1, az));
      by = fmaf(x2b, by, fmaf(d2b, my, by));
      bz = fmaf(x1b, bz, bz);
      my = fmaf(x2b, my, my);
      mz = fmaf(x1b, zm1, mz);
    }
  }
  if (!valid) return;
  const float m = on ? 1.f : 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    coef[(size_t)r * nv + j] = c0[r] * m;
    coef[(size_t)(R + r) * nv + j] = c1[r] * m;
    coef[(size_t)(2 * R + r) * nv + j] = c2[r] * m;
  }
}

// h_r,j for J.v, written as the K-major split-BF16 operand of the readout GEMM:
// row r * ny + iy, columns 2 ix (re) and 2 ix + 1 (im)
__global__ void lr_prep_jvp_kernel(const float* __restrict__ v, const float* __restrict__ coef,
                                   const float2* __restrict__ rho, const float* __restrict__ maskf, int nx,
                                   int ny, int nv, int R, __nv_bfloat16* __restrict__ hi,
                                   __nv_bfloat16* __restrict__ lo, int ldk, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const int iy = j / nx, ix = j - iy * nx;
  const float m = maskf[j];
  const float2 rh = rho[j];
  const float v0 = v[j], v1 = v[nv + j], v2 = v[2 * (size_t)nv + j] * m, v3 = v[3 * (size_t)nv + j] * m;
  for (int r = 0; r < R; ++r) {
    const float c = coef[(size_t)r * nv + j];
    const float t = fmaf(v0, coef[(size_t)(R + r) * nv + j], v1 * coef[(size_t)(2 * R + r) * nv + j]);
    // q = rho t + (v2 + i v3) c ; h = i q
    const float qr = rh.x * t + v2 * c, qi = rh.y * t + v3 * c;
    const size_t row = (size_t)(r * ny + iy) * ldk;
    put_split(hi, lo, row + 2 * ix, -qi);
    put_split(hi, lo, row + 2 * ix + 1, qr);
  }
}

// complex rows (r, a) x B columns of src (row stride 2B floats) -> split-BF16 rows (r, b)
// x A complex columns of dst (row stride ldk); tiles of 32 x 32 through shared memory
__global__ void lr_transpose_split_kernel(const float* __restrict__ src, int A, int B,
                                          __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldk,
                                          const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  __shared__ float2 tile[32][33];
  const int r = blockIdx.z;
  const int b0 = blockIdx.x * 32, a0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const float2* s2 = reinterpret_cast<const float2*>(src) + (size_t)r * A * B;
  for (int k = ty; k < 32; k += 8) {
    const int a = a0 + k, b = b0 + tx;
    tile[k][tx] = (a < A && b < B) ? s2[(size_t)a * B + b] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int b = b0 + k, a = a0 + tx;
    if (a < A && b < B) {
      const float2 v = tile[tx][k];
      const size_t row = ((size_t)r * B + b) * ldk;
      put_split(hi, lo, row + 2 * a, v.x);
      put_split(hi, lo, row + 2 * a + 1, v.y);
    }
  }
}

// s[n][kx] = sum_r U[n][r] H[(r nkx + kx)][ky(n)]   (H rows: ny complex values)
__global__ void lr_expand_kernel(const float* __restrict__ H, const float* __restrict__ U,
                                 const int* __restrict__ kyi, int ntr, int nkx, int ny, int R,
                                 float2* __restrict__ s) {
  const int kx = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = blockIdx.y;
  if (kx >= nkx || n >= ntr) return;
  const int ky = kyi[n];
  const float2* H2 = reinterpret_cast<const float2*>(H);
  float sr = 0.f, si = 0.f;
  for (int r = 0; r < R; ++r) {
    const float u = __ldg(U + (size_t)n * R + r);
    const float2 h = H2[((size_t)r * nkx + kx) * ny + ky];
    sr = fmaf(u, h.x, sr);
    si = fmaf(u, h.y, si);
  }
  s[(size_t)n * nkx + kx] = make_float2(sr, si);
}

// G_r[ky][kx] = sum_r' M_ky[r][r'] H_r'[ky][kx], written as the split operand of the
// phase-encode adjoint GEMM (rows (r, kx), columns 2 ky + re/im).  One block per ky.
__global__ void lr_gram_kernel(const float* __restrict__ H, const float* __restrict__ Mky, int nkx, int ny,
                               int R, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldk,
                               const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ float msh[];  // R x R
  const int ky = blockIdx.x;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) msh[e] = Mky[(size_t)ky * R * R + e];
  __syncthreads();
  const float2* H2 = reinterpret_cast<const float2*>(H);
  for (int kx = threadIdx.x; kx < nkx; kx += blockDim.x) {
    float2 h[kMaxRank];
    for (int r = 0; r < R; ++r) h[r] = H2[((size_t)r * nkx + kx) * ny + ky];
    for (int r = 0; r < R; ++r) {
      float gr = 0.f, gi = 0.f;
      for (int q = 0; q < R; ++q) {
        const float mm = msh[r * R + q];
        gr = fmaf(mm, h[q].x, gr);
        gi = fmaf(mm, h[q].y, gi);
      }
      const size_t row = ((size_t)r * nkx + kx) * ldk;
      put_split(hi, lo, row + 2 * ky, gr);
      put_split(hi, lo, row + 2 * ky + 1, gi);
    }
  }
}

// G_r[ky][kx] = sum_{n: ky(n) = ky} U[n][r] w[n][kx] into the same operand layout
__global__ void lr_gather_kernel(const float2* __restrict__ w, const float* __restrict__ U,
                                 const int* __restrict__ kyptr, const int* __restrict__ kytr, int nkx, int R,
                                 __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldk) {
  const int ky = blockIdx.x;
  const int na = kyptr[ky], ne = kyptr[ky + 1];
  for (int kx = threadIdx.x; kx < nkx; kx += blockDim.x) {
    float2 g[kMaxRank];
    for (int r = 0; r < R; ++r) g[r] = make_float2(0.f, 0.f);
    for (int t = na; t < ne; ++t) {
      const int n = kytr[t];
      const float2 wv = w[(size_t)n * nkx + kx];
      for (int r = 0; r < R; ++r) {
        const float u = __ldg(U + (size_t)n * R + r);
        g[r].x = fmaf(u, wv.x, g[r].x);
        g[r].y = fmaf(u, wv.y, g[r].y);
      }
    }
    for (int r = 0; r < R; ++r) {
      const size_t row = ((size_t)r * nkx + kx) * ldk;
      put_split(hi, lo, row + 2 * ky, g[r].x);
      put_split(hi, lo, row + 2 * ky + 1, g[r].y);
    }
  }
}

// g_k,j = Re sum_r conj(dh_r,j/dv_k) P_r,j with P rows (r ny + iy), columns 2 ix + re/im
__global__ void lr_final_kernel(const float* __restrict__ P, const float* __restrict__ coef,
                                const float2* __restrict__ rho, const float* __restrict__ maskf, int nx, int ny,
                                int nv, int R, float* __restrict__ g, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const int iy = j / nx, ix = j - iy * nx;
  const float2* P2 = reinterpret_cast<const float2*>(P);
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  const float2 rh = rho[j];
  for (int r = 0; r < R; ++r) {
    const float2 p = P2[(size_t)(r * ny + iy) * nx + ix];
    const float c = coef[(size_t)r * nv + j];
    const float t1 = coef[(size_t)(R + r) * nv + j], t2 = coef[(size_t)(2 * R + r) * nv + j];
    const float imcp = rh.x * p.y - rh.y * p.x;  // Im(conj(rho) P)
    a0 = fmaf(t1, imcp, a0);
    a1 = fmaf(t2, imcp, a1);
    a2 = fmaf(c, p.y, a2);
    a3 = fmaf(-c, p.x, a3);
  }
  const float m = maskf[j];
  g[j] = a0 * m;
  g[nv + j] = a1 * m;
  g[2 * (size_t)nv + j] = a2 * m;
  g[3 * (size_t)nv + j] = a3 * m;
}

// ---------------------------------------------------------------------------
// J^H J v with a fully sampled readout (nkx == nx).  The readout DFT and its adjoint
// cancel (F^H F = nx I), so per image column ix only the phase-encode DFT, the per-ky
// Gram and its adjoint remain:  P_r = nx F_y^H (M_ky (F_y h)).  Operands are stored
// with rows (ix, r) = ix R + r and columns 2 iy (or 2 ky) + re/im, so every kernel below
// reads and writes whole rows; the voxel-order inputs and outputs go through 32 x 32
// shared-memory tiles.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void put_split_pair(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t idx, float2 v) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
  const float2 hf = __bfloat1622float2(h);
  *reinterpret_cast<__nv_bfloat162*>(hi + idx) = h;
  *reinterpret_cast<__nv_bfloat162*>(lo + idx) = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
}

// h_r,j = i (rho_j (v0 dc1_r,j + v1 dc2_r,j) + (v2 + i v3) c_r,j) mask_j into rows (ix, r).
// Block: a 32 x 32 voxel tile and 4 basis functions (blockIdx.z).
__global__ void __launch_bounds__(256)
lr_prep_t_kernel(const float* __restrict__ v, const float* __restrict__ coef, const float2* __restrict__ rho,
                 const float* __restrict__ maskf, int nx, int ny, int nv, int R, __nv_bfloat16* __restrict__ hi,
                 __nv_bfloat16* __restrict__ lo, int ldk, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  __shared__ float2 S[4][32][33];  // [r - r0][ix - ix0][iy - iy0]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int ix0 = blockIdx.x * 32, iy0 = blockIdx.y * 32;
  const int ix = ix0 + tx;
  float v0[4], v1[4], v2[4], v3[4];
  float2 rh[4];
  int jj[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int iy = iy0 + ty + 8 * k;
    const bool ok = ix < nx && iy < ny;
    const int j = ok ? iy * nx + ix : -1;
    jj[k] = j;
    const float m = ok ? maskf[j] : 0.f;
    rh[k] = ok ? rho[j] : make_float2(0.f, 0.f);
    v0[k] = ok ? v[j] : 0.f;
    v1[k] = ok ? v[nv + j] : 0.f;
    v2[k] = ok ? v[2 * (size_t)nv + j] * m : 0.f;
    v3[k] = ok ? v[3 * (size_t)nv + j] * m : 0.f;
  }
  {
    const int r0 = blockIdx.z * 4;  // this block's chunk of 4 basis functions
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = r0 + rr;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float2 h = make_float2(0.f, 0.f);
        const int j = jj[k];
        if (j >= 0 && r < R) {
          const float c = coef[(size_t)r * nv + j];
          const float t = fmaf(v0[k], coef[(size_t)(R + r) * nv + j], v1[k] * coef[(size_t)(2 * R + r) * nv + j]);
          const float qr = rh[k].x * t + v2[k] * c, qi = rh[k].y * t + v3[k] * c;
          h = make_float2(-qi, qr);
        }
        S[rr][tx][ty + 8 * k] = h;
      }
    }
    __syncthreads();
    const int iy = iy0 + tx;
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const int rl = ty + 8 * i, a = rl >> 2, rr = rl & 3;
      const int ixa = ix0 + a, r = r0 + rr;
      if (ixa < nx && r < R && iy < ny) put_split_pair(hi, lo, (size_t)(ixa * R + r) * ldk + 2 * iy, S[rr][a][tx]);
    }
  }
}

// G[(ix, r)][ky] = sum_{n : ky(n) = ky} U[n][r] sum_q U[n][q] H[(ix, q)][ky]: the per-ky
// Gram applied through the TR axis (2 |S(ky)| R multiply-adds per value instead of R^2).
// Block (32, 8): 32 consecutive ky (lanes) x 8 image columns; the rows of U of the TRs
// of its 32 ky values (contiguous in Ug, U gathered in ky order) sit in shared memory,
// rows padded to R + 1 floats.
template <int R, bool SPLIT>
__global__ void __launch_bounds__(256)
lr_gram_t_kernel(const float* __restrict__ HT, int ldh, const float* __restrict__ Ug, const int* __restrict__ kyptr,
                 int nx, int ny, __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldk,
                 float2* __restrict__ gout, const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ float us[];  // [rows of this ky tile][R + 1]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int ky0 = blockIdx.x * 32;
  const int t0 = kyptr[ky0], t1 = kyptr[min(ky0 + 32, ny)];
  for (int e = tid; e < (t1 - t0) * R; e += 256) {
    const int t = e / R, r = e - t * R;
    us[t * (R + 1) + r] = Ug[(size_t)t0 * R + e];
  }
  __syncthreads();
  const int ky = ky0 + tx, ix = blockIdx.y * 8 + ty;
  if (ky >= ny || ix >= nx) return;
  const float2* H2 = reinterpret_cast<const float2*>(HT);
  const int ld2 = ldh / 2;
  float2 in[R], out[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    in[q] = H2[(size_t)(ix * R + q) * ld2 + ky];
    out[q] = make_float2(0.f, 0.f);
  }
  const int ta = kyptr[ky], te = kyptr[ky + 1];
  for (int t = ta; t < te; ++t) {
    const float* un = us + (t - t0) * (R + 1);
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      sr = fmaf(un[q], in[q].x, sr);
      si = fmaf(un[q], in[q].y, si);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      out[r].x = fmaf(un[r], sr, out[r].x);
      out[r].y = fmaf(un[r], si, out[r].y);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (SPLIT) put_split_pair(hi, lo, (size_t)(ix * R + r) * ldk + 2 * ky, out[r]);
    else gout[(size_t)(ix * R + r) * ny + ky] = out[r];
  }
}

// The same Gram product when no ky value has more than kGramShort TRs (one TR per fill
// for up to 8 fills, the usual sequence): the TR-axis sums s_t stay in registers and each
// output G[(ix, r)][ky] is written as soon as it is formed, so no R-long output array is
// held (about half the registers of the general kernel, twice the resident warps).
constexpr int kGramShort = 8;

template <int R, bool SPLIT>
__global__ void __launch_bounds__(256)
lr_gram_short_kernel(const float* __restrict__ HT, int ldh, const float* __restrict__ Ug,
                     const int* __restrict__ kyptr, int nx, int ny, __nv_bfloat16* __restrict__ hi,
                     __nv_bfloat16* __restrict__ lo, int ldk, float2* __restrict__ gout,
                     const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  extern __shared__ float us[];  // [rows of this ky tile][R + 1]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int ky0 = blockIdx.x * 32;
  const int t0 = kyptr[ky0], t1 = kyptr[min(ky0 + 32, ny)];
  for (int e = tid; e < (t1 - t0) * R; e += 256) {
    const int t = e / R, r = e - t * R;
    us[t * (R + 1) + r] = Ug[(size_t)t0 * R + e];
  }
  __syncthreads();
  const int ky = ky0 + tx, ix = blockIdx.y * 8 + ty;
  if (ky >= ny || ix >= nx) return;
  const float2* H2 = reinterpret_cast<const float2*>(HT);
  const int ld2 = ldh / 2;
  const int ta = kyptr[ky], ns = kyptr[ky + 1] - ta;  // ns <= kGramShort
  float2 sv[kGramShort];
#pragma unroll
  for (int k = 0; k < kGramShort; ++k) sv[k] = make_float2(0.f, 0.f);
  {
    float2 in[R];
#pragma unroll
    for (int q = 0; q < R; ++q) in[q] = H2[(size_t)(ix * R + q) * ld2 + ky];
#pragma unroll
    for (int k = 0; k < kGramShort; ++k) {
      if (k < ns) {
        const float* un = us + (ta + k - t0) * (R + 1);
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          sr = fmaf(un[q], in[q].x, sr);
          si = fmaf(un[q], in[q].y, si);
        }
        sv[k] = make_float2(sr, si);
      }
    }
  }
#pragma unroll 4
  for (int r = 0; r < R; ++r) {
    float2 o = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kGramShort; ++k) {
      if (k < ns) {
        const float u = us[(ta + k - t0) * (R + 1) + r];
        o.x = fmaf(u, sv[k].x, o.x);
        o.y = fmaf(u, sv[k].y, o.y);
      }
    }
    if (SPLIT) put_split_pair(hi, lo, (size_t)(ix * R + r) * ldk + 2 * ky, o);
    else gout[(size_t)(ix * R + r) * ny + ky] = o;
  }
}

// ---------------------------------------------------------------------------
// Phase-encode DFT by factorisation, for ny = 16 M with M = 2 N1 (N1 <= 8): with
// iy = 16 i1 + i2 and ky = k1 + M k2 (i1, k1 < M; i2, k2 < 16) the exponent ky iy (mod ny)
// splits into M-point, twiddle and 16-point parts,
//     X[k1 + M k2] = sum_i2 W16^(k2 i2) w^(k1 i2) sum_i1 wM^(k1 i1) x[16 i1 + i2],
// with w = exp(-2 pi i / ny), wM = w^16 and W16 = w^M.  The M-point DFT is one radix-2
// step over two N1-point DFTs, each formed by the symmetries of its matrix; the 16-point
// DFT is a radix-2 FFT held in one thread's registers.  The adjoint runs the same steps
// with conjugate roots in the reverse order.  Everything stays in float32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// N1-point DFT of x (sign -; CONJ: sign +) by the two symmetries of its matrix: with
// u_i = x_i + x_(N1 - i), d_i = x_i - x_(N1 - i) for 0 < i < N1 / 2,
//     A_k = x_0 + sum_i cos(2 pi k i / N1) u_i  [+ (-1)^k x_(N1/2) for even N1],
//     B_k = sum_i sin(2 pi k i / N1) d_i,
// X_k = A_k - i B_k and X_(N1 - k) = A_k + i B_k (swapped for CONJ); X_0 is the plain
// sum and, for even N1, X_(N1/2) the alternating one.
template <int N1, bool CONJ>
__device__ __forceinline__ void dft_n1(const DftSmall& W, const float2 (&x)[N1], float2 (&X)[N1]) {
  constexpr int P = (N1 - 1) / 2;
  constexpr bool EVEN = N1 % 2 == 0;
  float2 u[P + 1], d[P + 1];
#pragma unroll
  for (int i = 1; i <= P; ++i) {
    u[i] = cadd(x[i], x[N1 - i]);
    d[i] = csub(x[i], x[N1 - i]);
  }
  float2 s0 = x[0];
#pragma unroll
  for (int i = 1; i <= P; ++i) s0 = cadd(s0, u[i]);
  if (EVEN) s0 = cadd(s0, x[N1 / 2]);
  X[0] = s0;
#pragma unroll
  for (int k = 1; k <= P; ++k) {
    float ax = x[0].x, ay = x[0].y, bx = 0.f, by = 0.f;
    if (EVEN) {
      const float sg = (k & 1) ? -1.f : 1.f;
      ax = fmaf(sg, x[N1 / 2].x, ax);
      ay = fmaf(sg, x[N1 / 2].y, ay);
    }
#pragma unroll
    for (int i = 1; i <= P; ++i) {
      const float c = W.c[k - 1][i - 1], s = W.s[k - 1][i - 1];
      ax = fmaf(c, u[i].x, ax);
      ay = fmaf(c, u[i].y, ay);
      bx = fmaf(s, d[i].x, bx);
      by = fmaf(s, d[i].y, by);
    }
    const float2 minus_ib = make_float2(ax + by, ay - bx), plus_ib = make_float2(ax - by, ay + bx);
    X[k] = CONJ ? plus_ib : minus_ib;
    X[N1 - k] = CONJ ? minus_ib : plus_ib;
  }
  if (EVEN) {
    float2 a = x[0];
#pragma unroll
    for (int i = 1; i <= P; ++i) a = (i & 1) ? csub(a, u[i]) : cadd(a, u[i]);
    a = ((N1 / 2) & 1) ? csub(a, x[N1 / 2]) : cadd(a, x[N1 / 2]);
    X[N1 / 2] = a;
  }
}

// M-point DFT (M = 2 N1) by one radix-2 step in time: the N1-point DFTs E of the even and
// O of the odd samples, Y_k = E_k + wM^k O_k and Y_(k + N1) = E_k - wM^k O_k.
template <int N1, bool CONJ>
__device__ __forceinline__ void dft_m(const DftSmall& W, const float2 (&x)[2 * N1], float2 (&Y)[2 * N1]) {
  float2 xe[N1], xo[N1], E[N1], O[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) {
    xe[i] = x[2 * i];
    xo[i] = x[2 * i + 1];
  }
  dft_n1<N1, CONJ>(W, xe, E);
  dft_n1<N1, CONJ>(W, xo, O);
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    const float2 t = k == 0 ? O[0] : (CONJ ? cmulc(O[k], W.wm[k]) : cmul(O[k], W.wm[k]));
    Y[k] = cadd(E[k], t);
    Y[k + N1] = csub(E[k], t);
  }
}

// z times W16^m = exp(-2 pi i m / 16) (CONJ: exp(+2 pi i m / 16)), 0 <= m < 8; m is a
// compile-time constant once the callers' loops are unrolled, so the branches fold.
template <bool CONJ>
__device__ __forceinline__ float2 tw16(float2 z, int m) {
  constexpr float C1 = 0.923879532511286756f;  // cos(pi / 8)
  constexpr float S1 = 0.382683432365089772f;  // sin(pi / 8)
  constexpr float R2 = 0.707106781186547524f;  // cos(pi / 4)
  if (m == 0) return z;
  if (m == 4) return CONJ ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
  if (m == 2 || m == 6) {
    // (1 -/+ i) / sqrt 2 for m = 2, (-1 -/+ i) / sqrt 2 for m = 6
    const float p = (z.x + z.y) * R2, q = (z.y - z.x) * R2;
    if (m == 2) return CONJ ? make_float2(-q, p) : make_float2(p, q);
    return CONJ ? make_float2(-p, -q) : make_float2(q, -p);
  }
  const float c = m == 1 ? C1 : m == 3 ? S1 : m == 5 ? -S1 : -C1;
  const float s = m == 1 ? S1 : m == 3 ? C1 : m == 5 ? C1 : S1;
  // forward: (x + i y)(c - i s); CONJ: (x + i y)(c + i s)
  return CONJ ? make_float2(fmaf(z.x, c, -z.y * s), fmaf(z.y, c, z.x * s))
              : make_float2(fmaf(z.x, c, z.y * s), fmaf(z.y, c, -z.x * s));
}

__host__ __device__ constexpr int brev4(int k) {
  return ((k & 1) << 3) | ((k & 2) << 1) | ((k & 4) >> 1) | ((k & 8) >> 3);
}

// One radix-2 stage of span H of the 16-point FFT below (H a template argument, so that
// every index and twiddle is a compile-time constant).
template <bool CONJ, int H>
__device__ __forceinline__ void fft16_stage(float2 (&a)[16]) {
#pragma unroll
  for (int g = 0; g < 16; g += 2 * H) {
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const float2 u = a[g + j], v = a[g + j + H];
      a[g + j] = cadd(u, v);
      a[g + j + H] = tw16<CONJ>(csub(u, v), j * (8 / H));
    }
  }
}

// 16-point DFT in registers, radix-2 decimation in frequency: a in natural order on entry,
// X_k in a[brev4(k)] on return.
template <bool CONJ>
__device__ __forceinline__ void fft16(float2 (&a)[16]) {
  fft16_stage<CONJ, 8>(a);
  fft16_stage<CONJ, 4>(a);
  fft16_stage<CONJ, 2>(a);
  fft16_stage<CONJ, 1>(a);
}

// Row stride (complex values) of the per-basis-function rows of the column kernels: the
// M-point stage stores Z[k1][i2] at 17 k1 + i2, so that the lanes of the 16-point stage
// (one per (row, k1)) read and write distinct banks.
__host__ __device__ constexpr int col_row(int ny) { return 17 * (ny / 16); }

// coefT[(k R + r)][ix][iy] = coef[(k R + r)][iy nx + ix]: the coefficients in image-column
// order, so that a block working on one column ix reads them contiguously (32 x 32 tiles)
__global__ void lr_coef_transpose_kernel(const float* __restrict__ coef, int nx, int ny, float* __restrict__ coefT) {
  __shared__ float tile[32][33];
  const int plane = blockIdx.z;
  const int ix0 = blockIdx.x * 32, iy0 = blockIdx.y * 32;
  const size_t nv = (size_t)nx * ny;
  const float* src = coef + plane * nv;
  float* dst = coefT + plane * nv;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int iy = iy0 + k, ix = ix0 + threadIdx.x;
    tile[k][threadIdx.x] = (iy < ny && ix < nx) ? src[(size_t)iy * nx + ix] : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int ix = ix0 + k, iy = iy0 + threadIdx.x;
    if (ix < nx && iy < ny) dst[(size_t)ix * ny + iy] = tile[threadIdx.x][k];
  }
}

// ---------------------------------------------------------------------------
// The whole low-rank J^H J v for one image column ix in one cluster of two blocks
// (ny = 32 N1); block c of the pair owns the basis functions r in [c RC, (c + 1) RC),
// RC = ceil(R / 2), and the R columns h_r(iy) never leave shared memory.
//   0. each block loads the column's voxel data (v and rho);
//   1. warp w owns the rows r = 2w, 2w + 1: lane (r, i2) forms h_r(16 i1 + i2) for i1 < M
//      in registers, applies the M-point DFT and the twiddle, and lane (r, k1) the
//      16-point FFT of the factorised phase-encode DFT -> H_r(ky) (warp barriers only);
//   2. the per-ky Gram through the TR axis, one thread per phase-encode line ky: it forms
//      the block's part of s_t = sum_q U[t][q] H_q(ky) for the TRs t of its line and
//      stores it into the peer; after a cluster barrier it adds the peer's part (the same
//      sum in both blocks) and forms G_r(ky) = sum_t U[t][r] s_t for the block's r (the
//      rows of U in batches of eight basis functions whose loads issue together, each
//      pass's first batch before the barrier that precedes it);
//   3. the same warps apply the adjoint DFT -> P_r(iy);
//   4. one thread per iy contracts with the tangents over the block's r (coefficients in
//      two batches, the first loaded before step 3's barrier), keeping the part for its
//      own half of the column and storing the rest into the peer; after a second cluster
//      barrier each block adds the two parts for its half, writes g (masked, times nx)
//      and its part of <v, g>; the last block adds the parts.
// Two blocks per column (448 for 224 columns, three per SM) balance the SMs better than
// one block of twice the size (224 blocks on 152 SMs).
// ---------------------------------------------------------------------------
constexpr int kColThreads = 256, kColWarps = kColThreads / 32;
constexpr int kColMaxRc = 16;  // basis functions per block: R <= 32

// TR slots per phase-encode line that the per-line Gram step keeps in registers; with more
// slots a line's part of s also goes through shared memory (sbuf).
constexpr int kSlotRegs = 8;

__host__ __device__ inline int sbuf_slots(int kmax) { return kmax > kSlotRegs ? kmax : 0; }

size_t column_smem_bytes(int ny, int R, int kmax) {
  const size_t rc = (size_t)(R + 1) / 2;
  return sizeof(float2) * ((size_t)ny + rc * col_row(ny) + (size_t)(kmax + sbuf_slots(kmax)) * ny) +
         sizeof(float) * 14 * (size_t)ny;
}

// Shared-memory layout of the column kernels and the peer's exchange buffers.
struct ColShared {
  float2* rt;      // [NY] w^k
  float2* hs;      // [RC][col_row(NY)]: Z, H, G, T, P (see column_core)
  float2* sbuf;    // [kmax][NY] this block's part of s (only with kmax > kSlotRegs)
  float2* sin;     // [kmax][NY] the peer's part (written by it)
  float* vox;      // [6][NY]: v0, v1, m v2, m v3, Re rho, Im rho
  float* red4;     // [4][NY] contraction over this block's r
  float* rin;      // [4][NY] the peer's contraction (written by it)
  float2* sin_peer;
  float* rin_peer;
};

// Steps 1-4 of the column product for image column ix (the voxel data in S.vox): on return
// red4 (this block's half of iy) and rin hold the two parts of the contraction.
// KM > 0 and RCT > 0: kmax == KM and nr == RCT known at compile time (the benchmark's
// shapes); 0: taken from the arguments.
template <int N1, int KM = 0, int RCT = 0>
__device__ __forceinline__ void column_core(const DftSmall& W, const ColShared& S, const float* __restrict__ coefT,
                                            const float* __restrict__ UgS, int kmax, int ix, int nx, int R, int r0,
                                            int nr, int ya, int ye) {
  namespace cgp = cooperative_groups;
  cgp::cluster_group cl = cgp::this_cluster();
  constexpr int NY = 32 * N1, M = 2 * N1, RS = col_row(NY);
  constexpr int SC = KM > 0 ? KM : 8;              // TR slots per pass of step 2
  constexpr int RCM = RCT > 0 ? RCT : kColMaxRc;   // basis functions per block, at most
  const int km = KM > 0 ? KM : kmax;
  const int nrr = RCT > 0 ? RCT : nr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t plane = (size_t)nx * NY;
  const float2* rt = S.rt;
  float2* hs = S.hs;
  float2* sbuf = S.sbuf;
  const float2* sin = S.sin;
  const float* vox = S.vox;
  float* red4 = S.red4;
  float2* sin_peer = S.sin_peer;
  float* red4_peer_in = S.rin_peer;
  // 1. h_r and its phase-encode DFT.  Warp w owns the rows rl = 2w, 2w + 1 of hs.
  //    (a) lane (rl = 2w + lane / 16, i2 = lane mod 16) forms x[i1] = h_r(16 i1 + i2) for
  //        i1 < M, the M-point DFT over i1 and the twiddle w^(k1 i2), and stores
  //        Z[k1][i2] at 17 k1 + i2 of its row;
  //    (b) lane (rl = 2w + (lane >= M), k1 = lane mod M) reads Z[k1][.], applies the
  //        16-point FFT and, once every lane of the warp has read its inputs, stores
  //        H_r(k1 + M k2) at k1 + M k2 (natural ky order).
  //    Lanes without a row of their own (rl >= nr, or lane >= 2 M) compute on a clamped
  //    row and store nothing, so the warp stays converged at its barriers.
  const int rlast = max(nrr - 1, 0);
  {
    const int rl = 2 * warp + (lane >> 4), i2 = lane & 15, rlc = min(rl, rlast);
    const float* ca = coefT + (size_t)(r0 + rlc) * plane + (size_t)ix * NY;
    // the coefficients of all M samples are loaded together (one L2 round trip); the
    // M-point DFT as its radix-2 step: the N1-point DFTs of the even and then of the odd
    // samples (each formed just before its DFT), then the combination
    float cf[M], d1[M], d2[M];
#pragma unroll
    for (int i1 = 0; i1 < M; ++i1) {
      const int iy = 16 * i1 + i2;
      cf[i1] = ca[iy];
      d1[i1] = ca[(size_t)R * plane + iy];
      d2[i1] = ca[(size_t)2 * R * plane + iy];
    }
    float2 E[N1], O[N1];
#pragma unroll
    for (int par = 0; par < 2; ++par) {
      float2 x[N1];
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const int i1 = 2 * i + par, iy = 16 * i1 + i2;
        const float v0 = vox[iy], v1 = vox[NY + iy], v2 = vox[2 * NY + iy], v3 = vox[3 * NY + iy];
        const float rr = vox[4 * NY + iy], ri = vox[5 * NY + iy];
        const float c = cf[i1], t = fmaf(v0, d1[i1], v1 * d2[i1]);
        x[i] = make_float2(-(ri * t + v3 * c), rr * t + v2 * c);
      }
      if (par == 0) dft_n1<N1, false>(W, x, E);
      else dft_n1<N1, false>(W, x, O);
    }
    float2* row = hs + rl * RS;
    const bool own = rl < nrr;
#pragma unroll
    for (int k = 0; k < N1; ++k) {
      const float2 t = k == 0 ? O[0] : cmul(O[k], W.wm[k]);
      const float2 ya = cadd(E[k], t), yb = csub(E[k], t);  // Y_k and Y_(k + N1)
      const float2 za = k == 0 ? ya : cmul(ya, rt[k * i2]), zb = cmul(yb, rt[(k + N1) * i2]);  // (M - 1) 15 < NY
      if (own) {
        row[17 * k + i2] = za;
        row[17 * (k + N1) + i2] = zb;
      }
    }
  }
  __syncwarp();
  {
    const int rl2 = 2 * warp + (lane >= M ? 1 : 0), k1 = lane >= M ? lane - M : lane;
    const bool act = lane < 2 * M && rl2 < nrr;
    const float2* src = hs + min(rl2, rlast) * RS + 17 * (act ? k1 : 0);
    float2 a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = src[j];
    fft16<false>(a);
    __syncwarp();  // the rows' Z are read before H overwrites them
    float2* row = hs + rl2 * RS + k1;
    if (act) {
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) row[M * k2] = a[brev4(k2)];
    }
  }
  // The first batch of step 2a's rows of U, loaded before the barrier so that the L2
  // latency overlaps the wait (the register path of step 2 only)
  constexpr int QB = SC <= 5 ? 8 : 4;  // basis functions per batch of U loads in step 2
  const int kyt = tid;
  const float* ub = UgS + (size_t)r0 * km * NY + kyt;
  float u[QB][SC];
  auto load_u = [&](int q0) {
    if constexpr (KM >= 4 && KM <= 8) {
      // the slot planes (UgS is then the plan's UgQ): one 16-byte load for slots 0-3 and
      // one 4- or 16-byte load for the rest, per basis function
      const float4* p0 = reinterpret_cast<const float4*>(UgS) + (size_t)r0 * NY + kyt;
      const float4* p1 = reinterpret_cast<const float4*>(UgS) + (size_t)R * NY + (size_t)r0 * NY + kyt;
      const float* p1f = UgS + (size_t)4 * R * NY + (size_t)r0 * NY + kyt;  // plane 1 of floats (KM = 5)
#pragma unroll
      for (int b = 0; b < QB; ++b) {
        const bool in = q0 + b < nrr && kyt < NY;
        const float4 a = in ? __ldg(p0 + (size_t)(q0 + b) * NY) : make_float4(0.f, 0.f, 0.f, 0.f);
        u[b][0] = a.x;
        u[b][1] = a.y;
        u[b][2] = a.z;
        u[b][3] = a.w;
        if constexpr (KM == 5) {
          u[b][4] = in ? __ldg(p1f + (size_t)(q0 + b) * NY) : 0.f;
        } else if constexpr (KM > 5) {
          const float4 c = in ? __ldg(p1 + (size_t)(q0 + b) * NY) : make_float4(0.f, 0.f, 0.f, 0.f);
          const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int i = 4; i < KM; ++i) u[b][i] = cv[i - 4];
        }
      }
    } else {
#pragma unroll
      for (int b = 0; b < QB; ++b)
#pragma unroll
        for (int i = 0; i < SC; ++i)
          u[b][i] = (i < km && q0 + b < nrr && kyt < NY) ? __ldg(ub + ((size_t)(q0 + b) * km + i) * NY) : 0.f;
    }
  };
  if (km <= SC) load_u(0);
  __syncthreads();
  // 2. per-ky Gram through the TR axis, thread per ky: U as UgS[r][i][ky] (the TRs of each
  //    ky in slots i < kmax, zero past a ky's TRs), so consecutive threads read consecutive
  //    ky (coalesced); every s and G a thread forms belongs to its own ky, so the phase
  //    needs no block barrier, only the cluster barrier of the exchange.
  if (km <= SC) {
    // one pass over the slots: this thread's part of s stays in registers across the
    // exchange (NY <= kColThreads: at most one line per thread); U in batches of QB rows,
    // each batch's loads issued together
    const int ky = kyt;
    float2 acc[SC];
#pragma unroll
    for (int i = 0; i < SC; ++i) acc[i] = make_float2(0.f, 0.f);
    //  2a. this block's part of s[i][ky] = sum_q U[q][i][ky] H_q(ky), stored into the peer's sin
    for (int q0 = 0; q0 < nrr; q0 += QB) {
      if (q0 > 0) load_u(q0);
      if (ky < NY) {
#pragma unroll
        for (int b = 0; b < QB; ++b) {
          if (q0 + b < nrr) {
            const float2 h = hs[(q0 + b) * RS + ky];
#pragma unroll
            for (int i = 0; i < SC; ++i) {
              acc[i].x = fmaf(u[b][i], h.x, acc[i].x);
              acc[i].y = fmaf(u[b][i], h.y, acc[i].y);
            }
          }
        }
      }
    }
    if (ky < NY) {
#pragma unroll
      for (int i = 0; i < SC; ++i)
        if (i < km) sin_peer[i * NY + ky] = acc[i];
    }
    // both parts of every s are in both blocks after the wait; the first batch of U for
    // 2b is loaded between the arrival and the wait
    cl.barrier_arrive();
    load_u(0);
    cl.barrier_wait();
    //  2b. G_r(ky) = sum_i U[r][i][ky] s[i][ky] with s the sum of the two parts
    //      (commutative: the same s in both blocks); G overwrites H_r(ky), which only this
    //      thread read
    if (ky < NY) {
#pragma unroll
      for (int i = 0; i < SC; ++i) {
        if (i < km) {
          const float2 sb = sin[i * NY + ky];
          acc[i] = make_float2(acc[i].x + sb.x, acc[i].y + sb.y);
        }
      }
    }
    for (int q0 = 0; q0 < nrr; q0 += QB) {
      if (q0 > 0) load_u(q0);
      if (ky < NY) {
#pragma unroll
        for (int b = 0; b < QB; ++b) {
          if (q0 + b < nrr) {
            float2 g = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < SC; ++i) {
              g.x = fmaf(u[b][i], acc[i].x, g.x);
              g.y = fmaf(u[b][i], acc[i].y, g.y);
            }
            hs[(q0 + b) * RS + ky] = g;
          }
        }
      }
    }
  } else {
    //    2a. this block's part of s[i][ky] = sum_q U[q][i][ky] H_q(ky), slots in chunks of
    //        SC, kept in sbuf and stored into the peer's sin
    for (int ky = tid; ky < NY; ky += kColThreads) {
      const float* ub = UgS + (size_t)r0 * km * NY + ky;
      for (int i0 = 0; i0 < km; i0 += SC) {
        float2 acc[SC];
#pragma unroll
        for (int i = 0; i < SC; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int q = 0; q < nrr; ++q) {
          const float2 h = hs[q * RS + ky];
#pragma unroll
          for (int i = 0; i < SC; ++i) {
            if (i0 + i < km) {
              const float u = __ldg(ub + ((size_t)q * km + i0 + i) * NY);
              acc[i].x = fmaf(u, h.x, acc[i].x);
              acc[i].y = fmaf(u, h.y, acc[i].y);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < SC; ++i) {
          if (i0 + i < km) {
            sbuf[(i0 + i) * NY + ky] = acc[i];
            sin_peer[(i0 + i) * NY + ky] = acc[i];  // the peer's copy of this block's part
          }
        }
      }
    }
    cl.sync();  // both parts of every s are in both blocks
    //    2b. G_r(ky) = sum_i U[r][i][ky] s[i][ky], with s the sum of the two parts
    //        (commutative: the same s in both blocks), over the slots in chunks of SC; G
    //        overwrites H_r(ky), which only this thread read
    for (int ky = tid; ky < NY; ky += kColThreads) {
      const float* ub = UgS + (size_t)r0 * km * NY + ky;
      for (int i0 = 0; i0 < km; i0 += SC) {
        float2 sv[SC];
#pragma unroll
        for (int i = 0; i < SC; ++i) {
          sv[i] = make_float2(0.f, 0.f);
          if (i0 + i < km) {
            const float2 sa = sbuf[(i0 + i) * NY + ky], sb = sin[(i0 + i) * NY + ky];
            sv[i] = make_float2(sa.x + sb.x, sa.y + sb.y);
          }
        }
#pragma unroll 4
        for (int r = 0; r < nrr; ++r) {
          float2 g = i0 == 0 ? make_float2(0.f, 0.f) : hs[r * RS + ky];
#pragma unroll
          for (int i = 0; i < SC; ++i) {
            if (i0 + i < km) {
              const float u = __ldg(ub + ((size_t)r * km + i0 + i) * NY);
              g.x = fmaf(u, sv[i].x, g.x);
              g.y = fmaf(u, sv[i].y, g.y);
            }
          }
          hs[r * RS + ky] = g;
        }
      }
    }

  }
  __syncthreads();  // the adjoint below reads whole rows of hs
  // 3. adjoint phase-encode DFT on the same rows as step 1, in the reverse order (lanes
  //    without a row compute on a clamped one and store nothing):
  //    (a) lane (rl, k1) reads G(k1 + M k2) for k2 < 16, applies the conjugate 16-point FFT
  //        and stores T[k1][i2] at 17 k1 + i2;
  //    (b) lane (rl, i2) reads T[k1][i2] for k1 < M, applies the conjugate twiddle and the
  //        conjugate M-point DFT and stores P_r(16 i1 + i2) at 16 i1 + i2.
  {
    const int rl2 = 2 * warp + (lane >= M ? 1 : 0), k1 = lane >= M ? lane - M : lane;
    const bool act = lane < 2 * M && rl2 < nrr;
    const float2* src = hs + min(rl2, rlast) * RS + (act ? k1 : 0);
    float2 a[16];
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) a[k2] = src[M * k2];
    fft16<true>(a);
    __syncwarp();  // the rows' G are read before T overwrites them
    float2* row = hs + rl2 * RS + 17 * k1;
    if (act) {
#pragma unroll
      for (int j = 0; j < 16; ++j) row[j] = a[brev4(j)];
    }
  }
  __syncwarp();
  {
    const int rl = 2 * warp + (lane >> 4), i2 = lane & 15;
    const float2* src = hs + min(rl, rlast) * RS + i2;
    float2 z[M];
    z[0] = src[0];
#pragma unroll
    for (int q = 1; q < M; ++q) z[q] = cmulc(src[17 * q], rt[q * i2]);
    __syncwarp();  // the rows' T are read before P overwrites them
    float2 out[M];
    dft_m<N1, true>(W, z, out);
    float2* row = hs + rl * RS + i2;
    if (rl < nrr) {
#pragma unroll
      for (int i1 = 0; i1 < M; ++i1) row[16 * i1] = out[i1];
    }
  }
  // 4. contraction with the tangents over this block's r, one thread per iy (NY <=
  //    kColThreads), the coefficients in batches of 8 r whose loads issue together; the
  //    first batch is loaded before the barrier that ends step 3
  {
    constexpr int RB = 8;
    const int iy = tid;
    const float* cc = coefT + (size_t)ix * NY + iy;
    float c4[RB], e1[RB], e2[RB];
    auto load_c = [&](int rb0) {
#pragma unroll
      for (int b = 0; b < RB; ++b) {
        const bool in = rb0 + b < nrr && iy < NY;
        const int r = r0 + rb0 + b;
        c4[b] = in ? cc[(size_t)r * plane] : 0.f;
        e1[b] = in ? cc[(size_t)(R + r) * plane] : 0.f;
        e2[b] = in ? cc[(size_t)(2 * R + r) * plane] : 0.f;
      }
    };
    load_c(0);
    __syncthreads();
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const float rhx = iy < NY ? vox[4 * NY + iy] : 0.f, rhy = iy < NY ? vox[5 * NY + iy] : 0.f;
    for (int rb0 = 0; rb0 < RCM; rb0 += RB) {
      if (rb0 > 0) load_c(rb0);
      if (iy < NY) {
#pragma unroll
        for (int b = 0; b < RB; ++b) {
          if (rb0 + b < nrr) {
            const float2 pv = hs[(rb0 + b) * RS + iy];
            const float imcp = rhx * pv.y - rhy * pv.x;  // Im(conj(rho) P)
            a0 = fmaf(e1[b], imcp, a0);
            a1 = fmaf(e2[b], imcp, a1);
            a2 = fmaf(c4[b], pv.y, a2);
            a3 = fmaf(-c4[b], pv.x, a3);
          }
        }
      }
    }
    // the part for this block's half of the column stays here, the rest goes to the peer
    if (iy < NY) {
      float* dst = (iy >= ya && iy < ye) ? red4 : red4_peer_in;
      dst[iy] = a0;
      dst[NY + iy] = a1;
      dst[2 * NY + iy] = a2;
      dst[3 * NY + iy] = a3;
    }
  }
  cl.sync();  // the peer's part of this block's half has arrived
}

template <int N1, int KM, int RCT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kColThreads, 3)
lr_jhjv_column_kernel(const __grid_constant__ DftSmall W, const float* __restrict__ v,
                      const float* __restrict__ coefT, const float2* __restrict__ rho,
                      const float* __restrict__ maskf, const float2* __restrict__ roots, const float* __restrict__ UgS,
                      int kmax, int nx, int ny, int nv, int R, float scale,
                      float* __restrict__ g, double* red_part, unsigned* ticket, double* __restrict__ vdot,
                      double* __restrict__ vv, const int* __restrict__ gate) {
  red::pdl_trigger();  // the successor may stage its own set-up meanwhile
  namespace cgp = cooperative_groups;
  cgp::cluster_group cl = cgp::this_cluster();
  const int crank = (int)cl.block_rank(), peer = crank ^ 1;
  constexpr int NY = 32 * N1, RS = col_row(NY);  // the launch passes ny == NY
  const int RC = (R + 1) / 2, r0 = crank * RC, nr = min(R, r0 + RC) - r0;
  extern __shared__ float2 fsm[];
  float2* rt = fsm;                                      // [NY] w^k
  float2* hs = rt + NY;                                  // [RC][RS] rows of the DFTs
  float2* sbuf = hs + RC * RS;                           // [kmax][NY] this block's part of s, then s
  float2* sin = sbuf + sbuf_slots(kmax) * NY;            // [kmax][NY] the peer's part (written by it)
  float* vox = reinterpret_cast<float*>(sin + kmax * NY);  // [6][NY]: v0, v1, m v2, m v3, Re rho, Im rho
  float* red4 = vox + 6 * NY;                            // [4][NY] contraction over this block's r
  float* rin = red4 + 4 * NY;                            // [4][NY] the peer's contraction (written by it)
  const ColShared S = {rt, hs, sbuf, sin, vox, red4, rin, cl.map_shared_rank(sin, peer), cl.map_shared_rank(rin, peer)};
  const int tid = threadIdx.x;
  const int hy = (NY + 1) / 2, ya = crank * hy, ye = min(NY, ya + hy);  // this block's half of iy
  for (int e = tid; e < NY; e += kColThreads) rt[e] = roots[e];  // plan constants: before the wait
  cl.sync();  // both blocks are running before either stores into the other's shared memory
  red::pdl_wait();  // v, rho, the coefficients and the gate come from earlier launches
  // the gate is written by earlier launches only: both blocks of a cluster take the same
  // branch, so every cluster barrier below is reached by both
  if (gate != nullptr && *gate == 0) return;
  float sf = 0.f, sv = 0.f;
  for (int ix = blockIdx.x >> 1; ix < nx; ix += gridDim.x >> 1) {
    // 0. the column's voxel data (each block loads all of it)
    int inside = 0;
    for (int iy = tid; iy < NY; iy += kColThreads) {
      const int j = iy * nx + ix;
      const float m = maskf[j];
      const float2 rh = rho[j];
      float vk[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) vk[k] = v[(size_t)k * nv + j];
      const float val[6] = {vk[0], vk[1], vk[2] * m, vk[3] * m, rh.x, rh.y};
#pragma unroll
      for (int c = 0; c < 6; ++c) vox[c * NY + iy] = val[c];
      inside |= m != 0.f;
    }
    if (!__syncthreads_or(inside)) {
      // no voxel of the column lies inside the mask, so g is zero on it (the product is
      // column by column); both blocks of the cluster see the same column and skip it
      for (int iy = ya + tid; iy < ye; iy += kColThreads) {
        const int j = iy * nx + ix;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          g[(size_t)k * nv + j] = 0.f;
          if (vdot != nullptr) {
            const float vk = v[(size_t)k * nv + j];
            sv = fmaf(vk, vk, sv);
          }
        }
      }
      continue;
    }
    column_core<N1, KM, RCT>(W, S, coefT, UgS, kmax, ix, nx, R, r0, nr, ya, ye);
    for (int iy = ya + tid; iy < ye; iy += kColThreads) {
      const int j = iy * nx + ix;
      const float m = maskf[j] * scale;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float val = (red4[k * NY + iy] + rin[k * NY + iy]) * m;
        g[(size_t)k * nv + j] = val;
        if (vdot != nullptr) {
          const float vk = v[(size_t)k * nv + j];
          sf = fmaf(vk, val, sf);
          sv = fmaf(vk, vk, sv);
        }
      }
    }
    // No block reads the other's shared memory: every exchange is a store into the peer
    // followed by a cluster barrier.  The next column's store into the peer's sin comes
    // after this column's second barrier, and its store into the peer's rin after the
    // next column's first barrier; the peer reaches those barriers only after it has read
    // sin and rin for this column.
    __syncthreads();
  }
  if (vdot == nullptr) return;
  __shared__ double ws[kColWarps];
  const double t = red::block_sum<kColThreads>((double)sf, ws);
  if (vv == nullptr) {
    if (threadIdx.x == 0) red_part[blockIdx.x] = t;
    red::finish_reduction<kColThreads>(red_part, ticket, vdot, ws);
    return;
  }
  const double t2 = red::block_sum<kColThreads>((double)sv, ws);
  if (threadIdx.x == 0) {
    red_part[blockIdx.x] = t;
    red_part[gridDim.x + blockIdx.x] = t2;
  }
  red::finish_reduction2<kColThreads>(red_part, ticket, vdot, vv, ws);
}

// ---------------------------------------------------------------------------
// Fixed-count CG on the low-rank B = Re(J^H J) in one persistent launch: one cluster of
// two blocks per image column for the whole solve, every cluster resident (cooperative
// launch).  J^H J is block diagonal in the image columns when the readout DFT pair
// cancels, so each cluster multiplies its own column and the CG vectors of its column
// never leave shared memory (each block keeps its half of iy).
// The iteration is the pipelined form of CG (Ghysels and Vanroose, Parallel Computing
// 40, 2014): with w = B r carried by recurrence, the two inner products of iteration k
// depend only on r_k and w_k, so their grid-wide sum runs while the cluster applies B to
// w_k.  Before the loop w_0 = B r_0; per iteration k:
//   the block's parts of gamma = <r, r> and delta = <w, r> go to part[k mod 2] and the
//   block arrives at the grid counter (no wait); q = B w (not in the last iteration);
//   the block waits until every block has arrived k + 1 times and adds the parts itself
//   in block order (the same sums in every block); beta = gamma / gamma_prev,
//   pq = delta - beta gamma / alpha_prev, alpha = gamma / pq (an iteration with pq <= 0
//   or gamma = 0 freezes the rest, and block 0 records where); z = q + beta z, s = w + beta s, p = r + beta p,
//   x += alpha p, r -= alpha s, w -= alpha z on the block's half; the new w of each half
//   goes into both blocks' voxel data (a store into the peer and a cluster barrier).
// Two parity buffers of partials suffice: a block writes part[k mod 2] again only after
// passing the wait of iteration k + 1, when every block has finished reading it.
// The wait is bounded (2 s): a block that gives up sets the error flag, and both blocks of
// a cluster leave together at the next cluster barrier.
// ---------------------------------------------------------------------------
constexpr uint64_t kGridWaitNs = 2000000000ull;

__device__ __forceinline__ uint64_t col_global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// The persistent kernels' inner products are summed in float-float arithmetic (an
// unevaluated sum hi + lo of two floats, about 44 significant bits): GB300 issues float64
// at a small fraction of the float32 rate, and the float64 block and grid sums of an
// earlier version cost 15 us per Steihaug step.  Addition of two float-float values:
// Knuth's TwoSum of the high parts, the low parts added to the error, then a Fast2Sum
// renormalisation (Dekker 1971; Shewchuk 1997).  No multiplications: nothing for the
// compiler to contract.
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ FF ff_shfl_xor(FF a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Products and quotients of float-float values for the CG scalars (GB300 issues float64
// at a small fraction of the float32 rate, and a float64 division on one thread sat on the
// critical path of every iteration): the exact product of two floats by one fused
// multiply-add (Dekker's TwoProduct), Fast2Sum renormalisation, and a quotient with one
// correction step (q1 = a / b in float, then q2 from the float-float remainder a - q1 b).
__device__ __forceinline__ FF ff_fast2sum(float s, float e) {  // |s| >= |e|
  const float h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);  // the exact rounding error of a.hi b.hi
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ff_fast2sum(p, e);
}

__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, FF{-b.hi, -b.lo}); }

__device__ __forceinline__ FF ff_div(FF a, FF b) {
  // q1 needs no correct rounding (the remainder below is exact for any q1 near a / b), so
  // the fast approximate division serves; q2 corrects it
  const float q1 = __fdividef(a.hi, b.hi);
  const FF r = ff_sub(a, ff_mul(b, FF{q1, 0.f}));
  return ff_fast2sum(q1, __fdividef(r.hi, b.hi));
}

// Sums of NV values over the block, valid in thread 0 (two block barriers); ws holds
// NV kColWarps values.
template <int NV>
__device__ __forceinline__ void block_sums(FF (&v)[NV], FF* ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = ff_add(v[k], ff_shfl_xor(v[k], o));
    if (lane == 0) ws[k * kColWarps + w] = v[k];
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < kColWarps ? ws[k * kColWarps + lane] : FF{0.f, 0.f};
#pragma unroll
      for (int o = kColWarps / 2; o > 0; o >>= 1) v[k] = ff_add(v[k], ff_shfl_xor(v[k], o));
    }
  }
  __syncthreads();
}

// The first half of block_sums without a barrier: each warp's sums of its NV values go
// to ws[k kColWarps + warp]; after the next block barrier warp_finish gives the block sums
// in lane 0 of warp 0.
template <int NV>
__device__ __forceinline__ void warp_partials(FF (&v)[NV], FF* ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] = ff_add(v[k], ff_shfl_xor(v[k], o));
    if (lane == 0) ws[k * kColWarps + w] = v[k];
  }
}

template <int NV>
__device__ __forceinline__ void warp_finish(FF (&v)[NV], const FF* ws) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    v[k] = lane < kColWarps ? ws[k * kColWarps + lane] : FF{0.f, 0.f};
#pragma unroll
    for (int o = kColWarps / 2; o > 0; o >>= 1) v[k] = ff_add(v[k], ff_shfl_xor(v[k], o));
  }
}

// Thread 0 stores the block's NV partials (block sums in thread 0) into part[k G + block]
// and arrives at the grid counter; it does not wait.
template <int NV>
__device__ __forceinline__ void grid_arrive(FF* part, unsigned* bar, const FF (&v)[NV]) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[(size_t)k * gridDim.x + blockIdx.x] = v[k];
    // a release reduction: the partials (and the earlier stores of this thread) are
    // visible to whoever acquires a count that includes this arrival
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until the grid counter reaches `target` (bounded), then the block adds
// part[k G .. (k + 1) G) in block order for each k < NV; the sums are valid in thread 0
// and the same in every block.  Returns false in a block whose wait ran out.
template <int NV>
__device__ __forceinline__ bool grid_wait_sums(const FF* part, const unsigned* bar, unsigned target, int* err, FF* ws,
                               double (&out)[NV]) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_acquire(bar) < target) {
      // polls back off (32 ns doubling to 512 ns): blocks that arrive early, e.g. those
      // of image columns outside the mask, neither take issue slots from the SM's other
      // blocks nor flood the counter's L2 slice while the rest compute
      const uint64_t t0 = col_global_ns();
      uint32_t spins = 0, ns = 32;
      while (ld_acquire(bar) < target) {
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
        if ((++spins & 63u) == 0 && col_global_ns() - t0 > kGridWaitNs) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();  // the acquire in thread 0 orders the other threads' reads after it
  const int G = gridDim.x;  // at most 2 kColThreads (checked at launch)
  FF acc[NV];
  // other blocks wrote the partials: read them from L2 (ld.global.cg), not from L1; both
  // blocks of a thread are loaded before any is added
  const float2* vp = reinterpret_cast<const float2*>(part);
  const int i0 = threadIdx.x, i1 = threadIdx.x + kColThreads;
  float2 t0v[NV], t1v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    t0v[k] = i0 < G ? __ldcg(vp + (size_t)k * G + i0) : make_float2(0.f, 0.f);
    t1v[k] = i1 < G ? __ldcg(vp + (size_t)k * G + i1) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = ff_add(FF{t0v[k].x, t0v[k].y}, FF{t1v[k].x, t1v[k].y});
  block_sums<NV>(acc, ws);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = (double)acc[k].hi + (double)acc[k].lo;
  return s_ok != 0;
}

// The same wait and sums for warp 0 alone (no block barrier): lane 0 waits, the warp adds
// the partials in the same order as above (lane l takes blocks l, l + 32, ...; then the
// butterfly of commutative float-float additions) and every lane of warp 0 holds the sums,
// the same in every block.  Returns false (in every lane) where the wait ran out.
template <int NV>
__device__ __forceinline__ bool grid_wait_sums_w0(const FF* part, const unsigned* bar, unsigned target, int* err,
                                                  FF (&out)[NV]) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  if (lane == 0 && ld_acquire(bar) < target) {
    const uint64_t t0 = col_global_ns();
    uint32_t spins = 0, ns = 32;
    while (ld_acquire(bar) < target) {
      __nanosleep(ns);
      if (ns < 256) ns <<= 1;
      if ((++spins & 63u) == 0 && col_global_ns() - t0 > kGridWaitNs) {
        atomicExch(err, 1);
        ok = 0;
        break;
      }
    }
  }
  __syncwarp();  // lane 0's acquire orders the other lanes' reads after it
  ok = __shfl_sync(0xffffffffu, ok, 0);
  const int G = gridDim.x;
  const float2* vp = reinterpret_cast<const float2*>(part);
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    // G <= 2 kColThreads = 512 (checked at launch): 16 blocks per lane, loaded together
    float2 t[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int i = lane + 32 * j;
      t[j] = i < G ? __ldcg(vp + (size_t)k * G + i) : make_float2(0.f, 0.f);
    }
    FF f[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) f[j] = FF{t[j].x, t[j].y};
    // pairwise: four dependent additions instead of sixteen
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = ff_add(f[j], f[j + 8]);
#pragma unroll
    for (int j = 0; j < 4; ++j) f[j] = ff_add(f[j], f[j + 4]);
#pragma unroll
    for (int j = 0; j < 2; ++j) f[j] = ff_add(f[j], f[j + 2]);
    f[0] = ff_add(f[0], f[1]);
    FF acc = f[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = ff_add(acc, ff_shfl_xor(acc, o));
    out[k] = acc;
  }
  return ok != 0;
}

// Shared memory of the persistent fixed-count CG with cpc image columns per cluster: the
// column kernel's, then per column the mask and the CG vectors (and, for the second
// column on, its own product input and rho rows and its product q = B w).
size_t cg_column_smem_bytes(int ny, int R, int kmax, int cpc = 1) {
  const size_t hy = (size_t)(ny + 1) / 2;
  return column_smem_bytes(ny, R, kmax) + sizeof(float) * ((size_t)ny + 20 * hy) +
         (size_t)(cpc - 1) * sizeof(float) * (6 * (size_t)ny + ny + 20 * hy + 4 * hy);
}

// CPC image columns per cluster (1, or 2 where the grid of one cluster per column does
// not fit at once: every column's CG state stays in shared memory, the products of the
// cluster's columns run one after the other, and the grid-wide sums add all of them).
template <int N1, int KM, int RCT, int CPC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kColThreads, CPC == 1 ? 3 : 2)
lr_cg_columns_kernel(const __grid_constant__ DftSmall W, const float* __restrict__ rhs, float* __restrict__ xout,
                     const float* __restrict__ coefT, const float2* __restrict__ rho,
                     const float* __restrict__ maskf, const float2* __restrict__ roots,
                     const float* __restrict__ UgS, int kmax, int nx, int nv, int R, float scale, int iters,
                     int stall_block, double* part, unsigned* bar, double* sums, int* frozen_at, int* err) {
  namespace cgp = cooperative_groups;
  cgp::cluster_group cl = cgp::this_cluster();
  const int crank = (int)cl.block_rank(), peer = crank ^ 1;
  constexpr int NY = 32 * N1, RS = col_row(NY), HY = (NY + 1) / 2;
  const int RC = (R + 1) / 2, r0 = crank * RC, nr = min(R, r0 + RC) - r0;
  extern __shared__ float2 fsm[];
  float2* rt = fsm;
  float2* hs = rt + NY;
  float2* sbuf = hs + RC * RS;
  float2* sin = sbuf + sbuf_slots(kmax) * NY;
  float* vox0 = reinterpret_cast<float*>(sin + kmax * NY);  // rows 0..3: the product's input
  float* red4 = vox0 + 6 * NY;
  float* rin = red4 + 4 * NY;
  // per column c: vox[c] [6][NY] (w and rho), mk[c] [NY], cgv[c] [5 vectors r, p, s, z, x]
  // [4 rows][HY] of this block's half, and (c >= 1) qv[c] [4][HY], its product q = B w
  float* vox[CPC];
  float* mk[CPC];
  float* cgv[CPC];
  float* qv[CPC];
  {
    float* q = rin + 4 * NY;
#pragma unroll
    for (int c = 0; c < CPC; ++c) {
      if (c > 0) {
        vox[c] = q;
        q += 6 * NY;
      } else {
        vox[c] = vox0;
      }
      mk[c] = q;
      q += NY;
      cgv[c] = q;
      q += 20 * HY;
      if (c > 0) {
        qv[c] = q;
        q += 4 * HY;
      } else {
        qv[c] = nullptr;
      }
    }
  }
  float2* const sin_peer = cl.map_shared_rank(sin, peer);
  float* const rin_peer = cl.map_shared_rank(rin, peer);
  __shared__ int s_ok_peer[2];  // written by the peer, slot it mod 2 in iteration it
  int* ok_peer_remote = cl.map_shared_rank(s_ok_peer, peer);
  __shared__ FF ws[2 * kColWarps];
  __shared__ float s_al, s_be;
  __shared__ int s_apply;
  const int tid = threadIdx.x;
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;  // column c of this cluster: cid + c ncl
  const int G = gridDim.x;
  const int ya = crank * HY, nh = min(NY, ya + HY) - ya;  // this block's half of iy: ya .. ya + nh
  for (int e = tid; e < NY; e += kColThreads) rt[e] = roots[e];
  cl.sync();

  // rho and the mask of each whole column; r = rhs and p = s = z = x = 0 on this block's
  // half; the product's input is r (rows 2, 3 masked)
  bool inside[CPC];
#pragma unroll
  for (int c = 0; c < CPC; ++c) {
    const int ix = cid + c * ncl;
    int in = 0;
    if (ix < nx) {
      for (int iy = tid; iy < NY; iy += kColThreads) {
        const int j = iy * nx + ix;
        const float2 rh = rho[j];
        const float m = maskf[j];
        vox[c][4 * NY + iy] = rh.x;
        vox[c][5 * NY + iy] = rh.y;
        mk[c][iy] = m;
        in |= m != 0.f;
      }
    }
    inside[c] = __syncthreads_or(in) != 0;  // the same column in both blocks: the same answer
    float* const cg = cgv[c];
    float* const vp = cl.map_shared_rank(vox[c], peer);
    if (tid < nh) {
      const int iy = ya + tid, j = iy * nx + ix;
      const float m = ix < nx ? mk[c][iy] : 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float r = ix < nx ? rhs[(size_t)k * nv + j] : 0.f;
        cg[k * HY + tid] = r;
        cg[(4 + k) * HY + tid] = 0.f;
        cg[(8 + k) * HY + tid] = 0.f;
        cg[(12 + k) * HY + tid] = 0.f;
        cg[(16 + k) * HY + tid] = 0.f;
        const float vv = k >= 2 ? r * m : r;
        vox[c][k * NY + iy] = vv;
        vp[k * NY + iy] = vv;
      }
    }
  }
  cl.sync();

  // the product q = B w of column c (masked, like every product), into qv[c] for c >= 1
  auto product = [&](int c) {
    const ColShared S = {rt, hs, sbuf, sin, vox[c], red4, rin, sin_peer, rin_peer};
    column_core<N1, KM, RCT>(W, S, coefT, UgS, kmax, cid + c * ncl, nx, R, r0, nr, ya, ya + nh);
    if (c > 0 && tid < nh) {
      const int iy = ya + tid;
      const float m = mk[c][iy] * scale;
#pragma unroll
      for (int k = 0; k < 4; ++k) qv[c][k * HY + tid] = (red4[k * NY + iy] + rin[k * NY + iy]) * m;
    }
  };
  // column c's q at this thread's element (k, iy): column 0 reads the product's output
  // in place (its product is the last of an iteration), the others their copy
  auto qval = [&](int c, int k, int iy) {
    return c == 0 ? (red4[k * NY + iy] + rin[k * NY + iy]) * (mk[0][iy] * scale) : qv[c][k * HY + (iy - ya)];
  };

  // w_0 = B r_0 becomes the product's input
#pragma unroll
  for (int c = CPC - 1; c >= 0; --c)
    if (inside[c]) product(c);
#pragma unroll
  for (int c = 0; c < CPC; ++c) {
    float* const vp = cl.map_shared_rank(vox[c], peer);
    if (tid < nh) {
      const int iy = ya + tid;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float wv = inside[c] ? qval(c, k, iy) : 0.f;
        vox[c][k * NY + iy] = wv;
        vp[k * NY + iy] = wv;
      }
    }
  }
  // the thread's parts of delta = <w, r> and gamma = <r, r> over the cluster's columns
  // (formed with every update, on the thread's own elements) and their warp sums, which
  // warp 0 finishes after the cluster barrier below
  auto partials = [&]() {
    float sd = 0.f, sg = 0.f;
    if (tid < nh) {
#pragma unroll
      for (int c = 0; c < CPC; ++c) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float r = cgv[c][k * HY + tid];
          sd = fmaf(r, vox[c][k * NY + ya + tid], sd);
          sg = fmaf(r, r, sg);
        }
      }
    }
    FF v[2] = {{sd, 0.f}, {sg, 0.f}};
    warp_partials<2>(v, ws);
  };
  partials();
  cl.sync();

  // pq_prev = p.Bp of the previous iteration: beta gamma / alpha_prev = beta^2 pq_prev
  // (float-float, thread 0)
  FF gam_prev{0.f, 0.f}, pq_prev{0.f, 0.f};
  bool frozen = false;
  int applied = 0;  // iterations that moved x (thread 0)
  __shared__ int s_okb;
  __shared__ FF s_dg[2];  // this iteration's delta and gamma (for the record)
  for (int it = 0; it < iters; ++it) {
    FF* pk = reinterpret_cast<FF*>(part) + (size_t)(it & 1) * 2 * G;
    // q = B w while the other blocks arrive (not needed in the last iteration)
    const bool more = it + 1 < iters;
    // warp 0 finishes the block's parts of delta and gamma (the warps' sums, written before
    // the last cluster barrier) and arrives, before the product: the other blocks' waits
    // end as early as possible.  A block named by the test hook withholds its first
    // arrival, and every wait runs out.
    const bool arrive = it > 0 || (int)blockIdx.x != stall_block;
    if ((tid >> 5) == 0) {
      FF b[2];
      warp_finish<2>(b, ws);
      if (arrive) grid_arrive<2>(pk, bar, b);
    }
    // the products, column 0 last (the update reads its output in place)
#pragma unroll
    for (int c = CPC - 1; c >= 0; --c)
      if (inside[c] && more) product(c);
    // warp 0 waits, sums and decides; the other warps go straight to the block barrier
    if ((tid >> 5) == 0) {
      FF sums2[2];
      const bool okw = grid_wait_sums_w0<2>(pk, bar, (unsigned)G * (unsigned)(it + 1), err, sums2);
      const FF delta = sums2[0], gamma = sums2[1];
      if (tid == 0) {
        s_dg[0] = delta;
        s_dg[1] = gamma;
        int apply = 0;
        float al = 0.f, be = 0.f;
        if (okw) {
          FF beta{0.f, 0.f}, pq = delta;
          if (it > 0) {
            beta = ff_div(gamma, gam_prev);
            pq = ff_sub(delta, ff_mul(ff_mul(beta, beta), pq_prev));
          }
          apply = !frozen && pq.hi > 0.f && gamma.hi > 0.f;
          if (apply) {
            al = ff_div(gamma, pq).hi;
            be = beta.hi;
            gam_prev = gamma;
            pq_prev = pq;
            ++applied;
          } else {
            frozen = true;
          }
        }
        s_apply = apply;
        s_al = al;
        s_be = be;
        s_okb = okw;
        ok_peer_remote[it & 1] = okw;
      }
    }
    __syncthreads();
    const bool ok = s_okb != 0;
    if (tid == kColThreads - 1 && ok && blockIdx.x == 0) {  // the record, off warp 0's path
      sums[2 * it] = (double)s_dg[0].hi + (double)s_dg[0].lo;
      sums[2 * it + 1] = (double)s_dg[1].hi + (double)s_dg[1].lo;
    }
    if (s_apply && tid < nh) {
      const int iy = ya + tid;
      const float al = s_al, be = s_be;
#pragma unroll
      for (int c = 0; c < CPC; ++c) {
        float* const cg = cgv[c];
        float* const vp = cl.map_shared_rank(vox[c], peer);
        const bool pc = inside[c] && more;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = k * HY + tid;
          const float wv = vox[c][k * NY + iy];
          const float q = pc ? qval(c, k, iy) : 0.f;  // q = B w
          const float zv = fmaf(be, cg[12 * HY + e], q);
          const float sv = fmaf(be, cg[8 * HY + e], wv);
          const float pv = fmaf(be, cg[4 * HY + e], cg[e]);
          cg[12 * HY + e] = zv;
          cg[8 * HY + e] = sv;
          cg[4 * HY + e] = pv;
          cg[16 * HY + e] = fmaf(al, pv, cg[16 * HY + e]);
          cg[e] = fmaf(-al, sv, cg[e]);
          const float wn = fmaf(-al, zv, wv);
          vox[c][k * NY + iy] = wn;
          vp[k * NY + iy] = wn;
        }
      }
    }
    // the next iteration's parts from r and w as they now stand, summed over each warp
    partials();
    cl.sync();  // the new w of both halves is in both blocks; the peer's flag has arrived
    // both blocks of the cluster leave together; the slot is written again only after the
    // peer has passed the next cluster barrier, i.e. after this read
    if (!ok || !s_ok_peer[it & 1]) break;
  }
  // every block took the same decisions; block 0 reports where the solve froze (the
  // iteration index + 1; 0 when all iterations were applied)
  if (blockIdx.x == 0 && tid == 0) *frozen_at = applied < iters ? applied + 1 : 0;
#pragma unroll
  for (int c = 0; c < CPC; ++c) {
    const int ix = cid + c * ncl;
    if (tid < nh && ix < nx) {
      const int j = (ya + tid) * nx + ix;
#pragma unroll
      for (int k = 0; k < 4; ++k) xout[(size_t)k * nv + j] = cgv[c][(16 + k) * HY + tid];
    }
  }
}

// ---------------------------------------------------------------------------
// Steihaug's truncated CG (Nocedal & Wright Alg. 7.2, the inner solve of Algorithm 6) on
// the low-rank B = Re(J^H J) in one persistent launch, laid out like the fixed-count CG
// above: one cluster per image column, the column's res, dir, z and q = B dir in shared
// memory (each block its half of iy), every block taking the same decisions from the
// same grid-wide sums.  The product is applied to the residual, u = B res, so that one
// grid wait per step carries every sum (the direction's product follows by recurrence,
// B dir' = -u + beta q, as in the pipelined CG above).  Before the loop q = B dir_0 and
// one wait gives g.g and dir.q.  Per step:
//   the step decision from dir.q (negative curvature or the trust boundary end CG with z
//   on the boundary); z += c dir, and while CG continues res += c q; u = B res (not after
//   the last step); the parts of res.res, res.dir, z.res, z.dir, z.z, res.u, dir.u,
//   res.q go to one grid wait; the tolerance and step-count test and beta; then
//   dir' = -res + beta dir, q' = -u + beta q, and the next decision's sums follow from
//   the definitions: res.dir' = -res.res + beta res.dir,
//   dir'.dir' = res.res - 2 beta res.dir + beta^2 dir.dir, z.dir' = -z.res + beta z.dir,
//   dir'.q' = res.u - beta (dir.u + res.q) + beta^2 dir.q.
// Each grid wait is followed by an exchange of the two blocks' wait flags, so both blocks
// of a cluster leave together when one wait ran out (2 s: the error flag is set).
// ---------------------------------------------------------------------------
size_t st_column_smem_bytes(int ny, int R, int kmax) {
  const int hy = (ny + 1) / 2;
  return column_smem_bytes(ny, R, kmax) + sizeof(float) * ((size_t)ny + 16 * (size_t)hy);
}

template <int N1, int KM, int RCT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kColThreads, 3)
lr_steihaug_columns_kernel(const __grid_constant__ DftSmall W, const float* __restrict__ grad,
                           float* __restrict__ zout, const float* __restrict__ coefT,
                           const float2* __restrict__ rho, const float* __restrict__ maskf,
                           const float2* __restrict__ roots, const float* __restrict__ UgS, int kmax, int nx, int nv,
                           int R, float scale, double delta, double rel_tol, int max_steps, double* sc, int* si,
                           int stall_block, double* part, unsigned* bar, int* err) {
  namespace cgp = cooperative_groups;
  cgp::cluster_group cl = cgp::this_cluster();
  const int crank = (int)cl.block_rank(), peer = crank ^ 1;
  constexpr int NY = 32 * N1, RS = col_row(NY), HY = (NY + 1) / 2;
  constexpr int NP = 8;  // partials per block and grid wait, at most
  const int RC = (R + 1) / 2, r0 = crank * RC, nr = min(R, r0 + RC) - r0;
  extern __shared__ float2 fsm[];
  float2* rt = fsm;
  float2* hs = rt + NY;
  float2* sbuf = hs + RC * RS;
  float2* sin = sbuf + sbuf_slots(kmax) * NY;
  float* vox = reinterpret_cast<float*>(sin + kmax * NY);  // rows 0..3: the product's input
  float* red4 = vox + 6 * NY;
  float* rin = red4 + 4 * NY;
  float* mk = rin + 4 * NY;  // [NY] mask of the column
  float* const cr = mk + NY;  // [4 vectors res, dir, z, q][4 rows][HY] this block's half
  float* const cd = cr + 4 * HY;
  float* const cz = cr + 8 * HY;
  float* const cq = cr + 12 * HY;
  const ColShared S = {rt, hs, sbuf, sin, vox, red4, rin, cl.map_shared_rank(sin, peer), cl.map_shared_rank(rin, peer)};
  float* vox_peer = cl.map_shared_rank(vox, peer);
  // the wait flags of the two blocks, exchanged after every grid wait: slot n mod 2 in
  // exchange n, written again only after the peer has passed the next cluster barrier
  __shared__ int s_ok_peer[2];  // written by the peer
  int* ok_peer_remote = cl.map_shared_rank(s_ok_peer, peer);
  unsigned xch = 0;
  __shared__ FF ws[NP * kColWarps];
  __shared__ double lsc[S_COUNT];
  __shared__ int lsi[I_COUNT];
  __shared__ int s_ok, s_go, s_cont, s_prod;
  __shared__ float s_c, s_beta;
  const int tid = threadIdx.x;
  const int ix = blockIdx.x >> 1;  // one column per cluster
  const int G = gridDim.x;
  const int ya = crank * HY, nh = min(NY, ya + HY) - ya;  // this block's half of iy: ya .. ya + nh
  const int own = tid < nh;
  const int iy = ya + min(tid, nh - 1);
  unsigned waits = 0;  // grid waits passed; wait n uses part[(n mod 2) NP G ..]
  for (int e = tid; e < NY; e += kColThreads) rt[e] = roots[e];
  cl.sync();  // both blocks run (before any store into the peer) and hold the roots

  // rho and the mask of the whole column; res = g, dir = -g, z = 0 on this block's half;
  // the product's input is dir (rows 2, 3 masked)
  int inside = 0;
  for (int y = tid; y < NY; y += kColThreads) {
    const int j = y * nx + ix;
    const float2 rh = rho[j];
    const float m = maskf[j];
    vox[4 * NY + y] = rh.x;
    vox[5 * NY + y] = rh.y;
    mk[y] = m;
    inside |= m != 0.f;
  }
  inside = __syncthreads_or(inside);  // the same column in both blocks: the same answer
  const float mq = mk[iy] * scale;
  if (own) {
    const int j = iy * nx + ix;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float gv = grad[(size_t)k * nv + j];
      cr[k * HY + tid] = gv;
      cd[k * HY + tid] = -gv;
      cz[k * HY + tid] = 0.f;
      const float dv = k >= 2 ? -gv * mk[iy] : -gv;
      vox[k * NY + iy] = dv;
      vox_peer[k * NY + iy] = dv;
    }
  }
  cl.sync();  // dir of both halves is in both blocks
  // q = B dir_0, then g.g and dir.q
  if (inside) column_core<N1, KM, RCT>(W, S, coefT, UgS, kmax, ix, nx, R, r0, nr, ya, ya + nh);
  {
    float sg = 0.f, sq = 0.f;
    if (own) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float qv = inside ? (red4[k * NY + iy] + rin[k * NY + iy]) * mq : 0.f;
        const float gv = cr[k * HY + tid];
        cq[k * HY + tid] = qv;
        sg = fmaf(gv, gv, sg);
        sq = fmaf(cd[k * HY + tid], qv, sq);
      }
    }
    FF v[2] = {{sg, 0.f}, {sq, 0.f}};
    double t[2];
    block_sums<2>(v, ws);
    FF* pk = reinterpret_cast<FF*>(part) + (size_t)(waits & 1) * NP * G;
    if ((int)blockIdx.x != stall_block) grid_arrive<2>(pk, bar, v);  // the test hook withholds it
    const bool ok = grid_wait_sums<2>(pk, bar, (unsigned)G * ++waits, err, ws, t);
    if (tid == 0) {
      const double rr = t[0];
      for (int k = 0; k < S_COUNT; ++k) lsc[k] = 0.0;
      for (int k = 0; k < I_COUNT; ++k) lsi[k] = 0;
      lsc[S_RR] = rr;
      lsc[S_RD] = -rr;
      lsc[S_DD] = rr;
      lsc[S_DBD] = t[1];
      lsc[S_GNORM] = sqrt(rr);
      lsi[I_ACTIVE] = rr > 0.0 ? 1 : 0;
      lsi[I_EXIT] = rr > 0.0 ? MRSTAT_CG_MAX_ITER : MRSTAT_CG_ZERO_GRADIENT;
      s_ok = ok;
      s_go = lsi[I_ACTIVE];
      ok_peer_remote[xch & 1] = ok;
    }
  }
  cl.sync();  // the peer's flag has arrived
  bool failed = !s_ok || !s_ok_peer[xch++ & 1];
  for (int step = 0; step < max_steps && s_go && !failed; ++step) {
    // the step decision from dir.q (the same sums in every block)
    if (tid == 0) {
      st_step(lsc, lsi, delta);
      s_cont = lsi[I_CONT];
      s_c = (float)lsc[S_COEF];
      s_prod = lsi[I_STEPS] < max_steps;  // a next step can follow: its product is needed
    }
    __syncthreads();
    const float c = s_c;
    const int cont = s_cont;
    // z += c dir; while continuing res += c q, which is the next product's input
    float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (own) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = k * HY + tid;
        const float dv = cd[e];
        const float zv = fmaf(c, dv, cz[e]);
        cz[e] = zv;
        if (cont) {
          const float rv = fmaf(c, cq[e], cr[e]);
          cr[e] = rv;
          const float vv = k >= 2 ? rv * mk[iy] : rv;
          vox[k * NY + iy] = vv;
          vox_peer[k * NY + iy] = vv;
          a[0] = fmaf(rv, rv, a[0]);
          a[1] = fmaf(rv, dv, a[1]);
          a[2] = fmaf(zv, rv, a[2]);
          a[3] = fmaf(zv, dv, a[3]);
          a[4] = fmaf(zv, zv, a[4]);
        }
      }
    }
    if (!cont) break;  // negative curvature or the trust boundary: the same in every block
    FF* pk = reinterpret_cast<FF*>(part) + (size_t)(waits & 1) * NP * G;
    {
      // the block's first five parts go out now (thread 0 stores them; the arrival after
      // the product publishes them), so that nothing is held across the product
      FF v[5] = {{a[0], 0.f}, {a[1], 0.f}, {a[2], 0.f}, {a[3], 0.f}, {a[4], 0.f}};
      block_sums<5>(v, ws);
      if (tid == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) pk[(size_t)k * G + blockIdx.x] = v[k];
      }
    }
    cl.sync();  // res of both halves is in both blocks
    // u = B res, and its parts res.u, dir.u, res.q
    const bool prod = inside && s_prod;
    float b[3] = {0.f, 0.f, 0.f};
    if (prod) {
      column_core<N1, KM, RCT>(W, S, coefT, UgS, kmax, ix, nx, R, r0, nr, ya, ya + nh);
      if (own) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int e = k * HY + tid;
          const float uv = (red4[k * NY + iy] + rin[k * NY + iy]) * mq, rv = cr[e];
          b[0] = fmaf(rv, uv, b[0]);
          b[1] = fmaf(cd[e], uv, b[1]);
          b[2] = fmaf(rv, cq[e], b[2]);
        }
      }
    }
    {
      FF v[3] = {{b[0], 0.f}, {b[1], 0.f}, {b[2], 0.f}};
      double t[NP];
      block_sums<3>(v, ws);
      grid_arrive<3>(pk + (size_t)5 * G, bar, v);
      const bool ok = grid_wait_sums<NP>(pk, bar, (unsigned)G * ++waits, err, ws, t);
      if (tid == 0) {
        float be = 0.f;
        if (ok) {
          lsc[S_RR_NEW] = t[0];
          st_beta(lsc, lsi, rel_tol, max_steps);
          if (lsi[I_ACTIVE]) {
            const double beta = lsc[S_BETA], rr = t[0], rd = t[1], dd = lsc[S_DD], dq = lsc[S_DBD];
            lsc[S_RD] = -rr + beta * rd;
            lsc[S_DD] = rr - 2.0 * beta * rd + beta * beta * dd;
            lsc[S_ZD] = -t[2] + beta * t[3];
            lsc[S_ZZ] = t[4];
            lsc[S_DBD] = t[5] - beta * (t[6] + t[7]) + beta * beta * dq;
            be = (float)beta;
          }
        }
        s_ok = ok;
        s_go = ok && lsi[I_ACTIVE];
        s_beta = be;
        ok_peer_remote[xch & 1] = ok;
      }
      cl.sync();  // the peer's flag has arrived
      if (!s_ok || !s_ok_peer[xch++ & 1]) {
        failed = true;
        break;
      }
    }
    // dir' = -res + beta dir, q' = -u + beta q
    if (s_go && own) {
      const float be = s_beta;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = k * HY + tid;
        const float uv = prod ? (red4[k * NY + iy] + rin[k * NY + iy]) * mq : 0.f;
        cd[e] = fmaf(be, cd[e], -cr[e]);
        cq[e] = fmaf(be, cq[e], -uv);
      }
    }
    __syncthreads();
  }
  if (own) {
    const int j = iy * nx + ix;
#pragma unroll
    for (int k = 0; k < 4; ++k) zout[(size_t)k * nv + j] = cz[k * HY + tid];
  }
  if (blockIdx.x == 0 && tid == 0 && !failed) {
    for (int k = S_RR; k <= S_ZZ; ++k) sc[k] = lsc[k];
    si[I_ACTIVE] = 0;
    si[I_CONT] = 0;
    si[I_EXIT] = lsi[I_EXIT];
    si[I_STEPS] = lsi[I_STEPS];
  }
}

// Partial sums over one chunk of 8 basis functions (blockIdx.z) of
//   g_k,j = Re sum_r conj(dh_r,j/dv_k) P[(ix, r)][iy]   (P rows (ix, r), columns 2 iy + re/im)
// into part[z][4][nv].  Block (16, 16): a 16 x 16 voxel tile, one voxel per thread; P
// arrives through shared memory in whole 128-byte row pieces.
__global__ void __launch_bounds__(256)
lr_final_t_kernel(const float* __restrict__ PT, int ldp, const float* __restrict__ coef,
                  const float2* __restrict__ rho, int nx, int ny, int nv, int R, float* __restrict__ part,
                  const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  __shared__ float2 S[8][16][17];  // [r - r0][ix - ix0][iy - iy0]
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  const int ix0 = blockIdx.x * 16, iy0 = blockIdx.y * 16, r0 = blockIdx.z * 8;
  const float2* P2 = reinterpret_cast<const float2*>(PT);
  const int ld2 = ldp / 2;
  // load mapping: 16 lanes along iy, 128 rows (16 ix x 8 r) in 8 passes of 16
  const int ly = tid & 15, lrow = tid >> 4;
#pragma unroll
  for (int pass = 0; pass < 8; ++pass) {
    const int rl = lrow + 16 * pass, a = rl >> 3, rr = rl & 7;
    const int ixa = ix0 + a, r = r0 + rr, iyl = iy0 + ly;
    S[rr][a][ly] =
        (ixa < nx && r < R && iyl < ny) ? P2[(size_t)(ixa * R + r) * ld2 + iyl] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int ix = ix0 + tx, iy = iy0 + ty;
  if (ix >= nx || iy >= ny) return;
  const int j = iy * nx + ix;
  const float2 rh = rho[j];
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    const int r = r0 + rr;
    if (r < R) {
      const float2 pv = S[rr][tx][ty];
      const float c = coef[(size_t)r * nv + j];
      const float t1 = coef[(size_t)(R + r) * nv + j], t2 = coef[(size_t)(2 * R + r) * nv + j];
      const float imcp = rh.x * pv.y - rh.y * pv.x;  // Im(conj(rho) P)
      a0 = fmaf(t1, imcp, a0);
      a1 = fmaf(t2, imcp, a1);
      a2 = fmaf(c, pv.y, a2);
      a3 = fmaf(-c, pv.x, a3);
    }
  }
  float* pz = part + (size_t)blockIdx.z * 4 * nv;
  pz[j] = a0;
  pz[(size_t)nv + j] = a1;
  pz[2 * (size_t)nv + j] = a2;
  pz[3 * (size_t)nv + j] = a3;
}

// g = scale * mask * (sum of the chunk partials, in chunk order); with vdot, also
// *vdot = sum_e v[e] g[e] (the CG inner product <p, Re(J^H J) p>: float32 per thread,
// float64 from the warp level up, last-block finish over red / ticket)
constexpr int kSumThreads = 256;
__global__ void __launch_bounds__(kSumThreads)
lr_final_sum_kernel(const float* __restrict__ part, int nchunk, const float* __restrict__ maskf, int nv, float scale,
                    float* __restrict__ g, const int* __restrict__ gate, const float* __restrict__ v,
                    double* red_part, unsigned* ticket, double* __restrict__ vdot) {
  if (gate != nullptr && *gate == 0) return;
  const int64_t n4 = 4 * (int64_t)nv;
  float sf = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < nchunk; ++z) s += part[(size_t)z * n4 + e];
    const int j = (int)(e % nv);
    const float val = s * maskf[j] * scale;
    g[e] = val;
    if (vdot != nullptr) sf = fmaf(v[e], val, sf);
  }
  if (vdot == nullptr) return;
  __shared__ double ws[kSumThreads / 32];
  const double t = red::block_sum<kSumThreads>((double)sf, ws);
  if (threadIdx.x == 0) red_part[blockIdx.x] = t;
  red::finish_reduction<kSumThreads>(red_part, ticket, vdot, ws);
}

// training time courses [3][nq][ns] (quads) -> Y [ntr][3 ns] and Yt [3 ns][ntr] (complex
// storage with zero imaginary part), columns c * ns + s
__global__ void lr_train_matrix_kernel(const float4* __restrict__ D, int ns, int nq, int ntr,
                                       float2* __restrict__ Y, float2* __restrict__ Yt) {
  const int64_t K = 3 * (int64_t)ns;
  const int64_t total = (int64_t)ntr * K;
  const float* Df = reinterpret_cast<const float*>(D);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / K;
    const int64_t col = e - n * K;
    const int64_t c = col / ns, s = col - c * ns;
    const float v = Df[(((size_t)c * nq + (n >> 2)) * ns + s) * 4 + (n & 3)];
    Y[e] = make_float2(v, 0.f);
    Yt[col * ntr + n] = make_float2(v, 0.f);
  }
}

template <int R>
cudaError_t launch_project_t(const Plan& p, const LowRank& L, const float* alpha, const float* b1,
                             const uint8_t* mask, float* coef, cudaStream_t st) {
  const int blocks = (p.nv + 127) / 128;
  lr_project_kernel<R><<<blocks, 128, 0, st>>>(alpha, b1, mask, p.cs, p.phi, L.U, p.nv, p.ntr, (float)p.te_ms,
                                               (float)(p.tr_ms - p.te_ms), p.inversion ? -1.f : 1.f, coef);
  return cudaGetLastError();
}

inline int pad8(int k) { return (k + 7) / 8 * 8; }

}  // namespace

cudaError_t lowrank_project(const Plan& p, const LowRank& L, const float* alpha, const float* b1,
                            const uint8_t* mask, float* coef, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  switch (L.R) {
    case 8: return launch_project_t<8>(p, L, alpha, b1, mask, coef, st);
    case 16: return launch_project_t<16>(p, L, alpha, b1, mask, coef, st);
    case 24: return launch_project_t<24>(p, L, alpha, b1, mask, coef, st);
    case 32: return launch_project_t<32>(p, L, alpha, b1, mask, coef, st);
    default: return cudaErrorInvalidValue;
  }
}

void lowrank_free(LowRank* L) {
  if (L == nullptr) return;
  void* ptrs[] = {L->U, L->Ug, L->UgT, L->UgS, L->UgQ, L->kyof, L->Mky, L->kyptr, L->kytr, L->coef, L->coef2, L->gpart, L->coefT, L->a1_hi, L->a1_lo, L->a23_hi, L->a23_lo,
                  L->a4_hi, L->a4_lo, L->by_hi, L->by_lo, L->bya_hi, L->bya_lo, L->X1, L->H, L->Y3, L->P};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete L;
}

// Allocates the low-rank work space and builds the phase-encode DFT operands and the
// per-ky tables for basis U (device [ntr][R]); the readout DFT operands are the plan's
// split-BF16 tables.
int lowrank_setup(Plan* p, const float* U_dev, int R, cudaStream_t st) {
  if (R != 8 && R != 16 && R != 24 && R != 32)
    return fail(MRSTAT_ERR_INVALID_ARG, "rank %d not in {8, 16, 24, 32}", R);
  if (!p->tc) {
    const int s = build_split_tables(p);
    if (s != MRSTAT_OK) return s;
  }
  if (p->lr) {
    lowrank_free(p->lr);
    p->lr = nullptr;
  }
  LowRank* L = new LowRank();
  L->R = R;
  {
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    L->sms = sms > 0 ? sms : 1;
    L->smem_optin = optin;
  }
  const int nx = p->nx, ny = p->ny, nkx = p->nkx, ntr = p->ntr;
  L->k1 = pad8(2 * nx);
  L->k23 = pad8(2 * ny);
  L->k4 = pad8(2 * nkx);
  // host copies of U (float64 for the Gram tables)
  std::vector<float> Uh((size_t)ntr * R);
  cudaError_t e = cudaMemcpyAsync(Uh.data(), U_dev, Uh.size() * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    delete L;
    return cuda_fail(e, "basis copy");
  }
  std::vector<int> kyi_h(p->ntr_pad);
  e = cudaMemcpy(kyi_h.data(), p->kyi, kyi_h.size() * sizeof(int), cudaMemcpyDeviceToHost);
  std::vector<int> ptr(ny + 1, 0), trs(ntr);
  for (int n = 0; n < ntr; ++n) ptr[kyi_h[n] + 1]++;
  for (int k = 0; k < ny; ++k) ptr[k + 1] += ptr[k];
  {
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (int n = 0; n < ntr; ++n) trs[fill[kyi_h[n]]++] = n;
  }
  // U gathered in ky order (and transposed), the ky of each gathered TR, and the largest
  // number of TRs of any 32 consecutive ky values
  std::vector<float> Ug((size_t)ntr * R), UgT((size_t)ntr * R);
  std::vector<int> kyof(ntr);
  for (int t = 0; t < ntr; ++t)
    for (int r = 0; r < R; ++r) {
      Ug[(size_t)t * R + r] = Uh[(size_t)trs[t] * R + r];
      UgT[(size_t)r * ntr + t] = Uh[(size_t)trs[t] * R + r];
    }
  for (int k = 0; k < ny; ++k)
    for (int t = ptr[k]; t < ptr[k + 1]; ++t) kyof[t] = k;
  for (int k0 = 0; k0 < ny; k0 += 32) L->gram_rows_max = std::max(L->gram_rows_max, ptr[std::min(k0 + 32, ny)] - ptr[k0]);
  for (int k = 0; k < ny; ++k) L->ky_count_max = std::max(L->ky_count_max, ptr[k + 1] - ptr[k]);
  // U by (r, slot, ky): the i-th TR of ky at [r][i][ky], zero past the ky's TRs
  const int kmax = L->ky_count_max;
  std::vector<float> UgS((size_t)R * kmax * ny, 0.f);
  for (int k = 0; k < ny; ++k)
    for (int t = ptr[k]; t < ptr[k + 1]; ++t)
      for (int r = 0; r < R; ++r) UgS[((size_t)r * kmax + (t - ptr[k])) * ny + k] = Uh[(size_t)trs[t] * R + r];
  // the same in slot planes for the specialised column kernels (kmax <= 8): slots 0-3 as
  // float4 [R][ny], then slot 4 as float [R][ny] (kmax 5) or slots 4-7 as float4 [R][ny]
  const int w1 = kmax <= 4 ? 0 : (kmax == 5 ? 1 : 4);
  std::vector<float> UgQ(kmax <= 8 ? (size_t)R * ny * (4 + w1) : 0, 0.f);
  if (kmax <= 8)
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < ny; ++k)
        for (int i = 0; i < kmax; ++i) {
          const float v = UgS[((size_t)r * kmax + i) * ny + k];
          if (i < 4) UgQ[((size_t)r * ny + k) * 4 + i] = v;
          else UgQ[(size_t)R * ny * 4 + ((size_t)r * ny + k) * w1 + (i - 4)] = v;
        }
  // the cancelled readout DFT pair needs nkx == nx; the Gram kernel keeps a ky tile's rows of U
  // in shared memory
  L->full_readout = p->nkx == p->nx && (size_t)L->gram_rows_max * (R + 1) * sizeof(float) <= (size_t)L->smem_optin;
  // factorised phase-encode DFT: ny = 32 N1 with N1 <= 8
  L->fft_y = L->full_readout && ny % 32 == 0 && ny / 32 <= 8;
  // one pair of blocks per image column: ceil(R / 2) x ny values and two copies of the ntr
  // TR-axis sums in each block's shared memory
  L->column_path =
      L->fft_y && R <= 2 * kColMaxRc && column_smem_bytes(ny, R, L->ky_count_max) <= (size_t)L->smem_optin;
  if (L->fft_y) {
    const int n1 = ny / 32;
    std::memset(&L->dft_small, 0, sizeof(DftSmall));
    for (int k = 1; 2 * k < n1; ++k)
      for (int i = 1; 2 * i < n1; ++i) {
        const double ang = 2.0 * M_PI * (double)((k * i) % n1) / (double)n1;
        L->dft_small.c[k - 1][i - 1] = (float)std::cos(ang);
        L->dft_small.s[k - 1][i - 1] = (float)std::sin(ang);
      }
    for (int k = 0; k < n1; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)(2 * n1);
      L->dft_small.wm[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  }
  std::vector<float> M((size_t)ny * R * R, 0.f);
  for (int k = 0; k < ny; ++k)
    for (int a = 0; a < R; ++a)
      for (int b = 0; b < R; ++b) {
        double s = 0.0;
        for (int t = ptr[k]; t < ptr[k + 1]; ++t) s += (double)Uh[(size_t)trs[t] * R + a] * Uh[(size_t)trs[t] * R + b];
        M[((size_t)k * R + a) * R + b] = (float)s;
      }
  // phase-encode DFT operands (K-major real embeddings, split into bf16 hi + lo)
  const size_t nby = (size_t)2 * ny * L->k23;
  std::vector<uint16_t> byh(nby, 0), byl(nby, 0), bah(nby, 0), bal(nby, 0);
  auto put = [](std::vector<uint16_t>& hi, std::vector<uint16_t>& lo, size_t idx, double v) {
    const uint16_t h = host_bf16((float)v);
    hi[idx] = h;
    lo[idx] = host_bf16((float)(v - (double)host_bf16_to_float(h)));
  };
  for (int ky = 0; ky < ny; ++ky)
    for (int iy = 0; iy < ny; ++iy) {
      const long long r = ((long long)ky * iy) % ny;
      const double ang = -2.0 * M_PI * (double)r / (double)ny;
      const double er = std::cos(ang), ei = std::sin(ang);  // Ey = exp(-2 pi i ky iy / ny)
      // forward: output rows 2 ky (+1), inputs 2 iy (+1)
      put(byh, byl, (size_t)(2 * ky) * L->k23 + 2 * iy, er);
      put(byh, byl, (size_t)(2 * ky) * L->k23 + 2 * iy + 1, -ei);
      put(byh, byl, (size_t)(2 * ky + 1) * L->k23 + 2 * iy, ei);
      put(byh, byl, (size_t)(2 * ky + 1) * L->k23 + 2 * iy + 1, er);
      // adjoint (conj, transposed): output rows 2 iy (+1), inputs 2 ky (+1)
      put(bah, bal, (size_t)(2 * iy) * L->k23 + 2 * ky, er);
      put(bah, bal, (size_t)(2 * iy) * L->k23 + 2 * ky + 1, ei);
      put(bah, bal, (size_t)(2 * iy + 1) * L->k23 + 2 * ky, -ei);
      put(bah, bal, (size_t)(2 * iy + 1) * L->k23 + 2 * ky + 1, er);
    }
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const size_t rny = (size_t)R * ny, rnk = (size_t)R * nkx;
  chk(cudaMalloc(&L->U, (size_t)ntr * R * sizeof(float)));
  chk(cudaMalloc(&L->Ug, (size_t)ntr * R * sizeof(float)));
  chk(cudaMalloc(&L->UgT, (size_t)ntr * R * sizeof(float)));
  chk(cudaMalloc(&L->UgS, std::max<size_t>(UgS.size(), 1) * sizeof(float)));
  chk(cudaMalloc(&L->UgQ, std::max<size_t>(UgQ.size(), 4) * sizeof(float)));
  chk(cudaMalloc(&L->kyof, (size_t)ntr * sizeof(int)));
  chk(cudaMalloc(&L->Mky, M.size() * sizeof(float)));
  chk(cudaMalloc(&L->kyptr, ptr.size() * sizeof(int)));
  chk(cudaMalloc(&L->kytr, trs.size() * sizeof(int)));
  chk(cudaMalloc(&L->coef, (size_t)3 * R * p->nv * sizeof(float)));
  chk(cudaMalloc(&L->coef2, (size_t)3 * R * p->nv * sizeof(float)));
  chk(cudaMalloc(&L->gpart, (size_t)((R + 7) / 8) * 4 * p->nv * sizeof(float)));
  if (L->fft_y) chk(cudaMalloc(&L->coefT, (size_t)3 * R * p->nv * sizeof(float)));
  chk(cudaMalloc(&L->a1_hi, rny * L->k1 * 2));
  chk(cudaMalloc(&L->a1_lo, rny * L->k1 * 2));
  chk(cudaMalloc(&L->a23_hi, rnk * L->k23 * 2));
  chk(cudaMalloc(&L->a23_lo, rnk * L->k23 * 2));
  chk(cudaMalloc(&L->a4_hi, rny * L->k4 * 2));
  chk(cudaMalloc(&L->a4_lo, rny * L->k4 * 2));
  chk(cudaMalloc(&L->by_hi, nby * 2));
  chk(cudaMalloc(&L->by_lo, nby * 2));
  chk(cudaMalloc(&L->bya_hi, nby * 2));
  chk(cudaMalloc(&L->bya_lo, nby * 2));
  chk(cudaMalloc(&L->X1, rny * 2 * nkx * sizeof(float)));
  chk(cudaMalloc(&L->H, rnk * 2 * ny * sizeof(float)));
  chk(cudaMalloc(&L->Y3, rnk * 2 * ny * sizeof(float)));
  chk(cudaMalloc(&L->P, rny * 2 * nx * sizeof(float)));
  if (e != cudaSuccess) {
    lowrank_free(L);
    return cuda_fail(e, "low-rank allocation");
  }
  chk(cudaMemcpyAsync(L->U, U_dev, (size_t)ntr * R * sizeof(float), cudaMemcpyDeviceToDevice, st));
  chk(cudaMemcpy(L->Mky, M.data(), M.size() * sizeof(float), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->Ug, Ug.data(), Ug.size() * sizeof(float), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->UgT, UgT.data(), UgT.size() * sizeof(float), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->UgS, UgS.data(), UgS.size() * sizeof(float), cudaMemcpyHostToDevice));
  if (!UgQ.empty()) chk(cudaMemcpy(L->UgQ, UgQ.data(), UgQ.size() * sizeof(float), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->kyof, kyof.data(), kyof.size() * sizeof(int), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->kyptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->kytr, trs.data(), trs.size() * sizeof(int), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->by_hi, byh.data(), nby * 2, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->by_lo, byl.data(), nby * 2, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->bya_hi, bah.data(), nby * 2, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(L->bya_lo, bal.data(), nby * 2, cudaMemcpyHostToDevice));
  // padding columns of the operands must read as zero
  chk(cudaMemset(L->a1_hi, 0, rny * L->k1 * 2));
  chk(cudaMemset(L->a1_lo, 0, rny * L->k1 * 2));
  chk(cudaMemset(L->a23_hi, 0, rnk * L->k23 * 2));
  chk(cudaMemset(L->a23_lo, 0, rnk * L->k23 * 2));
  chk(cudaMemset(L->a4_hi, 0, rny * L->k4 * 2));
  chk(cudaMemset(L->a4_lo, 0, rny * L->k4 * 2));
  chk(make_split_operand(&L->op_a1, L->a1_hi, L->a1_lo, (int)rny, 2 * nx, L->k1, true));
  chk(make_split_operand(&L->op_a23, L->a23_hi, L->a23_lo, (int)rnk, 2 * ny, L->k23, true));
  chk(make_split_operand(&L->op_a4, L->a4_hi, L->a4_lo, (int)rny, 2 * nkx, L->k4, true));
  chk(make_split_operand(&L->op_by, L->by_hi, L->by_lo, 2 * ny, 2 * ny, L->k23, false));
  chk(make_split_operand(&L->op_bya, L->bya_hi, L->bya_lo, 2 * ny, 2 * ny, L->k23, false));
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    lowrank_free(L);
    return cuda_fail(e, "low-rank set-up");
  }
  p->bytes += (int64_t)((size_t)2 * ntr * R * 4 + M.size() * 4 + (size_t)6 * R * p->nv * 4 +
                        2 * 2 * (rny * L->k1 + rnk * L->k23 + rny * L->k4) + 4 * nby * 2 +
                        (rny * 2 * nkx + 2 * rnk * 2 * ny + rny * 2 * nx) * 4);
  p->lr = L;
  return MRSTAT_OK;
}

// ---- the three stages shared by the products ----
static int lr_forward_dft(Plan* p, const int* gate, cudaStream_t st) {
  LowRank& L = *p->lr;
  const int R = L.R, nx = p->nx, ny = p->ny, nkx = p->nkx;
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_XDFT, st);
    e = launch_tc_gemm(L.op_a1, p->tc[1], L.X1, R * ny, 2 * nkx, 2 * nx, 2 * nkx, 3, gate, p->dev_err, st);
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_VECTOR, st);
    dim3 grid((nkx + 31) / 32, (ny + 31) / 32, R);
    lr_transpose_split_kernel<<<grid, dim3(32, 8), 0, st>>>(L.X1, ny, nkx, (__nv_bfloat16*)L.a23_hi,
                                                            (__nv_bfloat16*)L.a23_lo, L.k23, gate);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_XDFT, st);
    e = launch_tc_gemm(L.op_a23, L.op_by, L.H, R * nkx, 2 * ny, 2 * ny, 2 * ny, 3, gate, p->dev_err, st);
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "low-rank DFT");
}

static int lr_adjoint_dft_and_final(Plan* p, float* g, const int* gate, cudaStream_t st) {
  LowRank& L = *p->lr;
  const int R = L.R, nx = p->nx, ny = p->ny, nkx = p->nkx;
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_XDFT_ADJ, st);
    e = launch_tc_gemm(L.op_a23, L.op_bya, L.Y3, R * nkx, 2 * ny, 2 * ny, 2 * ny, 3, gate, p->dev_err, st);
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_VECTOR, st);
    dim3 grid((ny + 31) / 32, (nkx + 31) / 32, R);
    lr_transpose_split_kernel<<<grid, dim3(32, 8), 0, st>>>(L.Y3, nkx, ny, (__nv_bfloat16*)L.a4_hi,
                                                            (__nv_bfloat16*)L.a4_lo, L.k4, gate);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_XDFT_ADJ, st);
    e = launch_tc_gemm(L.op_a4, p->tc[3], L.P, R * ny, 2 * nx, 2 * nkx, 2 * nx, 3, gate, p->dev_err, st);
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_JHW_DOT, st);
    lr_final_kernel<<<(p->nv + 255) / 256, 256, 0, st>>>(L.P, L.coef, p->rho, p->maskf, nx, ny, p->nv, R, g, gate);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "low-rank adjoint DFT");
}

static int lr_prep(Plan* p, const float* v, const int* gate, cudaStream_t st) {
  LowRank& L = *p->lr;
  Span sp(p, MRSTAT_K_YCONTRACT, st);
  lr_prep_jvp_kernel<<<(p->nv + 255) / 256, 256, 0, st>>>(v, L.coef, p->rho, p->maskf, p->nx, p->ny, p->nv, L.R,
                                                          (__nv_bfloat16*)L.a1_hi, (__nv_bfloat16*)L.a1_lo, L.k1,
                                                          gate);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "low-rank prep");
}

int lowrank_jvp(Plan* p, const float* v, float2* jv, cudaStream_t st) {
  LowRank& L = *p->lr;
  int s = lr_prep(p, v, p->gate, st);
  if (s == MRSTAT_OK) s = lr_forward_dft(p, p->gate, st);
  if (s != MRSTAT_OK) return s;
  Span sp(p, MRSTAT_K_VECTOR, st);
  dim3 grid((p->nkx + 127) / 128, p->ntr);
  lr_expand_kernel<<<grid, 128, 0, st>>>(L.H, L.U, p->kyi, p->ntr, p->nkx, p->ny, L.R, jv);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "low-rank expand");
}

int lowrank_jhw(Plan* p, const float2* w, float* g, cudaStream_t st) {
  LowRank& L = *p->lr;
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    lr_gather_kernel<<<p->ny, 128, 0, st>>>(w, L.U, L.kyptr, L.kytr, p->nkx, L.R, (__nv_bfloat16*)L.a23_hi,
                                            (__nv_bfloat16*)L.a23_lo, L.k23);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "low-rank gather");
  }
  return lr_adjoint_dft_and_final(p, g, p->gate, st);
}

// SPLIT: write G as the split-BF16 operand of the adjoint phase-encode GEMM; else as
// float2 rows [(ix, r)][ky] into gout (the FFT path)
template <int R, bool SPLIT>
static cudaError_t launch_gram_t(const Plan& p, const LowRank& L, float2* gout, const int* gate, cudaStream_t st) {
  const size_t sm = (size_t)L.gram_rows_max * (R + 1) * sizeof(float);
  const dim3 grid((p.ny + 31) / 32, (p.nx + 7) / 8);
  __nv_bfloat16* hi = (__nv_bfloat16*)L.a23_hi;
  __nv_bfloat16* lo = (__nv_bfloat16*)L.a23_lo;
  if (L.ky_count_max <= kGramShort) {
    cudaError_t e = cudaFuncSetAttribute(lr_gram_short_kernel<R, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    lr_gram_short_kernel<R, SPLIT><<<grid, dim3(32, 8), sm, st>>>(L.H, 2 * p.ny, L.Ug, L.kyptr, p.nx, p.ny, hi, lo,
                                                                   L.k23, gout, gate);
  } else {
    cudaError_t e =
        cudaFuncSetAttribute(lr_gram_t_kernel<R, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    lr_gram_t_kernel<R, SPLIT><<<grid, dim3(32, 8), sm, st>>>(L.H, 2 * p.ny, L.Ug, L.kyptr, p.nx, p.ny, hi, lo, L.k23,
                                                               gout, gate);
  }
  return cudaGetLastError();
}

template <bool SPLIT>
static cudaError_t launch_gram(const Plan& p, const LowRank& L, float2* gout, const int* gate, cudaStream_t st) {
  switch (L.R) {
    case 8: return launch_gram_t<8, SPLIT>(p, L, gout, gate, st);
    case 16: return launch_gram_t<16, SPLIT>(p, L, gout, gate, st);
    case 24: return launch_gram_t<24, SPLIT>(p, L, gout, gate, st);
    default: return launch_gram_t<32, SPLIT>(p, L, gout, gate, st);
  }
}

// J^H J v for a fully sampled readout: prep -> phase-encode DFT -> Gram through the TR axis
// -> adjoint phase-encode DFT -> final, times nx for the cancelled readout DFT pair.
static int lowrank_jhjv_full_readout(Plan* p, const float* v, float* out, double* vdot, cudaStream_t st) {
  LowRank& L = *p->lr;
  const int R = L.R, nx = p->nx, ny = p->ny;
  const int* gate = p->gate;
  const dim3 tiles((nx + 31) / 32, (ny + 31) / 32), tb(32, 8);
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_YCONTRACT, st);
    const dim3 grid(tiles.x, tiles.y, (R + 3) / 4);
    lr_prep_t_kernel<<<grid, tb, 0, st>>>(v, L.coef, p->rho, p->maskf, nx, ny, p->nv, R, (__nv_bfloat16*)L.a23_hi,
                                          (__nv_bfloat16*)L.a23_lo, L.k23, gate);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_XDFT, st);
    e = launch_tc_gemm(L.op_a23, L.op_by, L.H, R * nx, 2 * ny, 2 * ny, 2 * ny, 3, gate, p->dev_err, st);
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = launch_gram<true>(*p, L, nullptr, gate, st);
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_XDFT_ADJ, st);
    e = launch_tc_gemm(L.op_a23, L.op_bya, L.Y3, R * nx, 2 * ny, 2 * ny, 2 * ny, 3, gate, p->dev_err, st);
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_JHW_DOT, st);
    const int nchunk = (R + 7) / 8;
    const dim3 t16((nx + 15) / 16, (ny + 15) / 16, nchunk);
    lr_final_t_kernel<<<t16, dim3(16, 16), 0, st>>>(L.Y3, 2 * ny, L.coef, p->rho, nx, ny, p->nv, R, L.gpart, gate);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      const int64_t n4 = 4 * (int64_t)p->nv;
      // one float64 partial per block in the plan's reduction scratch
      const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n4 + kSumThreads - 1) / kSumThreads, kRedBlocks));
      lr_final_sum_kernel<<<blocks, kSumThreads, 0, st>>>(L.gpart, nchunk, p->maskf, p->nv, (float)nx, out, gate, v,
                                                          p->red, p->ticket, vdot);
      e = cudaGetLastError();
    }
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "low-rank J^H J v");
}

// The image-column copy of the coefficients, refreshed when they changed.
static cudaError_t ensure_coef_columns(Plan* p, cudaStream_t st) {
  LowRank& L = *p->lr;
  if (!L.coefT_dirty && L.coefT_src == L.coef) return cudaSuccess;
  const dim3 grid((p->nx + 31) / 32, (p->ny + 31) / 32, 3 * L.R);
  lr_coef_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(L.coef, p->nx, p->ny, L.coefT);
  L.coefT_src = L.coef;
  L.coefT_dirty = false;
  return cudaGetLastError();
}

// Shapes with a compiled specialisation of the column kernels (kmax TR slots per ky and
// R / 2 basis functions per block fixed at compile time): 224 rows with five or eight TRs
// per phase-encode line and 256 rows with five, rank 32.  Others take the generic kernels.
enum ColSpec { kSpecGeneric, kSpec7x5, kSpec7x8, kSpec8x5 };

static ColSpec col_spec(const Plan* p) {
  const LowRank& L = *p->lr;
  if (L.R != 32) return kSpecGeneric;
  if (p->ny == 224 && L.ky_count_max == 5) return kSpec7x5;
  if (p->ny == 224 && L.ky_count_max == 8) return kSpec7x8;
  if (p->ny == 256 && L.ky_count_max == 5) return kSpec8x5;
  return kSpecGeneric;
}

template <int N1, int KM, int RCT>
static cudaError_t launch_column_k(Plan* p, const float* v, double* vdot, double* vv, float* out, cudaStream_t st) {
  LowRank& L = *p->lr;
  const int nx = p->nx, ny = p->ny, R = L.R;
  const size_t sm = column_smem_bytes(ny, R, L.ky_count_max);
  cudaError_t e =
      cudaFuncSetAttribute(lr_jhjv_column_kernel<N1, KM, RCT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // two blocks per column (cluster pairs), one float64 partial per block
  const int grid = 2 * std::min(nx, kRedBlocks / 2);
  // programmatic dependent launch: the set-up above the kernel's pdl_wait overlaps the
  // tail of the previous launch in the stream
  return launch_pdl(lr_jhjv_column_kernel<N1, KM, RCT>, dim3(grid), dim3(kColThreads), sm, st, L.dft_small, v,
                    L.coefT, p->rho, p->maskf, p->roots, KM > 0 ? L.UgQ : L.UgS, L.ky_count_max, nx, ny, p->nv, R, (float)nx, out,
                    p->red, p->ticket, vdot, vv, p->gate);
}

template <int N1>
static cudaError_t launch_column_t(Plan* p, const float* v, double* vdot, double* vv, float* out, cudaStream_t st) {
  switch (col_spec(p)) {
    case kSpec7x5: return launch_column_k<7, 5, 0>(p, v, vdot, vv, out, st);
    case kSpec7x8: return launch_column_k<7, 8, 0>(p, v, vdot, vv, out, st);
    case kSpec8x5: return launch_column_k<8, 5, 0>(p, v, vdot, vv, out, st);
    default: return launch_column_k<N1, 0, 0>(p, v, vdot, vv, out, st);
  }
}

static cudaError_t launch_column(Plan* p, const float* v, double* vdot, double* vv, float* out, cudaStream_t st) {
  switch (p->ny / 32) {
    case 1: return launch_column_t<1>(p, v, vdot, vv, out, st);
    case 2: return launch_column_t<2>(p, v, vdot, vv, out, st);
    case 3: return launch_column_t<3>(p, v, vdot, vv, out, st);
    case 4: return launch_column_t<4>(p, v, vdot, vv, out, st);
    case 5: return launch_column_t<5>(p, v, vdot, vv, out, st);
    case 6: return launch_column_t<6>(p, v, vdot, vv, out, st);
    case 7: return launch_column_t<7>(p, v, vdot, vv, out, st);
    default: return launch_column_t<8>(p, v, vdot, vv, out, st);
  }
}

// A persistent column kernel: one cluster of two blocks per image column, all resident at
// once (cooperative launch).  With launch = false only checks that every cluster fits.
template <typename... KArgs, typename... Args>
static cudaError_t launch_persistent_columns(Plan* p, void (*kernel)(KArgs...), size_t sm, int clusters, bool launch,
                                             cudaStream_t st, Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * clusters);
  cfg.blockDim = dim3(kColThreads);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  if (!launch) {
    // every cluster must be resident at once (the grid waits wait for all of them)
    int max_clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&max_clusters, kernel, &cfg);
    if (e != cudaSuccess) return e;
    return max_clusters >= clusters ? cudaSuccess : cudaErrorCooperativeLaunchTooLarge;
  }
  e = cudaMemsetAsync(p->cg_bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int N1, int KM, int RCT>
static cudaError_t launch_cg_columns_k(Plan* p, const float* rhs, float* x, int iters, bool launch, cudaStream_t st) {
  LowRank& L = *p->lr;
  // one cluster per image column when all of them fit at once, else two columns per cluster
  auto go = [&](auto kernel, int cpc, bool now) {
    const size_t sm = cg_column_smem_bytes(p->ny, L.R, L.ky_count_max, cpc);
    return launch_persistent_columns(p, kernel, sm, (p->nx + cpc - 1) / cpc, now, st, L.dft_small, rhs, x,
                                     (const float*)L.coefT, (const float2*)p->rho, (const float*)p->maskf,
                                     (const float2*)p->roots, (const float*)(KM > 0 ? L.UgQ : L.UgS), L.ky_count_max, p->nx, p->nv,
                                     L.R, (float)p->nx, iters, p->grid_stall_block, p->red, p->cg_bar, p->cg_s,
                                     p->cg_frozen, p->dev_err);
  };
  cudaError_t e = go(lr_cg_columns_kernel<N1, KM, RCT, 1>, 1, false);
  if (e == cudaSuccess) return launch ? go(lr_cg_columns_kernel<N1, KM, RCT, 1>, 1, true) : e;
  if constexpr (KM > 0) {  // two columns per cluster: compiled for the specialised shapes only
    cudaGetLastError();
    e = go(lr_cg_columns_kernel<N1, KM, RCT, 2>, 2, false);
    if (e != cudaSuccess || !launch) return e;
    return go(lr_cg_columns_kernel<N1, KM, RCT, 2>, 2, true);
  }
  return e;
}

template <int N1>
static cudaError_t launch_cg_columns_t(Plan* p, const float* rhs, float* x, int iters, bool launch, cudaStream_t st) {
  switch (col_spec(p)) {
    case kSpec7x5: return launch_cg_columns_k<7, 5, 0>(p, rhs, x, iters, launch, st);
    case kSpec7x8: return launch_cg_columns_k<7, 8, 0>(p, rhs, x, iters, launch, st);
    case kSpec8x5: return launch_cg_columns_k<8, 5, 0>(p, rhs, x, iters, launch, st);
    default: return launch_cg_columns_k<N1, 0, 0>(p, rhs, x, iters, launch, st);
  }
}

static cudaError_t launch_cg_columns(Plan* p, const float* rhs, float* x, int iters, bool launch, cudaStream_t st) {
  switch (p->ny / 32) {
    case 1: return launch_cg_columns_t<1>(p, rhs, x, iters, launch, st);
    case 2: return launch_cg_columns_t<2>(p, rhs, x, iters, launch, st);
    case 3: return launch_cg_columns_t<3>(p, rhs, x, iters, launch, st);
    case 4: return launch_cg_columns_t<4>(p, rhs, x, iters, launch, st);
    case 5: return launch_cg_columns_t<5>(p, rhs, x, iters, launch, st);
    case 6: return launch_cg_columns_t<6>(p, rhs, x, iters, launch, st);
    case 7: return launch_cg_columns_t<7>(p, rhs, x, iters, launch, st);
    default: return launch_cg_columns_t<8>(p, rhs, x, iters, launch, st);
  }
}

struct SteihaugArgs {
  double delta, rel_tol;
  int max_steps;
  double* sc;
  int* si;
};

template <int N1, int KM, int RCT>
static cudaError_t launch_st_columns_k(Plan* p, const float* g, float* z, const SteihaugArgs& a, bool launch,
                                       cudaStream_t st) {
  LowRank& L = *p->lr;
  const size_t sm = st_column_smem_bytes(p->ny, L.R, L.ky_count_max);
  return launch_persistent_columns(p, lr_steihaug_columns_kernel<N1, KM, RCT>, sm, p->nx, launch, st, L.dft_small, g, z,
                                   (const float*)L.coefT, (const float2*)p->rho, (const float*)p->maskf,
                                   (const float2*)p->roots, (const float*)(KM > 0 ? L.UgQ : L.UgS), L.ky_count_max, p->nx, p->nv, L.R,
                                   (float)p->nx, a.delta, a.rel_tol, a.max_steps, a.sc, a.si, p->grid_stall_block,
                                   p->red, p->cg_bar, p->dev_err);
}

template <int N1>
static cudaError_t launch_st_columns_t(Plan* p, const float* g, float* z, const SteihaugArgs& a, bool launch,
                                       cudaStream_t st) {
  switch (col_spec(p)) {
    case kSpec7x5: return launch_st_columns_k<7, 5, 0>(p, g, z, a, launch, st);
    case kSpec7x8: return launch_st_columns_k<7, 8, 0>(p, g, z, a, launch, st);
    case kSpec8x5: return launch_st_columns_k<8, 5, 0>(p, g, z, a, launch, st);
    default: return launch_st_columns_k<N1, 0, 0>(p, g, z, a, launch, st);
  }
}

static cudaError_t launch_st_columns(Plan* p, const float* g, float* z, const SteihaugArgs& a, bool launch,
                                     cudaStream_t st) {
  switch (p->ny / 32) {
    case 1: return launch_st_columns_t<1>(p, g, z, a, launch, st);
    case 2: return launch_st_columns_t<2>(p, g, z, a, launch, st);
    case 3: return launch_st_columns_t<3>(p, g, z, a, launch, st);
    case 4: return launch_st_columns_t<4>(p, g, z, a, launch, st);
    case 5: return launch_st_columns_t<5>(p, g, z, a, launch, st);
    case 6: return launch_st_columns_t<6>(p, g, z, a, launch, st);
    case 7: return launch_st_columns_t<7>(p, g, z, a, launch, st);
    default: return launch_st_columns_t<8>(p, g, z, a, launch, st);
  }
}

// Steihaug's truncated CG on the low-rank Gauss-Newton matrix in one persistent launch
// where the column kernel applies and every cluster fits on the device at once; returns
// false (and nothing was launched) otherwise.  On return z holds the step and sc / si the
// solver's scalars (S_RR .. S_ZZ, I_EXIT, I_STEPS; I_ACTIVE = I_CONT = 0).
bool lowrank_steihaug_persistent(Plan* p, const float* g, float* z, double delta, int max_steps, double rel_tol,
                                 double* sc, int* si, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  if (p->lr == nullptr || !p->lr->active || !p->lr->column_path || p->cg_bar == nullptr || max_steps < 0)
    return false;
  // two parity buffers of eight partials per block in p->red; a grid counter that
  // reaches 2 nx (max_steps + 1)
  const int64_t G = 2 * (int64_t)p->nx;
  if (16 * G > kRedSlots || G > 2 * kColThreads || G * ((int64_t)max_steps + 1) >= (int64_t)1 << 31)
    return false;
  const SteihaugArgs a = {delta, rel_tol, max_steps, sc, si};
  cudaError_t e = launch_st_columns(p, g, z, a, false, st);
  if (e != cudaSuccess) {
    cudaGetLastError();  // does not fit (or cannot be asked): the caller iterates launch by launch
    return false;
  }
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = ensure_coef_columns(p, st);
  }
  if (e != cudaSuccess) {
    *err = e;
    return true;
  }
  {
    Span sp(p, MRSTAT_K_JHW_DOT, st);
    e = launch_st_columns(p, g, z, a, true, st);
  }
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorInvalidConfiguration || e == cudaErrorNotSupported) {
    cudaGetLastError();  // refused at launch (nothing ran): iterate launch by launch
    return false;
  }
  *err = e;
  return true;
}

// Fixed-count CG on the low-rank Gauss-Newton matrix in one persistent launch where the
// column kernel applies and every cluster fits on the device at once; returns false (and
// nothing was launched) otherwise.
bool lowrank_cg_fixed_persistent(Plan* p, const float* rhs, float* x, int iters, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  if (p->lr == nullptr || !p->lr->active || !p->lr->column_path || iters < 1 || p->cg_bar == nullptr) return false;
  // two parity buffers of two partials per block in p->red, and a grid counter that
  // reaches 2 nx iters
  const int64_t G = 2 * (int64_t)p->nx;
  if (4 * G > kRedSlots || G > 2 * kColThreads || G * iters >= (int64_t)1 << 31) return false;
  cudaError_t e = launch_cg_columns(p, rhs, x, iters, false, st);
  if (e != cudaSuccess) {
    cudaGetLastError();  // does not fit (or cannot be asked): the caller iterates launch by launch
    return false;
  }
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = ensure_coef_columns(p, st);
  }
  if (e != cudaSuccess) {
    *err = e;
    return true;
  }
  {
    Span sp(p, MRSTAT_K_JHW_DOT, st, iters, 1);  // one launch, counted as `iters` products
    e = launch_cg_columns(p, rhs, x, iters, true, st);
  }
  if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorInvalidConfiguration || e == cudaErrorNotSupported) {
    cudaGetLastError();  // refused at launch (nothing ran): iterate launch by launch
    return false;
  }
  *err = e;
  return true;
}

// J^H J v for a fully sampled readout and ny = 32 N1: the column kernel (factorised
// phase-encode DFT, Gram through the TR axis, adjoint, contraction and <v, J^H J v>), times
// nx for the cancelled readout DFT pair.
static int lowrank_jhjv_columns(Plan* p, const float* v, float* out, double* vdot, double* vv, cudaStream_t st) {
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = ensure_coef_columns(p, st);
  }
  if (e == cudaSuccess) {
    Span sp(p, MRSTAT_K_JHW_DOT, st);
    e = launch_column(p, v, vdot, vv, out, st);
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "low-rank J^H J v (column kernel)");
}

int lowrank_jhjv(Plan* p, const float* v, float* out, cudaStream_t st, double* vdot, double* vv) {
  LowRank& L = *p->lr;
  if (vv != nullptr && vdot == nullptr) {
    const int s = lowrank_jhjv(p, v, out, st);
    if (s != MRSTAT_OK) return s;
    const cudaError_t e = do_dot(p, v, v, 4 * (int64_t)p->nv, vv, st);
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "dot launch");
  }
  if (L.column_path) return lowrank_jhjv_columns(p, v, out, vdot, vv, st);
  if (vv != nullptr) {
    const int s = lowrank_jhjv(p, v, out, st, vdot);
    if (s != MRSTAT_OK) return s;
    const cudaError_t e = do_dot(p, v, v, 4 * (int64_t)p->nv, vv, st);
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "dot launch");
  }
  if (L.full_readout) return lowrank_jhjv_full_readout(p, v, out, vdot, st);
  if (vdot != nullptr) {
    const int s = lowrank_jhjv(p, v, out, st, nullptr);
    if (s != MRSTAT_OK) return s;
    const cudaError_t e = do_dot(p, v, out, 4 * (int64_t)p->nv, vdot, st);
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "dot launch");
  }
  int s = lr_prep(p, v, p->gate, st);
  if (s == MRSTAT_OK) s = lr_forward_dft(p, p->gate, st);
  if (s != MRSTAT_OK) return s;
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    lr_gram_kernel<<<p->ny, 128, (size_t)L.R * L.R * sizeof(float), st>>>(
        L.H, L.Mky, p->nkx, p->ny, L.R, (__nv_bfloat16*)L.a23_hi, (__nv_bfloat16*)L.a23_lo, L.k23, p->gate);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "low-rank Gram");
  }
  return lr_adjoint_dft_and_final(p, out, p->gate, st);
}

cudaError_t lowrank_train_matrix(const float4* D, int ns, int nq, int ntr, float2* Y, float2* Yt,
                                 cudaStream_t st) {
  const int64_t total = (int64_t)ntr * 3 * ns;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  lr_train_matrix_kernel<<<blocks, 256, 0, st>>>(D, ns, nq, ntr, Y, Yt);
  return cudaGetLastError();
}

}  // namespace mrstat
