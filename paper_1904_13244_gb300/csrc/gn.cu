// Inexact Gauss-Newton reconstruction (Algorithm 6) with a Steihaug trust region,
// the CGLS proton-density initialisation and the mask (Methods, "Reconstructions").
//
// The truncated CG runs entirely on the device: its float64 scalars live in a small
// device block, the last block of each reduction takes the Steihaug decisions (negative
// curvature, trust boundary, tolerance, iteration count) from the sums it has just
// formed, and once CG has stopped the product kernels return at once through the plan's
// gate flag.  The host waits
// once per outer iteration, to evaluate the trust-region ratio in float64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include <type_traits>

#include "internal.cuh"
#include "reduce.cuh"
#include "steihaug.cuh"

namespace mrstat {
namespace {


constexpr int kT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* ws /* [NV][8] */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) ws[k * 8 + w] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = (threadIdx.x < 8) ? ws[k * 8 + threadIdx.x] : 0.0;
    if (w == 0) x = warp_sum(x);
    v[k] = x;
  }
  __syncthreads();
}

// After thread 0 of every block stored its NV partials in part[k * gridDim.x + block], the
// last block sums them in block order into out[0..NV) and resets the ticket; returns true
// in the last block (where thread 0 may then act on the sums).
template <int NV>
__device__ __forceinline__ bool finish_n(double* part, unsigned* ticket, double* out, double* ws) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kT) s += ((volatile double*)part)[k * gridDim.x + i];
    v[k] = s;
  }
  block_sum_n<NV>(v, ws);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = v[k];
    *ticket = 0u;
  }
  return true;
}

// About four elements per thread (float32 partial sums over those, float64 from the warp
// level up), at most kRedBlocks blocks: the plan's reduction scratch holds five partial
// vectors of that length.
int grid_for(int64_t n) {
  int64_t b = (n + 4 * kT - 1) / (4 * kT);
  if (b > kRedBlocks) b = kRedBlocks;
  return (int)(b > 0 ? b : 1);
}

#define GRID_STRIDE(i, n) \
  _Pragma("unroll 4") for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kT)

// r = s - d (complex as float pairs, n floats) and f = 1/2 ||r||^2
__global__ void __launch_bounds__(kT)
residual_kernel(const float* __restrict__ s, const float* __restrict__ d, float* __restrict__ r,
                int64_t n, double* part, unsigned* ticket, double* f) {
  __shared__ double ws[8];
  float a = 0.f;
  GRID_STRIDE(i, n) {
    const float v = s[i] - d[i];
    r[i] = v;
    a = fmaf(v, v, a);
  }
  double acc[1] = {(double)a};
  block_sum_n<1>(acc, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = 0.5 * acc[0];
  finish_n<1>(part, ticket, f, ws);
}

// ||alpha * mask||^2 over all npar parameter rows
__global__ void __launch_bounds__(kT)
masked_norm_kernel(const float* __restrict__ alpha, const uint8_t* __restrict__ mask, int nv, int npar,
                   double* part, unsigned* ticket, double* out) {
  __shared__ double ws[8];
  double acc[1] = {0.0};
  GRID_STRIDE(j, nv) {
    if (mask[j]) {
      for (int k = 0; k < npar; ++k) {
        const double a = alpha[k * (int64_t)nv + j];
        acc[0] = fma(a, a, acc[0]);
      }
    }
  }
  block_sum_n<1>(acc, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
  finish_n<1>(part, ticket, out, ws);
}

// Steihaug initialisation: z = 0, res = g, dir = -g, rr = g.g
__global__ void __launch_bounds__(kT)
st_init_kernel(const float* __restrict__ g, float* __restrict__ z, float* __restrict__ res,
               float* __restrict__ dir, int64_t n, double* part, unsigned* ticket, double* rr) {
  __shared__ double ws[8];
  float a = 0.f;
  GRID_STRIDE(i, n) {
    const float v = g[i];
    z[i] = 0.f;
    res[i] = v;
    dir[i] = -v;
    a = fmaf(v, v, a);
  }
  double acc[1] = {(double)a};
  block_sum_n<1>(acc, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
  finish_n<1>(part, ticket, rr, ws);
}

__global__ void st_start_kernel(double* sc, int* si) {
  const double rr = sc[S_RR];
  // the sums the first step decision needs besides dir.B dir: res = g, dir = -g, z = 0
  sc[S_RD] = -rr;
  sc[S_DD] = rr;
  sc[S_ZD] = 0.0;
  sc[S_ZZ] = 0.0;
  sc[S_GNORM] = sqrt(rr);
  sc[S_MVAL] = 0.0;
  sc[S_COEF] = 0.0;
  sc[S_BETA] = 0.0;
  si[I_STEPS] = 0;
  si[I_CONT] = 0;
  si[I_ACTIVE] = rr > 0.0 ? 1 : 0;
  si[I_EXIT] = rr > 0.0 ? MRSTAT_CG_MAX_ITER : MRSTAT_CG_ZERO_GRADIENT;
}

__device__ __forceinline__ float4 ld4(const float* p, int64_t i) { return reinterpret_cast<const float4*>(p)[i]; }
__device__ __forceinline__ void st4(float* p, int64_t i, float4 v) { reinterpret_cast<float4*>(p)[i] = v; }
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {  // a x + y
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float dot4(float4 a, float4 b, float s) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
}

// One Steihaug iteration after the product q = B dir (which also left dir.q in S_DBD):
// the step decision from S_DBD..S_ZZ, then z += coef dir and, while continuing,
// res += coef q and rr_new = res.res.  Every block takes the same decision from the same
// sums (read before its ticket); the last block commits it, adds rr_new and takes the
// tolerance and iteration-count test.  Vectors as float4 over [0, 4 n4), then element by
// element; a block's first loads are issued before its thread 0 reads the scalars.
__global__ void __launch_bounds__(kT)
st_update_kernel(float* __restrict__ z, float* __restrict__ res, const float* __restrict__ dir,
                 const float* __restrict__ q, int64_t n, int64_t n4, double* sc, int* si, double delta,
                 double rel_tol, int max_steps, double* part, unsigned* ticket) {
  red::pdl_trigger();
  red::pdl_wait();  // q, the sums and the flags come from the previous launches
  const int64_t t0 = blockIdx.x * (int64_t)kT + threadIdx.x, stride = (int64_t)gridDim.x * kT;
  float4 zv, rv, dv, qv;
  if (t0 < n4) {
    zv = ld4(z, t0);
    rv = ld4(res, t0);
    dv = ld4(dir, t0);
    qv = ld4(q, t0);
  }
  __shared__ double lsc[S_COUNT];
  __shared__ int lsi[I_COUNT];
  __shared__ int s_go;
  if (threadIdx.x == 0) {
    for (int k = 0; k < S_COUNT; ++k) lsc[k] = sc[k];
    for (int k = 0; k < I_COUNT; ++k) lsi[k] = si[k];
    s_go = lsi[I_ACTIVE] != 0;  // CG stopped before this step: nothing to do, nothing to commit
    if (s_go) st_step(lsc, lsi, delta);
  }
  __syncthreads();
  if (!s_go) return;
  const float c = (float)lsc[S_COEF];
  const int cont = lsi[I_CONT];
  float sf = 0.f;
  for (int64_t i = t0; i < n4; i += stride) {
    if (i != t0) {
      zv = ld4(z, i);
      rv = ld4(res, i);
      dv = ld4(dir, i);
      qv = ld4(q, i);
    }
    st4(z, i, axpy4(c, dv, zv));
    if (cont) {
      rv = axpy4(c, qv, rv);
      st4(res, i, rv);
      sf = dot4(rv, rv, sf);
    }
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
    z[i] = fmaf(c, dir[i], z[i]);
    if (cont) {
      const float r = fmaf(c, q[i], res[i]);
      res[i] = r;
      sf = fmaf(r, r, sf);
    }
  }
  __shared__ double ws[8];
  double acc[1] = {(double)sf};
  block_sum_n<1>(acc, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
  if (finish_n<1>(part, ticket, sc + S_RR_NEW, ws) && threadIdx.x == 0) {
    sc[S_MVAL] = lsc[S_MVAL];
    sc[S_COEF] = lsc[S_COEF];
    si[I_STEPS] = lsi[I_STEPS];
    si[I_CONT] = lsi[I_CONT];
    si[I_ACTIVE] = lsi[I_ACTIVE];
    si[I_EXIT] = lsi[I_EXIT];
    if (cont) st_beta(sc, si, rel_tol, max_steps);
  }
}

// dir = -res + beta dir while CG continues, and the sums of the next step decision:
// res.dir, dir.dir, z.dir, z.z into S_RD..S_ZZ (dir.B dir comes with the next product)
__global__ void __launch_bounds__(kT)
st_dir_kernel(float* __restrict__ dir, const float* __restrict__ res, const float* __restrict__ z, int64_t n,
              int64_t n4, double* sc, const int* __restrict__ si, double* part, unsigned* ticket) {
  red::pdl_trigger();
  red::pdl_wait();  // res, z and the flags come from the update launch
  const int64_t t0 = blockIdx.x * (int64_t)kT + threadIdx.x, stride = (int64_t)gridDim.x * kT;
  float4 dv, rv, zv;
  if (t0 < n4) {
    dv = ld4(dir, t0);
    rv = ld4(res, t0);
    zv = ld4(z, t0);
  }
  __shared__ float s_beta;
  __shared__ int s_go;
  if (threadIdx.x == 0) {
    s_go = si[I_CONT] != 0 && si[I_ACTIVE] != 0;
    s_beta = (float)sc[S_BETA];
  }
  __syncthreads();
  if (!s_go) return;
  const float beta = s_beta;
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  for (int64_t i = t0; i < n4; i += stride) {
    if (i != t0) {
      dv = ld4(dir, i);
      rv = ld4(res, i);
      zv = ld4(z, i);
    }
    dv = axpy4(beta, dv, make_float4(-rv.x, -rv.y, -rv.z, -rv.w));
    st4(dir, i, dv);
    a[0] = dot4(rv, dv, a[0]);
    a[1] = dot4(dv, dv, a[1]);
    a[2] = dot4(zv, dv, a[2]);
    a[3] = dot4(zv, zv, a[3]);
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
    const float d = fmaf(beta, dir[i], -res[i]), r = res[i], zz = z[i];
    dir[i] = d;
    a[0] = fmaf(r, d, a[0]);
    a[1] = fmaf(d, d, a[1]);
    a[2] = fmaf(zz, d, a[2]);
    a[3] = fmaf(zz, zz, a[3]);
  }
  __shared__ double ws[4 * 8];
  double acc[4] = {(double)a[0], (double)a[1], (double)a[2], (double)a[3]};
  block_sum_n<4>(acc, ws);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) part[k * gridDim.x + blockIdx.x] = acc[k];
  }
  finish_n<4>(part, ticket, sc + S_RD, ws);
}

__device__ __forceinline__ float reflect(float x, float lo, float hi) {
  if (x > hi) x = 2.f * hi - x;
  if (x < lo) x = 2.f * lo - x;
  return fminf(fmaxf(x, lo), hi);
}

// trial = alpha + z inside the mask, with ln T1, ln T2 (and B1) reflected into their box
__global__ void trial_kernel(const float* __restrict__ alpha, const float* __restrict__ z,
                             const uint8_t* __restrict__ mask, int nv, int npar, float lt1a, float lt1b,
                             float lt2a, float lt2b, float b1a, float b1b, float* __restrict__ trial) {
  GRID_STRIDE(j, nv) {
    const bool on = mask[j] != 0;
    for (int k = 0; k < npar; ++k) {
      const int64_t i = k * (int64_t)nv + j;
      float v = alpha[i];
      if (on) {
        v += z[i];
        if (k == 0) v = reflect(v, lt1a, lt1b);
        if (k == 1) v = reflect(v, lt2a, lt2b);
        if (k == 4) v = reflect(v, b1a, b1b);
      }
      trial[i] = v;
    }
  }
}

__global__ void z_norm_kernel(const float* __restrict__ z, int64_t n, double* part, unsigned* ticket,
                              double* out) {
  __shared__ double ws[8];
  float a = 0.f;
  GRID_STRIDE(i, n) a = fmaf(z[i], z[i], a);
  double acc[1] = {(double)a};
  block_sum_n<1>(acc, ws);
  if (threadIdx.x == 0) part[blockIdx.x] = acc[0];
  finish_n<1>(part, ticket, out, ws);
}

// ---- rho initialisation (CGLS on the rho block) ----
__global__ void fill_rows_kernel(float* __restrict__ alpha, int nv, int npar, float lt1, float lt2) {
  GRID_STRIDE(j, nv) {
    alpha[j] = lt1;
    alpha[nv + j] = lt2;
    alpha[2 * (int64_t)nv + j] = 0.f;
    alpha[3 * (int64_t)nv + j] = 0.f;
    if (npar > 4) alpha[4 * (int64_t)nv + j] = 1.f;  // B1 = 1 (Methods, "Reconstructions")
  }
}

__global__ void fill_u8_kernel(uint8_t* __restrict__ m, int nv, uint8_t v) {
  GRID_STRIDE(j, nv) m[j] = v;
}

// y += sign * (num / den) * x, the coefficient formed once per block; a non-positive
// denominator or numerator freezes the iteration (flag set by block 0)
__global__ void __launch_bounds__(kT)
scaled_axpy_kernel(float* __restrict__ y, const float* __restrict__ x, int64_t n, const double* num,
                   const double* den, float sign, int* frozen, int may_freeze) {
  __shared__ float s_coef;
  __shared__ int s_apply;
  if (threadIdx.x == 0) {
    const bool ok = !*frozen && *den > 0.0 && *num > 0.0;
    s_apply = ok;
    s_coef = ok ? (float)(*num / *den) * sign : 0.f;
    if (!ok && may_freeze && blockIdx.x == 0) *frozen = 1;
  }
  __syncthreads();
  if (!s_apply) return;
  const float c = s_coef;
  GRID_STRIDE(i, n) y[i] = fmaf(c, x[i], y[i]);
}

// p = s + (num / den) * p unless frozen
__global__ void __launch_bounds__(kT)
xpby_kernel(float* __restrict__ p, const float* __restrict__ s, int64_t n, const double* num,
            const double* den, const int* frozen) {
  __shared__ float s_beta;
  __shared__ int s_apply;
  if (threadIdx.x == 0) {
    s_apply = !*frozen && *den > 0.0;
    s_beta = s_apply ? (float)(*num / *den) : 0.f;
  }
  __syncthreads();
  if (!s_apply) return;
  const float b = s_beta;
  GRID_STRIDE(i, n) p[i] = fmaf(b, p[i], s[i]);
}

__global__ void copy_scalar_kernel(double* dst, const double* src) { *dst = *src; }

// The exact minimum-norm least-squares rho at a uniform linearisation (one time course
// m_n shared by every voxel, as at alpha_0 of the Methods) with a fully sampled Cartesian
// readout (nkx = nx): M = diag(m) (F_y x F_x) row by row, so M^H M = F^H W F with W(ky) =
// sum over the TRs of ky of |m_n|^2, diagonal in k-space.  First the per-k-space solution
//   P[ky][kx] = sum_{n: ky(n) = ky} conj(m_n) d[n][kx] / W(ky)   (0 where W(ky) = 0),
// block per ky, thread per kx; m_n = i m_y,n is voxel 0's channel-0 time course.
__global__ void rho_ls_kspace_kernel(const float* __restrict__ D, int nv, const float2* __restrict__ d, int nkx,
                                     const int* __restrict__ ky_ptr, const int* __restrict__ ky_tr,
                                     float2* __restrict__ P) {
  const int ky = blockIdx.x;
  const int ta = ky_ptr[ky], te = ky_ptr[ky + 1];
  float w = 0.f;
  for (int i = ta; i < te; ++i) {
    const int n = ky_tr[i];
    const float m = D[(size_t)(n >> 2) * nv * 4 + (n & 3)];
    w = fmaf(m, m, w);
  }
  const float inv = w > 0.f ? 1.f / w : 0.f;
  for (int kx = threadIdx.x; kx < nkx; kx += blockDim.x) {
    float re = 0.f, im = 0.f;
    for (int i = ta; i < te; ++i) {
      const int n = ky_tr[i];
      const float m = D[(size_t)(n >> 2) * nv * 4 + (n & 3)];
      const float2 dv = d[(size_t)n * nkx + kx];
      re = fmaf(m, dv.y, re);  // conj(i m) d = m Im d - i m Re d
      im = fmaf(-m, dv.x, im);
    }
    P[(size_t)ky * nkx + kx] = make_float2(re * inv, im * inv);
  }
}

// Then rho = F^H P / (nx ny): Q = P F_x^H (readout adjoint, a complex GEMM) and here the
// phase-encode adjoint, rho[iy][ix] = sum_ky conj(w^(ky iy)) Q[ky][ix] / (nx ny), written
// as the (Re, Im) rows x[0..nv) and x[nv..2 nv).
__global__ void rho_ls_y_kernel(const float2* __restrict__ Q, const float2* __restrict__ roots, int nx, int ny,
                                float scale, float* __restrict__ x) {
  const int nv = nx * ny;
  GRID_STRIDE(j, nv) {
    const int iy = (int)(j / nx), ix = (int)(j - (int64_t)iy * nx);
    float re = 0.f, im = 0.f;
    int e = 0;  // (ky iy) mod ny
    for (int ky = 0; ky < ny; ++ky) {
      const float2 w = roots[e];
      const float2 q = Q[(size_t)ky * nx + ix];
      re = fmaf(w.x, q.x, fmaf(w.y, q.y, re));  // conj(w) q
      im = fmaf(w.x, q.y, fmaf(-w.y, q.x, im));
      e += iy;
      if (e >= ny) e -= ny;
    }
    x[j] = re * scale;
    x[nv + j] = im * scale;
  }
}

__global__ void rho_max_kernel(const float* __restrict__ x, int nv, double* part, unsigned* ticket,
                               double* out) {
  // max |rho|^2 via the same deterministic two-level pattern (max instead of sum)
  __shared__ double ws[8];
  __shared__ bool last;
  double m = 0.0;
  GRID_STRIDE(j, nv) {
    const double a = x[j], b = x[nv + j];
    m = fmax(m, a * a + b * b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kT / 32; ++w) b = fmax(b, ws[w]);
    part[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double b = 0.0;
  for (int i = 0; i < (int)gridDim.x; ++i) b = fmax(b, ((volatile double*)part)[i]);
  *out = b;
  *ticket = 0u;
}

// mask = |rho|^2 > thr^2 max|rho|^2; rho rows of alpha set to the masked CGLS solution
__global__ void draw_mask_kernel(const float* __restrict__ x, int nv, const double* rmax2, double thr,
                                 uint8_t* __restrict__ mask, float* __restrict__ alpha, int* count) {
  const double lim = thr * thr * (*rmax2);
  int c = 0;
  GRID_STRIDE(j, nv) {
    const float a = x[j], b = x[nv + j];
    const bool on = (double)a * a + (double)b * b > lim;
    mask[j] = on ? 1 : 0;
    alpha[2 * (int64_t)nv + j] = on ? a : 0.f;
    alpha[3 * (int64_t)nv + j] = on ? b : 0.f;
    c += on;
  }
  atomicAdd(count, c);
}

__global__ void set_rho_rows_kernel(const float* __restrict__ x, int nv, float* __restrict__ alpha) {
  GRID_STRIDE(j, nv) {
    alpha[2 * (int64_t)nv + j] = x[j];
    alpha[3 * (int64_t)nv + j] = x[nv + j];
  }
}

// v = (0, 0, Re rho, Im rho): J_s v is the signal itself (s is linear in rho)
__global__ void rho_direction_kernel(const float* __restrict__ alpha, int nv, float* __restrict__ v) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += gridDim.x * blockDim.x) {
    v[j] = 0.f;
    v[nv + j] = 0.f;
    v[2 * (size_t)nv + j] = alpha[2 * (size_t)nv + j];
    v[3 * (size_t)nv + j] = alpha[3 * (size_t)nv + j];
  }
}

__global__ void count_mask_kernel(const uint8_t* __restrict__ mask, int nv, int* count) {
  int c = 0;
  GRID_STRIDE(j, nv) c += mask[j] != 0;
  atomicAdd(count, c);
}

template <typename T>
void swap_ptr(T*& a, T*& b) {
  T* t = a;
  a = b;
  b = t;
}

cudaError_t ensure_workspace(Plan* p) {
  if (p->gn_ready) return cudaSuccess;
  if (ensure_timecourses(p) != cudaSuccess) return cudaErrorMemoryAllocation;
  const size_t nv = p->nv, nk = (size_t)p->ntr * p->nkx;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const size_t npv = (size_t)p->npar * nv;
  chk(dalloc(p, &p->D2, (size_t)p->nch * p->nq * nv));
  chk(dalloc(p, &p->rho2, nv));
  chk(dalloc(p, &p->gn_g, npv));
  chk(dalloc(p, &p->gn_z, npv));
  chk(dalloc(p, &p->gn_res, npv));
  chk(dalloc(p, &p->gn_dir, npv));
  chk(dalloc(p, &p->gn_q, npv));
  chk(dalloc(p, &p->gn_alpha, npv));
  chk(dalloc(p, &p->gn_trial, npv));
  chk(dalloc(p, &p->gn_s, nk));
  chk(dalloc(p, &p->gn_r, nk));
  chk(dalloc(p, &p->gn_st, nk));
  chk(dalloc(p, &p->gn_rt, nk));
  chk(dalloc(p, &p->gn_jv, nk));
  chk(dalloc(p, &p->gn_mask, nv));
  chk(dalloc(p, &p->gn_sc, S_COUNT));
  chk(dalloc(p, &p->gn_si, I_COUNT));
  if (e == cudaSuccess) p->gn_ready = true;
  return e;
}

struct Solver {
  Plan* p;
  cudaStream_t st;
  int64_t n4;    // npar nv (the GN vector length)
  int64_t nkf;   // k-space floats 2 ntr nkx
  double* sc;
  int* si;

  // vector kernel launch bookkeeping
  template <typename F>
  cudaError_t vec(F&& launch, int nlaunch = 1) {
    Span sp(p, MRSTAT_K_VECTOR, st, nlaunch);
    if constexpr (std::is_same_v<decltype(launch()), cudaError_t>) {
      const cudaError_t e = launch();
      if (e != cudaSuccess) return e;
    } else {
      launch();
    }
    return cudaGetLastError();
  }

  int residual(const float2* s, const float* d, float2* r, double* f) {
    cudaError_t e = vec([&] {
      residual_kernel<<<grid_for(nkf), kT, 0, st>>>(reinterpret_cast<const float*>(s), d,
                                                      reinterpret_cast<float*>(r), nkf, p->red, p->ticket, f);
    });
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "residual");
  }

  // Steihaug truncated CG on B = Re(J^H J) with gradient p->gn_g; result in p->gn_z
  int steihaug(double delta, int inner, double rel_tol) {
    cudaError_t e;
    {
      // the low-rank column path: the whole solve in one persistent launch
      cudaError_t pe;
      if (lowrank_steihaug_persistent(p, p->gn_g, p->gn_z, delta, inner, rel_tol, sc, si, st, &pe)) {
        if (pe != cudaSuccess) return cuda_fail(pe, "persistent Steihaug launch");
        e = vec([&] { z_norm_kernel<<<grid_for(n4), kT, 0, st>>>(p->gn_z, n4, p->red, p->ticket, sc + S_PNORM2); });
        return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "step norm");
      }
    }
    e = vec([&] {
      st_init_kernel<<<grid_for(n4), kT, 0, st>>>(p->gn_g, p->gn_z, p->gn_res, p->gn_dir, n4, p->red,
                                                  p->ticket, sc + S_RR);
    });
    if (e == cudaSuccess) e = vec([&] { st_start_kernel<<<1, 1, 0, st>>>(sc, si); });
    if (e != cudaSuccess) return cuda_fail(e, "Steihaug init");
    p->gate = si + I_ACTIVE;
    // the GN vectors are whole allocations (16-byte aligned): float4 over all of them
    const int64_t v4 = n4 / 4;
    int status = MRSTAT_OK;
    for (int it = 0; it < inner && status == MRSTAT_OK; ++it) {
      // q = B dir and dir.B dir (gated like the product once CG has stopped)
      status = do_jhjv(p, p->gn_dir, p->gn_q, st, sc + S_DBD);
      if (status != MRSTAT_OK) break;
      // programmatic dependent launches: each kernel's launch overlaps the previous one's tail
      e = vec([&] {
        return launch_pdl(st_update_kernel, dim3(grid_for(n4)), dim3(kT), 0, st, p->gn_z, p->gn_res, p->gn_dir,
                          p->gn_q, n4, v4, sc, si, delta, rel_tol, inner, p->red, p->ticket);
      });
      if (e == cudaSuccess)
        e = vec([&] {
          return launch_pdl(st_dir_kernel, dim3(grid_for(n4)), dim3(kT), 0, st, p->gn_dir, p->gn_res, p->gn_z, n4,
                            v4, sc, si, p->red, p->ticket);
        });
      if (e != cudaSuccess) status = cuda_fail(e, "Steihaug iteration");
    }
    p->gate = nullptr;
    if (status != MRSTAT_OK) return status;
    e = vec([&] { z_norm_kernel<<<grid_for(n4), kT, 0, st>>>(p->gn_z, n4, p->red, p->ticket, sc + S_PNORM2); });
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "step norm");
  }

  // The exact least-squares rho at the current (uniform) linearisation, nkx = nx and
  // ny <= ntr (the k-space work arrays hold ny rows); solution rows 2..3 of gn_z
  int ls_rho(const float* d) {
    const int nx = p->nx, ny = p->ny, nkx = p->nkx;
    cudaError_t e = cudaMemsetAsync(p->gn_z, 0, (size_t)p->npar * p->nv * sizeof(float), st);
    if (e == cudaSuccess)
      e = vec([&] {
        rho_ls_kspace_kernel<<<ny, 256, 0, st>>>(reinterpret_cast<const float*>(p->D), p->nv,
                                                 reinterpret_cast<const float2*>(d), nkx, p->ky_ptr, p->ky_tr,
                                                 p->gn_jv);
      });
    if (e == cudaSuccess) {
      Span sp(p, MRSTAT_K_XDFT_ADJ, st);
      e = launch_cgemm(p->gn_jv, p->fh, p->gn_r, ny, nx, nkx, nullptr, st);
    }
    if (e == cudaSuccess)
      e = vec([&] {
        // one voxel per thread: each runs a whole ny-term sum
        rho_ls_y_kernel<<<(int)((p->nv + kT - 1) / kT), kT, 0, st>>>(p->gn_r, p->roots, nx, ny,
                                                                     (float)(1.0 / ((double)nx * ny)),
                                                                     p->gn_z + 2 * (int64_t)p->nv);
      });
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "exact rho initialisation");
  }

  // CGLS for rho at the current linearisation (rho rows only); solution rows 2..3 of gn_z
  int cgls_rho(const float* d, int iters) {
    const int64_t n2 = 2 * (int64_t)p->nv;
    float* x = p->gn_z + n2;       // rows 2..3 of the solution
    float* pr = p->gn_dir;          // direction, rows 0..1 stay zero
    float* s = p->gn_g;             // A^H r
    float2* r = p->gn_r;            // k-space residual d - A x
    float2* q = p->gn_jv;
    cudaError_t e = cudaMemsetAsync(p->gn_z, 0, (size_t)p->npar * p->nv * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pr, 0, (size_t)p->npar * p->nv * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r, d, nkf * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(si + I_FROZEN, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "CGLS init");
    int status = do_jhw(p, r, s, st);
    if (status != MRSTAT_OK) return status;
    e = cudaMemcpyAsync(pr + n2, s + n2, n2 * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = do_dot(p, s + n2, s + n2, n2, sc + S_GAMMA, st);
    if (e != cudaSuccess) return cuda_fail(e, "CGLS init");
    for (int it = 0; it < iters; ++it) {
      status = do_jvp(p, pr, q, st);
      if (status != MRSTAT_OK) return status;
      e = do_dot(p, reinterpret_cast<const float*>(q), reinterpret_cast<const float*>(q), nkf, sc + S_QQ, st);
      if (e == cudaSuccess)
        e = vec([&] {
          scaled_axpy_kernel<<<grid_for(n2), kT, 0, st>>>(x, pr + n2, n2, sc + S_GAMMA, sc + S_QQ, 1.f,
                                                          si + I_FROZEN, 1);
        });
      if (e == cudaSuccess)
        e = vec([&] {
          scaled_axpy_kernel<<<grid_for(nkf), kT, 0, st>>>(reinterpret_cast<float*>(r),
                                                           reinterpret_cast<const float*>(q), nkf,
                                                           sc + S_GAMMA, sc + S_QQ, -1.f, si + I_FROZEN, 0);
        });
      if (e != cudaSuccess) return cuda_fail(e, "CGLS update");
      status = do_jhw(p, r, s, st);
      if (status != MRSTAT_OK) return status;
      e = do_dot(p, s + n2, s + n2, n2, sc + S_GAMMA_NEW, st);
      if (e == cudaSuccess)
        e = vec([&] {
          xpby_kernel<<<grid_for(n2), kT, 0, st>>>(pr + n2, s + n2, n2, sc + S_GAMMA_NEW, sc + S_GAMMA,
                                                   si + I_FROZEN);
        });
      if (e == cudaSuccess) e = vec([&] { copy_scalar_kernel<<<1, 1, 0, st>>>(sc + S_GAMMA, sc + S_GAMMA_NEW); });
      if (e != cudaSuccess) return cuda_fail(e, "CGLS direction");
    }
    return MRSTAT_OK;
  }
};

}  // namespace
}  // namespace mrstat

using namespace mrstat;

extern "C" {

void mrstat_gn_default_opts(mrstat_gn_opts* o) {
  if (o == nullptr) return;
  std::memset(o, 0, sizeof(*o));
  o->outer_iters = 10;
  o->inner_iters = 20;
  o->delta0 = 0.0;
  o->delta_max = 0.0;
  o->eta = 1e-4;
  o->cg_rel_tol = 0.0;
  o->t1_min_ms = 50.0;
  o->t1_max_ms = 6000.0;
  o->t2_min_ms = 5.0;
  o->t2_max_ms = 3000.0;
  o->rho_init_iters = 0;
  o->t1_init_ms = 1000.0;
  o->t2_init_ms = 100.0;
  o->mask_threshold = 0.0;
  o->b1_min = 0.5;
  o->b1_max = 1.5;
}

int mrstat_gn_solve(mrstat_plan* plan_, const float* d, float* alpha, const float* b1, uint8_t* mask,
                    const mrstat_gn_opts* o, mrstat_gn_report* rep, void* stream) {
  MRSTAT_ABI_RANGE();
  Plan* p = reinterpret_cast<Plan*>(plan_);
  if (p == nullptr || d == nullptr || alpha == nullptr || o == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, d, alpha or opts");
  if (o->outer_iters < 0 || o->outer_iters > MRSTAT_GN_MAX_OUTER || o->inner_iters < 1 ||
      o->rho_init_iters < 0 || !(o->t1_min_ms > 0) || !(o->t1_max_ms > o->t1_min_ms) ||
      !(o->t2_min_ms > 0) || !(o->t2_max_ms > o->t2_min_ms) || !std::isfinite(o->eta))
    return fail(MRSTAT_ERR_INVALID_ARG, "invalid Gauss-Newton options");
  const bool rho_init = o->rho_init_iters > 0 || o->rho_init_exact != 0;
  if (rho_init && (!(o->t1_init_ms > 0) || !(o->t2_init_ms > 0)))
    return fail(MRSTAT_ERR_INVALID_ARG, "invalid rho initialisation point");
  if (rho_init && o->mask_threshold > 0 && mask == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "drawing a mask needs a mask buffer");
  if (o->rho_init_exact != 0 && (p->nkx != p->nx || b1 != nullptr || p->ny > p->ntr))
    return fail(MRSTAT_ERR_UNSUPPORTED,
                "the exact rho initialisation needs nkx == nx, no B1 map and at least ny TRs");
  if (o->hessian != 0 && o->hessian != 1) return fail(MRSTAT_ERR_INVALID_ARG, "hessian must be 0 or 1");
  if (p->npar == 5) {
    if (b1 != nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "B1 is estimated (alpha row 4): pass b1 = NULL");
    if (!(o->b1_min > 0) || !(o->b1_max > o->b1_min)) return fail(MRSTAT_ERR_INVALID_ARG, "need 0 < b1_min < b1_max");
    if (o->hessian != 0 || o->surrogate_iters != 0)
      return fail(MRSTAT_ERR_UNSUPPORTED, "the low-rank and surrogate models do not estimate B1");
  }
  if (p->rc_seg > 0)
    return fail(MRSTAT_ERR_UNSUPPORTED, "the Gauss-Newton solve uses cached time courses (mrstat_set_recompute 0)");
  if (p->slice_iso > 0 && (o->hessian != 0 || o->surrogate_iters != 0 || b1 != nullptr))
    return fail(MRSTAT_ERR_UNSUPPORTED, "with the slice profile: exact Hessian, no surrogate, B1 = 1");
  if (o->hessian == 1 && p->lr == nullptr)
    return fail(MRSTAT_ERR_NOT_LINEARIZED, "the low-rank Hessian needs mrstat_lowrank_set_basis first");
  if (o->iteration_offset < 0) return fail(MRSTAT_ERR_INVALID_ARG, "iteration_offset must be >= 0");
  const int k0 = o->iteration_offset;  // schedule index of this call's first iteration
  if (o->surrogate_iters < 0 || o->surrogate_iters > (1 << 20))
    return fail(MRSTAT_ERR_INVALID_ARG, "surrogate_iters must lie in 0..2^20");
  // outer iterations of this call that run on the surrogate: schedule iterations below
  // surrogate_iters
  const int sur_iters = std::max(0, std::min(o->outer_iters, o->surrogate_iters - k0));
  Mlp* net = nullptr;
  if (sur_iters > 0) {
    if (o->surrogate == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "surrogate_iters > 0 needs a surrogate");
    if (p->lr == nullptr)
      return fail(MRSTAT_ERR_NOT_LINEARIZED, "the surrogate phase needs mrstat_lowrank_set_basis first");
    net = reinterpret_cast<Mlp*>(const_cast<mrstat_mlp*>(o->surrogate));
    if (net->R != p->lr->R)
      return fail(MRSTAT_ERR_INVALID_ARG, "surrogate rank %d differs from the basis rank %d", net->R, p->lr->R);
    if (net->device != p->device) return fail(MRSTAT_ERR_INVALID_ARG, "surrogate and plan live on different devices");
  }
  DeviceGuard guard(p->device);
  const auto t_start = std::chrono::steady_clock::now();
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = ensure_workspace(p);
  if (e != cudaSuccess) return cuda_fail(e, "Gauss-Newton work space");

  Solver S{p, st, (int64_t)p->npar * p->nv, 2 * (int64_t)p->ntr * p->nkx, p->gn_sc, p->gn_si};
  if (p->lr) p->lr->active = false;
  bool coef_stale = true;  // low-rank coefficients of the current point
  const int nv = p->nv;
  const int g = grid_for(nv);
  mrstat_gn_report local;
  std::memset(&local, 0, sizeof(local));
  int status = MRSTAT_OK;

  e = cudaMemcpyAsync(p->gn_alpha, alpha, (size_t)p->npar * nv * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->gn_si, 0, I_COUNT * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "Gauss-Newton setup");

  // -- rho initialisation and mask (Methods, "Reconstructions") --
  if (rho_init) {
    e = S.vec([&] {
      fill_rows_kernel<<<g, kT, 0, st>>>(p->gn_alpha, nv, p->npar, (float)std::log(o->t1_init_ms),
                                         (float)std::log(o->t2_init_ms));
    });
    if (e != cudaSuccess) return cuda_fail(e, "rho init fill");
    status = do_linearize(p, p->gn_alpha, b1, nullptr, p->D, p->rho, st);
    if (status == MRSTAT_OK) status = o->rho_init_exact ? S.ls_rho(d) : S.cgls_rho(d, o->rho_init_iters);
    if (status != MRSTAT_OK) return status;
    const float* x = p->gn_z + 2 * (int64_t)nv;
    if (o->mask_threshold > 0) {
      e = S.vec([&] { rho_max_kernel<<<g, kT, 0, st>>>(x, nv, p->red, p->ticket, p->gn_sc + S_RHOMAX); });
      if (e == cudaSuccess)
        e = S.vec([&] {
          draw_mask_kernel<<<g, kT, 0, st>>>(x, nv, p->gn_sc + S_RHOMAX, o->mask_threshold, p->gn_mask,
                                             p->gn_alpha, p->gn_si + I_MASKCOUNT);
        });
      if (e == cudaSuccess) e = cudaMemcpyAsync(mask, p->gn_mask, nv, cudaMemcpyDeviceToDevice, st);
    } else {
      if (mask) e = cudaMemcpyAsync(p->gn_mask, mask, nv, cudaMemcpyDeviceToDevice, st);
      else e = S.vec([&] { fill_u8_kernel<<<g, kT, 0, st>>>(p->gn_mask, nv, 1); });
      if (e == cudaSuccess) e = S.vec([&] { set_rho_rows_kernel<<<g, kT, 0, st>>>(x, nv, p->gn_alpha); });
      if (e == cudaSuccess) e = S.vec([&] { count_mask_kernel<<<g, kT, 0, st>>>(p->gn_mask, nv, p->gn_si + I_MASKCOUNT); });
    }
  } else {
    if (mask) e = cudaMemcpyAsync(p->gn_mask, mask, nv, cudaMemcpyDeviceToDevice, st);
    else e = S.vec([&] { fill_u8_kernel<<<g, kT, 0, st>>>(p->gn_mask, nv, 1); });
    if (e == cudaSuccess) e = S.vec([&] { count_mask_kernel<<<g, kT, 0, st>>>(p->gn_mask, nv, p->gn_si + I_MASKCOUNT); });
  }
  if (e != cudaSuccess) return cuda_fail(e, "mask");

  // -- the surrogate's low-rank model: coefficients from one MLP inference --
  auto sur_linearize = [&](const float* a, float2* rho_out, float* coef_out) -> int {
    cudaError_t r;
    {
      Span sp(p, MRSTAT_K_VECTOR, st);
      r = launch_prep_linearize(*p, a, p->gn_mask, rho_out, st);
    }
    if (r != cudaSuccess) return cuda_fail(r, "prep_linearize launch");
    Span sp(p, MRSTAT_K_BLOCH, st);
    return mlp_infer(net, a, b1, nv, coef_out, st);
  };
  auto sur_signal = [&](const float* a, float2* s_out) -> int {
    cudaError_t r = S.vec([&] { rho_direction_kernel<<<g, kT, 0, st>>>(a, nv, p->gn_q); });
    if (r != cudaSuccess) return cuda_fail(r, "rho direction");
    return lowrank_jvp(p, p->gn_q, s_out, st);
  };
  auto exact_point = [&]() -> int {
    int r = do_linearize(p, p->gn_alpha, b1, p->gn_mask, p->D, p->rho, st);
    if (r == MRSTAT_OK) r = do_signal(p, p->D, p->rho, p->gn_s, st);
    if (r == MRSTAT_OK) r = S.residual(p->gn_s, d, p->gn_r, p->gn_sc + S_F);
    return r;
  };

  // -- current point --
  if (sur_iters > 0) {
    status = sur_linearize(p->gn_alpha, p->rho, p->lr->coef);
    p->lr->coefT_dirty = true;
    if (status == MRSTAT_OK) status = sur_signal(p->gn_alpha, p->gn_s);
    if (status == MRSTAT_OK) status = S.residual(p->gn_s, d, p->gn_r, p->gn_sc + S_F);
  } else {
    status = exact_point();
  }
  if (status != MRSTAT_OK) return status;
  e = S.vec([&] {
    masked_norm_kernel<<<g, kT, 0, st>>>(p->gn_alpha, p->gn_mask, nv, p->npar, p->red, p->ticket,
                                         p->gn_sc + S_ANORM2);
  });
  if (e != cudaSuccess) return cuda_fail(e, "alpha norm");
  double hs[S_COUNT];
  int hi[I_COUNT];
  int herr = 0;
  auto fetch = [&]() -> int {
    cudaError_t r = cudaMemcpyAsync(hs, p->gn_sc, sizeof hs, cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(hi, p->gn_si, sizeof hi, cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaMemcpyAsync(&herr, p->dev_err, sizeof herr, cudaMemcpyDeviceToHost, st);
    if (r == cudaSuccess) r = cudaStreamSynchronize(st);
    if (r != cudaSuccess) return cuda_fail(r, "Gauss-Newton scalars");
    if (herr) {
      cudaMemsetAsync(p->dev_err, 0, sizeof(int), st);
      return fail(MRSTAT_ERR_TIMEOUT, "a kernel's bounded wait ran out (tensor-core pipeline or grid barrier)");
    }
    return MRSTAT_OK;
  };
  if ((status = fetch()) != MRSTAT_OK) return status;
  double f = hs[S_F];
  local.mask_voxels = hi[I_MASKCOUNT];
  if (!std::isfinite(f)) return fail(MRSTAT_ERR_NONFINITE, "objective is not finite at the initial point");
  double delta = o->delta0 > 0 ? o->delta0 : 0.1 * std::sqrt(hs[S_ANORM2]);
  const double delta_max = o->delta_max > 0 ? o->delta_max : INFINITY;
  const float lt1a = (float)std::log(o->t1_min_ms), lt1b = (float)std::log(o->t1_max_ms);
  const float lt2a = (float)std::log(o->t2_min_ms), lt2b = (float)std::log(o->t2_max_ms);

  for (int k = 0; k < o->outer_iters; ++k) {
    const bool sur = k < sur_iters;
    if (k > 0 && k == sur_iters) {
      // leave the surrogate: exact objective at the current point from here on
      p->lr->active = false;
      status = exact_point();
      if (status == MRSTAT_OK) status = fetch();
      if (status != MRSTAT_OK) return status;
      f = hs[S_F];
      coef_stale = true;
    }
    // gradient g = Re(J_s^H (s - d)) at the current point
    if (sur) {
      p->lr->active = true;
      status = lowrank_jhw(p, p->gn_r, p->gn_g, st);
    } else {
      status = do_jhw(p, p->gn_r, p->gn_g, st);
    }
    if (status != MRSTAT_OK) return status;
    if (sur) {
      p->lr->active = true;  // Steihaug's products: the surrogate's low-rank model
    } else if (o->hessian == 1) {
      if (coef_stale) {
        Span sp(p, MRSTAT_K_BLOCH, st);
        e = lowrank_project(*p, *p->lr, p->gn_alpha, b1, p->gn_mask, p->lr->coef, st);
        p->lr->coefT_dirty = true;
        if (e != cudaSuccess) return cuda_fail(e, "low-rank projection");
        coef_stale = false;
      }
      p->lr->active = true;  // Steihaug's products use the per-ky Gram form
    }
    status = S.steihaug(delta, o->inner_iters, o->cg_rel_tol);
    if (p->lr) p->lr->active = false;
    if (status != MRSTAT_OK) return status;
    e = S.vec([&] {
      trial_kernel<<<g, kT, 0, st>>>(p->gn_alpha, p->gn_z, p->gn_mask, nv, p->npar, lt1a, lt1b, lt2a, lt2b,
                                     (float)o->b1_min, (float)o->b1_max, p->gn_trial);
    });
    if (e != cudaSuccess) return cuda_fail(e, "trial point");
    if (sur) {
      // the trial point's coefficients go to coef2, which the products read while the
      // trial signal is formed; a rejected step swaps them back
      status = sur_linearize(p->gn_trial, p->rho2, p->lr->coef2);
      if (status == MRSTAT_OK) {
        swap_ptr(p->lr->coef, p->lr->coef2);
        status = sur_signal(p->gn_trial, p->gn_st);
      }
    } else {
      status = do_linearize(p, p->gn_trial, b1, p->gn_mask, p->D2, p->rho2, st);
      if (status == MRSTAT_OK) status = do_signal(p, p->D2, p->rho2, p->gn_st, st);
    }
    if (status == MRSTAT_OK) status = S.residual(p->gn_st, d, p->gn_rt, p->gn_sc + S_F);
    if (status == MRSTAT_OK) status = fetch();
    if (status != MRSTAT_OK) return status;
    const double ft = hs[S_F];
    const double pred = -hs[S_MVAL];
    const double ratio = (pred > 0 && std::isfinite(ft)) ? (f - ft) / pred : -INFINITY;
    const double pnorm = std::sqrt(hs[S_PNORM2]);
    local.f[k] = f;
    local.gnorm[k] = hs[S_GNORM];
    local.delta[k] = delta;
    local.cg_steps[k] = hi[I_STEPS];
    local.cg_exit[k] = hi[I_EXIT];
    local.ratio[k] = ratio;
    if (ratio < 0.25) delta *= 0.25;
    else if (ratio > 0.75 && pnorm >= 0.99 * delta) delta = std::fmin(2.0 * delta, delta_max);
    const bool acc = ratio > o->eta;
    local.accepted[k] = acc;
    local.iterations = k + 1;
    if (sur && !acc) swap_ptr(p->lr->coef, p->lr->coef2);
    if (acc) {
      if (!sur) swap_ptr(p->D, p->D2);
      swap_ptr(p->rho, p->rho2);
      swap_ptr(p->gn_alpha, p->gn_trial);
      swap_ptr(p->gn_s, p->gn_st);
      swap_ptr(p->gn_r, p->gn_rt);
      f = ft;
      coef_stale = true;
    }
  }
  local.f_final = f;
  local.delta_final = delta;
  // the plan's cached linearisation is the one at the returned alpha (mask gn_mask): the
  // exact one, or the surrogate's low-rank one when every iteration used the surrogate
  if (p->lr) p->lr->active = sur_iters > 0 && sur_iters == o->outer_iters;
  e = cudaMemcpyAsync(alpha, p->gn_alpha, (size_t)p->npar * nv * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "Gauss-Newton result");
  p->linearized = true;
  local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (rep) *rep = local;
  return MRSTAT_OK;
}

}  // extern "C"
