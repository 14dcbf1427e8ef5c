// K1: per-voxel hard-pulse Bloch recursion with forward-mode tangents, storing the
// echo magnetisation time courses (Supporting Information S2; Algorithm 2 step 1).
//
// One thread per voxel keeps the state in registers for the whole TR train.  With
// RF phases 0/180 degrees the rotation axis is -x or +x (S2: a = [-|B1| Re RF,
// |B1| Im RF, 0] for dB0 = 0), which leaves m_x = 0 for ever, so the state is
// (m_y, m_z) and the echo signal is i * m_y.  Per TR n with signed flip
// phi_n = (+-1) alpha_n B1:
//     (m_y, m_z) <- (cos phi m_y + sin phi m_z, cos phi m_z - sin phi m_y)   (Rodrigues)
//     relax over TE:       m_y <- E2 m_y,  m_z <- 1 + E1 (m_z - 1)           (S2 decay)
//                          (evaluated as m += (E - 1)(m - m_eq) with E - 1 from expm1f)
//     store m_y (and the tangents) at the echo
//     relax over TR - TE.
// Tangents with respect to ln T1 and ln T2 (T1 and T2 times the S2 d/dT form):
//     the rotation acts on them unchanged (k and theta do not depend on T1, T2);
//     decay adds (dt/T1) E1 (m_z - 1) to dm_z/dlnT1 and (dt/T2) E2 m_y to dm_y/dlnT2.
// With B1 as an unknown (NCH = 4) a fourth channel carries dm/dB1: the rotation angle is
// phi_n B1, so the rotation maps the B1 tangent t to R t + phi_n (m_z', -m_y') with m'
// the rotated magnetisation (the derivative of R(theta) m with respect to theta), and
// the decay scales it like m without a source term.
// Four consecutive TRs are written as one float4 per channel: D[c][n/4][j] holds
// TRs 4(n/4)..4(n/4)+3 of voxel j, so a warp stores 512 contiguous bytes.
#include "internal.cuh"

namespace mrstat {
namespace {

template <int NCH, bool B1MAP>
__global__ void __launch_bounds__(128)
bloch_kernel(const float* __restrict__ alpha, const float* __restrict__ b1,
             const uint8_t* __restrict__ mask, const float2* __restrict__ cs,
             const float* __restrict__ phi, int nv, int nq, float te, float tb, float m0z,
             float4* __restrict__ D) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const size_t cstride = (size_t)nq * nv;
  float4* out = D + j;

  if (mask != nullptr && mask[j] == 0) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = 0; q < nq; ++q)
#pragma unroll
      for (int c = 0; c < NCH; ++c) __stcs(out + c * cstride + (size_t)q * nv, z);
    return;
  }

  const float t1 = expf(alpha[j]);
  const float t2 = expf(alpha[nv + j]);
  // Decay over TE (a) and TR - TE (b).  E = exp(-dt/T) is within a few 1e-4 of 1 for
  // long T1/T2, where a float32 E would keep only ~4 significant digits of the rate
  // 1 - E and bias every TR the same way; x = E - 1 from expm1f keeps it to 1 ulp and
  // the updates take the form m += x * (m - m_eq).  d = (dt/T) E = dE/dln T.
  const float ra1 = te / t1, ra2 = te / t2, rb1 = tb / t1, rb2 = tb / t2;
  const float x1a = expm1f(-ra1), x2a = expm1f(-ra2), x1b = expm1f(-rb1), x2b = expm1f(-rb2);
  const float d1a = ra1 * (1.f + x1a), d2a = ra2 * (1.f + x2a);
  const float d1b = rb1 * (1.f + x1b), d2b = rb2 * (1.f + x2b);
  const float bj = B1MAP ? b1[j] : 1.f;

  float my = 0.f, mz = m0z;   // magnetisation
  float ay = 0.f, az = 0.f;   // d m / d ln T1
  float by = 0.f, bz = 0.f;   // d m / d ln T2
  float cy = 0.f, cz = 0.f;   // d m / d B1 (NCH = 4)

  // the per-TR rotation data of the next quad is loaded while this quad runs, so the
  // recursion does not wait on the table loads (the tables hold ntr_pad = 4 nq entries)
  float2 csn[4];
  float phin[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    csn[k] = B1MAP ? make_float2(0.f, 0.f) : __ldg(cs + k);
    phin[k] = (B1MAP || NCH > 3) ? __ldg(phi + k) : 0.f;
  }
  for (int q = 0; q < nq; ++q) {
    float2 csq[4];
    float phq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      csq[k] = csn[k];
      phq[k] = phin[k];
    }
    if (q + 1 < nq) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!B1MAP) csn[k] = __ldg(cs + 4 * (q + 1) + k);
        if (B1MAP || NCH > 3) phin[k] = __ldg(phi + 4 * (q + 1) + k);
      }
    }
    float o0[4], o1[4], o2[4], o3[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float c, s;
      const float phn = phq[k];
      if (B1MAP) {
        sincosf(phn * bj, &s, &c);
      } else {
        c = csq[k].x;
        s = csq[k].y;
      }
      // rotation about the RF axis
      float ty = c * my + s * mz;
      mz = c * mz - s * my;
      my = ty;
      if (NCH > 1) {
        ty = c * ay + s * az;
        az = c * az - s * ay;
        ay = ty;
        ty = c * by + s * bz;
        bz = c * bz - s * by;
        by = ty;
      }
      if (NCH > 3) {
        ty = c * cy + s * cz;
        cz = c * cz - s * cy;
        cy = fmaf(phn, mz, ty);
        cz = fmaf(-phn, my, cz);
      }
      // decay and regrowth over TE: m += (E - 1) o (m - m_eq), tangents gain their source terms
      float zm1 = mz - 1.f;
      if (NCH > 1) {
        ay = fmaf(x2a, ay, ay);
        az = fmaf(x1a, az, fmaf(d1a, zm1, az));
        by = fmaf(x2a, by, fmaf(d2a, my, by));
        bz = fmaf(x1a, bz, bz);
      }
      if (NCH > 3) {
        cy = fmaf(x2a, cy, cy);
        cz = fmaf(x1a, cz, cz);
      }
      my = fmaf(x2a, my, my);
      mz = fmaf(x1a, zm1, mz);
      o0[k] = my;
      if (NCH > 1) {
        o1[k] = ay;
        o2[k] = by;
      }
      if (NCH > 3) o3[k] = cy;
      // decay and regrowth over TR - TE
      zm1 = mz - 1.f;
      if (NCH > 1) {
        ay = fmaf(x2b, ay, ay);
        az = fmaf(x1b, az, fmaf(d1b, zm1, az));
        by = fmaf(x2b, by, fmaf(d2b, my, by));
        bz = fmaf(x1b, bz, bz);
      }
      if (NCH > 3) {
        cy = fmaf(x2b, cy, cy);
        cz = fmaf(x1b, cz, cz);
      }
      my = fmaf(x2b, my, my);
      mz = fmaf(x1b, zm1, mz);
    }
    __stcs(out + (size_t)q * nv, make_float4(o0[0], o0[1], o0[2], o0[3]));
    if (NCH > 1) {
      __stcs(out + cstride + (size_t)q * nv, make_float4(o1[0], o1[1], o1[2], o1[3]));
      __stcs(out + 2 * cstride + (size_t)q * nv, make_float4(o2[0], o2[1], o2[2], o2[3]));
    }
    if (NCH > 3) __stcs(out + 3 * cstride + (size_t)q * nv, make_float4(o3[0], o3[1], o3[2], o3[3]));
  }
}

template <int NCH>
cudaError_t launch_t(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                     float4* D, cudaStream_t st) {
  const int threads = 128;
  const int blocks = (p.nv + threads - 1) / threads;
  const float te = (float)p.te_ms, tb = (float)(p.tr_ms - p.te_ms);
  const float m0z = p.inversion ? -1.f : 1.f;
  if (b1 != nullptr)
    bloch_kernel<NCH, true><<<blocks, threads, 0, st>>>(alpha, b1, mask, p.cs, p.phi, p.nv, p.nq,
                                                        te, tb, m0z, D);
  else
    bloch_kernel<NCH, false><<<blocks, threads, 0, st>>>(alpha, b1, mask, p.cs, p.phi, p.nv, p.nq,
                                                         te, tb, m0z, D);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bloch(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                         float4* D, int nch, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  // with B1 estimated, B1 is alpha row 4
  if (p.npar == 5) b1 = alpha + 4 * (size_t)p.nv;
  if (nch == 4) return launch_t<4>(p, alpha, b1, mask, D, st);
  return nch == 1 ? launch_t<1>(p, alpha, b1, mask, D, st)
                  : launch_t<kChannels>(p, alpha, b1, mask, D, st);
}

cudaError_t launch_bloch_n(const Plan& p, const float* alpha, const float* b1, float4* D, int nv_override,
                           cudaStream_t st) {
  if (nv_override <= 0) return cudaSuccess;
  Plan q = p;  // same sequence tables, different voxel count
  q.nv = nv_override;
  cudaError_t e = launch_t<kChannels>(q, alpha, b1, nullptr, D, st);
  q.marks.clear();
  q.event_pool.clear();
  return e;
}

}  // namespace mrstat

// ---------------------------------------------------------------------------
// Checkpointed form (differentiation by recomputation).
//
// bloch_ckpt_kernel: the recursion with tangents, storing only m_y (one channel, TR
// quads) for the signal, plus the whole state (m_y, m_z and the four tangent
// components) before TR s*interval for every segment s.
//
// segment_jhw_kernel: one thread per (voxel, segment) restarts the recursion from the
// segment's checkpoint, so the segments of a voxel run in parallel, and accumulates
// Z_c = sum_n y_c[n] conj(Ey[n][iy]) Wt[n][ix] over the segment's TRs without storing
// any time course.  A second kernel adds the segments and forms the gradient.
// ---------------------------------------------------------------------------
namespace mrstat {
namespace {

struct Relax {
  float x1a, x2a, d1a, d2a, x1b, x2b, d1b, d2b;
};

__device__ __forceinline__ Relax relax_factors(float t1, float t2, float te, float tb) {
  Relax r;
  const float ra1 = te / t1, ra2 = te / t2, rb1 = tb / t1, rb2 = tb / t2;
  r.x1a = expm1f(-ra1);
  r.x2a = expm1f(-ra2);
  r.x1b = expm1f(-rb1);
  r.x2b = expm1f(-rb2);
  r.d1a = ra1 * (1.f + r.x1a);
  r.d2a = ra2 * (1.f + r.x2a);
  r.d1b = rb1 * (1.f + r.x1b);
  r.d2b = rb2 * (1.f + r.x2b);
  return r;
}

struct State {
  float my, mz, ay, az, by, bz;
};

__device__ __forceinline__ void rotate(State& s, float c, float sn) {
  float t = c * s.my + sn * s.mz;
  s.mz = c * s.mz - sn * s.my;
  s.my = t;
  t = c * s.ay + sn * s.az;
  s.az = c * s.az - sn * s.ay;
  s.ay = t;
  t = c * s.by + sn * s.bz;
  s.bz = c * s.bz - sn * s.by;
  s.by = t;
}

__device__ __forceinline__ void decay(State& s, float x1, float x2, float d1, float d2) {
  const float zm1 = s.mz - 1.f;
  s.ay = fmaf(x2, s.ay, s.ay);
  s.az = fmaf(x1, s.az, fmaf(d1, zm1, s.az));
  s.by = fmaf(x2, s.by, fmaf(d2, s.my, s.by));
  s.bz = fmaf(x1, s.bz, s.bz);
  s.my = fmaf(x2, s.my, s.my);
  s.mz = fmaf(x1, zm1, s.mz);
}

__device__ __forceinline__ void rot_cs(const float2* cs, const float* phi, bool b1map, float bj, int n,
                                       float& c, float& s) {
  if (b1map) {
    sincosf(__ldg(phi + n) * bj, &s, &c);
  } else {
    const float2 t = __ldg(cs + n);
    c = t.x;
    s = t.y;
  }
}

__global__ void __launch_bounds__(128)
bloch_ckpt_kernel(const float* __restrict__ alpha, const float* __restrict__ b1,
                  const uint8_t* __restrict__ mask, const float2* __restrict__ cs,
                  const float* __restrict__ phi, int nv, int nq, int interval, int nseg, float te, float tb,
                  float m0z, float4* __restrict__ Dm, float* __restrict__ ckpt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const bool on = mask == nullptr || mask[j] != 0;
  const float t1 = expf(alpha[j]), t2 = expf(alpha[nv + j]);
  const Relax r = relax_factors(t1, t2, te, tb);
  const bool b1map = b1 != nullptr;
  const float bj = b1map ? b1[j] : 1.f;
  State s{0.f, m0z, 0.f, 0.f, 0.f, 0.f};
  const size_t cstride = (size_t)nv;
  // the next quad's rotations are fetched while this quad runs (tables hold 4 nq entries)
  float2 rn[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) rot_cs(cs, phi, b1map, bj, k, rn[k].x, rn[k].y);
  for (int q = 0; q < nq; ++q) {
    const int n0 = 4 * q;
    float2 rq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rq[k] = rn[k];
    if (q + 1 < nq) {
#pragma unroll
      for (int k = 0; k < 4; ++k) rot_cs(cs, phi, b1map, bj, n0 + 4 + k, rn[k].x, rn[k].y);
    }
    if (n0 % interval == 0) {
      float* c = ckpt + (size_t)(n0 / interval) * 6 * nv + j;
      c[0] = s.my;
      c[cstride] = s.mz;
      c[2 * cstride] = s.ay;
      c[3 * cstride] = s.az;
      c[4 * cstride] = s.by;
      c[5 * cstride] = s.bz;
    }
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      rotate(s, rq[k].x, rq[k].y);
      decay(s, r.x1a, r.x2a, r.d1a, r.d2a);
      o[k] = on ? s.my : 0.f;
      decay(s, r.x1b, r.x2b, r.d1b, r.d2b);
    }
    __stcs(Dm + (size_t)q * nv + j, make_float4(o[0], o[1], o[2], o[3]));
  }
}

__device__ __forceinline__ int mod_small_b(int a, int n, float inv_n) {
  int q = __float2int_rz(__int2float_rn(a) * inv_n);
  int r = a - q * n;
  r += (r < 0) ? n : 0;
  r -= (r >= n) ? n : 0;
  return r;
}

// grid (ceil(nv / 128), nseg)
__global__ void __launch_bounds__(128)
segment_jhw_kernel(const float* __restrict__ alpha, const float* __restrict__ b1,
                   const uint8_t* __restrict__ mask, const float2* __restrict__ cs,
                   const float* __restrict__ phi, const float* __restrict__ ckpt, const float2* __restrict__ wt,
                   const int* __restrict__ kyi, const float2* __restrict__ roots, int nx, int ny, int nv,
                   int ntr, int interval, float te, float tb, float inv_ny, float* __restrict__ zpart) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int seg = blockIdx.y;
  if (j >= nv) return;
  float* zp = zpart + (size_t)seg * 6 * nv + j;
  if (mask != nullptr && mask[j] == 0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) zp[(size_t)c * nv] = 0.f;
    return;
  }
  const float t1 = expf(alpha[j]), t2 = expf(alpha[nv + j]);
  const Relax r = relax_factors(t1, t2, te, tb);
  const bool b1map = b1 != nullptr;
  const float bj = b1map ? b1[j] : 1.f;
  const float* c = ckpt + (size_t)seg * 6 * nv + j;
  State s{c[0], c[nv], c[2 * (size_t)nv], c[3 * (size_t)nv], c[4 * (size_t)nv], c[5 * (size_t)nv]};
  const int iy = j / nx, ix = j - iy * nx;
  float z0r = 0.f, z0i = 0.f, z1r = 0.f, z1i = 0.f, z2r = 0.f, z2i = 0.f;
  const int na = seg * interval, ne = min(ntr, na + interval);
  for (int n = na; n < ne; ++n) {
    float cc, sn;
    rot_cs(cs, phi, b1map, bj, n, cc, sn);
    rotate(s, cc, sn);
    decay(s, r.x1a, r.x2a, r.d1a, r.d2a);
    const float2 e = __ldg(roots + mod_small_b(__ldg(kyi + n) * iy, ny, inv_ny));
    const float2 w = __ldg(wt + (size_t)n * nx + ix);
    const float ur = fmaf(e.x, w.x, e.y * w.y);
    const float ui = fmaf(e.x, w.y, -e.y * w.x);
    z0r = fmaf(s.my, ur, z0r);
    z0i = fmaf(s.my, ui, z0i);
    z1r = fmaf(s.ay, ur, z1r);
    z1i = fmaf(s.ay, ui, z1i);
    z2r = fmaf(s.by, ur, z2r);
    z2i = fmaf(s.by, ui, z2i);
    decay(s, r.x1b, r.x2b, r.d1b, r.d2b);
  }
  zp[0] = z0r;
  zp[(size_t)nv] = z0i;
  zp[2 * (size_t)nv] = z1r;
  zp[3 * (size_t)nv] = z1i;
  zp[4 * (size_t)nv] = z2r;
  zp[5 * (size_t)nv] = z2i;
}

__global__ void segment_sum_kernel(const float* __restrict__ zpart, const float* __restrict__ alpha,
                                   const uint8_t* __restrict__ mask, int nv, int nseg, float* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  float z[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int s = 0; s < nseg; ++s)
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] += zpart[((size_t)s * 6 + c) * nv + j];
  const float m = (mask == nullptr || mask[j]) ? 1.f : 0.f;
  const float rr = alpha[2 * (size_t)nv + j] * m, ri = alpha[3 * (size_t)nv + j] * m;
  g[j] = (rr * z[3] - ri * z[2]) * m;
  g[nv + j] = (rr * z[5] - ri * z[4]) * m;
  g[2 * (size_t)nv + j] = z[1] * m;
  g[3 * (size_t)nv + j] = -z[0] * m;
}

}  // namespace

cudaError_t launch_bloch_ckpt(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                              int interval, int nseg, float* ckpt, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  const int blocks = (p.nv + 127) / 128;
  bloch_ckpt_kernel<<<blocks, 128, 0, st>>>(alpha, b1, mask, p.cs, p.phi, p.nv, p.nq, interval, nseg,
                                            (float)p.te_ms, (float)(p.tr_ms - p.te_ms),
                                            p.inversion ? -1.f : 1.f, p.dfwd, ckpt);
  return cudaGetLastError();
}

cudaError_t launch_segment_jhw(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                               int interval, int nseg, const float* ckpt, float* zpart, float* g,
                               cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  dim3 grid((p.nv + 127) / 128, nseg);
  segment_jhw_kernel<<<grid, 128, 0, st>>>(alpha, b1, mask, p.cs, p.phi, ckpt, p.wt, p.kyi, p.roots, p.nx, p.ny,
                                           p.nv, p.ntr, interval, (float)p.te_ms, (float)(p.tr_ms - p.te_ms),
                                           1.0f / (float)p.ny, zpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  segment_sum_kernel<<<(p.nv + 255) / 256, 256, 0, st>>>(zpart, alpha, mask, p.nv, nseg, g);
  return cudaGetLastError();
}

}  // namespace mrstat
