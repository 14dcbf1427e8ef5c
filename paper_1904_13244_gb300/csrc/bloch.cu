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

  for (int q = 0; q < nq; ++q) {
    float o0[4], o1[4], o2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int n = 4 * q + k;
      float c, s;
      if (B1MAP) {
        sincosf(__ldg(phi + n) * bj, &s, &c);
      } else {
        const float2 t = __ldg(cs + n);
        c = t.x;
        s = t.y;
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
      // decay and regrowth over TE: m += (E - 1) o (m - m_eq), tangents gain their source terms
      float zm1 = mz - 1.f;
      if (NCH > 1) {
        ay = fmaf(x2a, ay, ay);
        az = fmaf(x1a, az, fmaf(d1a, zm1, az));
        by = fmaf(x2a, by, fmaf(d2a, my, by));
        bz = fmaf(x1a, bz, bz);
      }
      my = fmaf(x2a, my, my);
      mz = fmaf(x1a, zm1, mz);
      o0[k] = my;
      if (NCH > 1) {
        o1[k] = ay;
        o2[k] = by;
      }
      // decay and regrowth over TR - TE
      zm1 = mz - 1.f;
      if (NCH > 1) {
        ay = fmaf(x2b, ay, ay);
        az = fmaf(x1b, az, fmaf(d1b, zm1, az));
        by = fmaf(x2b, by, fmaf(d2b, my, by));
        bz = fmaf(x1b, bz, bz);
      }
      my = fmaf(x2b, my, my);
      mz = fmaf(x1b, zm1, mz);
    }
    __stcs(out + (size_t)q * nv, make_float4(o0[0], o0[1], o0[2], o0[3]));
    if (NCH > 1) {
      __stcs(out + cstride + (size_t)q * nv, make_float4(o1[0], o1[1], o1[2], o1[3]));
      __stcs(out + 2 * cstride + (size_t)q * nv, make_float4(o2[0], o2[1], o2[2], o2[3]));
    }
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
  return nch == 1 ? launch_t<1>(p, alpha, b1, mask, D, st)
                  : launch_t<kChannels>(p, alpha, b1, mask, D, st);
}

}  // namespace mrstat
