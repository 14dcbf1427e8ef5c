// K1 with the slice profile: Gaussian RF pulses played as sub-steps against a balanced
// slice-select gradient, averaged over isochromats across the slice (Methods, "Pulse
// Sequence": Gaussian envelopes; "Reconstructions": the Bloch solver takes the slice
// profile into account).  The model (the paper gives no pulse parameters):
//   isochromat k of n_iso sits at u_k = extent ((k + 1/2)/n_iso - 1/2) slice thicknesses;
//   the pulse is n_sub hard sub-pulses with Gaussian weights w_s (sum 1), sub-step s
//   turns about the TR's RF axis by phi_n w_s (phi_n the signed flip, as in the
//   hard-pulse kernel) and then precesses about z by beta_k = 2 pi tbw u_k / n_sub;
//   a pre-winder and a rewinder of -n_sub/2 beta_k each balance the gradient;
//   the rest of the TR as in the hard-pulse recursion, per isochromat; the echo is the
//   mean of m_y over the isochromats (the x components cancel by the slice's mirror
//   symmetry, so the signal stays i * mean m_y).
//
// One lane per isochromat (n_iso a power of two <= 32, 32 / n_iso voxels per warp), the
// whole 3-vector state and its ln T1 / ln T2 tangents in registers.  The pulse of a
// (TR, isochromat) pair does not depend on the voxel: mrstat_set_slice_profile composes
// each one once, in float64 on the host, into a 3 x 3 matrix (columns: the basis vectors
// pushed through pre-winder, sub-steps and rewinder); each block stages a chunk of TRs'
// matrices in shared memory and its lanes apply them; the per-voxel sum over the
// isochromats is a segmented shuffle reduction, written as TR quads like K1.
#include "internal.cuh"

namespace mrstat {
namespace {

constexpr int kSliceThreads = 512;
constexpr int kSliceChunk = 16;  // TRs per composed chunk: kSliceChunk * n_iso <= kSliceThreads
constexpr int kSliceMaxSub = 64;

__global__ void __launch_bounds__(kSliceThreads)
bloch_slice_kernel(const float* __restrict__ alpha, const uint8_t* __restrict__ mask,
                   const float* __restrict__ rotg, int n_iso, int log2_iso, int nv, int nq, float te, float tb,
                   float m0z, int nch, float4* __restrict__ D) {
  __shared__ float rot[kSliceChunk * 32 * 9];  // [TR in chunk][isochromat][3 x 3, column-major]
  const int tid = threadIdx.x, lane = tid & 31;
  const int k = lane & (n_iso - 1);                              // this lane's isochromat
  const int j = ((blockIdx.x * kSliceThreads + tid) >> 5) * (32 >> log2_iso) + (lane >> log2_iso);
  const bool live = j < nv;
  const bool on = live && (mask == nullptr || mask[j] != 0);
  const size_t cstride = (size_t)nq * nv;

  float t1 = 1000.f, t2 = 100.f;
  if (live) {
    t1 = expf(alpha[j]);
    t2 = expf(alpha[nv + j]);
  }
  // decay factors as in K1: m += (E - 1)(m - m_eq) with E - 1 from expm1f; d = dE/dln T
  const float ra1 = te / t1, ra2 = te / t2, rb1 = tb / t1, rb2 = tb / t2;
  const float x1a = expm1f(-ra1), x2a = expm1f(-ra2), x1b = expm1f(-rb1), x2b = expm1f(-rb2);
  const float d1a = ra1 * (1.f + x1a), d2a = ra2 * (1.f + x2a);
  const float d1b = rb1 * (1.f + x1b), d2b = rb2 * (1.f + x2b);

  float m[3] = {0.f, 0.f, m0z}, a[3] = {0.f, 0.f, 0.f}, b[3] = {0.f, 0.f, 0.f};
  float o0[4], o1[4], o2[4];
  const float inv_iso = 1.f / (float)n_iso;
  const int ntr4 = 4 * nq;

  for (int n0 = 0; n0 < ntr4; n0 += kSliceChunk) {
    __syncthreads();  // the previous chunk's matrices are no longer read
    // the chunk's composed pulses (TRs past the train are never applied)
    const int nrot = min(kSliceChunk, ntr4 - n0) * 32 * 9;
    const float* src = rotg + (size_t)n0 * 32 * 9;
    for (int e = tid; e < nrot; e += kSliceThreads) rot[e] = __ldg(src + e);
    __syncthreads();
    for (int nq4 = 0; nq4 < kSliceChunk; nq4 += 4) {
      if (n0 + nq4 >= ntr4) break;  // ntr4 and the quads are multiples of 4
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int nn = nq4 + u;
        const float* R = rot + (nn * 32 + k) * 9;  // columns R[0..2], R[3..5], R[6..8]
        float r[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) r[e] = R[e];
        float v[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = fmaf(r[i], m[0], fmaf(r[3 + i], m[1], r[6 + i] * m[2]));
        m[0] = v[0], m[1] = v[1], m[2] = v[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = fmaf(r[i], a[0], fmaf(r[3 + i], a[1], r[6 + i] * a[2]));
        a[0] = v[0], a[1] = v[1], a[2] = v[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = fmaf(r[i], b[0], fmaf(r[3 + i], b[1], r[6 + i] * b[2]));
        b[0] = v[0], b[1] = v[1], b[2] = v[2];
        // decay over TE with the tangents' source terms (taken from the state before decay)
        float zm1 = m[2] - 1.f;
        a[0] = fmaf(x2a, a[0], a[0]);
        a[1] = fmaf(x2a, a[1], a[1]);
        a[2] = fmaf(x1a, a[2], fmaf(d1a, zm1, a[2]));
        b[0] = fmaf(x2a, b[0], fmaf(d2a, m[0], b[0]));
        b[1] = fmaf(x2a, b[1], fmaf(d2a, m[1], b[1]));
        b[2] = fmaf(x1a, b[2], b[2]);
        m[0] = fmaf(x2a, m[0], m[0]);
        m[1] = fmaf(x2a, m[1], m[1]);
        m[2] = fmaf(x1a, zm1, m[2]);
        // echo: the mean of m_y (and tangents) over the voxel's isochromats; with 32
        // isochromats (one voxel per warp) the quad's twelve sums are formed together after
        // the quad, otherwise per TR here
        if (n_iso == 32) {
          o0[u] = m[1];
          o1[u] = a[1];
          o2[u] = b[1];
        } else {
          float sy = m[1], sa = a[1], sb = b[1];
          for (int o = n_iso >> 1; o > 0; o >>= 1) {
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sb += __shfl_xor_sync(0xffffffffu, sb, o);
          }
          o0[u] = sy * inv_iso;
          o1[u] = sa * inv_iso;
          o2[u] = sb * inv_iso;
        }
        // decay over TR - TE
        zm1 = m[2] - 1.f;
        a[0] = fmaf(x2b, a[0], a[0]);
        a[1] = fmaf(x2b, a[1], a[1]);
        a[2] = fmaf(x1b, a[2], fmaf(d1b, zm1, a[2]));
        b[0] = fmaf(x2b, b[0], fmaf(d2b, m[0], b[0]));
        b[1] = fmaf(x2b, b[1], fmaf(d2b, m[1], b[1]));
        b[2] = fmaf(x1b, b[2], b[2]);
        m[0] = fmaf(x2b, m[0], m[0]);
        m[1] = fmaf(x2b, m[1], m[1]);
        m[2] = fmaf(x1b, zm1, m[2]);
      }
      if (n_iso == 32) {
        // the quad's twelve sums v[3 u + channel] over the warp's lanes, by halving: after
        // the exchanges across lane bits 4 and 3, lane group g = lane / 8 holds TR u = g's
        // three values, summed over its partners; a butterfly over the low three lane bits
        // completes them (18 shuffles for the quad instead of 60)
        float v[12];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          v[3 * u] = o0[u];
          v[3 * u + 1] = o1[u];
          v[3 * u + 2] = o2[u];
        }
        const bool h4 = (lane & 16) != 0, h3 = (lane & 8) != 0;
        float w[6], x[3];
#pragma unroll
        for (int e = 0; e < 6; ++e) {
          const float send = h4 ? v[e] : v[6 + e], keep = h4 ? v[6 + e] : v[e];
          w[e] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const float send = h3 ? w[e] : w[3 + e], keep = h3 ? w[3 + e] : w[e];
          x[e] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)
#pragma unroll
          for (int e = 0; e < 3; ++e) x[e] += __shfl_xor_sync(0xffffffffu, x[e], o);
        if ((lane & 7) == 0 && live) {  // TR u of the quad: one float of each channel's float4
          const int u = lane >> 3;
          const size_t q = (size_t)((n0 + nq4) >> 2) * nv + j;
          __stcs(reinterpret_cast<float*>(D + q) + u, on ? x[0] * inv_iso : 0.f);
          if (nch > 1) {
            __stcs(reinterpret_cast<float*>(D + cstride + q) + u, on ? x[1] * inv_iso : 0.f);
            __stcs(reinterpret_cast<float*>(D + 2 * cstride + q) + u, on ? x[2] * inv_iso : 0.f);
          }
        }
      } else if (k == 0 && live) {  // one float4 per channel and TR quad, as K1 stores them
        const size_t q = (size_t)((n0 + nq4) >> 2) * nv + j;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        __stcs(D + q, on ? make_float4(o0[0], o0[1], o0[2], o0[3]) : z4);
        if (nch > 1) {  // the tangent channels (absent from the forward-only buffer)
          __stcs(D + cstride + q, on ? make_float4(o1[0], o1[1], o1[2], o1[3]) : z4);
          __stcs(D + 2 * cstride + q, on ? make_float4(o2[0], o2[1], o2[2], o2[3]) : z4);
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_bloch_slice(const Plan& p, const float* alpha, const uint8_t* mask, float4* D, int nch,
                               cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  const int vpb = (kSliceThreads / 32) * (32 / p.slice_iso);  // voxels per block
  const int blocks = (p.nv + vpb - 1) / vpb;
  const float te = (float)p.te_ms, tb = (float)(p.tr_ms - p.te_ms);
  int log2_iso = 0;
  while ((1 << log2_iso) < p.slice_iso) ++log2_iso;
  bloch_slice_kernel<<<blocks, kSliceThreads, 0, st>>>(alpha, mask, p.slice_rot, p.slice_iso, log2_iso, p.nv,
                                                      p.nq, te, tb, p.inversion ? -1.f : 1.f, nch, D);
  return cudaGetLastError();
}

}  // namespace mrstat

using namespace mrstat;

extern "C" {

int mrstat_set_slice_profile(mrstat_plan* plan, const mrstat_slice_profile* prof) {
  MRSTAT_ABI_RANGE();
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (p == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan");
  DeviceGuard g(p->device);
  if (prof == nullptr) {
    p->slice_iso = 0;
    p->linearized = false;
    return MRSTAT_OK;
  }
  const int ni = prof->n_iso, ns = prof->n_sub;
  if (ni < 1 || ni > 32 || (ni & (ni - 1)) != 0 || ns < 1 || ns > kSliceMaxSub || !(prof->sigma > 0) ||
      !(prof->extent > 0) || !std::isfinite(prof->tbw))
    return fail(MRSTAT_ERR_INVALID_ARG, "slice profile: n_iso a power of two in 1..32, n_sub in 1..%d, "
                                        "sigma > 0, extent > 0", kSliceMaxSub);
  if (p->npar != 4) return fail(MRSTAT_ERR_UNSUPPORTED, "the slice-profile model has no B1 tangent");
  // Gaussian sub-pulse weights (sum 1), in float64
  std::vector<double> w(ns);
  double sum = 0.0;
  for (int s = 0; s < ns; ++s) {
    const double x = (s + 0.5) / ns - 0.5;
    w[s] = std::exp(-x * x / (2.0 * prof->sigma * prof->sigma));
    sum += w[s];
  }
  cudaError_t e = cudaSuccess;
  if (p->slice_rot == nullptr) e = dalloc(p, &p->slice_rot, (size_t)p->ntr_pad * 32 * 9);
  // the composed pulse of every (TR, isochromat): pre-winder, then per sub-step the RF
  // rotation by phi_n w_s about the TR's axis (the hard-pulse kernel's convention) and the
  // precession by beta_k, then the rewinder; in float64 from the plan's signed flips
  std::vector<float> phi(p->ntr_pad);
  if (e == cudaSuccess) e = cudaMemcpy(phi.data(), p->phi, phi.size() * sizeof(float), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "slice profile tables");
  std::vector<float> rot((size_t)p->ntr_pad * 32 * 9, 0.f);
  for (int n = 0; n < p->ntr_pad; ++n)
    for (int k = 0; k < ni; ++k) {
      const double u = prof->extent * ((k + 0.5) / ni - 0.5);
      const double beta = 2.0 * M_PI * prof->tbw * u / ns, half = -0.5 * ns * beta;
      const double cb = std::cos(beta), sb = std::sin(beta), ch = std::cos(half), sh = std::sin(half);
      for (int c = 0; c < 3; ++c) {
        double x = c == 0, y = c == 1, z = c == 2;
        double t = ch * x - sh * y;  // pre-winder
        y = sh * x + ch * y;
        x = t;
        for (int s = 0; s < ns; ++s) {
          const double ang = (double)phi[n] * (w[s] / sum), cn = std::cos(ang), sn = std::sin(ang);
          t = cn * y + sn * z;  // RF sub-pulse
          z = cn * z - sn * y;
          y = t;
          t = cb * x - sb * y;  // gradient precession
          y = sb * x + cb * y;
          x = t;
        }
        t = ch * x - sh * y;  // rewinder
        y = sh * x + ch * y;
        x = t;
        float* R = rot.data() + ((size_t)n * 32 + k) * 9 + 3 * c;
        R[0] = (float)x;
        R[1] = (float)y;
        R[2] = (float)z;
      }
    }
  e = cudaMemcpy(p->slice_rot, rot.data(), rot.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "slice profile tables");
  p->slice_iso = ni;
  p->slice_sub = ns;
  p->linearized = false;
  return MRSTAT_OK;
}

}  // extern "C"
