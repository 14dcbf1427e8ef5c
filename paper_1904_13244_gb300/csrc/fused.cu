// Recompute form of the exact model: the Bloch recursion re-run inside every product
// instead of streaming cached time courses (Algorithms 2 and 4 evaluate the simulation
// inside every product; Supporting Information S2 for the recursion).
//
// The linearisation keeps, for every voxel, the relaxation factors and the state
// (m_y, m_z and their ln T1 / ln T2 tangents; m_x = 0 for RF phases 0/180) before every
// seg-th TR: 6 floats per voxel and segment instead of 3 floats per voxel and TR.  A
// product is one launch over (image column ix, segment s) blocks with one thread per
// row iy: each thread restarts its voxel's recursion from the segment's state, so the
// segments of a column run in parallel, and the block forms the phase-encode sums of its
// column TR by TR:
//   J.v:      A[n][ix] = sum_iy E[ky(n)][iy] q_n(iy), q_n = i (rho t_n + (v2 + i v3) m_y,n),
//             t_n = v0 dm_y,n/dlnT1 + v1 dm_y,n/dlnT2 (then the readout DFT of A);
//   J^H w:    b_n(iy) = conj(E[ky(n)][iy]) Wt[n][ix] with Wt the readout adjoint of w, and
//             g0 += dm1 Im(conj(rho) b), g1 += dm2 Im(conj(rho) b), g2 += m Im b,
//             g3 -= m Re b  (Re of conj(dq/dalpha_k) b);
//   J^H J v:  with nkx = nx the readout DFT pair cancels (F^H F = nx I), so Wt = nx A and
//             both halves run in one pass: A[n] is formed in the block and used at once.
// E[ky][iy] = roots[(ky iy) mod ny] is an exact table lookup.  TRs go in chunks of kChunk:
// each thread advances its recursion kChunk TRs, keeping the three echo values and phases
// in registers, the block adds the kChunk complex sums (a halving warp exchange, then the
// warps' partials through shared memory), and the gradient terms of the chunk follow.
// Per-segment gradients go to gpart[s][4][nv]; a second kernel adds the segments.
#include "internal.cuh"

namespace mrstat {
namespace {

constexpr int kChunk = 4;       // TRs per block reduction
constexpr int kMaxRows = 256;   // one thread per row of the column

enum { RC_JV = 0, RC_JHW = 1, RC_JHJV = 2 };

struct RcRelax {
  float x1a, x2a, d1a, d2a, x1b, x2b, d1b, d2b;
};

__device__ __forceinline__ RcRelax rc_relax(float t1, float t2, float te, float tb) {
  // E - 1 by expm1f (float32 keeps the small per-TR change of long T1/T2), and
  // d = (dt/T) E = dE/dln T
  RcRelax r;
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

struct RcState {
  float my, mz, ay, az, by, bz;
};

// rotation about the RF axis by the signed flip (cos c, sin s), on m and both tangents
__device__ __forceinline__ void rc_rotate(RcState& s, float c, float sn) {
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

// decay and regrowth m += (E - 1)(m - m_eq); the tangents gain their source terms
__device__ __forceinline__ void rc_decay(RcState& s, float x1, float x2, float d1, float d2) {
  const float zm1 = s.mz - 1.f;
  s.ay = fmaf(x2, s.ay, s.ay);
  s.az = fmaf(x1, s.az, fmaf(d1, zm1, s.az));
  s.by = fmaf(x2, s.by, fmaf(d2, s.my, s.by));
  s.bz = fmaf(x1, s.bz, s.bz);
  s.my = fmaf(x2, s.my, s.my);
  s.mz = fmaf(x1, zm1, s.mz);
}

__device__ __forceinline__ void rc_cs(const float2* cs, const float* phi, const float* b1, float bj, int n,
                                      float& c, float& s) {
  if (b1 != nullptr) {
    sincosf(__ldg(phi + n) * bj, &s, &c);
  } else {
    const float2 t = __ldg(cs + n);
    c = t.x;
    s = t.y;
  }
}

// a mod n for 0 <= a < n * n and n <= kMaxRows, with magic = ceil(2^32 / n) (0 for n = 1,
// where a is 0): the quotient umulhi(a, magic) is exact for every such a and n (the error
// a (magic - 2^32 / n) / 2^32 < n^2 / 2^32 stays below the gap 1 / n to the next integer;
// tests/test_host_arith.py checks this for every n <= 256 and a < n^2)
__device__ __forceinline__ int rc_mod(int a, int n, unsigned magic) {
  return a - (int)__umulhi((unsigned)a, magic) * n;
}

// Linearisation: relaxation factors and the state before every seg-th TR, per voxel.
//   rlx [8][nv]: x1a x2a d1a d2a x1b x2b d1b d2b;  ckpt [nseg][6][nv]
__global__ void __launch_bounds__(128)
rc_ckpt_kernel(const float* __restrict__ alpha, const float* __restrict__ b1, const float2* __restrict__ cs,
               const float* __restrict__ phi, int nv, int ntr, int seg, int nseg, float te, float tb, float m0z,
               float* __restrict__ rlx, float* __restrict__ ckpt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const float t1 = expf(alpha[j]), t2 = expf(alpha[nv + j]);
  const RcRelax r = rc_relax(t1, t2, te, tb);
  const float rv[8] = {r.x1a, r.x2a, r.d1a, r.d2a, r.x1b, r.x2b, r.d1b, r.d2b};
#pragma unroll
  for (int k = 0; k < 8; ++k) rlx[(size_t)k * nv + j] = rv[k];
  const float bj = b1 != nullptr ? b1[j] : 1.f;
  RcState s{0.f, m0z, 0.f, 0.f, 0.f, 0.f};
  for (int sg = 0; sg < nseg; ++sg) {
    float* c = ckpt + (size_t)sg * 6 * nv + j;
    c[0] = s.my;
    c[(size_t)nv] = s.mz;
    c[2 * (size_t)nv] = s.ay;
    c[3 * (size_t)nv] = s.az;
    c[4 * (size_t)nv] = s.by;
    c[5 * (size_t)nv] = s.bz;
    if (sg + 1 == nseg) break;  // the last segment's end state is never needed
    const int ne = min(ntr, (sg + 1) * seg);
    for (int n = sg * seg; n < ne; ++n) {
      float cc, sn;
      rc_cs(cs, phi, b1, bj, n, cc, sn);
      rc_rotate(s, cc, sn);
      rc_decay(s, r.x1a, r.x2a, r.d1a, r.d2a);
      rc_decay(s, r.x1b, r.x2b, r.d1b, r.d2b);
    }
  }
}

// Sum of K complex values (v[2k], v[2k+1]) over the 32 lanes of a warp by halving
// exchanges: at each offset 16, 8, ... a lane sends the half of its values it does not
// keep and adds the half it receives, until one complex value is left, that of slot
// (lane / (32 / K)) mod K; the remaining offsets finish the sum.  For K = 8: 18 shuffles
// instead of 80 for eight separate warp sums.
template <int K>
__device__ __forceinline__ float2 rc_warp_sum(float (&v)[2 * K], int lane) {
  static_assert(K == 1 || K == 2 || K == 4 || K == 8, "chunk of 1, 2, 4 or 8 TRs");
#pragma unroll
  for (int n = 2 * K, off = 16; n > 2; n >>= 1, off >>= 1) {
    const bool up = lane & off;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const float send = up ? v[i] : v[i + n / 2];
      const float keep = up ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  float re = v[0], im = v[1];
#pragma unroll
  for (int off = 16 / K; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  return make_float2(re, im);
}

// One row's voxel data and running sums in rc_product_kernel.
struct RcRow {
  bool on;        // the row exists (rows past ny contribute zeros)
  int iy, j;
  float m;        // mask
  float2 rh;      // rho * mask
  RcRelax r;
  RcState s;
  float bj;
  float v0, v1, v2, v3;
  float g0, g1, g2, g3;
};

// grid (nx, nseg), block = ceil(ny / kRows) rounded up to whole warps; thread t owns rows
// t + q H, q < kRows, H = ceil(ny / kRows): the recursions of its rows are independent
// chains (instruction-level parallelism), and the per-TR table loads and the block sums
// serve all of them.
constexpr int kRows = 2;

template <int MODE>
__global__ void __launch_bounds__(kMaxRows / kRows, 4)
rc_product_kernel(const float* __restrict__ rlx, const float* __restrict__ ckpt, const float2* __restrict__ rho,
                  const float* __restrict__ maskf, const float* __restrict__ b1, const float* __restrict__ v,
                  const float2* __restrict__ cs, const float* __restrict__ phi, const int* __restrict__ kyi,
                  const float2* __restrict__ roots, int nx, int ny, int nv, int ntr, int seg, unsigned magic,
                  float scale, float2* __restrict__ A, const float2* __restrict__ wt, float* __restrict__ gpart,
                  const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  __shared__ float2 part[kMaxRows / 32][kChunk];
  __shared__ float2 asum[kChunk];
  const int ix = blockIdx.x, sg = blockIdx.y;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
  const int H = (ny + kRows - 1) / kRows;
  RcRow w[kRows];
#pragma unroll
  for (int q = 0; q < kRows; ++q) {
    RcRow& x = w[q];
    x.iy = t + q * H;
    x.on = t < H && x.iy < ny;
    x.j = x.on ? x.iy * nx + ix : 0;
    x.m = x.on ? maskf[x.j] : 0.f;
    x.rh = x.on ? rho[x.j] : make_float2(0.f, 0.f);
    x.r = RcRelax{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    x.s = RcState{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    x.bj = 1.f;
    x.v0 = x.v1 = x.v2 = x.v3 = 0.f;
    x.g0 = x.g1 = x.g2 = x.g3 = 0.f;
    if (x.on) {
      const int j = x.j;
      x.r = {rlx[j], rlx[(size_t)nv + j], rlx[2 * (size_t)nv + j], rlx[3 * (size_t)nv + j],
             rlx[4 * (size_t)nv + j], rlx[5 * (size_t)nv + j], rlx[6 * (size_t)nv + j], rlx[7 * (size_t)nv + j]};
      const float* c = ckpt + (size_t)sg * 6 * nv + j;
      x.s = {c[0], c[(size_t)nv], c[2 * (size_t)nv], c[3 * (size_t)nv], c[4 * (size_t)nv], c[5 * (size_t)nv]};
      if (b1 != nullptr) x.bj = b1[j];
      if (MODE != RC_JHW) {
        x.v0 = v[j];
        x.v1 = v[(size_t)nv + j];
        x.v2 = v[2 * (size_t)nv + j] * x.m;
        x.v3 = v[3 * (size_t)nv + j] * x.m;
      }
    }
  }
  const int na = sg * seg, ne = min(ntr, na + seg);
  for (int n0 = na; n0 < ne; n0 += kChunk) {
    float y0[kRows][kChunk], y1[kRows][kChunk], y2[kRows][kChunk];
    float2 e[kRows][kChunk];
    float p[2 * kChunk];
#pragma unroll
    for (int k = 0; k < kChunk; ++k) {
      const int n = n0 + k;
      p[2 * k] = p[2 * k + 1] = 0.f;
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        y0[q][k] = y1[q][k] = y2[q][k] = 0.f;
        e[q][k] = make_float2(0.f, 0.f);
      }
      if (n < ne) {  // uniform across the block
        float2 csn = make_float2(1.f, 0.f);
        if (b1 == nullptr) csn = __ldg(cs + n);
        const int kyn = __ldg(kyi + n);
#pragma unroll
        for (int q = 0; q < kRows; ++q) {
          RcRow& x = w[q];
          float cc = csn.x, sn = csn.y;
          if (b1 != nullptr) sincosf(__ldg(phi + n) * x.bj, &sn, &cc);
          rc_rotate(x.s, cc, sn);
          rc_decay(x.s, x.r.x1a, x.r.x2a, x.r.d1a, x.r.d2a);
          y0[q][k] = x.s.my * x.m;
          y1[q][k] = x.s.ay * x.m;
          y2[q][k] = x.s.by * x.m;
          // rows that do not exist keep e = 0: their index would leave the table
          if (x.on) e[q][k] = __ldg(roots + rc_mod(kyn * x.iy, ny, magic));
          if (MODE != RC_JHW) {
            // q = i u, u = rho t + (v2 + i v3) m_y; p += E q (both rows of the thread)
            const float tt = fmaf(x.v0, y1[q][k], x.v1 * y2[q][k]);
            const float ur = fmaf(x.rh.x, tt, x.v2 * y0[q][k]);
            const float ui = fmaf(x.rh.y, tt, x.v3 * y0[q][k]);
            const float qr = -ui, qi = ur;
            p[2 * k] += fmaf(e[q][k].x, qr, -e[q][k].y * qi);
            p[2 * k + 1] += fmaf(e[q][k].x, qi, e[q][k].y * qr);
          }
          rc_decay(x.s, x.r.x1b, x.r.x2b, x.r.d1b, x.r.d2b);
        }
      }
    }
    float2 a[kChunk];
    if (MODE != RC_JHW) {
      const float2 ws = rc_warp_sum<kChunk>(p, lane);
      constexpr int kLanesPerSlot = 32 / kChunk;
      if ((lane & (kLanesPerSlot - 1)) == 0) part[warp][lane / kLanesPerSlot] = ws;
      __syncthreads();
      if (t < kChunk) {
        float2 u = make_float2(0.f, 0.f);
        for (int wi = 0; wi < nwarps; ++wi) {
          const float2 pw = part[wi][t];
          u.x += pw.x;
          u.y += pw.y;
        }
        asum[t] = u;
        if (MODE == RC_JV && n0 + t < ne) A[(size_t)(n0 + t) * nx + ix] = u;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kChunk; ++k) a[k] = asum[k];
    } else {
#pragma unroll
      for (int k = 0; k < kChunk; ++k)
        a[k] = n0 + k < ne ? __ldg(wt + (size_t)(n0 + k) * nx + ix) : make_float2(0.f, 0.f);
    }
    if (MODE != RC_JV) {
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        RcRow& x = w[q];
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
          // b = conj(E) a; Re conj(dq/dalpha) b for q = i rho m (tangents) and q = i m (rho)
          const float br = fmaf(e[q][k].x, a[k].x, e[q][k].y * a[k].y);
          const float bi = fmaf(e[q][k].x, a[k].y, -e[q][k].y * a[k].x);
          const float imcb = fmaf(x.rh.x, bi, -x.rh.y * br);
          x.g0 = fmaf(y1[q][k], imcb, x.g0);
          x.g1 = fmaf(y2[q][k], imcb, x.g1);
          x.g2 = fmaf(y0[q][k], bi, x.g2);
          x.g3 = fmaf(-y0[q][k], br, x.g3);
        }
      }
    }
  }
  if (MODE != RC_JV) {
#pragma unroll
    for (int q = 0; q < kRows; ++q) {
      const RcRow& x = w[q];
      if (!x.on) continue;
      float* gp = gpart + (size_t)sg * 4 * nv + x.j;
      gp[0] = x.g0 * scale;
      gp[(size_t)nv] = x.g1 * scale;
      gp[2 * (size_t)nv] = x.g2 * scale;
      gp[3 * (size_t)nv] = x.g3 * scale;
    }
  }
}

// g[k][j] = sum_s gpart[s][k][j] (the segments of each voxel, in segment order)
__global__ void rc_segment_sum_kernel(const float* __restrict__ gpart, int nv, int nseg, float* __restrict__ g,
                                      const int* __restrict__ gate) {
  if (gate != nullptr && *gate == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * nv) return;
  float t = 0.f;
  for (int s = 0; s < nseg; ++s) t += gpart[(size_t)s * 4 * nv + i];
  g[i] = t;
}

}  // namespace

bool recompute_supported(const Plan& p) { return p.ny <= kMaxRows && p.npar == 4 && p.slice_iso == 0; }

cudaError_t launch_rc_linearize(const Plan& p, const float* alpha, const float* b1, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  rc_ckpt_kernel<<<(p.nv + 127) / 128, 128, 0, st>>>(alpha, b1, p.cs, p.phi, p.nv, p.ntr, p.rc_seg, p.rc_nseg,
                                                     (float)p.te_ms, (float)(p.tr_ms - p.te_ms),
                                                     p.inversion ? -1.f : 1.f, p.rc_rlx, p.rc_ckpt);
  return cudaGetLastError();
}

// mode 0: J.v's phase-encode sums into A; 1: J^H w from the readout adjoint wt into g;
// 2: J^H J v into g (nkx == nx)
cudaError_t launch_rc_product(const Plan& p, int mode, const float* v, const float2* wt, float* g, cudaStream_t st) {
  if (p.nv == 0) return cudaSuccess;
  const int threads = ((p.ny + kRows - 1) / kRows + 31) / 32 * 32;
  const dim3 grid(p.nx, p.rc_nseg);
  const unsigned magic = p.ny > 1 ? (unsigned)((0x100000000ull + (unsigned)p.ny - 1) / (unsigned)p.ny) : 0u;
  const float scale = mode == RC_JHJV ? (float)p.nx : 1.f;
  const float* b1 = p.rc_has_b1 ? p.rc_b1 : nullptr;
  switch (mode) {
    case RC_JV:
      rc_product_kernel<RC_JV><<<grid, threads, 0, st>>>(p.rc_rlx, p.rc_ckpt, p.rho, p.maskf, b1, v, p.cs, p.phi,
                                                         p.kyi, p.roots, p.nx, p.ny, p.nv, p.ntr, p.rc_seg, magic,
                                                         scale, p.A, nullptr, nullptr, p.gate);
      return cudaGetLastError();
    case RC_JHW:
      rc_product_kernel<RC_JHW><<<grid, threads, 0, st>>>(p.rc_rlx, p.rc_ckpt, p.rho, p.maskf, b1, nullptr, p.cs,
                                                          p.phi, p.kyi, p.roots, p.nx, p.ny, p.nv, p.ntr, p.rc_seg,
                                                          magic, scale, nullptr, wt, p.rc_gpart, p.gate);
      break;
    default:
      rc_product_kernel<RC_JHJV><<<grid, threads, 0, st>>>(p.rc_rlx, p.rc_ckpt, p.rho, p.maskf, b1, v, p.cs,
                                                           p.phi, p.kyi, p.roots, p.nx, p.ny, p.nv, p.ntr, p.rc_seg,
                                                           magic, scale, nullptr, nullptr, p.rc_gpart, p.gate);
      break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n4 = 4 * p.nv;
  rc_segment_sum_kernel<<<(n4 + 255) / 256, 256, 0, st>>>(p.rc_gpart, p.nv, p.rc_nseg, g, p.gate);
  return cudaGetLastError();
}

}  // namespace mrstat
