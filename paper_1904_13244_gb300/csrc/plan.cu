// Host side of libmrstat: plan life cycle, per-TR tables and the C entry points.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace mrstat {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int fail(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? MRSTAT_ERR_OUT_OF_MEMORY : MRSTAT_ERR_CUDA;
}

namespace {

void free_plan(Plan* p) {
  if (p == nullptr) return;
  void* ptrs[] = {p->slice_rot, p->cs, p->phi, p->kyi, p->ky_ptr, p->ky_tr, p->roots, p->ft, p->fh, p->D, p->rho, p->maskf,
                  p->dfwd, p->cf, p->A, p->wt, p->red, p->ticket, p->cg_r, p->cg_p, p->cg_q, p->cg_w, p->cg_bar,
                  p->cg_jv, p->cg_s, p->cg_frozen, p->D2, p->rho2, p->gn_g, p->gn_z, p->gn_res,
                  p->gn_dir, p->gn_q, p->gn_alpha, p->gn_trial, p->gn_s, p->gn_r, p->gn_st,
                  p->gn_rt, p->gn_jv, p->gn_mask, p->gn_sc, p->gn_si, p->bf_ft_hi, p->bf_ft_lo,
                  p->bf_fh_hi, p->bf_fh_lo, p->bf_a_hi, p->bf_a_lo, p->bf_w_hi, p->bf_w_lo, p->dev_err, p->ckpt, p->zpart,
                  p->rc_rlx, p->rc_ckpt, p->rc_gpart, p->rc_b1};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  delete[] p->tc;
  lowrank_free(p->lr);
  delete p;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// exp(-2 pi i a / n) for an integer phase a, reduced exactly modulo n first
inline void unit_root(long long a, long long n, float2* out, bool conj) {
  long long r = a % n;
  if (r < 0) r += n;
  const double ang = -2.0 * M_PI * (double)r / (double)n;
  out->x = (float)std::cos(ang);
  out->y = (float)(conj ? -std::sin(ang) : std::sin(ang));
}

}  // namespace

cudaError_t ensure_timecourses(Plan* p) {
  if (p->D != nullptr) return cudaSuccess;
  const int64_t before = p->bytes;
  cudaError_t e = dalloc(p, &p->D, (size_t)p->nch * p->nq * p->nv);
  p->d_bytes = p->bytes - before;
  return e;
}

cudaError_t ensure_forward_scratch(Plan* p) {
  if (p->dfwd != nullptr) return cudaSuccess;
  return dalloc(p, &p->dfwd, (size_t)p->nq * p->nv);
}

int build_split_tables(Plan* p) {
  if (p->tc != nullptr) return MRSTAT_OK;
  p->kf_pad = (2 * p->nx + 7) / 8 * 8;
  p->ka_pad = (2 * p->nkx + 7) / 8 * 8;
  const size_t nf = (size_t)2 * p->nkx * p->kf_pad, na = (size_t)2 * p->nx * p->ka_pad;
  // real embeddings of the complex DFT matrices (K-major), split into bf16 hi + lo
  std::vector<uint16_t> bfh_f(nf, 0), bfl_f(nf, 0), bfh_a(na, 0), bfl_a(na, 0);
  auto put = [](std::vector<uint16_t>& hi, std::vector<uint16_t>& lo, size_t idx, double v) {
    const uint16_t h = host_bf16((float)v);
    hi[idx] = h;
    lo[idx] = host_bf16((float)(v - (double)host_bf16_to_float(h)));
  };
  for (int k = 0; k < p->nkx; ++k)
    for (int ix = 0; ix < p->nx; ++ix) {
      const long long kx = k - p->nkx / 2;
      long long r = (kx * ix) % p->nx;
      if (r < 0) r += p->nx;
      const double ang = -2.0 * M_PI * (double)r / (double)p->nx;
      const double fr = std::cos(ang), fi = std::sin(ang);  // F = exp(-2 pi i kx ix / nx)
      // forward: rows 2k (re), 2k+1 (im) of the output; columns 2ix (re A), 2ix+1 (im A)
      put(bfh_f, bfl_f, (size_t)(2 * k) * p->kf_pad + 2 * ix, fr);
      put(bfh_f, bfl_f, (size_t)(2 * k) * p->kf_pad + 2 * ix + 1, -fi);
      put(bfh_f, bfl_f, (size_t)(2 * k + 1) * p->kf_pad + 2 * ix, fi);
      put(bfh_f, bfl_f, (size_t)(2 * k + 1) * p->kf_pad + 2 * ix + 1, fr);
      // adjoint with G = conj(F): rows 2ix, 2ix+1 of the output; columns 2k, 2k+1 of w
      put(bfh_a, bfl_a, (size_t)(2 * ix) * p->ka_pad + 2 * k, fr);
      put(bfh_a, bfl_a, (size_t)(2 * ix) * p->ka_pad + 2 * k + 1, fi);
      put(bfh_a, bfl_a, (size_t)(2 * ix + 1) * p->ka_pad + 2 * k, -fi);
      put(bfh_a, bfl_a, (size_t)(2 * ix + 1) * p->ka_pad + 2 * k + 1, fr);
    }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  chk(cudaMalloc(&p->bf_ft_hi, nf * 2));
  chk(cudaMalloc(&p->bf_ft_lo, nf * 2));
  chk(cudaMalloc(&p->bf_fh_hi, na * 2));
  chk(cudaMalloc(&p->bf_fh_lo, na * 2));
  chk(cudaMalloc(&p->bf_a_hi, (size_t)p->ntr * p->kf_pad * 2));
  chk(cudaMalloc(&p->bf_a_lo, (size_t)p->ntr * p->kf_pad * 2));
  chk(cudaMalloc(&p->bf_w_hi, (size_t)p->ntr * p->ka_pad * 2));
  chk(cudaMalloc(&p->bf_w_lo, (size_t)p->ntr * p->ka_pad * 2));
  if (e != cudaSuccess) return cuda_fail(e, "split-BF16 table allocation");
  p->bytes += (int64_t)(2 * (nf + na) * 2 + 2 * (size_t)p->ntr * (p->kf_pad + p->ka_pad) * 2);
  chk(cudaMemcpy(p->bf_ft_hi, bfh_f.data(), nf * 2, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->bf_ft_lo, bfl_f.data(), nf * 2, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->bf_fh_hi, bfh_a.data(), na * 2, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->bf_fh_lo, bfl_a.data(), na * 2, cudaMemcpyHostToDevice));
  chk(cudaMemset(p->bf_a_hi, 0, (size_t)p->ntr * p->kf_pad * 2));
  chk(cudaMemset(p->bf_a_lo, 0, (size_t)p->ntr * p->kf_pad * 2));
  chk(cudaMemset(p->bf_w_hi, 0, (size_t)p->ntr * p->ka_pad * 2));
  chk(cudaMemset(p->bf_w_lo, 0, (size_t)p->ntr * p->ka_pad * 2));
  TcOperand* tc = new TcOperand[4];
  chk(make_split_operand(&tc[0], p->bf_a_hi, p->bf_a_lo, p->ntr, 2 * p->nx, p->kf_pad, true));
  chk(make_split_operand(&tc[1], p->bf_ft_hi, p->bf_ft_lo, 2 * p->nkx, 2 * p->nx, p->kf_pad, false));
  chk(make_split_operand(&tc[2], p->bf_w_hi, p->bf_w_lo, p->ntr, 2 * p->nkx, p->ka_pad, true));
  chk(make_split_operand(&tc[3], p->bf_fh_hi, p->bf_fh_lo, 2 * p->nx, 2 * p->nkx, p->ka_pad, false));
  if (e != cudaSuccess) {
    delete[] tc;
    return cuda_fail(e, "split-BF16 tables");
  }
  p->tc = tc;
  return MRSTAT_OK;
}

cudaEvent_t pool_event(Plan* p) {
  if (p->pool_used == p->event_pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    p->event_pool.push_back(e);
  }
  return p->event_pool[p->pool_used++];
}

int do_jvp(Plan* p, const float* v, float2* jv, cudaStream_t st) {
  cudaError_t e;
  if (p->rc_seg > 0) {
    {
      Span sp(p, MRSTAT_K_YCONTRACT, st);
      e = launch_rc_product(*p, 0, v, nullptr, nullptr, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "recompute J.v launch");
    return do_xdft(p, p->A, jv, p->gate, st);
  }
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = launch_prep_jvp(*p, v, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prep_jvp launch");
  {
    Span sp(p, MRSTAT_K_YCONTRACT, st);
    e = launch_ycontract(*p, p->D, p->nch, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ycontract launch");
  return do_xdft(p, p->A, jv, p->gate, st);
}

int do_jhw(Plan* p, const float2* w, float* g, cudaStream_t st) {
  const int status = do_xdft_adj(p, w, p->wt, p->gate, st);
  if (status != MRSTAT_OK) return status;
  cudaError_t e;
  if (p->rc_seg > 0) {
    {
      Span sp(p, MRSTAT_K_JHW_DOT, st, 1, 2);  // the product and the segment sum
      e = launch_rc_product(*p, 1, nullptr, p->wt, g, st);
    }
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "recompute J^H w launch");
  }
  {
    Span sp(p, MRSTAT_K_JHW_DOT, st);
    e = launch_jhw_dot(*p, g, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "jhw_dot launch");
  return MRSTAT_OK;
}

int do_signal(Plan* p, const float4* D, const float2* rho_masked, float2* s, cudaStream_t st) {
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = launch_prep_rho(*p, rho_masked, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prep_rho launch");
  {
    // the signal only needs channel 0 (m_y) and coefficient 0 (rho)
    Span sp(p, MRSTAT_K_YCONTRACT, st);
    e = launch_ycontract(*p, D, 1, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ycontract launch");
  return do_xdft(p, p->A, s, nullptr, st);
}

int do_xdft(Plan* p, const float2* A, float2* out, const int* gate, cudaStream_t st) {
  cudaError_t e;
  if (p->form == MRSTAT_FORM_SPLIT_BF16) {
    {
      Span sp(p, MRSTAT_K_VECTOR, st);
      e = launch_split_bf16(reinterpret_cast<const float*>(A), p->ntr, 2 * p->nx, 2 * p->nx, p->bf_a_hi,
                            p->bf_a_lo, p->kf_pad, gate, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "split launch");
    Span sp(p, MRSTAT_K_XDFT, st);
    e = launch_tc_gemm(p->tc[0], p->tc[1], reinterpret_cast<float*>(out), p->ntr, 2 * p->nkx, 2 * p->nx,
                       2 * p->nkx, 3, gate, p->dev_err, st);
  } else {
    Span sp(p, MRSTAT_K_XDFT, st);
    e = launch_cgemm(A, p->ft, out, p->ntr, p->nkx, p->nx, gate, st);
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "x-DFT launch");
}

int do_xdft_adj(Plan* p, const float2* w, float2* out, const int* gate, cudaStream_t st) {
  cudaError_t e;
  if (p->form == MRSTAT_FORM_SPLIT_BF16) {
    {
      Span sp(p, MRSTAT_K_VECTOR, st);
      e = launch_split_bf16(reinterpret_cast<const float*>(w), p->ntr, 2 * p->nkx, 2 * p->nkx, p->bf_w_hi,
                            p->bf_w_lo, p->ka_pad, gate, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "split launch");
    Span sp(p, MRSTAT_K_XDFT_ADJ, st);
    e = launch_tc_gemm(p->tc[2], p->tc[3], reinterpret_cast<float*>(out), p->ntr, 2 * p->nx, 2 * p->nkx,
                       2 * p->nx, 3, gate, p->dev_err, st);
  } else {
    Span sp(p, MRSTAT_K_XDFT_ADJ, st);
    e = launch_cgemm(w, p->fh, out, p->ntr, p->nx, p->nkx, gate, st);
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "x-DFT adjoint launch");
}

int do_linearize(Plan* p, const float* alpha, const float* b1, const uint8_t* mask, float4* D,
                 float2* rho, cudaStream_t st) {
  cudaError_t e;
  {
    Span sp(p, MRSTAT_K_VECTOR, st);
    e = launch_prep_linearize(*p, alpha, mask, rho, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prep_linearize launch");
  if (p->slice_iso > 0 && b1 != nullptr)
    return fail(MRSTAT_ERR_UNSUPPORTED, "the slice-profile model takes B1 = 1 (no map)");
  {
    Span sp(p, MRSTAT_K_BLOCH, st);
    e = p->slice_iso > 0 ? launch_bloch_slice(*p, alpha, mask, D, 3, st)
                         : launch_bloch(*p, alpha, b1, mask, D, p->nch, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "bloch launch");
  return MRSTAT_OK;
}

// J^H J v.  With a fully sampled readout (nkx == nx: kx runs over a whole period of the
// x frequencies) the readout DFT and its adjoint cancel, F^H F = nx I, so
// W~ = nx A and the two x-DFTs are skipped: exact, not an approximation.
int do_jhjv(Plan* p, const float* v, float* out, cudaStream_t st, double* vdot, double* vv) {
  if (p->lr && p->lr->active) return lowrank_jhjv(p, v, out, st, vdot, vv);
  if (vv != nullptr) {
    const int s = do_jhjv(p, v, out, st, vdot);
    if (s != MRSTAT_OK) return s;
    const cudaError_t e = do_dot(p, v, v, (int64_t)p->npar * p->nv, vv, st);
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "dot launch");
  }
  if (vdot != nullptr) {
    const int s = do_jhjv(p, v, out, st, nullptr);
    if (s != MRSTAT_OK) return s;
    const cudaError_t e = do_dot(p, v, out, (int64_t)p->npar * p->nv, vdot, st);
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "dot launch");
  }
  if (p->nkx == p->nx && p->rc_seg > 0) {
    // the simulation, both phase-encode sums and the tangent products in one pass
    cudaError_t e;
    {
      Span sp(p, MRSTAT_K_JHW_DOT, st, 1, 2);  // the product and the segment sum
      e = launch_rc_product(*p, 2, v, nullptr, out, st);
    }
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "recompute J^H J v launch");
  }
  if (p->nkx == p->nx) {
    cudaError_t e;
    {
      Span sp(p, MRSTAT_K_VECTOR, st);
      e = launch_prep_jvp(*p, v, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "prep_jvp launch");
    {
      Span sp(p, MRSTAT_K_YCONTRACT, st);
      e = launch_ycontract(*p, p->D, p->nch, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "ycontract launch");
    {
      Span sp(p, MRSTAT_K_JHW_DOT, st);
      e = launch_jhw_dot(*p, out, st, p->A, (float)p->nx);
    }
    return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "jhw_dot launch");
  }
  int s = do_jvp(p, v, p->cg_jv, st);
  if (s == MRSTAT_OK) s = do_jhw(p, p->cg_jv, out, st);
  return s;
}

cudaError_t do_dot(Plan* p, const float* a, const float* b, int64_t n, double* out, cudaStream_t st) {
  Span sp(p, MRSTAT_K_VECTOR, st);
  return launch_dot(a, b, n, p->red, p->ticket, out, st, p->gate);
}

}  // namespace mrstat

using namespace mrstat;

struct mrstat_plan : public Plan {};

extern "C" {

const char* mrstat_status_string(int status) {
  switch (status) {
    case MRSTAT_OK: return "ok";
    case MRSTAT_ERR_INVALID_ARG: return "invalid argument";
    case MRSTAT_ERR_SHAPE: return "invalid shape";
    case MRSTAT_ERR_NOT_LINEARIZED: return "plan not linearised";
    case MRSTAT_ERR_CUDA: return "CUDA error";
    case MRSTAT_ERR_NONFINITE: return "non-finite value";
    case MRSTAT_ERR_TIMEOUT: return "iteration budget exhausted";
    case MRSTAT_ERR_UNSUPPORTED: return "unsupported";
    case MRSTAT_ERR_OUT_OF_MEMORY: return "out of device memory";
    default: return "unknown status";
  }
}

const char* mrstat_last_error(void) { return g_last_error.c_str(); }

int mrstat_plan_inject_grid_stall(mrstat_plan* plan, int32_t block) {
  if (plan == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan");
  // the persistent launches have two blocks per image column
  if (block >= 2 * plan->nx) return fail(MRSTAT_ERR_INVALID_ARG, "stall block outside the persistent grid (2 nx blocks)");
  plan->grid_stall_block = block < 0 ? -1 : block;
  return MRSTAT_OK;
}

int mrstat_plan_check(mrstat_plan* plan) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan");
  DeviceGuard g(plan->device);
  int flag = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&flag, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "plan check");
  if (flag) {
    cudaMemset(plan->dev_err, 0, sizeof(int));
    return fail(MRSTAT_ERR_TIMEOUT, "a kernel's bounded wait ran out (tensor-core pipeline or grid counter)");
  }
  return MRSTAT_OK;
}

int mrstat_profile_start(mrstat_plan* plan, uint32_t kernel_mask) {
  if (plan == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan");
  for (int64_t& c : plan->launches) c = 0;
  for (int64_t& c : plan->kernel_launches) c = 0;
  plan->marks.clear();
  plan->pool_used = 0;
  plan->prof_mask = kernel_mask;
  plan->prof_on = true;
  return MRSTAT_OK;
}

int mrstat_profile_stop(mrstat_plan* plan, mrstat_kernel_stats* out) {
  if (plan == nullptr || out == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard g(plan->device);
  std::memset(out, 0, sizeof(*out));
  for (int k = 0; k < 8; ++k) {
    out->launches[k] = plan->launches[k];
    out->kernels[k] = plan->kernel_launches[k];
  }
  for (const Plan::Mark& m : plan->marks) {
    cudaError_t e = cudaEventSynchronize(m.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, m.a, m.b);
    if (e != cudaSuccess) {
      plan->prof_on = false;
      return cuda_fail(e, "profile events");
    }
    out->ms[m.kid] += ms;
    out->timed[m.kid] += m.n;
  }
  plan->marks.clear();
  plan->pool_used = 0;
  plan->prof_on = false;
  return MRSTAT_OK;
}

int mrstat_plan_create(const mrstat_seq* seq, int32_t form, mrstat_plan** out) {
  MRSTAT_ABI_RANGE();
  g_last_error.clear();
  if (out == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (seq == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "seq is NULL");
  const bool estimate_b1 = (form & MRSTAT_ESTIMATE_B1) != 0;
  form &= ~MRSTAT_ESTIMATE_B1;
  if (form != MRSTAT_FORM_PLAIN_FP32 && form != MRSTAT_FORM_SPLIT_BF16)
    return fail(MRSTAT_ERR_INVALID_ARG, "form %d not available", form);
  if (seq->nx < 1 || seq->nx > 2048 || seq->ny < 1 || seq->ny > 2048 || seq->nkx < 1 ||
      seq->nkx > 4096 || seq->ntr < 1 || seq->ntr > 65536)
    return fail(MRSTAT_ERR_SHAPE, "sizes out of range: nx=%d ny=%d nkx=%d ntr=%d", seq->nx, seq->ny,
                seq->nkx, seq->ntr);
  if (seq->flip_rad == nullptr || seq->ky == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "flip_rad or ky is NULL");
  if (!(seq->tr_ms > 0.0) || !(seq->te_ms > 0.0) || !(seq->te_ms < seq->tr_ms) ||
      !std::isfinite(seq->tr_ms))
    return fail(MRSTAT_ERR_INVALID_ARG, "need 0 < te_ms < tr_ms (te=%g tr=%g)", seq->te_ms, seq->tr_ms);
  const int lo = -(seq->ny / 2), hi = seq->ny - seq->ny / 2;
  for (int n = 0; n < seq->ntr; ++n) {
    if (!std::isfinite(seq->flip_rad[n]) || seq->flip_rad[n] < 0.f)
      return fail(MRSTAT_ERR_INVALID_ARG, "flip_rad[%d] = %g is not a finite non-negative angle", n,
                  (double)seq->flip_rad[n]);
    if (seq->ky[n] < lo || seq->ky[n] >= hi)
      return fail(MRSTAT_ERR_SHAPE, "ky[%d] = %d outside [%d, %d)", n, seq->ky[n], lo, hi);
  }

  mrstat_plan* p = new mrstat_plan();
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return fail(MRSTAT_ERR_CUDA, "no CUDA device");
  }
  p->nx = seq->nx;
  p->ny = seq->ny;
  p->nkx = seq->nkx;
  p->ntr = seq->ntr;
  p->ntr_pad = (seq->ntr + 3) / 4 * 4;
  p->nq = p->ntr_pad / 4;
  p->nv = seq->nx * seq->ny;
  p->form = form;
  p->npar = estimate_b1 ? 5 : 4;
  p->nch = estimate_b1 ? 4 : kChannels;
  p->tr_ms = seq->tr_ms;
  p->te_ms = seq->te_ms;
  p->inversion = seq->inversion != 0;
  p->alternate = seq->alternate_phase != 0;

  // host tables (float64, rounded once)
  std::vector<float2> cs(p->ntr_pad);
  std::vector<float> phi(p->ntr_pad, 0.f);
  std::vector<int> kyi(p->ntr_pad, 0);
  for (int n = 0; n < p->ntr_pad; ++n) {
    double ph = 0.0;
    if (n < p->ntr) {
      ph = (double)seq->flip_rad[n];
      if (p->alternate && (n & 1)) ph = -ph;  // RF phase 180 degrees rotates about +x
      kyi[n] = ((seq->ky[n] % p->ny) + p->ny) % p->ny;
    }
    phi[n] = (float)ph;
    cs[n] = make_float2((float)std::cos(ph), (float)std::sin(ph));
  }
  std::vector<int> ky_ptr(p->ny + 1, 0), ky_tr(std::max(p->ntr, 1), 0);
  for (int n = 0; n < p->ntr; ++n) ky_ptr[kyi[n] + 1]++;
  for (int k = 0; k < p->ny; ++k) ky_ptr[k + 1] += ky_ptr[k];
  {
    std::vector<int> fill(ky_ptr.begin(), ky_ptr.end() - 1);
    for (int n = 0; n < p->ntr; ++n) ky_tr[fill[kyi[n]]++] = n;
  }
  std::vector<float2> roots(p->ny), ft((size_t)p->nx * p->nkx), fh((size_t)p->nkx * p->nx);
  for (int k = 0; k < p->ny; ++k) unit_root(k, p->ny, &roots[k], false);
  for (int ix = 0; ix < p->nx; ++ix)
    for (int k = 0; k < p->nkx; ++k) {
      const long long kx = k - p->nkx / 2;
      unit_root(kx * ix, p->nx, &ft[(size_t)ix * p->nkx + k], false);
      unit_root(kx * ix, p->nx, &fh[(size_t)k * p->nx + ix], true);
    }

  const size_t nv = p->nv, nq = p->nq;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  chk(dalloc(p, &p->cs, p->ntr_pad));
  chk(dalloc(p, &p->phi, p->ntr_pad));
  chk(dalloc(p, &p->kyi, p->ntr_pad));
  chk(dalloc(p, &p->roots, p->ny));
  chk(dalloc(p, &p->ky_ptr, ky_ptr.size()));
  chk(dalloc(p, &p->ky_tr, ky_tr.size()));
  chk(dalloc(p, &p->ft, ft.size()));
  chk(dalloc(p, &p->fh, fh.size()));
  chk(dalloc(p, &p->rho, nv));
  chk(dalloc(p, &p->maskf, nv));
  chk(dalloc(p, &p->cf, (size_t)kMaxChannels * nv));
  // A has the padded TR rows too (zero, never written): J^H J v reads it as W~ over TR quads
  chk(dalloc(p, &p->A, (size_t)p->ntr_pad * p->nx));
  chk(dalloc(p, &p->wt, (size_t)p->ntr_pad * p->nx));
  chk(dalloc(p, &p->red, (size_t)kRedSlots));
  chk(dalloc(p, &p->ticket, 1));
  chk(dalloc(p, &p->cg_r, (size_t)p->npar * nv));
  chk(dalloc(p, &p->cg_p, (size_t)p->npar * nv));
  chk(dalloc(p, &p->cg_q, (size_t)p->npar * nv));
  chk(dalloc(p, &p->cg_w, (size_t)p->npar * nv));
  chk(dalloc(p, &p->cg_bar, 2));
  chk(dalloc(p, &p->cg_jv, (size_t)p->ntr * p->nkx));
  chk(dalloc(p, &p->cg_frozen, 1));
  chk(dalloc(p, &p->dev_err, 1));
  if (e != cudaSuccess) {
    int st = cuda_fail(e, "plan allocation");
    free_plan(p);
    return st;
  }
  chk(cudaMemcpy(p->cs, cs.data(), cs.size() * sizeof(float2), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->phi, phi.data(), phi.size() * sizeof(float), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->kyi, kyi.data(), kyi.size() * sizeof(int), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->roots, roots.data(), roots.size() * sizeof(float2), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->ky_ptr, ky_ptr.data(), ky_ptr.size() * sizeof(int), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->ky_tr, ky_tr.data(), ky_tr.size() * sizeof(int), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->ft, ft.data(), ft.size() * sizeof(float2), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(p->fh, fh.data(), fh.size() * sizeof(float2), cudaMemcpyHostToDevice));
  chk(cudaMemset(p->wt, 0, (size_t)p->ntr_pad * p->nx * sizeof(float2)));
  chk(cudaMemset(p->A, 0, (size_t)p->ntr_pad * p->nx * sizeof(float2)));
  chk(cudaMemset(p->ticket, 0, sizeof(unsigned)));
  chk(cudaMemset(p->dev_err, 0, sizeof(int)));
  if (e == cudaSuccess && form == MRSTAT_FORM_SPLIT_BF16) {
    const int st = build_split_tables(p);
    if (st != MRSTAT_OK) {
      free_plan(p);
      return st;
    }
  }
  chk(cudaDeviceSynchronize());
  if (e != cudaSuccess) {
    int st = cuda_fail(e, "plan tables");
    free_plan(p);
    return st;
  }
  *out = p;
  return MRSTAT_OK;
}

int mrstat_plan_destroy(mrstat_plan* plan) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr) return MRSTAT_OK;
  DeviceGuard g(plan->device);
  cudaDeviceSynchronize();
  free_plan(plan);
  return MRSTAT_OK;
}

int mrstat_plan_info(const mrstat_plan* plan, mrstat_plan_info_t* info) {
  if (plan == nullptr || info == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL argument");
  info->nx = plan->nx;
  info->ny = plan->ny;
  info->nkx = plan->nkx;
  info->ntr = plan->ntr;
  info->nv = plan->nv;
  info->form = plan->form;
  info->ntr_padded = plan->ntr_pad;
  info->device_bytes = plan->bytes;
  info->timecourse_bytes = plan->d_bytes;
  info->npar = plan->npar;
  return MRSTAT_OK;
}

int mrstat_linearize(mrstat_plan* plan, const float* alpha, const float* b1, const uint8_t* mask,
                     void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || alpha == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan or alpha");
  if (plan->npar == 5 && b1 != nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "B1 is estimated (alpha row 4): pass b1 = NULL");
  DeviceGuard g(plan->device);
  cudaStream_t st = as_stream(stream);
  plan->linearized = false;
  if (plan->lr) plan->lr->active = false;
  if (plan->rc_seg > 0) {
    // recompute form: rho, the mask, the B1 map, relaxation factors and segment states
    cudaError_t e;
    {
      Span sp(plan, MRSTAT_K_VECTOR, st);
      e = launch_prep_linearize(*plan, alpha, mask, plan->rho, st);
    }
    plan->rc_has_b1 = b1 != nullptr;
    if (e == cudaSuccess && b1 != nullptr)
      e = cudaMemcpyAsync(plan->rc_b1, b1, (size_t)plan->nv * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
      Span sp(plan, MRSTAT_K_BLOCH, st);
      e = launch_rc_linearize(*plan, alpha, b1, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "recompute linearisation");
    plan->linearized = true;
    return MRSTAT_OK;
  }
  cudaError_t ea = ensure_timecourses(plan);
  if (ea != cudaSuccess) return cuda_fail(ea, "time-course allocation");
  const int status = do_linearize(plan, alpha, b1, mask, plan->D, plan->rho, st);
  if (status != MRSTAT_OK) return status;
  plan->linearized = true;
  return MRSTAT_OK;
}

int mrstat_forward(mrstat_plan* plan, const float* alpha, const float* b1, const uint8_t* mask,
                   float* s, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || alpha == nullptr || s == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, alpha or s");
  if (plan->npar == 5 && b1 != nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "B1 is estimated (alpha row 4): pass b1 = NULL");
  if (plan->slice_iso > 0 && b1 != nullptr)
    return fail(MRSTAT_ERR_UNSUPPORTED, "the slice-profile model takes B1 = 1 (no map)");
  DeviceGuard g(plan->device);
  cudaStream_t st = as_stream(stream);
  cudaError_t e = ensure_forward_scratch(plan);
  if (e != cudaSuccess) return cuda_fail(e, "forward scratch allocation");
  {
    Span sp(plan, MRSTAT_K_BLOCH, st);
    e = plan->slice_iso > 0 ? launch_bloch_slice(*plan, alpha, mask, plan->dfwd, 1, st)
                            : launch_bloch(*plan, alpha, b1, mask, plan->dfwd, 1, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "bloch launch");
  {
    Span sp(plan, MRSTAT_K_VECTOR, st);
    e = launch_prep_forward(*plan, alpha, mask, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prep_forward launch");
  {
    Span sp(plan, MRSTAT_K_YCONTRACT, st);
    e = launch_ycontract(*plan, plan->dfwd, 1, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ycontract launch");
  return do_xdft(plan, plan->A, reinterpret_cast<float2*>(s), nullptr, st);
}

int mrstat_jvp(mrstat_plan* plan, const float* v, float* jv, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || v == nullptr || jv == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, v or jv");
  if (!plan->linearized) return fail(MRSTAT_ERR_NOT_LINEARIZED, "mrstat_jvp before mrstat_linearize");
  DeviceGuard g(plan->device);
  if (plan->lr && plan->lr->active) return lowrank_jvp(plan, v, reinterpret_cast<float2*>(jv), as_stream(stream));
  return do_jvp(plan, v, reinterpret_cast<float2*>(jv), as_stream(stream));
}

int mrstat_jhw(mrstat_plan* plan, const float* w, float* gout, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || w == nullptr || gout == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, w or g");
  if (!plan->linearized) return fail(MRSTAT_ERR_NOT_LINEARIZED, "mrstat_jhw before mrstat_linearize");
  DeviceGuard g(plan->device);
  if (plan->lr && plan->lr->active) return lowrank_jhw(plan, reinterpret_cast<const float2*>(w), gout, as_stream(stream));
  return do_jhw(plan, reinterpret_cast<const float2*>(w), gout, as_stream(stream));
}

int mrstat_timecourses(mrstat_plan* plan, int32_t channel, float* out, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || out == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan or out");
  if (channel < 0 || channel >= plan->nch)
    return fail(MRSTAT_ERR_INVALID_ARG, "channel %d not in [0, %d)", channel, plan->nch);
  if (plan->rc_seg > 0) return fail(MRSTAT_ERR_UNSUPPORTED, "the recompute form keeps no time courses");
  if (!plan->linearized || plan->D == nullptr || (plan->lr && plan->lr->active))
    return fail(MRSTAT_ERR_NOT_LINEARIZED, "timecourses need an exact mrstat_linearize");
  DeviceGuard g(plan->device);
  Span sp(plan, MRSTAT_K_VECTOR, as_stream(stream));
  cudaError_t e = launch_timecourse(*plan, channel, out, as_stream(stream));
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "timecourse launch");
}

int mrstat_dot(mrstat_plan* plan, const float* a, const float* b, int64_t n, double* out,
               void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || out == nullptr || n < 0 || (n > 0 && (a == nullptr || b == nullptr)))
    return fail(MRSTAT_ERR_INVALID_ARG, "bad argument to mrstat_dot");
  DeviceGuard g(plan->device);
  cudaError_t e = do_dot(plan, a, b, n, out, as_stream(stream));
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "dot launch");
}

int mrstat_forward_ckpt(mrstat_plan* plan, const float* alpha, const float* b1, const uint8_t* mask,
                        int32_t interval, float* s, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || alpha == nullptr || s == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, alpha or s");
  if (interval < 4 || interval % 4 != 0)
    return fail(MRSTAT_ERR_INVALID_ARG, "checkpoint interval %d is not a positive multiple of 4", interval);
  if (plan->npar != 4) return fail(MRSTAT_ERR_UNSUPPORTED, "the checkpointed form does not estimate B1");
  if (plan->slice_iso > 0) return fail(MRSTAT_ERR_UNSUPPORTED, "the checkpointed form uses the hard-pulse model");
  DeviceGuard g(plan->device);
  cudaStream_t st = as_stream(stream);
  cudaError_t e = ensure_forward_scratch(plan);
  if (e != cudaSuccess) return cuda_fail(e, "forward scratch allocation");
  const int nseg = (plan->ntr + interval - 1) / interval;
  if (nseg > plan->ckpt_cap) {
    cudaStreamSynchronize(st);
    if (plan->ckpt) {
      cudaFree(plan->ckpt);
      cudaFree(plan->zpart);
      plan->bytes -= 2 * (int64_t)plan->ckpt_cap * 6 * plan->nv * (int64_t)sizeof(float);
      plan->ckpt = plan->zpart = nullptr;
      plan->ckpt_cap = 0;
    }
    e = dalloc(plan, &plan->ckpt, (size_t)nseg * 6 * plan->nv);
    if (e == cudaSuccess) e = dalloc(plan, &plan->zpart, (size_t)nseg * 6 * plan->nv);
    if (e != cudaSuccess) return cuda_fail(e, "checkpoint allocation");
    plan->ckpt_cap = nseg;
  }
  plan->ckpt_ready = false;
  {
    Span sp(plan, MRSTAT_K_BLOCH, st);
    e = launch_bloch_ckpt(*plan, alpha, b1, mask, interval, nseg, plan->ckpt, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "checkpointed Bloch launch");
  {
    Span sp(plan, MRSTAT_K_VECTOR, st);
    e = launch_prep_forward(*plan, alpha, mask, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prep_forward launch");
  {
    Span sp(plan, MRSTAT_K_YCONTRACT, st);
    e = launch_ycontract(*plan, plan->dfwd, 1, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "ycontract launch");
  const int status = do_xdft(plan, plan->A, reinterpret_cast<float2*>(s), nullptr, st);
  if (status != MRSTAT_OK) return status;
  plan->ckpt_interval = interval;
  plan->ckpt_nseg = nseg;
  plan->ckpt_alpha = alpha;
  plan->ckpt_b1 = b1;
  plan->ckpt_mask = mask;
  plan->ckpt_ready = true;
  return MRSTAT_OK;
}

int mrstat_jhw_ckpt(mrstat_plan* plan, const float* w, float* gout, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || w == nullptr || gout == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, w or g");
  if (!plan->ckpt_ready)
    return fail(MRSTAT_ERR_NOT_LINEARIZED, "mrstat_jhw_ckpt before mrstat_forward_ckpt");
  DeviceGuard g(plan->device);
  cudaStream_t st = as_stream(stream);
  int status = do_xdft_adj(plan, reinterpret_cast<const float2*>(w), plan->wt, nullptr, st);
  if (status != MRSTAT_OK) return status;
  cudaError_t e;
  {
    Span sp(plan, MRSTAT_K_JHW_DOT, st, 1, 2);  // the segment kernel and the segment sum
    e = launch_segment_jhw(*plan, plan->ckpt_alpha, plan->ckpt_b1, plan->ckpt_mask, plan->ckpt_interval,
                           plan->ckpt_nseg, plan->ckpt, plan->zpart, gout, st);
  }
  return e == cudaSuccess ? MRSTAT_OK : cuda_fail(e, "segment recompute launch");
}

int mrstat_jhjv(mrstat_plan* plan, const float* v, float* out, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || v == nullptr || out == nullptr)
    return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan, v or out");
  if (!plan->linearized) return fail(MRSTAT_ERR_NOT_LINEARIZED, "mrstat_jhjv before a linearisation");
  DeviceGuard g(plan->device);
  return do_jhjv(plan, v, out, as_stream(stream));
}

int mrstat_cg_fixed(mrstat_plan* plan, const float* rhs, float* x, int32_t iters, void* stream) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || rhs == nullptr || x == nullptr || iters < 0)
    return fail(MRSTAT_ERR_INVALID_ARG, "bad argument to mrstat_cg_fixed");
  if (!plan->linearized) return fail(MRSTAT_ERR_NOT_LINEARIZED, "mrstat_cg_fixed before mrstat_linearize");
  DeviceGuard g(plan->device);
  cudaStream_t st = as_stream(stream);
  if (plan->cg_s_cap < iters + 1) {
    if (plan->cg_s) {
      cudaStreamSynchronize(st);
      cudaFree(plan->cg_s);
      plan->bytes -= (int64_t)plan->cg_s_cap * 4 * sizeof(double);
      plan->cg_s = nullptr;
      plan->cg_s_cap = 0;
    }
    const int cap = iters + 1 < 64 ? 64 : iters + 1;
    cudaError_t e = dalloc(plan, &plan->cg_s, (size_t)cap * 4);
    if (e != cudaSuccess) return cuda_fail(e, "CG scalar allocation");
    plan->cg_s_cap = cap;
  }
  const int64_t n = (int64_t)plan->npar * plan->nv;
  double* sc = plan->cg_s;
  plan->cg_last_iters = -1;
  {
    // the low-rank column path runs the whole solve in one persistent launch
    cudaError_t pe;
    if (lowrank_cg_fixed_persistent(plan, rhs, x, iters, st, &pe)) {
      if (pe != cudaSuccess) return cuda_fail(pe, "persistent CG launch");
      plan->cg_last_iters = iters;
      return MRSTAT_OK;
    }
  }
  // Chronopoulos-Gear form: the product is applied to the residual, w = B r, with
  // delta = <r, w> and gamma = <r, r> formed in the same pass; one vector kernel then
  // updates p, q = B p, x and r.  Per iteration k the scalars sit at sc[4k..4k+2].
  cudaError_t e = cudaMemsetAsync(plan->cg_frozen, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    Span sp(plan, MRSTAT_K_VECTOR, st);
    e = launch_cg_init(rhs, x, plan->cg_r, plan->cg_p, plan->cg_q, n, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "CG init");
  for (int it = 0; it < iters; ++it) {
    double* sk = sc + 4 * it;
    const int s = do_jhjv(plan, plan->cg_r, plan->cg_w, st, sk, sk + 1);
    if (s != MRSTAT_OK) return s;
    {
      Span sp(plan, MRSTAT_K_VECTOR, st);
      e = launch_cg_cg_step(x, plan->cg_r, plan->cg_p, plan->cg_q, plan->cg_w, n, sk, it > 0 ? sk - 4 : nullptr,
                            plan->cg_frozen, it, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "CG iteration");
  }
  plan->cg_last_iters = iters;
  return MRSTAT_OK;
}

int mrstat_set_recompute(mrstat_plan* plan, int32_t segment) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || segment < 0) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan or negative segment");
  if (segment > 0 && !recompute_supported(*plan))
    return fail(MRSTAT_ERR_UNSUPPORTED, "the recompute form needs ny <= 256, B1 known (npar 4) and hard pulses");
  DeviceGuard g(plan->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "recompute set-up");
  auto release = [&](float*& q, size_t count) {
    if (q) {
      cudaFree(q);
      plan->bytes -= (int64_t)(count * sizeof(float));
      q = nullptr;
    }
  };
  const size_t nv = (size_t)plan->nv;
  release(plan->rc_rlx, 8 * nv);
  release(plan->rc_ckpt, (size_t)plan->rc_nseg * 6 * nv);
  release(plan->rc_gpart, (size_t)plan->rc_nseg * 4 * nv);
  release(plan->rc_b1, nv);
  plan->rc_seg = 0;
  plan->rc_nseg = 0;
  plan->linearized = false;
  if (plan->lr) plan->lr->active = false;
  if (segment == 0) return MRSTAT_OK;
  const int seg = std::min<int>(segment, plan->ntr);
  const int nseg = (plan->ntr + seg - 1) / seg;
  e = dalloc(plan, &plan->rc_rlx, 8 * nv);
  if (e == cudaSuccess) e = dalloc(plan, &plan->rc_ckpt, (size_t)nseg * 6 * nv);
  if (e == cudaSuccess) e = dalloc(plan, &plan->rc_gpart, (size_t)nseg * 4 * nv);
  if (e == cudaSuccess) e = dalloc(plan, &plan->rc_b1, nv);
  plan->rc_seg = seg;
  plan->rc_nseg = nseg;
  if (e != cudaSuccess) {
    const int s = cuda_fail(e, "recompute work space");
    mrstat_set_recompute(plan, 0);
    return s;
  }
  return MRSTAT_OK;
}

int mrstat_cg_applied(mrstat_plan* plan, int32_t* applied) {
  MRSTAT_ABI_RANGE();
  if (plan == nullptr || applied == nullptr) return fail(MRSTAT_ERR_INVALID_ARG, "NULL plan or applied");
  if (plan->cg_last_iters < 0) return fail(MRSTAT_ERR_NOT_LINEARIZED, "mrstat_cg_applied before mrstat_cg_fixed");
  DeviceGuard g(plan->device);
  int frozen = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&frozen, plan->cg_frozen, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "CG iteration count");
  *applied = frozen > 0 ? frozen - 1 : plan->cg_last_iters;
  return MRSTAT_OK;
}

}  // extern "C"
