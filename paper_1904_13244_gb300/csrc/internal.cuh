// Internal declarations shared by the translation units of libmrstat.so.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mrstat.h"
#include "tc_gemm.cuh"
#include "lowrank.cuh"
#include "mlp.cuh"

namespace mrstat {

// Number of channels of the cached time courses: m_y, dm_y/dlnT1, dm_y/dlnT2 (a plan
// that estimates B1 adds dm_y/dB1: Plan::nch = 4).
constexpr int kChannels = 3;
constexpr int kMaxChannels = 4;
// Maximum number of blocks of a float64 reduction (partials buffer size).
constexpr int kRedBlocks = 608;
// doubles in Plan::red: five partials per block of the vector kernels, or two parity
// buffers of up to eight partials per block of the persistent column kernels
constexpr int kRedSlots = 16 * kRedBlocks;

struct Plan {
  int nx = 0, ny = 0, nkx = 0, ntr = 0;
  int ntr_pad = 0;   // ntr rounded up to a multiple of 4
  int nq = 0;        // ntr_pad / 4 TR quads
  int nv = 0;
  int form = 0;
  int npar = 4;      // unknowns per voxel (5 with B1 estimated)
  int nch = 3;       // cached time-course channels (4 with B1 estimated)
  int device = 0;
  double tr_ms = 0, te_ms = 0;
  int inversion = 0, alternate = 0;

  // per-TR tables (device)
  float2* cs = nullptr;     // [ntr_pad] (cos phi_n, sin phi_n), phi_n the signed flip
  float* phi = nullptr;     // [ntr_pad] signed flip (radians)
  // slice profile (mrstat_set_slice_profile): 0 isochromats = hard pulses
  int slice_iso = 0, slice_sub = 0;
  float* slice_rot = nullptr;    // [ntr_pad][32][9] composed pulse of each (TR, isochromat), 3 x 3 column-major
  int* kyi = nullptr;       // [ntr_pad] ky mod ny in [0, ny)
  int* ky_ptr = nullptr;    // [ny + 1] TRs of each ky (CSR over ky_tr)
  int* ky_tr = nullptr;     // [ntr] TR indices grouped by ky, ascending within a ky
  float2* roots = nullptr;  // [ny] exp(-2 pi i k / ny)
  float2* ft = nullptr;     // [nx][nkx] exp(-2 pi i kx ix / nx)
  float2* fh = nullptr;     // [nkx][nx] exp(+2 pi i kx ix / nx)

  // cached linearisation
  float4* D = nullptr;      // [nch][nq][nv] four consecutive TRs per float4
  float2* rho = nullptr;    // [nv] rho * mask
  float* maskf = nullptr;   // [nv] 1 inside the mask, 0 outside
  bool linearized = false;

  // scratch
  float4* dfwd = nullptr;   // [nq][nv] m_y only, for mrstat_forward
  float2* cf = nullptr;     // [4][nv] per-voxel complex coefficients of the y-contraction
  float2* A = nullptr;      // [ntr_pad][nx] y-contracted image rows (padded rows zero)
  float2* wt = nullptr;     // [ntr_pad][nx] x-adjoint of a k-space vector (rows >= ntr zero)
  double* red = nullptr;    // [kRedSlots] reduction partials
  unsigned* ticket = nullptr;  // last-block ticket of the reductions (0 between launches)
  float* cg_r = nullptr;    // [npar][nv]
  float* cg_p = nullptr;    // [npar][nv]
  float* cg_q = nullptr;    // [npar][nv]
  float* cg_w = nullptr;    // [npar][nv] Re(J^H J) r
  unsigned* cg_bar = nullptr;  // [2] grid counter of the persistent column launches
  int grid_stall_block = -1;   // test hook: this block of those launches withholds an arrival
  float2* cg_jv = nullptr;  // [ntr][nkx]
  double* cg_s = nullptr;   // CG scalars, 4 per iteration
  int* cg_frozen = nullptr; // CG stop flag: 0, or the index + 1 of the iteration that froze the solve
  int cg_s_cap = 0;         // iterations the scalar buffer holds
  int cg_last_iters = -1;   // iters of the last mrstat_cg_fixed (-1: none yet)

  // Gauss-Newton work space (allocated by the first mrstat_gn_solve)
  bool gn_ready = false;
  float4* D2 = nullptr;     // trial-point time courses
  float2* rho2 = nullptr;   // trial-point rho * mask
  float *gn_g = nullptr, *gn_z = nullptr, *gn_res = nullptr, *gn_dir = nullptr, *gn_q = nullptr;
  float *gn_alpha = nullptr, *gn_trial = nullptr;
  float2 *gn_s = nullptr, *gn_r = nullptr, *gn_st = nullptr, *gn_rt = nullptr, *gn_jv = nullptr;
  uint8_t* gn_mask = nullptr;
  double* gn_sc = nullptr;  // scalar block
  int* gn_si = nullptr;     // integer state block

  // split-BF16 readout DFT (form MRSTAT_FORM_SPLIT_BF16)
  int kf_pad = 0, ka_pad = 0;       // padded K of the forward (2 nx) and adjoint (2 nkx) GEMMs
  void *bf_ft_hi = nullptr, *bf_ft_lo = nullptr;  // [2 nkx][kf_pad] forward DFT, K-major
  void *bf_fh_hi = nullptr, *bf_fh_lo = nullptr;  // [2 nx][ka_pad] adjoint DFT, K-major
  void *bf_a_hi = nullptr, *bf_a_lo = nullptr;    // [ntr][kf_pad] split rows A
  void *bf_w_hi = nullptr, *bf_w_lo = nullptr;    // [ntr][ka_pad] split k-space rows
  TcOperand* tc = nullptr;          // [4]: A rows, forward B, k-space rows, adjoint B
  LowRank* lr = nullptr;            // low-rank form (after mrstat_lowrank_set_basis)
  int* dev_err = nullptr;           // set by a kernel whose bounded wait ran out

  // checkpointed form
  float* ckpt = nullptr;        // [nseg][6][nv] Bloch states at segment starts
  float* zpart = nullptr;       // [nseg][6][nv] per-segment partial inner products
  int ckpt_interval = 0, ckpt_nseg = 0, ckpt_cap = 0;
  const float* ckpt_alpha = nullptr;   // caller's alpha/b1/mask of the last checkpointed forward
  const float* ckpt_b1 = nullptr;
  const uint8_t* ckpt_mask = nullptr;
  bool ckpt_ready = false;

  // recompute form (mrstat_set_recompute): states every rc_seg TRs instead of D
  int rc_seg = 0, rc_nseg = 0;  // 0: cached time courses
  float* rc_rlx = nullptr;      // [8][nv] relaxation factors of the linearisation
  float* rc_ckpt = nullptr;     // [rc_nseg][6][nv] states before each segment
  float* rc_gpart = nullptr;    // [rc_nseg][4][nv] per-segment gradients
  float* rc_b1 = nullptr;       // [nv] copy of the linearisation's B1 map
  bool rc_has_b1 = false;

  // kernels of the products return at once while *gate == 0 (nullptr: always run)
  const int* gate = nullptr;

  int64_t bytes = 0;
  int64_t d_bytes = 0;

  // tracing
  int64_t launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t kernel_launches[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool prof_on = false;
  uint32_t prof_mask = 0;
  struct Mark {
    int kid;
    cudaEvent_t a, b;
    int n;  // launches (or, for a persistent kernel, products) the events bracket
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> event_pool;
  size_t pool_used = 0;
};

// error reporting (thread-local message)
void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

// Makes the plan's device current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

template <typename T>
inline cudaError_t dalloc(Plan* p, T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e == cudaSuccess) p->bytes += (int64_t)(count * sizeof(T));
  return e;
}

cudaEvent_t pool_event(Plan* p);

// Counts the launches of one kernel class and, while profiling it, brackets them with events.
// NVTX range over one C-ABI call (header-only NVTX3: a no-op unless a profiler injects
// itself), so that a timeline shows the library's calls around their kernels.
struct AbiRange {
  explicit AbiRange(const char* name) { nvtxRangePushA(name); }
  ~AbiRange() { nvtxRangePop(); }
  AbiRange(const AbiRange&) = delete;
  AbiRange& operator=(const AbiRange&) = delete;
};
#define MRSTAT_ABI_RANGE() ::mrstat::AbiRange mrstat_abi_range_(__func__)

struct Span {
  Plan* p;
  int kid;
  cudaStream_t st;
  int n;
  cudaEvent_t a = nullptr, b = nullptr;
  // nlaunch: launches, or products of a persistent launch, the span counts; nkernels: the
  // kernel launches it makes (default: nlaunch)
  Span(Plan* plan, int k, cudaStream_t s, int nlaunch = 1, int nkernels = -1) : p(plan), kid(k), st(s), n(nlaunch) {
    p->launches[kid] += nlaunch;
    p->kernel_launches[kid] += nkernels < 0 ? nlaunch : nkernels;
    if (p->prof_on && ((p->prof_mask >> kid) & 1u)) {
      a = pool_event(p);
      b = pool_event(p);
      if (a && b) cudaEventRecord(a, st);
    }
  }
  ~Span() {
    if (a && b) {
      cudaEventRecord(b, st);
      p->marks.push_back({kid, a, b, n});
    }
  }
};

// product building blocks on a plan (plan.cu); they return an mrstat_status
int do_jvp(Plan* p, const float* v, float2* jv, cudaStream_t st);
int do_jhw(Plan* p, const float2* w, float* g, cudaStream_t st);
int do_signal(Plan* p, const float4* D, const float2* rho_masked, float2* s, cudaStream_t st);
int do_linearize(Plan* p, const float* alpha, const float* b1, const uint8_t* mask, float4* D,
                 float2* rho, cudaStream_t st);
cudaError_t do_dot(Plan* p, const float* a, const float* b, int64_t n, double* out, cudaStream_t st);
// Re(J^H J) v with the plan's active linearisation (exact: J.v then J^H; low-rank: per-ky
// Gram); with vdot also *vdot = <v, Re(J^H J) v> and with vv also *vv = <v, v> (fused into
// the last pass where the path allows it, else one more inner-product launch each)
int do_jhjv(Plan* p, const float* v, float* out, cudaStream_t st, double* vdot = nullptr, double* vv = nullptr);
// readout DFT of rows A [ntr][nx] (complex) into out [ntr][nkx], and its adjoint
int do_xdft(Plan* p, const float2* A, float2* out, const int* gate, cudaStream_t st);
int do_xdft_adj(Plan* p, const float2* w, float2* out, const int* gate, cudaStream_t st);

cudaError_t ensure_timecourses(Plan* p);   // allocates D on first use
int build_split_tables(Plan* p);           // split-BF16 readout DFT operands (plan.cu)
// low-rank form (lowrank.cu)
int lowrank_setup(Plan* p, const float* U_dev, int R, cudaStream_t st);
void lowrank_free(LowRank* L);
cudaError_t lowrank_project(const Plan& p, const LowRank& L, const float* alpha, const float* b1,
                            const uint8_t* mask, float* coef, cudaStream_t st);
int lowrank_jvp(Plan* p, const float* v, float2* jv, cudaStream_t st);
int lowrank_jhw(Plan* p, const float2* w, float* g, cudaStream_t st);
// Re(J^H J) v; with vdot also *vdot = <v, Re(J^H J) v>, with vv also *vv = <v, v> (fused
// where the path allows)
int lowrank_jhjv(Plan* p, const float* v, float* out, cudaStream_t st, double* vdot = nullptr,
                 double* vv = nullptr);
// mrstat_cg_fixed in one persistent launch when the low-rank column path applies (false:
// not launched); *err: the launch's error
bool lowrank_cg_fixed_persistent(Plan* p, const float* rhs, float* x, int iters, cudaStream_t st, cudaError_t* err);
// Steihaug's truncated CG from the gradient g in one persistent launch when the low-rank
// column path applies (false: not launched): the step into z, the solver's scalars into
// sc / si; *err: the launch's error
bool lowrank_steihaug_persistent(Plan* p, const float* g, float* z, double delta, int max_steps, double rel_tol,
                                 double* sc, int* si, cudaStream_t st, cudaError_t* err);
cudaError_t lowrank_train_matrix(const float4* D, int ns, int nq, int ntr, float2* Y, float2* Yt,
                                 cudaStream_t st);
cudaError_t ensure_forward_scratch(Plan* p);

// Launch with programmatic stream serialization: the kernel may start while the previous
// launch in the stream runs (if that one allows it), so it must call red::pdl_wait()
// before it reads anything an earlier launch wrote.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- launchers (each returns the launch's cudaError_t) ----
// bloch.cu
cudaError_t launch_bloch(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                         float4* D, int nch, cudaStream_t st);
// slice.cu: the slice-profile recursion (B1 = 1; nch 1: m only, 3: m and the two tangents)
cudaError_t launch_bloch_slice(const Plan& p, const float* alpha, const uint8_t* mask, float4* D, int nch,
                               cudaStream_t st);
// the same recursion for nv_override voxels laid out [2][nv_override] (ln T1, ln T2)
cudaError_t launch_bloch_n(const Plan& p, const float* alpha, const float* b1, float4* D, int nv_override,
                           cudaStream_t st);
// recompute form (fused.cu)
bool recompute_supported(const Plan& p);
cudaError_t launch_rc_linearize(const Plan& p, const float* alpha, const float* b1, cudaStream_t st);
cudaError_t launch_rc_product(const Plan& p, int mode, const float* v, const float2* wt, float* g, cudaStream_t st);

cudaError_t launch_bloch_ckpt(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                              int interval, int nseg, float* ckpt, cudaStream_t st);
cudaError_t launch_segment_jhw(const Plan& p, const float* alpha, const float* b1, const uint8_t* mask,
                               int interval, int nseg, const float* ckpt, float* zpart, float* g,
                               cudaStream_t st);
// encode.cu
cudaError_t launch_prep_forward(const Plan& p, const float* alpha, const uint8_t* mask, cudaStream_t st);
cudaError_t launch_prep_rho(const Plan& p, const float2* rho, cudaStream_t st);
cudaError_t launch_prep_linearize(const Plan& p, const float* alpha, const uint8_t* mask, float2* rho,
                                  cudaStream_t st);
cudaError_t launch_prep_jvp(const Plan& p, const float* v, cudaStream_t st);
cudaError_t launch_ycontract(const Plan& p, const float4* D, int nch, cudaStream_t st);
// g from W~ = p.wt, or from wt (then times scale) when given
cudaError_t launch_jhw_dot(const Plan& p, float* g, cudaStream_t st, const float2* wt = nullptr, float scale = 1.f);
cudaError_t launch_timecourse(const Plan& p, int channel, float* out, cudaStream_t st);
// dft.cu
cudaError_t launch_cgemm(const float2* A, const float2* B, float2* C, int M, int N, int K,
                         const int* gate, cudaStream_t st);
// reduce.cu
cudaError_t launch_dot(const float* a, const float* b, int64_t n, double* partials, unsigned* ticket,
                       double* out, cudaStream_t st, const int* gate = nullptr);
cudaError_t launch_cg_init(const float* rhs, float* x, float* r, float* p, float* q, int64_t n, cudaStream_t st);
// one Chronopoulos-Gear CG step (see reduce.cu); sk = {delta_k, gamma_k, alpha_k, -} of
// this iteration, sp the previous iteration's (NULL in the first); an iteration that
// freezes the solve stores it + 1 in *frozen
cudaError_t launch_cg_cg_step(float* x, float* r, float* p, float* q, const float* w, int64_t n, double* sk,
                              const double* sp, int* frozen, int it, cudaStream_t st);

}  // namespace mrstat
