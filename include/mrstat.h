/*
 * mrstat.h -- C ABI of the GB300 MR-STAT hot path (libmrstat.so).
 *
 * MR-STAT (van der Heide et al., arXiv 1904.13244) fits T1, T2 and complex proton
 * density maps directly to time-domain k-space data by an inexact Gauss-Newton
 * method whose inner CG solve only needs the signal s(alpha) and the Jacobian
 * products J.v and Re(J^H w) (Theory, Eq. 4; Algorithms 2, 4 and 6).  This library
 * evaluates those products on one GPU with hand-written sm_103a kernels.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Image grid nx (readout, x) by ny (phase encode, y); nv = nx * ny voxels; voxel
 *    j = iy * nx + ix (ix fastest).
 *  - Parameter maps alpha are float32 [npar][nv] in DEVICE memory, parameter-major
 *    (Theory: index j + k Nv): k = 0 ln(T1/ms), 1 ln(T2/ms), 2 Re rho, 3 Im rho
 *    (log scaling of T1 and T2: Methods, "Reconstructions"), and k = 4 B1 for plans
 *    created with MRSTAT_ESTIMATE_B1 (npar = 5; otherwise npar = 4).
 *  - k-space vectors (s, d, J.v, w) are interleaved complex float32 [ntr][nkx][2]
 *    in DEVICE memory; TR n samples the phase-encode line ky[n] and readout points
 *    kx = k - nkx/2, k = 0..nkx-1; the encoding phase is exp(-2 pi i (kx ix/nx +
 *    ky iy/ny)) (Theory, Eqs. 1-2 with the gradient encoding of Supporting
 *    Information S2).
 *  - J denotes the SIGNAL Jacobian J_s = ds/dalpha.  The paper's J = dr/dalpha is
 *    -J_s (Theory, "Computing the gradient g"), so the gradient of
 *    f = 1/2 ||d - s||^2 is -Re(J_s^H (d - s)).
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).  Every
 *    call only enqueues work on that stream and returns; no call synchronises the
 *    device unless its comment says so.  Buffers belong to the caller and must stay
 *    valid until the enqueued work has finished.
 *  - A plan is bound to the CUDA device that was current when it was created; calls
 *    switch to that device and restore the caller's device before returning.
 *  - Every call returns an mrstat_status; mrstat_last_error() gives a message for
 *    the last failure on the calling thread.  A failed call leaves outputs
 *    undefined but the plan usable.
 *  - Calls on the same plan must not overlap in time on different host threads or
 *    different streams: the plan's work buffers are shared.
 */
#ifndef MRSTAT_H
#define MRSTAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mrstat_status {
  MRSTAT_OK = 0,
  MRSTAT_ERR_INVALID_ARG = 1,     /* null pointer, bad enum, bad option value          */
  MRSTAT_ERR_SHAPE = 2,           /* sizes out of range (see mrstat_plan_create)        */
  MRSTAT_ERR_NOT_LINEARIZED = 3,  /* jvp/jhw/timecourses before mrstat_linearize        */
  MRSTAT_ERR_CUDA = 4,            /* a CUDA runtime call or kernel launch failed        */
  MRSTAT_ERR_NONFINITE = 5,       /* NaN or Inf found where a finite value is required */
  MRSTAT_ERR_TIMEOUT = 6,         /* an iteration budget ran out                        */
  MRSTAT_ERR_UNSUPPORTED = 7,     /* valid request this build does not implement        */
  MRSTAT_ERR_OUT_OF_MEMORY = 8    /* device allocation failed                            */
} mrstat_status;

/* Numerical forms of the encoding contraction. */
typedef enum mrstat_form {
  MRSTAT_FORM_PLAIN_FP32 = 0,     /* every step in FP32 on the CUDA cores               */
  MRSTAT_FORM_SPLIT_BF16 = 1      /* readout DFT on tcgen05 tensor cores as split-BF16
                                     products (hi*hi + hi*lo + lo*hi), FP32 accumulation;
                                     everything else as in the plain form              */
} mrstat_form;

/*
 * Pulse-sequence description (Methods, "Pulse Sequence"; Supporting Information S1).
 * Balanced gradient echo with one phase-encode line per TR; the RF pulse of TR n is
 * an instantaneous rotation by flip_rad[n] * B1 about -x (RF phase 0) or +x (RF
 * phase 180 degrees; the phase alternates 0/180 between TRs when alternate_phase is
 * nonzero).  inversion != 0 applies an ideal non-selective inversion before TR 0.
 * The magnetisation is sampled at te_ms after each pulse and held constant across
 * the nkx readout samples of its TR.  flip_rad and ky are HOST arrays read only
 * during mrstat_plan_create.
 */
typedef struct mrstat_seq {
  int32_t nx, ny;          /* image grid, 1..2048 each                             */
  int32_t nkx;             /* readout samples per TR, 1..4096                       */
  int32_t ntr;             /* number of TRs, 1..65536                               */
  double tr_ms, te_ms;     /* 0 < te_ms < tr_ms                                    */
  int32_t inversion;       /* 0 or 1                                                */
  int32_t alternate_phase; /* 0 or 1                                                */
  const float* flip_rad;   /* host [ntr], finite, >= 0                              */
  const int32_t* ky;       /* host [ntr], each in [-(ny/2), ny - ny/2)              */
} mrstat_seq;

typedef struct mrstat_plan mrstat_plan;

/* Static description of a plan (host struct filled by mrstat_plan_info). */
typedef struct mrstat_plan_info_t {
  int32_t nx, ny, nkx, ntr, nv, form;
  int32_t ntr_padded;          /* ntr rounded up to a multiple of 4 (TR quads)      */
  int64_t device_bytes;        /* device memory owned by the plan                   */
  int64_t timecourse_bytes;    /* of which the cached time courses D                */
  int32_t npar;                /* unknowns per voxel: 4, or 5 with B1 estimated     */
} mrstat_plan_info_t;

/*
 * OR this flag into the form of mrstat_plan_create to make B1 the fifth unknown per
 * voxel (the paper estimates B1 along with T1, T2 and rho: Methods, "Reconstructions";
 * the derivative of the Bloch recursion with respect to B1 is the S2 forward-mode
 * derivative through the rotation angle).  Such a plan works on npar = 5 rows
 * alpha = (ln T1, ln T2, Re rho, Im rho, B1): every [4][nv] below becomes [5][nv], the
 * time courses carry a fourth channel dm_y/dB1, the b1 arguments must be NULL (B1 is
 * alpha row 4), and the low-rank and checkpointed entry points return UNSUPPORTED.
 */
#define MRSTAT_ESTIMATE_B1 0x100

/*
 * Create a plan: validates the sequence, builds the per-TR rotation and phase
 * tables and allocates the small work buffers (x-DFT matrices, reduction scratch,
 * CG vectors).  The large buffers are allocated by the first call that needs them:
 * the cached time courses D (3 x ntr_padded x nv float32, 4 x with B1 estimated) by
 * mrstat_linearize, the
 * m_y scratch (ntr_padded x nv float32) by mrstat_forward / mrstat_forward_ckpt.  Synchronises the current device once.  On failure *out is
 * set to NULL.  form: a mrstat_form, optionally | MRSTAT_ESTIMATE_B1.
 * Errors: INVALID_ARG (null seq/out/arrays, bad form, non-finite or
 * negative flips, te/tr), SHAPE (sizes outside the ranges above, ky out of range),
 * OUT_OF_MEMORY, CUDA.
 */
int mrstat_plan_create(const mrstat_seq* seq, int32_t form, mrstat_plan** out);

/* Free a plan and its device memory (synchronises the plan's device). NULL is a no-op. */
int mrstat_plan_destroy(mrstat_plan* plan);

int mrstat_plan_info(const mrstat_plan* plan, mrstat_plan_info_t* info);

/*
 * Wait for the plan's device work and report device-side failures: returns
 * MRSTAT_ERR_TIMEOUT (and clears the flag) when a tensor-core kernel stopped because a
 * bounded wait on its pipeline barriers ran out, or a persistent CG launch because its
 * bounded grid wait ran out (2 s); its outputs are then undefined.
 * Synchronises the plan's device.
 */
int mrstat_plan_check(mrstat_plan* plan);

/*
 * Test hook for the failure path of the persistent CG and Steihaug launches: with
 * block >= 0, block `block` of the next persistent launches withholds its first arrival
 * at the grid counter, so every block's bounded grid wait (2 s) runs out; the launch
 * ends early, x (or the Steihaug step) is undefined, and mrstat_plan_check /
 * mrstat_gn_solve report MRSTAT_ERR_TIMEOUT.  block < 0 turns it off (the default).
 * Nothing faults or hangs.  Errors: INVALID_ARG (NULL plan, or block >= 2 nx: the
 * persistent launches have two blocks per image column).
 */
int mrstat_plan_inject_grid_stall(mrstat_plan* plan, int32_t block);

/*
 * Linearise the model at alpha (Algorithm 2 step 1 for every voxel, with the
 * forward-mode derivatives of Supporting Information S2): runs the Bloch recursion
 * of every voxel and caches m_y and dm_y/dln T1, dm_y/dln T2 at every echo, plus
 * rho and the mask, for later mrstat_jvp / mrstat_jhw / mrstat_timecourses calls.
 *   alpha: device float [npar][nv] (see top; row 4 = B1 when B1 is estimated, and then
 *          a fourth channel dm_y/dB1 is cached).
 *   b1:    device float [nv] relative transmit field, or NULL for B1 = 1 (must be NULL
 *          when B1 is estimated).
 *   mask:  device uint8 [nv], nonzero = voxel takes part, or NULL for all voxels
 *          (Methods: voxels without significant proton density are excluded; a
 *          masked-out voxel contributes nothing to s and gets zero gradient).
 * Errors: INVALID_ARG (null plan/alpha, b1 given with B1 estimated), CUDA.
 */
int mrstat_linearize(mrstat_plan* plan, const float* alpha, const float* b1,
                     const uint8_t* mask, void* stream);

/*
 * s = sum_j rho_j m_j(theta_j) exp(-i k.r_j) (Algorithm 2; Eqs. 1-2) at alpha.
 *   s: device float [ntr][nkx][2] output.  Does not change the cached linearisation.
 * Errors: INVALID_ARG, CUDA.
 */
int mrstat_forward(mrstat_plan* plan, const float* alpha, const float* b1,
                   const uint8_t* mask, float* s, void* stream);

/*
 * jv = J_s v at the cached linearisation ("Similar techniques ... J v", text before
 * Eq. 4): jv = encode(rho (v0 dm/dlnT1 + v1 dm/dlnT2 [+ v4 dm/dB1]) + (v2 + i v3) m).
 *   v: device float [npar][nv];  jv: device float [ntr][nkx][2].
 * Errors: INVALID_ARG, NOT_LINEARIZED, CUDA.
 */
int mrstat_jvp(mrstat_plan* plan, const float* v, float* jv, void* stream);

/*
 * g = Re(J_s^H w) at the cached linearisation (Algorithm 4 with J_s = -J):
 * g[k][j] = Re sum_{n,kx} conj(d(rho_j m_j[n])/dalpha_k exp(-i k.r_j)) w[n][kx].
 *   w: device float [ntr][nkx][2];  g: device float [npar][nv] (zero outside the mask).
 * Errors: INVALID_ARG, NOT_LINEARIZED, CUDA.
 */
int mrstat_jhw(mrstat_plan* plan, const float* w, float* g, void* stream);

/*
 * Copy one cached time course channel out of the plan: channel 0 = m_y, 1 =
 * dm_y/dln T1, 2 = dm_y/dln T2 (3 = dm_y/dB1 when B1 is estimated) at every echo (the echo signal is i * m_y because
 * the RF phases 0/180 keep m_x = 0; Supporting Information S2).
 *   out: device float [ntr][nv].  Masked-out voxels read as 0.
 * Errors: INVALID_ARG (bad channel), NOT_LINEARIZED, CUDA.
 */
int mrstat_timecourses(mrstat_plan* plan, int32_t channel, float* out, void* stream);

/*
 * Recompute form of the exact model.  The paper evaluates every matrix-free product by
 * running the Bloch simulation again (Algorithms 2 and 4); with segment > 0 the plan does
 * the same instead of caching the time courses: mrstat_linearize keeps, per voxel, the
 * relaxation factors and the Bloch state (m_y, m_z and their ln T1 / ln T2 tangents)
 * before every segment-th TR (6 floats per voxel and segment), and every mrstat_jvp,
 * mrstat_jhw, mrstat_jhjv and mrstat_cg_fixed product re-runs the recursion from those
 * states, all segments in parallel, fused with the phase-encode sums (and, for
 * Re(J^H J) v with nkx == nx, with both of them in one pass).  The results are those of
 * the cached form up to float32 rounding.  segment = 0 restores the cached time courses.
 * Either way the cached linearisation is dropped.  Synchronises the plan's device.
 *   segment: TRs per segment (>= 0; values above ntr mean one segment).
 * The recompute form needs ny <= 256, B1 known or 1 (not estimated) and hard pulses
 * (else UNSUPPORTED); mrstat_timecourses and mrstat_gn_solve return UNSUPPORTED while it
 * is on.  Errors: INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY, CUDA.
 */
int mrstat_set_recompute(mrstat_plan* plan, int32_t segment);

/*
 * Checkpointed signal and gradient (differentiation by recomputation).
 *
 * mrstat_forward_ckpt computes s like mrstat_forward and keeps, instead of the time
 * courses, the full Bloch state of every voxel (m_y, m_z and their ln T1 / ln T2
 * tangents) before every `interval`-th TR: 6 * ceil(ntr / interval) floats per voxel.
 * mrstat_jhw_ckpt then returns Re(J_s^H w) at that point by re-running each segment of
 * the recursion from its checkpoint (Supporting Information S2), all segments in
 * parallel, fused with the inner products of Algorithm 4; no time course is stored.
 * mrstat_jhw_ckpt reads alpha, b1 and mask from the caller's buffers given to the last
 * mrstat_forward_ckpt, which must still hold the same values.
 *   interval: positive multiple of 4 (64 is the usual choice).
 * Errors: INVALID_ARG, NOT_LINEARIZED (jhw_ckpt before forward_ckpt), OUT_OF_MEMORY, CUDA.
 */
int mrstat_forward_ckpt(mrstat_plan* plan, const float* alpha, const float* b1,
                        const uint8_t* mask, int32_t interval, float* s, void* stream);
int mrstat_jhw_ckpt(mrstat_plan* plan, const float* w, float* g, void* stream);

/*
 * out = Re(J_s^H J_s) v, the Gauss-Newton matrix-vector product of the inner CG
 * (Eq. 4: first y = J v, then Re(J^H y)), with the plan's current linearisation:
 * mrstat_jvp then mrstat_jhw after mrstat_linearize, or the per-ky Gram product of the
 * low-rank form after mrstat_lowrank_linearize.
 *   v, out: device float [npar][nv].
 * Errors: INVALID_ARG, NOT_LINEARIZED, CUDA.
 */
int mrstat_jhjv(mrstat_plan* plan, const float* v, float* out, void* stream);

/*
 * Low-rank (compressed) form.  Every echo time course is represented in a real time
 * basis U [ntr][R]: m_j[n] ~ i sum_r U[n][r] c_r,j, and likewise dm_j/dln T1 and
 * dm_j/dln T2 with coefficients dc1, dc2.  This is the SVD compression the paper's
 * comparison pipeline applies to its dictionary (Methods, "Numerical Brain
 * Simulation"), applied to the signal model itself; the encoding sum of Eqs. 1-2 then
 * becomes R two-dimensional DFTs, and Re(J^H J) v uses the per-ky Gram matrices
 * M_ky = sum_{n: ky(n) = ky} U[n]^T U[n] so that it never touches the TR axis.  All
 * DFTs run as split-BF16 tcgen05 products with float32 accumulation.
 *
 * mrstat_lowrank_basis: U = leading R left singular vectors of the training time courses
 *   [m_y | dm_y/dlnT1 | dm_y/dlnT2] of ns voxels (Bloch recursion on the device, then
 *   subspace iteration Q <- orth(Y (Y^T Q)) with float32 products on the device and
 *   float64 orthonormalisation and Rayleigh-Ritz on the host).
 *   train: device float [2][ns] (ln T1, ln T2 in ms); train_b1: device float [ns] or
 *   NULL; U_out: device float [ntr][R]; sv_out: host double [R] singular values or NULL.
 *   1 <= R <= 32.  Allocates and frees its own work space; synchronises.
 * mrstat_lowrank_set_basis: adopts U (device float [ntr][R], R in {8, 16, 24, 32},
 *   orthonormal columns) and allocates the form's work space; synchronises.
 * mrstat_lowrank_linearize: makes the low-rank model at alpha the plan's linearisation
 *   for mrstat_jvp, mrstat_jhw, mrstat_jhjv and mrstat_cg_fixed.  coef = NULL projects
 *   the exact Bloch recursion onto U on the fly (no time course is stored); otherwise
 *   coef is device float [3][R][nv] (c, dc1, dc2), e.g. from a learned surrogate.  A
 *   later mrstat_linearize switches the plan back to the exact model.
 * mrstat_lowrank_coefficients: copies the current coefficients to device [3][R][nv].
 * mrstat_lowrank_rank: R of the adopted basis (0 if none).
 * Errors: INVALID_ARG, NOT_LINEARIZED (no basis / no low-rank linearisation),
 * OUT_OF_MEMORY, TIMEOUT (a tensor-core kernel's bounded wait ran out), CUDA.
 */
int mrstat_lowrank_basis(mrstat_plan* plan, const float* train, const float* train_b1, int32_t ns,
                         int32_t rank, float* U_out, double* sv_out, void* stream);
int mrstat_lowrank_set_basis(mrstat_plan* plan, const float* U, int32_t rank, void* stream);
int mrstat_lowrank_linearize(mrstat_plan* plan, const float* alpha, const float* b1,
                             const uint8_t* mask, const float* coef, void* stream);
int mrstat_lowrank_coefficients(mrstat_plan* plan, float* coef, void* stream);
int mrstat_lowrank_rank(const mrstat_plan* plan);

/*
 * Coefficients of the exact time courses of ns parameter samples in the plan's time
 * basis (training targets of the learned surrogate): the Bloch recursion with its
 * tangents projected onto U on the fly, as in mrstat_lowrank_linearize.
 *   params: device float [2][ns] (ln T1, ln T2); b1: device float [ns] or NULL;
 *   coef: device float [3][R][ns] (c, dc/dlnT1, dc/dlnT2).
 * Errors: INVALID_ARG, NOT_LINEARIZED (no basis), CUDA.
 */
int mrstat_lowrank_project_samples(mrstat_plan* plan, const float* params, const float* b1, int32_t ns,
                                   float* coef, void* stream);

/*
 * Learned surrogate of the compressed Bloch model.  The paper names surrogate models as
 * a way to cut the cost of its partial-derivative computations (Discussion).  The MLP
 * maps u = ((ln T1 - mu1)/s1, (ln T2 - mu2)/s2, (B1 - mu3)/s3) through three tanh
 * layers of width `hidden` to R coefficients c = scale * (W4 a3 + b4) of the echo time
 * course in the plan's time basis; dc/dln T1 and dc/dln T2 come from forward-mode
 * tangents through the same layers, all three streams sharing one BF16 tcgen05 GEMM
 * per layer (float32 accumulation).  Training minimises the Sobolev loss
 *   L = 1/B sum_b sum_r [(c - c*)^2 + lam ((dc1 - dc1*)^2 + (dc2 - dc2*)^2)] / scale_r^2
 * by Adam with hand-written forward, backward and update kernels; float32 master
 * weights, BF16 copies for the GEMMs.  Parameters are flat float32 in the order
 * W1 [hidden][3], b1, W2, b2, W3, b3, W4 [R][hidden], b4.
 *
 * All pointers are device memory unless marked host.  lnT: [2][n] (ln T1, ln T2 in
 * ms); b1: [n] or NULL (B1 = 1); target/coef: [3][R][n] (c, dc/dlnT1, dc/dlnT2).
 * mrstat_mlp_train_step: one Adam step on a batch (lr = 0: gradient only); *loss
 *   (device double, may be NULL) receives the batch loss before the step.
 * mrstat_mlp_loss_grad: loss (host double) and gradient (device float [num_params], may
 *   be NULL) of a batch at the current weights; synchronises.
 * mrstat_mlp_infer: coefficients and their ln T1 / ln T2 derivatives for n samples.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, TIMEOUT, CUDA.
 */
typedef struct mrstat_mlp mrstat_mlp;

typedef struct mrstat_mlp_config {
  int32_t hidden;          /* 64, 128 or 256                                           */
  int32_t rank;            /* R, 1..32                                                 */
  float norm[6];           /* mu1, s1, mu2, s2, mu3, s3 (s > 0)                         */
  float sobolev_weight;    /* lam                                                      */
  uint64_t seed;           /* Glorot-uniform initial weights, zero biases              */
} mrstat_mlp_config;

int mrstat_mlp_create(const mrstat_mlp_config* cfg, mrstat_mlp** out);
int mrstat_mlp_destroy(mrstat_mlp* mlp);
int64_t mrstat_mlp_num_params(const mrstat_mlp* mlp);
int mrstat_mlp_set_output_scale(mrstat_mlp* mlp, const float* scale /* host [R] */);
int mrstat_mlp_get_params(mrstat_mlp* mlp, float* params /* host [num_params] */);
int mrstat_mlp_set_params(mrstat_mlp* mlp, const float* params /* host [num_params] */);
int mrstat_mlp_train_step(mrstat_mlp* mlp, const float* lnT, const float* b1, const float* target,
                          int32_t batch, float lr, double* loss, void* stream);
int mrstat_mlp_loss_grad(mrstat_mlp* mlp, const float* lnT, const float* b1, const float* target,
                         int32_t batch, double* loss /* host */, float* grad, void* stream);
int mrstat_mlp_infer(mrstat_mlp* mlp, const float* lnT, const float* b1, int32_t n, float* coef,
                     void* stream);

/*
 * *out = sum_i a[i] * b[i] (the CG inner products of the inner Gauss-Newton loop,
 * Algorithm 6): each thread adds its few products (a grid-stride handful) in float32,
 * all partial sums are added in float64; the relative error is ~1e-7 of sum |a b|.  a, b: device float [n]; out: device double.
 * Uses the plan's reduction scratch.  n may be 0 (result 0).
 * Errors: INVALID_ARG (null pointer, n < 0), CUDA.
 */
int mrstat_dot(mrstat_plan* plan, const float* a, const float* b, int64_t n,
               double* out, void* stream);

/*
 * Allocation-free variant of mrstat_dot: *out = sum_i a[i] * b[i] with the same
 * arithmetic (float32 per-thread partials over 16 elements, float64 from the warp level
 * up, deterministic order), needing no plan.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, such as code running while
 * another framework owns the device allocator, inside a memory-pool budget that must not
 * grow, or in a process that forbids allocation after start-up.  It allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine): its scratch is a file-scope
 * device array of 4128 doubles (33 KB) holding one partial per block of 4096 elements
 * and a ticket counter.
 *   a, b: device float [n]; out: device double; stream: cudaStream_t or NULL.
 *   n: 0 .. 16,777,216 (4096 blocks x 4096 elements); larger n is rejected with
 *   INVALID_ARG (use mrstat_dot for those).
 * The first call on each device looks up the array's address on that device
 * (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture.  Every call on a device shares the one array, which keeps the last
 * call's contents; each call clears the ticket before its kernel.  Calls that overlap on
 * the GPU (concurrent streams, or several threads) race on the array and give wrong
 * results: serialise them.
 * Errors: INVALID_ARG (null pointer, n < 0, n above the limit), UNSUPPORTED (device index
 * >= 64), CUDA.
 */
int mrstat_dot_static(const float* a, const float* b, int64_t n, double* out, void* stream);

/*
 * Slice profile (Methods, "Pulse Sequence": every RF pulse has a Gaussian envelope;
 * "Reconstructions": the Bloch solver takes the slice profile into account).  With a
 * profile set, mrstat_linearize / mrstat_forward (and the Gauss-Newton solver) simulate
 * every voxel as n_iso isochromats across the slice, at u_k = extent ((k + 1/2)/n_iso
 * - 1/2) slice thicknesses; each RF pulse is n_sub hard sub-pulses with Gaussian weights
 * exp(-((s + 1/2)/n_sub - 1/2)^2 / (2 sigma^2)) (normalised to sum 1, so the slice centre
 * turns by the nominal flip), sub-step s followed by a slice-select precession of
 * 2 pi tbw u_k / n_sub, with a pre-winder and a rewinder of half the pulse's gradient
 * area each (a balanced sequence); relaxation as in the hard-pulse model; the echo is
 * the mean over the isochromats.  The paper gives no pulse parameters: these are the
 * build's readings.  profile = NULL restores hard pulses.  Either way the cached
 * linearisation is dropped.
 *   n_iso: a power of two in 1..32; n_sub: 1..64; sigma > 0; extent > 0.
 * The slice-profile model takes B1 = 1: a b1 map, B1 estimation, the low-rank and
 * surrogate forms and the checkpointed form are UNSUPPORTED with it.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
typedef struct mrstat_slice_profile {
  int32_t n_iso;   /* isochromats across the slice */
  int32_t n_sub;   /* RF sub-steps */
  double sigma;    /* Gaussian width, fraction of the pulse */
  double tbw;      /* time-bandwidth product */
  double extent;   /* the isochromats span this many slice thicknesses */
} mrstat_slice_profile;

int mrstat_set_slice_profile(mrstat_plan* plan, const mrstat_slice_profile* profile);

/*
 * Fixed-count conjugate gradients on Re(J_s^H J_s) x = rhs at the cached
 * linearisation (the inner CG of Algorithm 6 without trust-region exits): x_0 = 0,
 * then exactly `iters` iterations, each one J^H J v product plus float64 inner products;
 * every scalar stays on the device.  The iteration is written in the Chronopoulos-Gear
 * form (the product is applied to the residual r, and <r, Hr>, <r, r> come with it;
 * p.Hp follows from them), which has textbook CG's iterates in exact arithmetic and one
 * vector update per iteration.  Where the low-rank model's column form applies and all
 * of its image columns fit on the device at once, the whole solve is one persistent
 * launch in the pipelined form of the same recurrences (Ghysels and Vanroose 2014: Hr is
 * carried by recurrence, so the grid-wide inner products overlap the next product);
 * also textbook CG's iterates in exact arithmetic, with `iters` products in all.  An
 * iteration whose curvature p.Hp is not positive, or whose residual is exactly zero,
 * freezes x for the remaining iterations.  A persistent launch whose grid wait ran out
 * sets the flag mrstat_plan_check reports.
 *   rhs, x: device float [npar][nv].  iters >= 0.
 * Errors: INVALID_ARG, NOT_LINEARIZED, CUDA.
 */
int mrstat_cg_fixed(mrstat_plan* plan, const float* rhs, float* x, int32_t iters,
                    void* stream);

/*
 * Number of iterations the last mrstat_cg_fixed on this plan applied to x: its `iters`
 * unless an iteration froze the solve (non-positive curvature p.Hp, or a residual that
 * is exactly zero; the inner solve of Algorithm 6 ends there), in which case x holds the
 * iterate of the iterations before it.  A caller that times or trusts a fixed-count
 * solve checks this equals iters.  Synchronises the plan's device.
 *   applied: host int32 out.
 * Errors: INVALID_ARG (NULL pointer), NOT_LINEARIZED (no mrstat_cg_fixed has run on
 * the plan), CUDA.
 */
int mrstat_cg_applied(mrstat_plan* plan, int32_t* applied);

/*
 * Inexact Gauss-Newton reconstruction (Algorithm 6) with a trust region.
 *
 * Minimises f(alpha) = 1/2 ||d - s(alpha)||^2 (Theory, Eq. argmin) by outer
 * iterations, each of which linearises the model, forms g = grad f = -Re(J_s^H (d - s))
 * and solves Re(J_s^H J_s) p = -g approximately by Steihaug's truncated CG inside the
 * trust region ||p|| <= Delta (Eq. 4; Methods: trust-region framework of Steihaug and
 * Nocedal & Wright Alg. 7.2).  A trial point alpha + p, reflected into the T1/T2 box
 * (Methods: reflection at feasible boundaries), is accepted when the actual reduction
 * exceeds eta times the CG model's predicted reduction; Delta shrinks by 4 when the
 * ratio is below 1/4 and doubles (up to delta_max) when it is above 3/4 with the step
 * on the boundary.  With rho_init_iters > 0 the complex proton density is first
 * initialised as the least-squares solution of M(alpha_0) rho = d by CGLS at
 * T1 = t1_init_ms, T2 = t2_init_ms (Methods), and with mask_threshold > 0 the mask
 * |rho| > mask_threshold * max |rho| is drawn and written to `mask`.  With
 * rho_init_exact != 0 that least-squares solution is computed exactly instead (the
 * minimum-norm one, which the paper's LSQR from zero approaches): every voxel shares the
 * time course m_n at alpha_0, so M^H M is diagonal in k-space and rho = F^H P / (nx ny)
 * with P(kx, ky) = sum_{n: ky(n) = ky} conj(m_n) d_n(kx) / sum |m_n|^2 (P = 0 on a ky no TR
 * samples); this needs nkx == nx, b1 == NULL and ntr >= ny (else UNSUPPORTED).
 *
 * With opts->surrogate_iters = k > 0 the first k outer iterations replace the Bloch
 * simulation by the learned surrogate (mrstat_mlp_*), the remedy for the cost of the
 * derivative computations the paper names (Discussion): the coefficients of every
 * voxel's time course and tangents in the plan's basis come from one MLP inference, and
 * objective, gradient and CG products are those of that low-rank model.  At iteration k
 * the solver re-evaluates the objective with the exact model and continues with it, so
 * the result is the exact model's minimiser; the report's f[] shows the switch.
 *
 * With B1 estimated (MRSTAT_ESTIMATE_B1) every vector has npar = 5 rows; hessian = 1 and
 * surrogate_iters > 0 are then UNSUPPORTED.
 *
 * With opts->hessian = 1 the CG uses the low-rank Gauss-Newton matrix of the plan's
 * time basis (the compressed model's Re(J^H J), recomputed at every accepted point by
 * projecting the exact recursion onto the basis), while gradient, objective and the
 * trust-region ratio stay exact, so the iteration converges to the exact model's
 * solution.
 *
 * Resuming: the state of a solve between outer iterations is alpha, the mask, the trust
 * radius and the iteration count.  A call with alpha = the previous call's result, that
 * call's mask as input (no rho initialisation, mask_threshold = 0), delta0 = its
 * report->delta_final and iteration_offset = the iterations run so far continues the
 * solve exactly where it stopped (the surrogate schedule included), so a long
 * reconstruction can be checkpointed on the host and restarted.
 *
 * Every CG scalar lives on the device in float64; the host synchronises once per
 * outer iteration to evaluate the trust-region ratio.  Where the CG matrix is the
 * low-rank one (hessian = 1 or the surrogate phase) on a fully sampled readout with
 * ny = 32 N1 (N1 <= 8) and every image column's pair of blocks fits on the device at
 * once, each Steihaug solve is one persistent launch (the residual's product carries the
 * direction's by recurrence; the same decisions in exact arithmetic); if its grid waits
 * run out (2 s) the call returns TIMEOUT.  On return the plan holds the linearisation
 * at the returned alpha.
 *   d:      device float [ntr][nkx][2] measured k-space data.
 *   alpha:  device float [npar][nv], initial guess in, estimate out (B1 in row 4 when
 *           estimated; reflected into [b1_min, b1_max] like T1 and T2).
 *   b1:     device float [nv] or NULL (B1 = 1); a known map, not estimated.
 *   mask:   device uint8 [nv]: in, the voxels to fit (NULL = all), unless a mask is
 *           drawn, in which case it is written (must then be non-NULL).
 *   report: host struct filled with the per-iteration history (may be NULL).
 * Errors: INVALID_ARG (bad pointers or options), UNSUPPORTED (see above),
 * OUT_OF_MEMORY (the solver's work space: a second set of time courses plus a few
 * vectors), TIMEOUT (a bounded device wait ran out), CUDA.
 */
#define MRSTAT_GN_MAX_OUTER 64

typedef enum mrstat_cg_exit {
  MRSTAT_CG_MAX_ITER = 0,
  MRSTAT_CG_BOUNDARY = 1,
  MRSTAT_CG_NEGATIVE_CURVATURE = 2,
  MRSTAT_CG_CONVERGED = 3,
  MRSTAT_CG_ZERO_GRADIENT = 4
} mrstat_cg_exit;

typedef struct mrstat_gn_opts {
  int32_t outer_iters;         /* 0..MRSTAT_GN_MAX_OUTER                               */
  int32_t inner_iters;         /* CG iterations per outer iteration, >= 1              */
  double delta0;               /* initial radius; <= 0: 0.1 ||alpha_0|| over the mask  */
  double delta_max;            /* <= 0: unbounded                                      */
  double eta;                  /* acceptance threshold on the reduction ratio          */
  double cg_rel_tol;           /* CG stops when ||res|| <= cg_rel_tol ||g|| (0: never) */
  double t1_min_ms, t1_max_ms; /* T1 box                                               */
  double t2_min_ms, t2_max_ms; /* T2 box                                               */
  int32_t rho_init_iters;      /* CGLS iterations of the rho initialisation (0: none)  */
  double t1_init_ms, t2_init_ms;
  double mask_threshold;       /* > 0: draw the mask after the rho initialisation       */
  int32_t hessian;             /* 0: exact Re(J^H J); 1: low-rank per-ky Gram product of
                                  the plan's time basis (mrstat_lowrank_set_basis) for the
                                  CG, with the exact gradient and objective              */
  int32_t surrogate_iters;     /* >= 0: the first surrogate_iters outer iterations of the
                                  schedule run on the learned surrogate's low-rank model
                                  (objective, gradient, CG products and the trust-region
                                  ratio); the rest on the exact model.  A call that ends
                                  inside the surrogate phase returns the surrogate model's
                                  iterate (a later call with iteration_offset continues) */
  const mrstat_mlp* surrogate; /* required when surrogate_iters > 0; its rank must equal
                                  the plan's basis rank                                  */
  double b1_min, b1_max;       /* B1 box when B1 is estimated                           */
  int32_t rho_init_exact;      /* != 0: the rho initialisation is the exact least-squares
                                  solution instead of rho_init_iters CGLS steps (needs
                                  nkx == nx, b1 == NULL and ntr >= ny)                   */
  int32_t iteration_offset;    /* >= 0: outer iterations already run by earlier calls of a
                                  solve this call resumes; iteration k of this call is
                                  iteration iteration_offset + k of the schedule (the
                                  surrogate phase covers schedule iterations
                                  0..surrogate_iters-1)                                  */
} mrstat_gn_opts;

typedef struct mrstat_gn_report {
  int32_t iterations;                      /* outer iterations run                  */
  int32_t mask_voxels;                     /* voxels inside the mask                */
  int32_t cg_steps[MRSTAT_GN_MAX_OUTER];
  int32_t cg_exit[MRSTAT_GN_MAX_OUTER];    /* mrstat_cg_exit                         */
  int32_t accepted[MRSTAT_GN_MAX_OUTER];
  double f[MRSTAT_GN_MAX_OUTER];           /* objective at the start of iteration   */
  double gnorm[MRSTAT_GN_MAX_OUTER];
  double delta[MRSTAT_GN_MAX_OUTER];
  double ratio[MRSTAT_GN_MAX_OUTER];
  double f_final;
  double seconds;                          /* wall time of the call                 */
  double delta_final;                      /* trust radius after the last iteration  */
} mrstat_gn_report;

/* Fill opts with the defaults: 10 x 20 iterations, delta0 from alpha_0, eta = 1e-4,
   no CG tolerance, T1 in [50, 6000] ms, T2 in [5, 3000] ms, no rho initialisation
   (t1_init 1000 ms, t2_init 100 ms, 50 CGLS steps and threshold 0.1 when enabled),
   B1 in [0.5, 1.5] (start B1 = 1 with the rho initialisation). */
void mrstat_gn_default_opts(mrstat_gn_opts* opts);

int mrstat_gn_solve(mrstat_plan* plan, const float* d, float* alpha, const float* b1,
                    uint8_t* mask, const mrstat_gn_opts* opts, mrstat_gn_report* report,
                    void* stream);

/*
 * Tracing of the plan's own kernel launches.  Launch counts are always kept; while
 * profiling is on, every launch of a kernel whose bit is set in kernel_mask is
 * bracketed by two CUDA events on its stream.  mrstat_profile_start clears the
 * counters and turns profiling on; mrstat_profile_stop waits for the recorded events,
 * fills *out (launches and summed event time per kernel) and turns profiling off.
 * Instrumentation for roofline reporting; it does not change any result.
 */
typedef enum mrstat_kernel_id {
  MRSTAT_K_BLOCH = 0,        /* Bloch recursion + tangents (K1)                    */
  MRSTAT_K_YCONTRACT = 1,    /* phase-encode contraction of s and J.v (K2)         */
  MRSTAT_K_XDFT = 2,         /* readout DFT (K3)                                   */
  MRSTAT_K_XDFT_ADJ = 3,     /* readout DFT adjoint (K3^H)                         */
  MRSTAT_K_JHW_DOT = 4,      /* phase-encode adjoint + tangent inner products (K4) */
  MRSTAT_K_VECTOR = 5,       /* coefficient preparation, reductions, CG updates    */
  MRSTAT_K_COUNT = 6
} mrstat_kernel_id;

typedef struct mrstat_kernel_stats {
  int64_t launches[8];       /* indexed by mrstat_kernel_id; a persistent CG or
                                Steihaug launch counts its products                  */
  double ms[8];              /* summed event time of the profiled launches           */
  int64_t timed[8];          /* launches that were bracketed by events               */
  int64_t kernels[8];        /* kernel launches (a persistent launch counts once, a
                                call that launches two kernels counts two)            */
} mrstat_kernel_stats;

int mrstat_profile_start(mrstat_plan* plan, uint32_t kernel_mask);
int mrstat_profile_stop(mrstat_plan* plan, mrstat_kernel_stats* out);

const char* mrstat_status_string(int status);

/* Message of the last failed call on the calling thread ("" if none). */
const char* mrstat_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MRSTAT_H */
