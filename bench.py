#!/usr/bin/env python
"""Benchmark of the MR-STAT hot path: J^H.J.v products per second.

One step = one pass of the inner Gauss-Newton solve (Algorithm 6) on a 224x224 grid
with 1120 TRs: linearise the Bloch model (all voxels, with tangents), then a fixed
number of CG iterations on Re(J^H J) x = b, each one J^H J v product plus the CG
inner products.  value = CG products per second summed over ranks, for the form
selected with --form:

* surrogate (default): the compressed model in a rank-32 time basis whose coefficients
  come from the learned surrogate (one MLP inference on the tensor cores per step);
  every J^H J v is the per-ky Gram product between the phase-encode DFT and its
  adjoint (factorised 224 = 7 x 32 on the CUDA cores, fused into the first and last
  pass; the readout DFT pair cancels: nkx = nx);
* lowrank: the same products, the linearisation projects the exact Bloch recursion
  onto the basis;
* plain: exact FP32 model; the linearisation caches m_y and its tangents
  (3 x 1120 x 50176 float32 = 674 MB, more than the 126 MB L2) and every J^H J v
  streams them twice (J.v, then Re(J^H w)) with an FP32 readout DFT between;
* split: as plain, readout DFT as split-BF16 tcgen05 products.

The run also times the plain form on the same inputs (key "plain") and runs the full
reconstruction (15 Gauss-Newton x 30 CG from T1 = 1000 ms, T2 = 100 ms with the exact
least-squares rho initialisation and mask, SNR 30 data) with the exact CG matrix, the low-rank CG
matrix, and 10 surrogate iterations followed by 5 exact ones (key "recon": seconds
and T1/T2/rho NRMSE against the ground truth, and whether the fast runs reach the
plain run's NRMSE: |NRMSE_fast - NRMSE_plain| <= max(0.1 NRMSE_plain, 1e-3)), plus one
reconstruction with B1 as a fifth unknown on the phantom with a smooth B1 field
(key "recon.b1_estimated"), and the same step in the low-rank form on the paper's other
sequence shapes: 224 x 224 with 1792 TRs and the sine-squared train, and the 112 x 88,
16-fill constant-flip scan (key "shapes": products/s), and the slice-profile Bloch model
(32 isochromats, 16 Gaussian RF sub-steps): one linearisation and the plain-form step with
it (key "slice_profile").
Inputs are the seeded brain-like phantom and flip train of ``synth``.

Multi-GPU: N independent replicas (one per rank), weak scaling, no collective on
the data path; the timing takes the maximum over ranks.

``--impl reference`` times the FP64 oracle (the reference of this build) on the
host cores on a bounded sample of the same workload and extrapolates to the full
step; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import math
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "J^H·J·v products/s and recon seconds at 224² vs plain FP32 GPU, equal T1/T2 NRMSE"
HBM_FALLBACK_GBS = 6800.0

# DRAM traffic per launch from one ncu capture, keyed by the SHA-256 prefix of the
# kernel's source file at capture time; reported only while the source is unchanged.
NCU_TRAFFIC = {
    # (kernel class, source hash): dram__bytes_read.sum + dram__bytes_write.sum per launch
    # profiles/tc_gemm_persistent_brain224.md
    ("xdft", "0728f575d9d96a3d"): 13670656.0,
    ("xdft_adj", "0728f575d9d96a3d"): 13668608.0,
    # profiles/lr_cg_columns_kernel_brain224.md: one persistent CG launch of 30 products
    # read 20 971 520 B and wrote 0 B (caches flushed before it), per product
    ("jhw_dot", "4ac33d5f5257c6e2"): (20971520.0 + 0.0) / 30,
    # profiles/rc_product_kernel_brain224.md: one recompute J^H J v read 12 698 624 B
    ("jhw_dot_rc", "43b010ca1597d1da"): 12698624.0,
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="brain224")
    ap.add_argument("--cg-iters", type=int, default=30)
    ap.add_argument("--segment", type=int, default=140,
                    help="TRs per segment of the plain form's recompute variant")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-plan", action="store_true",
                    help="also run the oracle's full CPU baseline plan (single-threaded and all cores; minutes)")
    ap.add_argument("--oracle-plan-worker", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--form", default="surrogate", choices=["surrogate", "lowrank", "plain", "recompute", "split"])
    ap.add_argument("--hidden", type=int, default=256)
    ap.add_argument("--train-steps", type=int, default=24000)
    ap.add_argument("--rank", type=int, default=32)
    ap.add_argument("--no-recon", action="store_true")
    ap.add_argument("--no-shapes", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the split-BF16 (precision form) legs")
    ap.add_argument("--no-fp64-errors", action="store_true",
                    help="skip the error of every form against the FP64 oracle on sampled outputs")
    ap.add_argument("--no-diff", action="store_true", help="skip the differentiation-form leg (autograd)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-part legs (224x224 and 256x256 with a B1 map)")
    ap.add_argument("--clock-log", default=os.environ.get("MRSTAT_CLOCK_LOG"),
                    help="CSV file for the nvidia-smi clock samples of the timed region "
                         "(default: a file in the system temp directory)")
    ap.add_argument("--profile-recon", default=None, choices=["plain", "lowrank", "surrogate"],
                    help="run that reconstruction once more first and bracket the timed one with "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


def alpha_of(ph):
    return np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                     ph.rho.imag.ravel()]).astype(np.float32)


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample(workload: str, ntr_sample: int, products: int, seed: int = 0, rows: int | None = None):
    """Time the oracle's linearisation and products on the first ntr_sample TRs (and the
    first ``rows`` image rows) of the workload; returns (seconds for linearise, seconds
    per product, scale) where scale = full work / sampled work (linear in TRs and rows)."""
    from oracle import model
    seq, ph = synth.config(workload, seed)
    rows = seq.ny if rows is None else min(rows, seq.ny)
    sub = synth.Sequence(nx=seq.nx, ny=rows, nkx=seq.nkx, tr_ms=seq.tr_ms, te_ms=seq.te_ms,
                         flip_rad=seq.flip_rad[:ntr_sample],
                         ky=np.clip(seq.ky[:ntr_sample], -(rows // 2), rows - rows // 2 - 1),
                         inversion=seq.inversion, alternate_phase=seq.alternate_phase)
    scale = (seq.ntr / ntr_sample) * (seq.ny / rows)
    alpha = alpha_of(ph).astype(np.float64)[:, :rows * seq.nx]
    v = synth.random_params(rows * seq.nx, 7)
    t0 = time.perf_counter()
    lin = model.linearize(sub, alpha)
    t1 = time.perf_counter()
    for _ in range(products):
        v = model.gauss_newton_product(lin, v)
        v = v / max(np.linalg.norm(v), 1e-30)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / max(products, 1), scale


def oracle_plan_worker(seeds: int = 3):
    """The oracle's CPU timings on this process's thread settings (the caller sets
    OMP_NUM_THREADS and friends before numpy loads): forward, J.v, Re(J^H w) and
    Re(J^H J) v in full on the 64 x 64 / 320-TR workload; a 10 x 20 Gauss-Newton solve on
    the 16 x 16 / 64-TR workload (SNR 50), one outer iteration of it on the 64 x 64
    workload (scaled by 10: a full solve takes minutes); the 224 x 224 /
    1120-TR linearisation and product on 8 of its TRs, extrapolated linearly in TRs.
    Medians over `seeds` seeded runs after one warm-up run where the item is short."""
    from oracle import model, solver
    res = {}

    def med(fn, n, warm=True):
        if warm:
            fn()
        ts = []
        for i in range(n):
            t0 = time.perf_counter()
            fn(i)
            ts.append(time.perf_counter() - t0)
        return float(np.median(ts))

    seq, ph = synth.config("ellipse64")
    alpha = alpha_of(ph).astype(np.float64)
    lin = model.linearize(seq, alpha)
    v = synth.random_params(seq.nv, 1)
    w = synth.random_kspace(seq.ntr, seq.nkx, 2)
    res["ellipse64_forward_s"] = med(lambda i=0: model.forward(seq, alpha), seeds)
    res["ellipse64_linearize_s"] = med(lambda i=0: model.linearize(seq, alpha), seeds)
    res["ellipse64_jvp_s"] = med(lambda i=0: model.jvp(lin, v), seeds)
    res["ellipse64_jhw_s"] = med(lambda i=0: model.jhw(lin, w), seeds)
    res["ellipse64_jhjv_s"] = med(lambda i=0: model.gauss_newton_product(lin, v), seeds)

    def gn(name, outer, inner, snr, n):
        sq, p = synth.config(name)
        a = alpha_of(p).astype(np.float64)
        d = synth.add_noise(model.forward(sq, a), snr, 3)

        def run(i=0):
            a0, mask = solver.initial_alpha(sq, d, sq.nv, exact=True)
            solver.gauss_newton(sq, d, a0, mask=mask, opts=solver.GNOptions(outer_iters=outer, inner_iters=inner))
        return med(run, n, warm=n > 1)
    res["quad16_gn_10x20_s"] = gn("quad16", 10, 20, 50.0, seeds)
    # 64 x 64: one outer iteration (with the rho initialisation) timed, scaled by 10
    res["ellipse64_gn_1x20_s"] = gn("ellipse64", 1, 20, 50.0, 1)
    res["ellipse64_gn_10x20_s_extrapolated"] = 10 * res["ellipse64_gn_1x20_s"]
    t_lin, t_prod, scale = oracle_sample("brain224", 8, 1)
    res["brain224_linearize_s_extrapolated"] = t_lin * scale
    res["brain224_jhjv_s_extrapolated"] = t_prod * scale
    res["brain224_note"] = "224 x 224 / 1120 TRs timed on 8 TRs and scaled by 140 (linear in TRs)"
    return res


def fp64_errors(mr, torch, seq, ph, alpha_h, U, net):
    """Normwise relative error of every form against the FP64 oracle on sampled outputs of
    the workload, which the oracle computes one by one (this runs the oracle, so it belongs
    to the cpu_baseline leg): s and J.v on 12 TRs, Re(J^H w) on 64 voxels and Re(J^H J) v on
    3 image columns (with nkx = nx the readout DFT pair cancels, so a column of the product
    is nx times the product of that column alone).  The low-rank and surrogate forms are
    compared with the exact model (their model error included) and, for Re(J^H w) and
    Re(J^H J) v, with the oracle's projection on the same basis (the low-rank form's
    arithmetic error; the surrogate's fit error)."""
    from oracle import bloch, encoding, metrics, model
    rng = np.random.default_rng(53)
    rows = np.sort(rng.choice(seq.ntr, 12, replace=False))
    vox = np.sort(rng.choice(seq.nv, 64, replace=False))
    cols = [40, seq.nx // 2, seq.nx - 50]
    alpha = alpha_h.astype(np.float64)
    v = synth.random_params(seq.nv, 51)
    w = synth.random_kspace(seq.ntr, seq.nkx, 52)
    Ud = U.cpu().numpy().astype(np.float64)
    # oracle: s and J.v on the sampled TRs
    sim = bloch.simulate(seq, np.exp(alpha[0]), np.exp(alpha[1]), rows=rows)
    rho = alpha[2] + 1j * alpha[3]
    ref = {"s": encoding.encode(seq, rho[None, :] * sim["m"], rows),
           "jv": encoding.encode(seq, rho[None, :] * (v[0][None, :] * sim["dm_dlnT1"] + v[1][None, :] * sim["dm_dlnT2"])
                                 + (v[2] + 1j * v[3])[None, :] * sim["m"], rows)}
    del sim
    # Re(J^H w) on the sampled voxels: exact and projected time courses
    simv = bloch.simulate(seq, np.exp(alpha[0, vox]), np.exp(alpha[1, vox]))
    W = encoding.encode_adjoint(seq, w, vox)
    rv = rho[vox]

    def gdot(m, d1, d2):
        return np.stack([np.real(np.sum(np.conj(rv[None] * d1) * W, 0)), np.real(np.sum(np.conj(rv[None] * d2) * W, 0)),
                         np.real(np.sum(np.conj(m) * W, 0)), np.real(np.sum(np.conj(1j * m) * W, 0))])
    P = Ud @ Ud.T
    ref["g"] = gdot(simv["m"], simv["dm_dlnT1"], simv["dm_dlnT2"])
    ref_g_proj = gdot(P @ simv["m"], P @ simv["dm_dlnT1"], P @ simv["dm_dlnT2"])
    # Re(J^H J) v on the sampled columns
    v3 = v.reshape(4, seq.ny, seq.nx)
    h_ref, h_proj = [], []
    for ix in cols:
        sub = synth.Sequence(nx=1, ny=seq.ny, nkx=1, tr_ms=seq.tr_ms, te_ms=seq.te_ms, flip_rad=seq.flip_rad,
                             ky=seq.ky, inversion=seq.inversion, alternate_phase=seq.alternate_phase)
        a1 = alpha.reshape(4, seq.ny, seq.nx)[:, :, ix]
        lin = model.linearize(sub, a1)
        h_ref.append(seq.nx * model.gauss_newton_product(lin, v3[:, :, ix]))
        h_proj.append(seq.nx * model.gauss_newton_product(model.project_onto_basis(lin, Ud), v3[:, :, ix]))
    ref["h"] = np.stack(h_ref, -1)
    ref_h_proj = np.stack(h_proj, -1)

    a_dev = torch.tensor(alpha_h, device="cuda")
    v_dev = torch.tensor(v.astype(np.float32), device="cuda")
    w_dev = torch.tensor(w, dtype=torch.complex64, device="cuda")

    def outputs(pl, with_s):
        o = {}
        if with_s:
            o["s"] = pl.forward(a_dev).cpu().numpy()[rows]
        o["jv"] = pl.jvp(v_dev).cpu().numpy()[rows]
        o["g"] = pl.jhw(w_dev).cpu().numpy()[:, vox]
        o["h"] = pl.jhjv(v_dev).cpu().numpy().reshape(4, seq.ny, seq.nx)[:, :, cols]
        pl.check()
        return o

    res = {"sample": "12 TRs (s, J.v), 64 voxels (Re(J^H w)), 3 image columns (Re(J^H J) v) of the workload"}
    for name, form in (("plain", mr.MRSTAT_FORM_PLAIN_FP32), ("split", mr.MRSTAT_FORM_SPLIT_BF16)):
        pl = mr.Plan(seq, form=form)
        pl.linearize(a_dev)
        o = outputs(pl, True)
        pl.close()
        res[name] = {k: metrics.relerr(o[k], ref[k]) for k in o}
    pl = mr.Plan(seq)
    pl.lowrank_set_basis(U)
    for name in ("lowrank", "surrogate"):
        if name == "surrogate":
            if net is None:
                continue
            pl.lowrank_linearize(a_dev, coef=net.infer(a_dev[:2]))
        else:
            pl.lowrank_linearize(a_dev)
        o = outputs(pl, False)
        res[name] = {k: metrics.relerr(o[k], ref[k]) for k in o}
        res[name]["g_vs_projected"] = metrics.relerr(o["g"], ref_g_proj)
        res[name]["h_vs_projected"] = metrics.relerr(o["h"], ref_h_proj)
    pl.close()
    return res


def run_oracle_plan():
    """The oracle's CPU baseline plan, single-threaded and on all host cores, each in a
    fresh interpreter so that the thread settings take effect before numpy loads."""
    out = {"cores": cpu_cores()}
    for label, threads in (("one_thread", 1), ("all_cores", cpu_cores())):
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-plan-worker"], env=env,
                           capture_output=True, text=True)
        if r.returncode != 0:
            out[label] = {"error": r.stderr[-500:]}
            continue
        out[label] = json.loads(r.stdout.strip().splitlines()[-1])
        out[label]["threads"] = threads
    return out


def max_over_ranks(x: float, dist=None) -> float:
    """Maximum of a per-rank float over the process group (the timing rule for N > 1);
    the tensor lives on the current CUDA device under NCCL, on the CPU under gloo."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_products_per_s(t_lin, t_prod, scale, iters):
    """Extrapolate the sample linearly to the full step (linearise + iters products)."""
    return iters / ((t_lin + iters * t_prod) * scale)


def run_reference(args, rank: int):
    if rank != 0:
        return
    seq, _ = synth.config(args.workload)
    # one step is about 1 s of oracle work on a full-grid single-TR sample; shrink the
    # sampled image rows so that warm-up + steps stay within about two minutes
    n = max(args.steps + args.warmup, 1)
    rows = max(8, min(seq.ny, int(seq.ny * 100.0 / n)))
    ntr_sample = 1
    times = []
    for i in range(n):
        t_lin, t_prod, scale = oracle_sample(args.workload, ntr_sample, 1, rows=rows)
        if i >= args.warmup:
            times.append((t_lin, t_prod))
    if not times:
        times.append((t_lin, t_prod))
    t_lin = float(np.median([t[0] for t in times]))
    t_prod = float(np.median([t[1] for t in times]))
    value = oracle_products_per_s(t_lin, t_prod, scale, args.cg_iters)
    step_s = args.cg_iters / value
    sample = (f"FP64 NumPy oracle: linearise + 1 J^H J v product on the first {ntr_sample} of {seq.ntr} TRs "
              f"and the first {rows} of {seq.ny} image rows of {args.workload}, extrapolated linearly in TRs "
              f"and rows to linearise + {args.cg_iters} products")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "products/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {seq.nx}x{seq.ny} grid, {seq.ntr} TRs, {seq.nkx} readout "
                                   "samples, exact Bloch model (the oracle)",
                       "form": "oracle", "step": f"linearize + {args.cg_iters} CG iterations (one J^H J v each)",
                       "cg_iters": args.cg_iters, "parallelism": "rank 0 on the host cores"},
            "cpu_baseline": {"value": value, "unit": "products/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# learned surrogate: trained on device on exact projections of the Bloch model
# ---------------------------------------------------------------------------
def training_params(torch, n, seed):
    """Parameter samples of the learned part: T1 log-U(100, 6000) ms, T2 log-U(10, 3000) ms
    (the paper's training ranges widened so that CSF does not extrapolate) and B1 U(0.8,
    1.2); returns (ln T1 / ln T2 [2, n], B1 [n]) on the device."""
    rng = np.random.default_rng(seed)
    x = np.stack([rng.uniform(np.log(100), np.log(6000), n), rng.uniform(np.log(10), np.log(3000), n)])
    b1 = rng.uniform(0.8, 1.2, n)
    return (torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(b1, dtype=torch.float32, device="cuda"))


def train_surrogate(mr, torch, plan, rank, hidden, steps, n_train=1 << 20, batch=4096, seed=0):
    """MLP fitted to the plan's projected Bloch model on n_train samples (T1, T2, B1 drawn
    by training_params); targets from mrstat_lowrank_project_samples, i.e. the Bloch kernel
    itself.  Returns the network and a summary (training seconds, held-out relative errors
    of c, dc/dlnT1, dc/dlnT2 on B1-varied samples and at B1 = 1)."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, xb = training_params(torch, n_train, seed + 77)
    tgt = plan.lowrank_project_samples(x, b1=xb)
    scale = tgt[0].abs().amax(dim=1).clamp_min(1e-6).cpu().numpy()
    net = mr.Surrogate(hidden, rank, (np.log(1000.0), 1.0, np.log(100.0), 1.2, 1.0, 0.2), 0.5, seed=seed)
    net.set_output_scale(scale)
    for it in range(steps):
        idx = torch.randint(0, n_train, (batch,), device="cuda", generator=gen)
        lr = 2e-3 if it < steps * 0.6 else (6e-4 if it < steps * 0.85 else 2e-4)
        net.train_step(x[:, idx].contiguous(), tgt[:, :, idx].contiguous(), lr, b1=xb[idx].contiguous())
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    del tgt
    xt, xtb = training_params(torch, 16384, seed + 78)

    def held_out(b1):
        tt = plan.lowrank_project_samples(xt, b1=b1)
        pred = net.infer(xt, b1=b1)
        return {k: float(torch.linalg.vector_norm(pred[i] - tt[i]) / torch.linalg.vector_norm(tt[i]))
                for i, k in enumerate(("c", "dc_dlnT1", "dc_dlnT2"))}
    return net, {"hidden": hidden, "train_seconds": secs, "train_samples": n_train, "steps": steps,
                 "batch": batch, "b1_range": [0.8, 1.2], "holdout_relerr": held_out(xtb),
                 "holdout_relerr_b1_1": held_out(None)}


# ---------------------------------------------------------------------------
# the timed solve's result, checked after the timed region
# ---------------------------------------------------------------------------
def check_cg(torch, plan, rhs, x, iters):
    """After the timed steps: no device wait ran out (mrstat_plan_check raises), every CG
    iteration was applied, and x of the last step against CG run product by product
    through mrstat_jhjv at the same linearisation with float64 vectors and scalars."""
    plan.check()
    applied = plan.cg_applied()
    xr = torch.zeros_like(rhs, dtype=torch.float64)
    r = rhs.double().clone()
    p = r.clone()
    rr = float(torch.sum(r * r))
    rr0 = rr
    for _ in range(iters):
        q = plan.jhjv(p.float()).double()
        a = rr / float(torch.sum(p * q))
        xr += a * p
        r -= a * q
        rr_new = float(torch.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    err = float(torch.linalg.vector_norm(x.double() - xr) / torch.linalg.vector_norm(xr))
    res = plan.jhjv(x).double() - rhs.double()
    return {"iterations_applied": applied, "iterations": iters,
            "relerr_vs_product_by_product_cg_f64": err,
            "true_residual_rel": float(torch.linalg.vector_norm(res)) / np.sqrt(rr0),
            "f64_cg_recursive_residual_rel": float(np.sqrt(rr / rr0)),
            "plan_check": "ok"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, path: str | None = None):
        self.gpu = gpu_index
        self.proc = None
        if path is None:
            import tempfile
            path = os.path.join(tempfile.gettempdir(), f"mrstat_clocks_{os.getpid()}.csv")
        self.path = path

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


# ---------------------------------------------------------------------------
# reconstructions (Algorithm 6)
# ---------------------------------------------------------------------------
def noisy_data(torch, plan, truth, b1, snr=30.0):
    """d = s(truth) + complex Gaussian noise with ||s|| / ||noise|| = snr (seeded)."""
    s_true = plan.forward(truth, b1=b1)
    gen = torch.Generator(device="cpu").manual_seed(7)
    noise = torch.complex(torch.randn(s_true.shape, generator=gen), torch.randn(s_true.shape, generator=gen))
    noise = noise.to("cuda").to(torch.complex64)
    return s_true + noise * (torch.linalg.vector_norm(s_true) / (snr * torch.linalg.vector_norm(noise))), noise


def reconstruct(torch, plan, seq, ph, truth, d, b1, runs, rho_kw, profile=None, outer=15, inner=30):
    """One 15 x 30 Gauss-Newton reconstruction per entry of runs (name, gn options) from
    T1 = 1000 ms, T2 = 100 ms with the rho initialisation rho_kw and the 0.1 mask; seconds
    and T1 / T2 / rho NRMSE against the truth over the drawn mask inside the support, and
    whether each run reaches the "plain" run's T1 and T2 NRMSE:
    |NRMSE - NRMSE_plain| <= max(0.1 NRMSE_plain, 1e-3)."""
    out = {}
    sup = torch.tensor(ph.support.ravel(), device="cuda")
    for name, kw in runs:
        a = torch.zeros((4, seq.nv), dtype=torch.float32, device="cuda")
        mask = torch.zeros(seq.nv, dtype=torch.uint8, device="cuda")
        if profile == name:
            plan.gn_solve(d, a.clone(), b1=b1, mask=mask.clone(), outer_iters=outer, inner_iters=inner,
                          mask_threshold=0.1, **rho_kw, **kw)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = plan.gn_solve(d, a, b1=b1, mask=mask, outer_iters=outer, inner_iters=inner, mask_threshold=0.1,
                            **rho_kw, **kw)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        if profile == name:
            torch.cuda.profiler.stop()
        m = mask.bool() & sup

        def nrmse(x, y):
            return float(torch.linalg.vector_norm((x - y)[m]) / torch.linalg.vector_norm(y[m]))
        out[name] = {"seconds": secs, "nrmse_t1": nrmse(torch.exp(a[0]), torch.exp(truth[0])),
                     "nrmse_t2": nrmse(torch.exp(a[1]), torch.exp(truth[1])),
                     "nrmse_rho": float(torch.linalg.vector_norm(torch.complex(a[2] - truth[2], a[3] - truth[3])[m])
                                        / torch.linalg.vector_norm(torch.complex(truth[2], truth[3])[m])),
                     "f_final": rep["f_final"], "accepted": sum(rep["accepted"]),
                     "cg_steps": sum(rep["cg_steps"]), "mask_voxels": rep["mask_voxels"]}
    for name in out:
        if name != "plain" and "plain" in out:
            out[name]["equal_nrmse"] = all(abs(out[name][k] - out["plain"][k]) <= max(0.1 * out["plain"][k], 1e-3)
                                           for k in ("nrmse_t1", "nrmse_t2"))
    return out


def gn_rhs(torch, plan, alpha, b1, seq, rank):
    """A Gauss-Newton right-hand side: Re(J^H w) of the exact model at alpha for a seeded
    complex Gaussian k-space vector w, scaled to unit RMS.  It lies in the range of
    Re(J^H J), so CG solves a consistent system (the background voxels' ln T1 / ln T2 rows,
    where rho = 0, are in the null space)."""
    plan.linearize(alpha, b1=b1)
    w = torch.tensor(synth.random_kspace(seq.ntr, seq.nkx, 100 + rank), dtype=torch.complex64, device="cuda")
    g = plan.jhw(w)
    return (g / torch.sqrt(torch.mean(g * g))).contiguous()


def differentiation(mr, torch, seq, ph, reps=10):
    """The differentiation form at the workload's size: s(alpha) as a torch.autograd.Function
    with the loss 1/2 ||s - d||^2, forward and backward timed with CUDA events (median of
    reps after a warm-up), with Bloch-state checkpoints every 64 TRs (the backward re-runs
    the recursion segment by segment) and without (the forward caches the time courses);
    device memory held by the plan after the forward, and torch's peak over the pass."""
    from paper_1904_13244_gb300.autograd import signal
    a0 = torch.tensor(alpha_of(ph), device="cuda")
    d = torch.zeros((seq.ntr, seq.nkx), dtype=torch.complex64, device="cuda")
    out = {}
    for ck in (64, 0):
        plan = mr.Plan(seq)
        fw, bw = [], []
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        for i in range(reps + 1):
            a = a0.clone().requires_grad_(True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            s = signal(a, plan, checkpoint=ck)
            loss = 0.5 * torch.sum(torch.abs(s - d) ** 2)
            e1.record()
            loss.backward()
            e2.record()
            torch.cuda.synchronize()
            if i > 0:
                fw.append(e0.elapsed_time(e1))
                bw.append(e1.elapsed_time(e2))
            del s, loss
        plan.check()
        out[f"checkpoint_{ck}" if ck else "no_checkpoint"] = {
            "forward_ms": float(np.median(fw)), "backward_ms": float(np.median(bw)),
            "plan_device_bytes": int(plan.info()["device_bytes"]),
            "torch_peak_bytes": int(torch.cuda.max_memory_allocated() - base)}
        plan.close()
    out["note"] = ("loss 1/2 ||s - d||^2 through paper_1904_13244_gb300.autograd.signal; forward = "
                   "Bloch recursion + encoding (+ the loss), backward = Re(J^H grad_s)")
    return out


def plain_products(mr, torch, names=("ellipse64", "brain224"), reps=20):
    """The plain FP32 form's single products per second (cached time courses): J.v,
    Re(J^H w) and Re(J^H J) v on the 64 x 64 / 320-TR ellipse workload and on brain224, CUDA
    events around reps back-to-back calls after a warm-up; the linearisation (K1) timed on
    its own."""
    out = {}
    for name in names:
        seq, ph = synth.config(name)
        pl = mr.Plan(seq)
        a = torch.tensor(alpha_of(ph), device="cuda")
        v = torch.tensor(synth.random_params(seq.nv, 3).astype(np.float32), device="cuda")
        w = torch.tensor(synth.random_kspace(seq.ntr, seq.nkx, 4), dtype=torch.complex64, device="cuda")
        jv = torch.empty((seq.ntr, seq.nkx), dtype=torch.complex64, device="cuda")
        g = torch.empty((4, seq.nv), dtype=torch.float32, device="cuda")
        res = {"grid": [seq.nx, seq.ny], "ntr": seq.ntr}
        for key, fn in (("linearize", lambda: pl.linearize(a)), ("jvp", lambda: pl.jvp(v, out=jv)),
                        ("jhw", lambda: pl.jhw(w, out=g)), ("jhjv", lambda: pl.jhjv(v, out=g))):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[key + "_ms"] = ms
            if key != "linearize":
                res[key + "_per_s"] = 1e3 / ms
        pl.check()
        pl.close()
        out[name] = res
    return out


def learned_part(mr, torch, args, name, rank, iters, timed, trained=None):
    """The learned-part form on a workload with a smooth, known B1 map in [0.8, 1.2]: a
    rank-R basis and the surrogate trained for this sequence on B1-varied samples, then the
    bench step (linearise + iters CG iterations) with the surrogate's coefficients, with the
    compressed-exact coefficients (the Bloch recursion projected on the basis) and with the
    plain FP32 model, and the three 15 x 30 reconstructions (rho initialised by 50 CGLS
    steps: the exact least-squares form needs B1 = 1)."""
    seq, ph = synth.config(name, seed=rank, b1_map=True)
    plan = mr.Plan(seq)
    own = trained is None
    if own:
        train, train_b1 = training_params(torch, 4096, 1000)
        U, _ = plan.lowrank_basis(train, args.rank, train_b1=train_b1)
        plan.lowrank_set_basis(U)
        net, info = train_surrogate(mr, torch, plan, args.rank, args.hidden, args.train_steps)
    else:
        # the same sequence as the headline workload: its basis and network (trained on the
        # same B1-varied distribution) serve here as they are
        U, net, info = trained
        plan.lowrank_set_basis(U)
    a = torch.tensor(alpha_of(ph), device="cuda")
    b1 = torch.tensor(ph.b1.ravel().astype(np.float32), device="cuda")
    rhs = gn_rhs(torch, plan, a, b1, seq, rank)
    x = torch.empty_like(rhs)
    coef = torch.empty((3, args.rank, seq.nv), dtype=torch.float32, device="cuda")

    def step_surrogate():
        net.infer(a[:2], b1=b1, out=coef)
        plan.lowrank_linearize(a, b1=b1, coef=coef)
        plan.cg_fixed(rhs, iters, out=x)

    def step_lowrank():
        plan.lowrank_linearize(a, b1=b1)
        plan.cg_fixed(rhs, iters, out=x)

    def step_plain():
        plan.linearize(a, b1=b1)
        plan.cg_fixed(rhs, iters, out=x)
    out = {"grid": [seq.nx, seq.ny], "ntr": seq.ntr, "rank": args.rank,
           "b1": "known map 1 + 0.2 smooth field clipped to [0.8, 1.2]", "surrogate": info}
    nsteps = max(5, args.steps // 4)
    for key, st in (("surrogate", step_surrogate), ("lowrank", step_lowrank), ("plain", step_plain)):
        ms, _, _ = timed(plan, st, nsteps, ())
        out[key + "_step"] = {"products_per_s": iters / (ms / 1e3), "ms_per_step": ms,
                              "cg_iterations_applied": plan.cg_applied()}
    out["surrogate_gain_vs_lowrank"] = out["surrogate_step"]["products_per_s"] / out["lowrank_step"]["products_per_s"]
    out["surrogate_gain_vs_plain"] = out["surrogate_step"]["products_per_s"] / out["plain_step"]["products_per_s"]
    if not args.no_recon:
        truth = a.clone()
        d, _ = noisy_data(torch, plan, truth, b1)
        runs = [("plain", dict(hessian=0)), ("lowrank", dict(hessian=1)),
                ("surrogate", dict(hessian=1, surrogate_iters=10, surrogate=net))]
        out["recon"] = reconstruct(torch, plan, seq, ph, truth, d, b1, runs, dict(rho_init_iters=50))
    if own:
        net.close()
    plan.close()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.oracle_plan_worker:
        print(json.dumps(oracle_plan_worker()), flush=True)
        return
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1904_13244_gb300 import build as _build
    _build.build()
    import paper_1904_13244_gb300 as mr

    seq, ph = synth.config(args.workload, seed=rank)
    iters = args.cg_iters
    alpha_h = alpha_of(ph)
    form_code = mr.MRSTAT_FORM_SPLIT_BF16 if args.form == "split" else mr.MRSTAT_FORM_PLAIN_FP32
    plan = mr.Plan(seq, form=form_code)
    a_dev = torch.tensor(alpha_h, device="cuda")
    rhs_dev = gn_rhs(torch, plan, a_dev, None, seq, rank)
    rhs_h = rhs_dev.cpu().numpy()
    if args.form == "recompute":
        plan.set_recompute(args.segment)
    x_dev = torch.empty_like(rhs_dev)
    stream = torch.cuda.current_stream()
    basis = None
    net = None
    surrogate_info = None
    if args.form in ("lowrank", "surrogate") or not args.no_recon:
        train, train_b1 = training_params(torch, 4096, 1000)
        basis, _ = plan.lowrank_basis(train, args.rank, train_b1=train_b1)
        plan.lowrank_set_basis(basis)
    if args.form == "surrogate" or not args.no_recon:
        net, surrogate_info = train_surrogate(mr, torch, plan, args.rank, args.hidden, args.train_steps)
    coef_dev = torch.empty((3, args.rank, seq.nv), dtype=torch.float32, device="cuda")

    def make_step(pl, form):
        def step():
            if form == "surrogate":
                net.infer(a_dev[:2], out=coef_dev)
                pl.lowrank_linearize(a_dev, coef=coef_dev)
            elif form == "lowrank":
                pl.lowrank_linearize(a_dev)
            else:
                pl.linearize(a_dev)
            pl.cg_fixed(rhs_dev, iters, out=x_dev)
        return step

    def timed(pl, step, nsteps, prof_kernels, sampler=None):
        for _ in range(max(args.warmup, 0)):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        pl.profile_start(())  # launch counters only: no events between the timed launches
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        st = pl.profile_stop()
        clk = sampler.stop() if sampler else None
        t = max_over_ranks(e0.elapsed_time(e1) / max(nsteps, 1), dist if world > 1 else None)
        if prof_kernels:
            # per-kernel times from a second pass of the same steps, CUDA events around each
            # launch of the listed kernel classes (outside the timed region)
            pl.profile_start(prof_kernels)
            for _ in range(nsteps):
                step()
            torch.cuda.synchronize()
            st = pl.profile_stop()
        if world > 1:
            dist.barrier()
        return t, st, clk

    all_kernels = ("bloch", "ycontract", "xdft", "xdft_adj", "jhw_dot")
    step = make_step(plan, args.form)
    ms, stats, clk = timed(plan, step, args.steps, all_kernels, ClockSampler(local, args.clock_log))
    value = world * iters / (ms / 1e3)
    cg_check = check_cg(torch, plan, rhs_dev, x_dev, iters)
    # what the learned surrogate buys: the same step with the coefficients of the exact
    # Bloch recursion projected on the basis (the compressed-exact form) on the same inputs
    compressed_exact = None
    if args.form == "surrogate":
        cms, _, _ = timed(plan, make_step(plan, "lowrank"), max(5, args.steps // 4), ())
        compressed_exact = {"value": world * iters / (cms / 1e3), "ms_per_step": cms,
                            "surrogate_gain": value / (world * iters / (cms / 1e3))}

    # the plain FP32 form on the same inputs, for the comparison the metric asks for
    plain = None
    if args.form not in ("plain", "recompute"):
        # the plain FP32 form in both variants, cached time courses and the recompute form
        # (the recursion re-run inside every product from states every `segment` TRs); the
        # faster one is the plain form the comparison uses
        pplan = mr.Plan(seq)
        nst = max(1, args.steps // 4)
        pms, pstats, _ = timed(pplan, make_step(pplan, "plain"), nst, all_kernels)
        stored = {"value": world * iters / (pms / 1e3), "ms_per_step": pms,
                  "kernel_ms_per_step": {k: pstats[k]["ms"] / nst for k in all_kernels}}
        pplan.set_recompute(args.segment)
        rms, rstats, _ = timed(pplan, make_step(pplan, "plain"), nst, all_kernels)
        pplan.check()
        recompute = {"value": world * iters / (rms / 1e3), "ms_per_step": rms, "segment": args.segment,
                     "kernel_ms_per_step": {k: rstats[k]["ms"] / nst for k in all_kernels},
                     "cg_iterations_applied": pplan.cg_applied()}
        pplan.close()
        best = "recompute" if recompute["value"] > stored["value"] else "stored"
        plain = dict((recompute if best == "recompute" else stored), variant=best, stored=stored,
                     recompute=recompute)

    # the precision form: the exact model with the readout DFTs as split-BF16 tcgen05
    # products (s, J.v and Re(J^H w); inside J^H J v the readout DFT pair cancels because
    # nkx = nx, so its CG products are the plain form's)
    precision = None
    if args.form != "split" and not args.no_precision:
        xplan = mr.Plan(seq, form=mr.MRSTAT_FORM_SPLIT_BF16)
        nst = max(1, args.steps // 4)
        xms, xstats, _ = timed(xplan, make_step(xplan, "split"), nst, all_kernels)
        # the encoding alone: forward (K1 + K2 + split x-DFT) and J^H w (split x-DFT^H + K4)
        w_dev = torch.tensor(synth.random_kspace(seq.ntr, seq.nkx, 5), dtype=torch.complex64, device="cuda")

        def enc():
            xplan.forward(a_dev)
            xplan.jhw(w_dev)
        ems, estats, _ = timed(xplan, enc, nst, all_kernels)
        xplan.check()
        precision = {"value": world * iters / (xms / 1e3), "ms_per_step": xms,
                     "kernel_ms_per_step": {k: xstats[k]["ms"] / nst for k in all_kernels},
                     "forward_plus_jhw_ms": ems,
                     "xdft_launch_ms": estats["xdft"]["ms"] / max(estats["xdft"]["timed"], 1),
                     "xdft_adj_launch_ms": estats["xdft_adj"]["ms"] / max(estats["xdft_adj"]["timed"], 1),
                     "xdft_tflops_split": 3 * 2 * seq.ntr * (2 * seq.nkx) * (2 * seq.nx) / 1e12
                     / (estats["xdft"]["ms"] / max(estats["xdft"]["timed"], 1) / 1e3)}
        xplan.close()

    # the paper's other sequence shapes (Supporting Information S1 / S3): the same step in
    # the low-rank form (coefficients by exact projection), products/s
    shapes = None
    if not args.no_shapes and world == 1:
        shapes = {}
        train_s, train_sb1 = training_params(torch, 4096, 1000)
        for name in ("brain224_1792", "const112x88"):
            sseq, sph = synth.config(name, seed=rank)
            splan = mr.Plan(sseq)
            sa = torch.tensor(alpha_of(sph), device="cuda")
            srhs = gn_rhs(torch, splan, sa, None, sseq, rank)
            sx = torch.empty_like(srhs)
            sU, _ = splan.lowrank_basis(train_s, args.rank, train_b1=train_sb1)
            splan.lowrank_set_basis(sU)

            def sstep(splan=splan, sa=sa, srhs=srhs, sx=sx):
                splan.lowrank_linearize(sa)
                splan.cg_fixed(srhs, iters, out=sx)
            sms, _, _ = timed(splan, sstep, max(3, args.steps // 6), ())
            shapes[name] = {"products_per_s": iters / (sms / 1e3), "ms_per_step": sms,
                            "grid": [sseq.nx, sseq.ny], "ntr": sseq.ntr,
                            "train": synth.CONFIGS[name].get("train", "smooth"),
                            "column_kernel": bool(sseq.ny % 32 == 0 and sseq.ny // 32 <= 8)}
            splan.close()

    # the slice-profile Bloch model (32 isochromats, 16 Gaussian RF sub-steps): one
    # linearisation of the same phantom, and the exact-form step with it
    slice_prof = None
    if not args.no_shapes and world == 1:
        sp_plan = mr.Plan(seq)
        sp_plan.set_slice_profile(32, 16)
        for _ in range(2):
            sp_plan.linearize(a_dev)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        reps = 5
        for _ in range(reps):
            sp_plan.linearize(a_dev)
        ev1.record(stream)
        torch.cuda.synchronize()
        lin_ms = ev0.elapsed_time(ev1) / reps
        # per voxel, TR and isochromat: the pulse applied to m and both tangents (3 x 15
        # flops) and two relaxations with the tangents' source terms (2 x 25 flops)
        flops = seq.nv * seq.ntr * 32 * 95.0
        fp32_peak = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * 2.07e9
        sms, _, _ = timed(sp_plan, make_step(sp_plan, "plain"), max(3, args.steps // 6), ())
        slice_prof = {"linearize_ms": lin_ms, "isochromats": 32, "rf_substeps": 16,
                      "achieved_tflops": flops / (lin_ms / 1e3) / 1e12,
                      "fp32_peak_tflops": fp32_peak / 1e12, "frac": flops / (lin_ms / 1e3) / fp32_peak,
                      "plain_step_products_per_s": iters / (sms / 1e3), "plain_step_ms": sms}
        sp_plan.close()

    # end to end through the C ABI from pinned host buffers: every step copies its inputs
    # (alpha, rhs) in from host memory and its result x out.  Serving order: two sets of
    # device buffers, the next step's inputs copied in on one stream while the current
    # step computes, the results copied out on another; the host waits once at the end.
    e2e = None
    if not args.no_e2e:
        a_host = torch.tensor(alpha_h).pin_memory()
        rhs_host = torch.tensor(rhs_h).pin_memory()
        x_host = [torch.empty_like(rhs_host).pin_memory() for _ in range(2)]
        bufs = [(torch.empty_like(a_dev), torch.empty_like(rhs_dev), torch.empty_like(x_dev),
                 None if coef_dev is None else torch.empty_like(coef_dev)) for _ in range(2)]

        def step_on(b):
            a_b, r_b, x_b, c_b = b
            if args.form == "surrogate":
                net.infer(a_b[:2], out=c_b)
                plan.lowrank_linearize(a_b, coef=c_b)
            elif args.form == "lowrank":
                plan.lowrank_linearize(a_b)
            else:
                plan.linearize(a_b)
            plan.cg_fixed(r_b, iters, out=x_b)

        comp = torch.cuda.current_stream()
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def copy_in(i):
            j = i % 2
            with torch.cuda.stream(h2d):
                if i >= 2:
                    h2d.wait_event(ev_done[j])  # step i - 2 has read these buffers
                bufs[j][0].copy_(a_host, non_blocking=True)
                bufs[j][1].copy_(rhs_host, non_blocking=True)
                ev_in[j].record(h2d)

        k = max(2, min(args.steps, 50))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        copy_in(0)
        for i in range(k):
            j = i % 2
            if i + 1 < k:
                copy_in(i + 1)
            comp.wait_event(ev_in[j])
            if i >= 2:
                comp.wait_event(ev_out[j])  # step i - 2's result has left this buffer
            step_on(bufs[j])
            ev_done[j].record(comp)
            with torch.cuda.stream(d2h):
                d2h.wait_event(ev_done[j])
                x_host[j].copy_(bufs[j][2], non_blocking=True)
                ev_out[j].record(d2h)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / k, dist if world > 1 else None)
        e2e = {"value": world * iters / dt, "unit": "products/s",
               "h2d_bytes_per_step": int(a_host.numel() * 4 + rhs_host.numel() * 4),
               "d2h_bytes_per_step": int(x_host[0].numel() * 4),
               "pipeline": "two buffer sets; inputs in on one stream, results out on another, "
                           "overlapping the previous step's compute; one host wait at the end"}

    # roofline of the dominant kernel class
    info = plan.info()
    nv, ntr_pad, nx, ny, ntr, nkx = info["nv"], info["ntr_padded"], info["nx"], info["ny"], info["ntr"], seq.nkx
    R = args.rank
    d_bytes = 3 * ntr_pad * nv * 4
    per_step_ms = {k: stats[k]["ms"] / max(args.steps, 1) for k in all_kernels}
    per_launch = {k: stats[k]["ms"] / max(stats[k]["timed"], 1) for k in all_kernels}
    lowrank_like = args.form in ("lowrank", "surrogate")
    full_readout = nkx == nx
    column_bytes = None
    max_trs_per_ky = int(np.bincount(np.mod(np.asarray(seq.ky), ny), minlength=ny).max())
    fft_y = full_readout and ny % 32 == 0 and ny // 32 <= 8
    if lowrank_like and fft_y and max_trs_per_ky <= 8:
        # the whole product in one kernel per image column (FP32 CUDA cores): count its
        # arithmetic against the FP32-pipe peak: h and the contraction (20 flops per
        # basis function and voxel), the forward and adjoint phase-encode DFTs at the
        # conventional 5 N log2 N flops of a complex N-point FFT (independent of how the
        # kernel factorises them), the Gram through the TR axis (8 per basis function and
        # TR); its algorithmic bytes are the coefficients, v, rho, mask in and g out
        col_flops = nx * (R * ny * 20 + 2 * R * 5 * ny * math.log2(ny) + 8 * ntr * R)
        col_bytes = nv * (12 * R + 16 + 8 + 4 + 16)
        work = {"jhw_dot": (col_flops, "alu")}
        column_bytes = col_bytes
    elif lowrank_like and fft_y:
        # factorised phase-encode DFT on the CUDA cores, fused into the first and last pass
        work = {"ycontract": (nv * (16 + 8 + 4) + 3 * R * nv * 4 + R * nv * 8, "hbm"),   # v, rho, mask, c -> H
                "jhw_dot": (R * nv * 8 + 3 * R * nv * 4 + nv * (8 + 4) + nv * 16 + nv * 16, "hbm")}  # G, c, v -> g
    elif lowrank_like and full_readout:
        # per J^H J v: one phase-encode DFT GEMM in each of xdft / xdft_adj, three split
        # BF16 products of the real-embedded [R nx x 2ny] x [2ny x 2ny] matrices
        gemm_flops = 3 * 2 * (R * nx) * (2 * ny) * (2 * ny)
        op_bytes = R * nx * 2 * ny * 2 * 2  # one BF16 hi + lo operand [R nx][2 ny]
        work = {"xdft": (gemm_flops, "tensor"), "xdft_adj": (gemm_flops, "tensor"),
                # prep: v, rho, mask and 3 R coefficient rows in, the split operand out
                "ycontract": (nv * (16 + 8 + 4) + 3 * R * nv * 4 + op_bytes, "hbm"),
                # final: the adjoint DFT output, coefficients, rho, mask in, g out
                "jhw_dot": (R * nx * 2 * ny * 4 + 3 * R * nv * 4 + nv * (8 + 4) + nv * 16, "hbm")}
    elif lowrank_like:
        gemm_flops = 3 * 2 * (R * ny * (2 * nkx) * (2 * nx) + R * nkx * (2 * ny) * (2 * ny))
        work = {"xdft": (gemm_flops / 2, "tensor"), "xdft_adj": (gemm_flops / 2, "tensor")}
    elif args.form == "recompute" and full_readout:
        # one fused launch per product: 86 flops per voxel-TR (the rotation of m and both
        # tangents 18, two relaxations with the tangents' sources 34, the combination with
        # v and the phase 15, the adjoint phase and the four tangent products 17, the block
        # sums 2)
        work = {"jhw_dot": (86.0 * nv * ntr, "alu")}
    else:
        work = {"jhw_dot": (d_bytes + ntr_pad * nx * 8 + nv * (8 + 4 + 16) + ntr_pad * 4, "hbm"),
                "ycontract": (d_bytes + nv * 24 + ntr * nx * 8 + ntr_pad * 4, "hbm"),
                "bloch": (d_bytes + nv * 16, "hbm")}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}

    def roof(k):
        amount, bound = work[k]
        if bound == "hbm":
            peak, peak_kind = measured_peak_hbm()
            achieved = amount / (per_launch[k] / 1e3) / 1e9
            unit = "GB/s"
        elif bound == "alu":
            # FP32 FMA pipes: SMs x 128 lanes x 2 flops x the maximum SM clock
            props = torch.cuda.get_device_properties(torch.cuda.current_device())
            mhz = (clk or {}).get("sm_max_mhz") or 2070.0
            peak = props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12
            peak_kind = f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz"
            achieved = amount / (per_launch[k] / 1e3) / 1e12
            unit = "TFLOP/s"
        else:
            # a kernel timed inside a long step: the sustained BF16 figure
            peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
            peak_kind = "measured sustained" if peaks else "fallback"
            achieved = amount / (per_launch[k] / 1e3) / 1e12
            unit = "TFLOP/s"
        return {"kernel": k, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "peak_source": peak_kind, "algorithmic_per_launch": amount,
                "launch_ms": per_launch[k]}

    cand = {k: per_step_ms[k] for k in work if stats[k]["timed"] > 0}
    if args.form == "surrogate":
        # the MLP inference is not one of the plan's kernel classes: time it on its own
        for _ in range(3):
            net.infer(a_dev[:2], out=coef_dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            net.infer(a_dev[:2], out=coef_dev)
        e1.record(stream)
        torch.cuda.synchronize()
        H = args.hidden
        # value + two tangent rows per voxel through 3 -> H -> H -> H -> R
        work["mlp_infer"] = (2 * 3 * nv * (3 * H + 2 * H * H + H * R), "tensor")
        per_launch["mlp_infer"] = e0.elapsed_time(e1) / 20
        per_step_ms["mlp_infer"] = per_launch["mlp_infer"]
        cand["mlp_infer"] = per_step_ms["mlp_infer"]
    dom = max(cand, key=cand.get)
    src = {"jhw_dot": "encode.cu", "ycontract": "encode.cu", "bloch": "bloch.cu", "xdft": "tc_gemm.cu",
           "xdft_adj": "tc_gemm.cu", "mlp_infer": "mlp.cu"}
    if lowrank_like:
        src.update({"jhw_dot": "lowrank.cu", "ycontract": "lowrank.cu"})
    if args.form == "recompute":
        src.update({"jhw_dot": "fused.cu"})
    if dom == "mlp_infer":
        src["mlp_infer"] = "mlp.cu"
    h = source_hash(os.path.join(ROOT, "paper_1904_13244_gb300", "csrc", src[dom]))
    roofline = roof(dom)
    roofline["traffic"] = NCU_TRAFFIC.get((dom + ("_rc" if args.form == "recompute" else ""), h))
    if column_bytes is not None and dom == "jhw_dot":
        hbm_peak, _ = measured_peak_hbm()
        gbs = column_bytes / (per_launch[dom] / 1e3) / 1e9
        roofline["hbm"] = {"algorithmic_bytes": column_bytes, "achieved_GBs": gbs, "frac": gbs / hbm_peak}
    roofline["other_kernels"] = {k: {kk: vv for kk, vv in roof(k).items() if kk in ("achieved", "unit", "frac",
                                                                                      "launch_ms")}
                                 for k in cand if k != dom}

    # full reconstructions (Algorithm 6, 15 x 30) with the exact and the low-rank CG matrix
    recon = None
    if not args.no_recon and rank == 0:
        if args.form == "recompute":
            plan.set_recompute(0)  # the Gauss-Newton solve keeps cached time courses
        truth = torch.tensor(alpha_h, device="cuda")
        d, noise = noisy_data(torch, plan, truth, None)
        runs = [("plain", dict(hessian=0)), ("lowrank", dict(hessian=1))]
        if net is not None:
            runs.append(("surrogate", dict(hessian=1, surrogate_iters=10, surrogate=net)))
        recon = reconstruct(torch, plan, seq, ph, truth, d, None, runs, dict(rho_init_exact=1),
                            profile=args.profile_recon)
        if not args.no_precision:
            # the precision form's reconstruction: exact model, split-BF16 readout DFTs
            xplan = mr.Plan(seq, form=mr.MRSTAT_FORM_SPLIT_BF16)
            recon["split"] = reconstruct(torch, xplan, seq, ph, truth, d, None, [("split", dict(hessian=0))],
                                         dict(rho_init_exact=1))["split"]
            xplan.check()
            xplan.close()
            recon["split"]["equal_nrmse"] = all(
                abs(recon["split"][k] - recon["plain"][k]) <= max(0.1 * recon["plain"][k], 1e-3)
                for k in ("nrmse_t1", "nrmse_t2"))
        # B1 as the fifth unknown (a known map before): brain phantom with a smooth B1 field
        # in [0.8, 1.2], the same noise level, B1 started at 1 with the rho initialisation
        seq_b, ph_b = synth.config(args.workload, seed=rank, b1_map=True)
        truth_b = torch.tensor(np.concatenate([alpha_of(ph_b), ph_b.b1.ravel()[None].astype(np.float32)]),
                               device="cuda")
        bplan = mr.Plan(seq_b, estimate_b1=True)
        s_b = bplan.forward(truth_b)
        d_b = s_b + noise * (torch.linalg.vector_norm(s_b) / (30.0 * torch.linalg.vector_norm(noise)))
        sup_b = torch.tensor(ph_b.support.ravel(), device="cuda")
        a = torch.zeros((5, seq_b.nv), dtype=torch.float32, device="cuda")
        mask = torch.zeros(seq_b.nv, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = bplan.gn_solve(d_b, a, mask=mask, outer_iters=15, inner_iters=30, rho_init_exact=1,
                             mask_threshold=0.1)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        mb = mask.bool() & sup_b

        def nrmse_b(x, y):
            return float(torch.linalg.vector_norm((x - y)[mb]) / torch.linalg.vector_norm(y[mb]))
        recon["b1_estimated"] = {"seconds": secs, "nrmse_t1": nrmse_b(torch.exp(a[0]), torch.exp(truth_b[0])),
                                 "nrmse_t2": nrmse_b(torch.exp(a[1]), torch.exp(truth_b[1])),
                                 "nrmse_b1": nrmse_b(a[4], truth_b[4]), "f_final": rep["f_final"],
                                 "accepted": sum(rep["accepted"]), "cg_steps": sum(rep["cg_steps"]),
                                 "mask_voxels": rep["mask_voxels"],
                                 "settings": "B1 = 1 + 0.2 smooth field in [0.8, 1.2] estimated with T1, T2, rho; "
                                             "15 GN x 30 CG, SNR 30"}
        bplan.close()
        recon["settings"] = ("15 GN x 30 CG, SNR 30, rho the exact least-squares solution at T1 1000 ms / T2 100 ms, mask 0.1; "
                             "surrogate: 10 surrogate + 5 exact iterations, low-rank CG matrix")

    # the plain form's single products at 64 x 64 and 224 x 224
    products = None
    if not args.no_shapes and rank == 0 and world == 1:
        products = plain_products(mr, torch)

    # the differentiation form (autograd, with and without Bloch-state checkpoints)
    diff = None
    if not args.no_diff and rank == 0 and world == 1:
        diff = differentiation(mr, torch, seq, ph)

    # the learned-part form (surrogate trained on B1-varied samples, known smooth B1 map) at
    # 224 x 224 / 1120 TRs and 256 x 256 / 1280 TRs: step rates of the surrogate, the
    # compressed-exact and the plain model, and the three reconstructions
    learned = None
    if not args.no_learned and rank == 0 and world == 1:
        learned = {}
        for n in ("brain224", "brain256"):
            reuse = (basis, net, surrogate_info) if (n == args.workload and net is not None) else None
            learned[n] = learned_part(mr, torch, args, n, rank, iters, timed, reuse)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ntr_sample = 8
        t_lin, t_prod, scale = oracle_sample(args.workload, ntr_sample, 2)
        cpu = {"value": oracle_products_per_s(t_lin, t_prod, scale, iters), "unit": "products/s",
               "cores": cpu_cores(), "kind": "oracle",
               "sample": f"FP64 NumPy oracle, linearise + 2 J^H J v products on the first {ntr_sample} of {seq.ntr} "
                         f"TRs ({t_lin + 2 * t_prod:.1f} s), extrapolated linearly in TRs to linearise + "
                         f"{iters} products; elementwise NumPy single-threaded, BLAS on all cores"}
        if args.cpu_plan:
            cpu["plan"] = run_oracle_plan()
        if not args.no_fp64_errors and basis is not None:
            t0 = time.perf_counter()
            cpu["fp64_errors"] = fp64_errors(mr, torch, seq, ph, alpha_h, basis, net)
            cpu["fp64_errors"]["oracle_seconds"] = time.perf_counter() - t0

    launches = int(sum(stats[k]["kernels"] for k in stats))
    if args.form == "surrogate":
        # MLP inference per step: the first layer on the CUDA cores and three fused
        # tensor-core layers (outside the plan's counters)
        launches += 4 * args.steps
    if rank == 0:
        dft = ("factorised FP32 phase-encode DFT" if fft_y else "split-BF16 tcgen05 DFTs")
        form_desc = {"surrogate": f"learned surrogate + low-rank form (rank {R} time basis, MLP {args.hidden}x3 "
                                  f"tcgen05 coefficients, {dft}, per-ky Gram J^H J v)",
                     "lowrank": f"low-rank form (rank {R} time basis, {dft}, per-ky Gram J^H J v)",
                     "plain": "plain FP32 form (cached time courses, FP32 readout DFT)",
                     "recompute": f"plain FP32 form, recompute variant (Bloch recursion re-run in every product "
                                  f"from states every {args.segment} TRs, fused with the phase-encode sums)",
                     "split": "split-BF16 form (cached time courses, tcgen05 readout DFT)"}[args.form]
        l2 = ("inputs larger than L2 (cached time courses %.0f MB)" % (d_bytes / 1e6) if not lowrank_like
              else "L2 not flushed: the low-rank operands (~%.0f MB) are L2-resident by design; the "
                   "linearisation streams the parameters and writes the coefficients each step"
              % ((R * ny * 2 * nx * 2 * 2 + R * nkx * 2 * ny * 4 * 3) / 1e6))
        line = {"metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": ("f32 (MLP bf16)" if args.form == "surrogate" else "f32") if (not lowrank_like or fft_y)
                else "bf16x3+f32",
                "data": "synthetic",
                "config": {"workload": f"{args.workload}: {seq.nx}x{seq.ny} grid, {seq.ntr} TRs, "
                                       f"{seq.nkx} readout samples, " + form_desc,
                           "form": args.form, "step": f"linearize + {iters} CG iterations (one J^H J v each)",
                           "cg_iters": iters, "l2": l2, "parallelism": f"replicas{world}"},
                "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "cpu_baseline": cpu, "cg_check": cg_check, "compressed_exact": compressed_exact, "plain": plain,
                "precision": precision,
                "speedup_vs_plain": (value / plain["value"]) if plain else None,
                "recon": recon, "learned_part": learned, "differentiation": diff, "plain_products": products,
                "surrogate": surrogate_info, "shapes": shapes, "slice_profile": slice_prof,
                "kernel_ms_per_step": {k: v for k, v in per_step_ms.items()}}
        print(json.dumps(line), flush=True)
    if net is not None:
        net.close()
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
