#!/usr/bin/env python
"""Benchmark of the MR-STAT hot path: J^H.J.v products per second.

One step = one pass of the inner Gauss-Newton solve (Algorithm 6) on a 224x224 grid
with 1120 TRs: linearise the Bloch model (all voxels, with tangents), then a fixed
number of CG iterations on Re(J^H J) x = b, each one J.v and one Re(J^H w) product
plus float64 inner products.  value = CG products per second summed over ranks.
Inputs are the seeded brain-like phantom and flip train of ``synth``; the cached
time courses (3 x 1120 x 50176 float32 = 674 MB) exceed the 126 MB L2, so every
product streams them from HBM.

Multi-GPU: N independent replicas (one per rank), weak scaling, no collective on
the data path; the timing takes the maximum over ranks.

``--impl reference`` times the FP64 oracle (the reference of this build) on the
host cores on a bounded sample of the same workload and extrapolates to the full
step; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
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
NCU_TRAFFIC = {}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="brain224")
    ap.add_argument("--cg-iters", type=int, default=30)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "cg_iters": args.cg_iters},
            "cpu_baseline": {"value": value, "unit": "products/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

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
# GPU arm
# ---------------------------------------------------------------------------
def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

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
    rhs_h = synth.random_params(seq.nv, 100 + rank).astype(np.float32)
    plan = mr.Plan(seq)
    a_dev = torch.tensor(alpha_h, device="cuda")
    rhs_dev = torch.tensor(rhs_h, device="cuda")
    x_dev = torch.empty_like(rhs_dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.linearize(a_dev)
        plan.cg_fixed(rhs_dev, iters, out=x_dev)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    plan.profile_start(("ycontract", "jhw_dot", "bloch"))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    stats = plan.profile_stop()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    if world > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    value = world * iters / (ms / 1e3)

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        a_host = torch.tensor(alpha_h).pin_memory()
        rhs_host = torch.tensor(rhs_h).pin_memory()
        x_host = torch.empty_like(rhs_host).pin_memory()
        k = max(1, min(args.steps, 50))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(k):
            a_dev.copy_(a_host, non_blocking=True)
            rhs_dev.copy_(rhs_host, non_blocking=True)
            step()
            x_host.copy_(x_dev, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        dt = (time.perf_counter() - t0) / k
        if world > 1:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": world * iters / dt, "unit": "products/s",
               "h2d_bytes_per_step": int(a_host.numel() * 4 + rhs_host.numel() * 4),
               "d2h_bytes_per_step": int(x_host.numel() * 4)}

    # roofline of the dominant kernel (HBM-bound streaming of the cached time courses)
    info = plan.info()
    nv, ntr_pad, nx, ny, ntr = info["nv"], info["ntr_padded"], info["nx"], info["ny"], info["ntr"]
    d_bytes = 3 * ntr_pad * nv * 4
    alg = {
        "jhw_dot": d_bytes + ntr_pad * nx * 8 + nv * (8 + 4 + 16) + ntr_pad * 4,
        "ycontract": d_bytes + nv * 24 + ntr * nx * 8 + ntr_pad * 4,
        "bloch": d_bytes + nv * 16,
    }
    src = {"jhw_dot": "encode.cu", "ycontract": "encode.cu", "bloch": "bloch.cu"}
    per_launch = {k: stats[k]["ms"] / max(stats[k]["timed"], 1) for k in alg}
    per_step_ms = {k: stats[k]["ms"] / max(args.steps, 1) for k in alg}
    dom = max(per_step_ms, key=per_step_ms.get)
    peak, peak_kind = measured_peak_hbm()
    achieved = alg[dom] / (per_launch[dom] / 1e3) / 1e9
    h = source_hash(os.path.join(ROOT, "paper_1904_13244_gb300", "csrc", src[dom]))
    traffic = NCU_TRAFFIC.get((dom, h))
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg[dom], "launch_ms": per_launch[dom],
                "other_kernels": {k: {"launch_ms": per_launch[k], "GB/s": alg[k] / (per_launch[k] / 1e3) / 1e9
                                      if per_launch[k] > 0 else None} for k in alg if k != dom}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ntr_sample = 8
        t_lin, t_prod, scale = oracle_sample(args.workload, ntr_sample, 2)
        cpu = {"value": oracle_products_per_s(t_lin, t_prod, scale, iters), "unit": "products/s",
               "cores": cpu_cores(), "kind": "oracle",
               "sample": f"FP64 NumPy oracle, linearise + 2 J^H J v products on the first {ntr_sample} of {seq.ntr} "
                         f"TRs ({t_lin + 2 * t_prod:.1f} s), extrapolated linearly in TRs to linearise + "
                         f"{iters} products; elementwise NumPy single-threaded, BLAS on all cores"}

    launches = int(sum(stats[k]["launches"] for k in stats))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "products/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": f"{args.workload}: {seq.nx}x{seq.ny} grid, {seq.ntr} TRs, "
                                       f"{seq.nkx} readout samples, plain FP32 form",
                           "form": "plain_fp32", "step": f"linearize + {iters} CG iterations (one J^H J v each)",
                           "cg_iters": iters, "l2": "inputs larger than L2 (cached time courses "
                                                    f"{d_bytes / 1e6:.0f} MB)",
                           "parallelism": f"replicas{world}"},
                "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "cpu_baseline": cpu,
                "kernel_ms_per_step": {k: v for k, v in per_step_ms.items()}}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
