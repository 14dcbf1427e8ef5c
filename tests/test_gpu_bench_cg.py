"""The timed fixed-count CG of the benchmark (30 iterations of the persistent launch on the
low-rank Re(J^H J), Eq. 4) against the FP64 oracle.

The benchmark step solves on the 224-row brain workload with 1120 TRs (five per
phase-encode line) and a rank-32 basis: the shared-memory layout of three 256-thread
blocks per SM.  With a fully sampled readout J^H J is block diagonal in the image columns,
so a few columns of the same workload (nx = nkx = 8, same rows, TRs, flips and basis rank)
run the same kernel instantiation and layout on a problem the oracle solves in seconds.
The persistent launch carries w = B r by the pipelined recurrences (Ghysels and Vanroose
2014), which in exact arithmetic are textbook CG; in float32 they can drift from the true
residual, so after 30 iterations the test checks

* x against textbook CG in float64 on the oracle's projected model,
* x against CG launched product by product through mrstat_jhjv with float64 scalars,
* the true residual ||b - B x|| of the GPU x (B the oracle's) against the recursive
  residual of float64 CG,
* that every iteration was applied (mrstat_cg_applied).

At the full 224 x 224 size the same launch is compared with the product-by-product CG,
and its true residual is checked on sampled image columns: with nkx = nx the readout DFT
pair cancels (F^H F = nx I), so B restricted to column ix is nx times the one-column
oracle operator.
"""
import numpy as np
import pytest

import synth
from oracle import metrics, model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ITERS = 30
RANK = 32


@pytest.fixture(scope="module")
def mr():
    import paper_1904_13244_gb300 as mr
    from paper_1904_13244_gb300 import build
    build.build()
    return mr


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def cuda(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def columns(seq, ph, cols):
    """The image columns `cols` of a workload as a workload of their own (same rows, TRs,
    flips and phase-encode order; nkx = the number of columns)."""
    nx = len(cols)
    sub = synth.Sequence(nx=nx, ny=seq.ny, nkx=nx, tr_ms=seq.tr_ms, te_ms=seq.te_ms, flip_rad=seq.flip_rad,
                         ky=seq.ky, inversion=seq.inversion, alternate_phase=seq.alternate_phase)
    alpha = np.stack([np.log(ph.t1_ms[:, cols].ravel()), np.log(ph.t2_ms[:, cols].ravel()),
                      ph.rho[:, cols].real.ravel(), ph.rho[:, cols].imag.ravel()])
    return sub, f32(alpha)


def basis(seq):
    rng = np.random.default_rng(1000)
    tr = f32(np.stack([rng.uniform(np.log(100), np.log(6000), 1000), rng.uniform(np.log(10), np.log(3000), 1000)]))
    return f32(model.time_basis(seq, np.exp(tr[0]), np.exp(tr[1]), RANK)[0])


def textbook_cg(apply_B, b, iters):
    """Textbook CG from x = 0 in float64; returns x and the recursive residual norms."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    norms = [np.sqrt(rr)]
    for _ in range(iters):
        q = apply_B(p)
        a = rr / float(np.sum(p * q))
        x = x + a * p
        r = r - a * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        norms.append(np.sqrt(rr))
    return x, np.array(norms)


def jhjv_cg(plan, b_dev, iters):
    """CG through mrstat_jhjv, one product launch per iteration, vectors and scalars in
    float64 (test code: the product is the library's, the recurrences torch's)."""
    x = torch.zeros_like(b_dev, dtype=torch.float64)
    r = b_dev.double().clone()
    p = r.clone()
    rr = float(torch.sum(r * r))
    for _ in range(iters):
        q = plan.jhjv(p.float()).double()
        a = rr / float(torch.sum(p * q))
        x += a * p
        r -= a * q
        rr_new = float(torch.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def test_bench_cg_on_a_few_columns_matches_oracle(mr):
    seq, ph = synth.config("brain224")
    sub, alpha = columns(seq, ph, list(range(108, 116)))
    U = basis(sub)
    exact = model.linearize(sub, alpha)
    lin = model.project_onto_basis(exact, U)
    # the bench's right-hand side: Re(J^H w) of the exact model for a seeded k-space w,
    # unit RMS (a consistent system: rho = 0 voxels' ln T1 / ln T2 rows are in the null space)
    g = model.jhw(exact, synth.random_kspace(sub.ntr, sub.nkx, 100))
    b = f32(g / np.sqrt(np.mean(g * g)))
    x_ref, norms = textbook_cg(lambda v: model.gauss_newton_product(lin, v), b, ITERS)
    with mr.Plan(sub) as plan:
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha))
        b_dev = cuda(b)
        plan.profile_start(kernels=("jhw_dot",))
        x_gpu = plan.cg_fixed(b_dev, ITERS)
        prof = plan.profile_stop()
        plan.check()
        applied = plan.cg_applied()
        x_lpi = jhjv_cg(plan, b_dev, ITERS).cpu().numpy()
        x_gpu = x_gpu.cpu().numpy().astype(np.float64)
    assert prof["jhw_dot"]["launches"] == ITERS  # counted as ITERS products ...
    assert prof["jhw_dot"]["kernels"] == 1       # ... made by one persistent launch
    assert applied == ITERS
    e_ref = metrics.relerr(x_gpu, x_ref)
    e_lpi = metrics.relerr(x_gpu, x_lpi)
    true_res = np.linalg.norm(b - model.gauss_newton_product(lin, x_gpu))
    ref_res = np.linalg.norm(b - model.gauss_newton_product(lin, x_ref))
    nb = np.linalg.norm(b)
    msg = (f"relerr vs float64 CG {e_ref:.2e}, vs product-by-product CG {e_lpi:.2e}; true residual "
           f"{true_res / nb:.3e}, float64 CG recursive {norms[-1] / nb:.3e} true {ref_res / nb:.3e}")
    print(msg)
    assert e_ref < 2e-3, msg
    assert e_lpi < 2e-3, msg
    # float64 CG's recursive and true residuals agree: the reference itself is sound
    assert abs(ref_res - norms[-1]) < 1e-6 * nb, msg
    # the pipelined float32 recurrences reach the residual exact CG reaches
    assert true_res < 1.2 * norms[-1] + 2e-5 * nb, msg


def test_bench_cg_full_size(mr):
    """The benchmark's launch itself (224 x 224, 448 blocks): against the product-by-product
    CG, and its true residual on sampled image columns through the one-column oracle."""
    seq, ph = synth.config("brain224")
    alpha = f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                          ph.rho.imag.ravel()]))
    U = basis(seq)
    with mr.Plan(seq) as plan:
        plan.linearize(cuda(alpha))
        g = plan.jhw(cuda(synth.random_kspace(seq.ntr, seq.nkx, 100), torch.complex64))
        b_dev = (g / torch.sqrt(torch.mean(g * g))).contiguous()
        b = b_dev.cpu().numpy().astype(np.float64)
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha))
        x_gpu = plan.cg_fixed(b_dev, ITERS)
        plan.check()
        assert plan.cg_applied() == ITERS
        x_lpi = jhjv_cg(plan, b_dev, ITERS)
        bx_gpu = plan.jhjv(x_gpu).cpu().numpy().astype(np.float64)
        e_lpi = float(torch.linalg.vector_norm(x_gpu.double() - x_lpi) / torch.linalg.vector_norm(x_lpi))
        x_gpu = x_gpu.cpu().numpy().astype(np.float64)
        x_lpi = x_lpi.cpu().numpy()
    assert e_lpi < 2e-3, e_lpi
    # residual on sampled columns: B restricted to column ix is nx times the oracle operator
    # of that column alone (a one-column workload with a one-point readout)
    cols = [40, 111, 170]
    x3 = x_gpu.reshape(4, seq.ny, seq.nx)
    l3 = x_lpi.reshape(4, seq.ny, seq.nx)
    b3 = b.reshape(4, seq.ny, seq.nx)
    bx3 = bx_gpu.reshape(4, seq.ny, seq.nx)
    for ix in cols:
        sub, a1 = columns(seq, ph, [ix])
        lin = model.project_onto_basis(model.linearize(sub, a1), U)
        bx = seq.nx * model.gauss_newton_product(lin, x3[:, :, ix])
        # the GPU product of the GPU x on that column is the oracle's
        assert metrics.relerr(bx3[:, :, ix], bx) < 1e-4, ix
        # and the persistent launch's x leaves the residual the float64 recurrences leave
        # (background voxels have rho = 0, so part of b is in the null space of B and
        # stays in every residual)
        res = np.linalg.norm(b3[:, :, ix] - bx)
        res_lpi = np.linalg.norm(b3[:, :, ix] - seq.nx * model.gauss_newton_product(lin, l3[:, :, ix]))
        assert res < 1.2 * res_lpi + 1e-4 * np.linalg.norm(b3[:, :, ix]), (ix, res, res_lpi)


def test_two_columns_per_cluster_full_size(mr):
    """256 x 256 with 1280 TRs: one cluster per image column (512 blocks) does not fit at
    once, so the persistent launch gives each cluster two columns (ix and ix + 128; their
    CG vectors stay in shared memory, the products run one after the other).  One launch
    for all 30 products, against the product-by-product CG, and its residual on sampled
    columns of both kinds through the one-column oracle."""
    seq, ph = synth.config("brain256")
    alpha = f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                          ph.rho.imag.ravel()]))
    U = basis(seq)
    with mr.Plan(seq) as plan:
        plan.linearize(cuda(alpha))
        g = plan.jhw(cuda(synth.random_kspace(seq.ntr, seq.nkx, 101), torch.complex64))
        b_dev = (g / torch.sqrt(torch.mean(g * g))).contiguous()
        b = b_dev.cpu().numpy().astype(np.float64)
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha))
        plan.profile_start(kernels=("jhw_dot",))
        x_gpu = plan.cg_fixed(b_dev, ITERS)
        prof = plan.profile_stop()
        plan.check()
        assert plan.cg_applied() == ITERS
        x_lpi = jhjv_cg(plan, b_dev, ITERS)
        bx_gpu = plan.jhjv(x_gpu).cpu().numpy().astype(np.float64)
        e_lpi = float(torch.linalg.vector_norm(x_gpu.double() - x_lpi) / torch.linalg.vector_norm(x_lpi))
        x_gpu = x_gpu.cpu().numpy().astype(np.float64)
        x_lpi = x_lpi.cpu().numpy()
    assert prof["jhw_dot"]["kernels"] == 1 and prof["jhw_dot"]["launches"] == ITERS
    assert e_lpi < 2e-3, e_lpi
    x3 = x_gpu.reshape(4, seq.ny, seq.nx)
    l3 = x_lpi.reshape(4, seq.ny, seq.nx)
    b3 = b.reshape(4, seq.ny, seq.nx)
    bx3 = bx_gpu.reshape(4, seq.ny, seq.nx)
    for ix in (60, 190):  # a first and a second column of a cluster
        sub, a1 = columns(seq, ph, [ix])
        lin = model.project_onto_basis(model.linearize(sub, a1), U)
        bx = seq.nx * model.gauss_newton_product(lin, x3[:, :, ix])
        assert metrics.relerr(bx3[:, :, ix], bx) < 1e-4, ix
        res = np.linalg.norm(b3[:, :, ix] - bx)
        res_lpi = np.linalg.norm(b3[:, :, ix] - seq.nx * model.gauss_newton_product(lin, l3[:, :, ix]))
        assert res < 1.2 * res_lpi + 1e-4 * np.linalg.norm(b3[:, :, ix]), (ix, res, res_lpi)
