"""B1 as the fifth unknown (plans created with MRSTAT_ESTIMATE_B1) against the oracle.

The oracle linearises with alpha of 5 rows (ln T1, ln T2, Re rho, Im rho, B1) and carries
dm/dB1 (S2 derivative through the rotation angle); the GPU caches a fourth time-course
channel and every vector has 5 rows.  Bars as for the 4-parameter products: 1e-5
normwise per output and per parameter row; Gauss-Newton as in test_gpu_gn.py.
"""
import numpy as np
import pytest

import synth
from oracle import model, solver, metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def alpha5(nx, ny, seed):
    rng = np.random.default_rng(seed)
    t1 = np.exp(rng.uniform(np.log(200), np.log(3000), nx * ny))
    t2 = np.exp(rng.uniform(np.log(20), np.log(300), nx * ny))
    rho = rng.uniform(0.5, 1.0, nx * ny) * np.exp(1j * rng.uniform(0, 2 * np.pi, nx * ny))
    b1 = synth.smooth_b1(nx, ny, seed + 1).ravel()
    return f32(np.stack([np.log(t1), np.log(t2), rho.real, rho.imag, b1]))


CASES = {
    # name: (nx, ny, fills, extra_trs, nkx)
    "square_16": (16, 16, 4, 0, 16),
    "ragged_40x24": (40, 24, 3, 5, 48),
    "odd_33x7": (33, 7, 2, 3, 33),
}


@pytest.mark.parametrize("name", list(CASES))
def test_products_with_b1_match_oracle(mr, name):
    nx, ny, fills, extra, nkx = CASES[name]
    seq = synth.make_sequence(nx, ny, fills, 7.8, 3.9, seed=2, nkx=nkx, extra_trs=extra)
    alpha = alpha5(nx, ny, 5)
    mask = np.random.default_rng(3).random(seq.nv) > 0.2
    lin = model.linearize(seq, alpha, mask=mask)
    v = synth.random_params(seq.nv, 11, 5)
    w = synth.random_kspace(seq.ntr, seq.nkx, 12)
    with mr.Plan(seq, estimate_b1=True) as plan:
        assert plan.info()["npar"] == 5
        a = cuda(alpha)
        mk = cuda(mask.astype(np.uint8), torch.uint8)
        plan.linearize(a, mask=mk)
        tcs = [plan.timecourses(c).cpu().numpy() for c in range(4)]
        s = plan.forward(a, mask=mk).cpu().numpy()
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        h = plan.jhjv(cuda(v)).cpu().numpy()
    for c, ref in enumerate([lin.m, lin.dm1, lin.dm2, lin.dmb]):
        assert metrics.relerr(tcs[c][:, mask], ref.imag[:, mask]) < TOL, c
        assert np.all(tcs[c][:, ~mask] == 0)
    assert metrics.relerr(s, model.signal(lin)) < TOL
    assert metrics.relerr(jv, model.jvp(lin, v)) < TOL
    gref = model.jhw(lin, w)
    href = model.gauss_newton_product(lin, v)
    for k in range(5):
        assert metrics.relerr(g[k], gref[k]) < TOL, k
        assert metrics.relerr(h[k], href[k]) < TOL, k


def test_b1_plan_rejects_what_it_does_not_support(mr):
    seq = synth.make_sequence(16, 16, 2, 7.8, 3.9, seed=0)
    alpha = alpha5(16, 16, 1)
    with mr.Plan(seq, estimate_b1=True) as plan:
        with pytest.raises(mr.MrstatError) as e:
            plan.linearize(cuda(alpha), b1=cuda(np.ones(seq.nv)))
        assert e.value.status == 1
        with pytest.raises(mr.MrstatError) as e:
            plan.lowrank_set_basis(cuda(np.eye(seq.ntr, 8)))
        assert e.value.status == 7
        d = cuda(np.zeros((seq.ntr, seq.nkx)), torch.complex64)
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(d, cuda(alpha), outer_iters=1, hessian=1)
        assert e.value.status == 7
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(d, cuda(alpha), outer_iters=1, b1_min=1.2, b1_max=1.1)
        assert e.value.status == 1


def _noisy_b1_quad():
    seq = synth.make_sequence(16, 16, 6, 7.8, 3.9, seed=4)
    ph = synth.quadrant_phantom(16, 4)
    b1 = synth.smooth_b1(16, 16, 6).ravel()
    truth = f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                          ph.rho.imag.ravel(), b1]))
    d = synth.add_noise(model.forward(seq, truth), 50.0, 3).astype(np.complex64).astype(np.complex128)
    a0 = truth + 0.05 * synth.random_params(seq.nv, 4, 5)
    a0[4] = np.clip(a0[4], 0.6, 1.4)
    return seq, truth, d, f32(a0)


def test_first_outer_iteration_with_b1_matches_oracle(mr):
    seq, truth, d, a0 = _noisy_b1_quad()
    opts = solver.GNOptions(outer_iters=1, inner_iters=10)
    a_ref, rep_ref = solver.gauss_newton(seq, d, a0, opts=opts)
    with mr.Plan(seq, estimate_b1=True) as plan:
        a = cuda(a0)
        rep = plan.gn_solve(cuda(d, torch.complex64), a, outer_iters=1, inner_iters=10)
        a_gpu = a.cpu().numpy()
    assert abs(rep["f"][0] - rep_ref.f[0]) / rep_ref.f[0] < 1e-5
    assert abs(rep["gnorm"][0] - rep_ref.gnorm[0]) / rep_ref.gnorm[0] < 1e-5
    assert rep["cg_exit"][0] == rep_ref.exit[0]
    assert rep["cg_steps"][0] == rep_ref.cg_steps[0]
    assert rep["accepted"][0] == rep_ref.accepted[0]
    assert metrics.relerr(a_gpu - a0, a_ref - a0) < 1e-3


def test_noiseless_recovery_with_b1_estimated(mr):
    """As the oracle pin: B1 with the tissue maps from T1 = 1000 ms, T2 = 100 ms, B1 = 1
    and the CGLS rho on the 16x16 phantom scanned with 24 fills."""
    seq = synth.make_sequence(16, 16, 24, 7.8, 3.9, seed=0)
    ph = synth.quadrant_phantom(16, 0)
    b1 = synth.smooth_b1(16, 16, 3).ravel()
    truth = np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel(),
                      b1])
    d = model.forward(seq, truth)
    with mr.Plan(seq, estimate_b1=True) as plan:
        a = cuda(np.zeros((5, seq.nv)))
        mask = torch.zeros(seq.nv, dtype=torch.uint8, device="cuda")
        rep = plan.gn_solve(cuda(d, torch.complex64), a, mask=mask, outer_iters=15, inner_iters=60,
                            rho_init_iters=50, mask_threshold=0.1)
        a_gpu = a.cpu().numpy().astype(np.float64)
    assert rep["mask_voxels"] == seq.nv
    assert rep["f_final"] < 1e-6 * rep["f"][0]
    assert metrics.nrmse(np.exp(a_gpu[0]), ph.t1_ms.ravel()) < 1e-3
    assert metrics.nrmse(np.exp(a_gpu[1]), ph.t2_ms.ravel()) < 1e-3
    assert metrics.nrmse(a_gpu[4], b1) < 1e-3
