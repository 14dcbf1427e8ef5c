"""Slice-profile Bloch model on the GPU (mrstat_set_slice_profile) against the oracle's
slice-averaged recursion (oracle/slice_profile.py).

The GPU composes each (TR, isochromat) pulse into a 3 x 3 matrix in float32 before
applying it; the oracle plays every sub-step in float64.  Bars as for the hard-pulse
products: 1e-5 normwise per output (and per parameter row of the gradients); the
Gauss-Newton step as in test_gpu_gn.py.
"""
import numpy as np
import pytest

import synth
from oracle import model, metrics, slice_profile as sp, solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def mr():
    import paper_1904_13244_gb300 as mr
    from paper_1904_13244_gb300 import build
    build.build()
    return mr


def cuda(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def random_alpha(nv, seed):
    rng = np.random.default_rng(seed)
    t1 = np.exp(rng.uniform(np.log(200), np.log(3000), nv))
    t2 = np.exp(rng.uniform(np.log(20), np.log(300), nv))
    rho = rng.uniform(0.5, 1.0, nv) * np.exp(1j * rng.uniform(0, 2 * np.pi, nv))
    return f32(np.stack([np.log(t1), np.log(t2), rho.real, rho.imag]))


CASES = {
    # name: (nx, ny, fills, extra_trs, nkx, train, SliceProfile)
    "square_32iso": (12, 16, 3, 0, 12, "smooth", sp.SliceProfile(n_iso=32, n_sub=16)),
    "ragged_8iso": (20, 12, 2, 5, 24, "sine2", sp.SliceProfile(n_iso=8, n_sub=12, sigma=0.25, tbw=3.0, extent=2.5)),
    "one_iso_constant": (9, 7, 3, 2, 9, "constant", sp.SliceProfile(n_iso=1, n_sub=4)),
    "two_iso_one_sub": (16, 8, 2, 1, 16, "smooth", sp.SliceProfile(n_iso=2, n_sub=1, tbw=2.0)),
}


def set_profile(plan, p):
    plan.set_slice_profile(p.n_iso, p.n_sub, p.sigma, p.tbw, p.extent)


@pytest.mark.parametrize("name", list(CASES))
def test_slice_products_match_oracle(mr, name):
    nx, ny, fills, extra, nkx, train, prof = CASES[name]
    seq = synth.make_sequence(nx, ny, fills, 7.8, 3.9, seed=3, nkx=nkx, extra_trs=extra, train=train)
    alpha = random_alpha(seq.nv, 4)
    mask = np.random.default_rng(5).random(seq.nv) > 0.15
    lin = model.linearize(seq, alpha, mask=mask, profile=prof)
    v = synth.random_params(seq.nv, 11)
    w = synth.random_kspace(seq.ntr, seq.nkx, 12)
    with mr.Plan(seq) as plan:
        set_profile(plan, prof)
        a = cuda(alpha)
        mk = cuda(mask.astype(np.uint8), torch.uint8)
        plan.linearize(a, mask=mk)
        tcs = [plan.timecourses(c).cpu().numpy() for c in range(3)]
        s = plan.forward(a, mask=mk).cpu().numpy()
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        h = plan.jhjv(cuda(v)).cpu().numpy()
    for c, ref in enumerate([lin.m, lin.dm1, lin.dm2]):
        assert metrics.relerr(tcs[c][:, mask], ref.imag[:, mask]) < TOL, c
        assert np.all(tcs[c][:, ~mask] == 0)
    assert metrics.relerr(s, model.signal(lin)) < TOL
    assert metrics.relerr(jv, model.jvp(lin, v)) < TOL
    gref, href = model.jhw(lin, w), model.gauss_newton_product(lin, v)
    for k in range(4):
        assert metrics.relerr(g[k], gref[k]) < TOL, k
        assert metrics.relerr(h[k], href[k]) < TOL, k


def test_hard_pulses_restored_and_one_isochromat_matches_them(mr):
    seq = synth.make_sequence(10, 8, 3, 7.8, 3.9, seed=6)
    a = cuda(random_alpha(seq.nv, 7))
    with mr.Plan(seq) as plan:
        plan.linearize(a)
        hard = plan.timecourses(0).cpu().numpy()
        plan.set_slice_profile(1, 8)
        plan.linearize(a)
        one = plan.timecourses(0).cpu().numpy()
        plan.set_slice_profile(16, 8)
        plan.linearize(a)
        sixteen = plan.timecourses(0).cpu().numpy()
        plan.set_slice_profile(None)
        plan.linearize(a)
        back = plan.timecourses(0).cpu().numpy()
    assert metrics.relerr(one, hard) < 2e-6
    assert metrics.relerr(sixteen, hard) > 1e-2
    assert np.array_equal(back, hard)


def test_slice_profile_rejects_what_it_does_not_cover(mr):
    seq = synth.make_sequence(16, 16, 2, 7.8, 3.9, seed=0)
    with mr.Plan(seq) as plan:
        with pytest.raises(mr.MrstatError) as e:
            plan.set_slice_profile(3, 8)
        assert e.value.status == 1
        with pytest.raises(mr.MrstatError) as e:
            plan.set_slice_profile(8, 65)
        assert e.value.status == 1
        plan.set_slice_profile(8, 8)
        a = cuda(random_alpha(seq.nv, 1))
        with pytest.raises(mr.MrstatError) as e:
            plan.linearize(a, b1=cuda(np.ones(seq.nv)))
        assert e.value.status == 7
        with pytest.raises(mr.MrstatError) as e:
            plan.lowrank_set_basis(cuda(np.eye(seq.ntr, 8)))
        assert e.value.status == 7
        with pytest.raises(mr.MrstatError) as e:
            plan.forward_ckpt(a)
        assert e.value.status == 7
        d = cuda(np.zeros((seq.ntr, seq.nkx)), torch.complex64)
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(d, a.clone(), outer_iters=1, hessian=1)
        assert e.value.status == 7
    with mr.Plan(seq, estimate_b1=True) as plan:
        with pytest.raises(mr.MrstatError) as e:
            plan.set_slice_profile(8, 8)
        assert e.value.status == 7


def test_first_gauss_newton_iteration_with_slice_profile(mr):
    seq = synth.make_sequence(12, 12, 4, 7.8, 3.9, seed=8)
    prof = sp.SliceProfile(n_iso=16, n_sub=8)
    truth = random_alpha(seq.nv, 9)
    d = synth.add_noise(model.forward(seq, truth, profile=prof), 50.0, 3).astype(np.complex64).astype(np.complex128)
    a0 = f32(truth + 0.05 * synth.random_params(seq.nv, 4))
    opts = solver.GNOptions(outer_iters=1, inner_iters=8)
    a_ref, rep_ref = solver.gauss_newton(seq, d, a0, opts=opts, profile=prof)
    with mr.Plan(seq) as plan:
        set_profile(plan, prof)
        a = cuda(a0)
        rep = plan.gn_solve(cuda(d, torch.complex64), a, outer_iters=1, inner_iters=8)
        a_gpu = a.cpu().numpy()
    assert abs(rep["f"][0] - rep_ref.f[0]) / rep_ref.f[0] < 1e-5
    assert abs(rep["gnorm"][0] - rep_ref.gnorm[0]) / rep_ref.gnorm[0] < 1e-5
    assert rep["cg_exit"][0] == rep_ref.exit[0]
    assert rep["cg_steps"][0] == rep_ref.cg_steps[0]
    assert rep["accepted"][0] == rep_ref.accepted[0]
    assert metrics.relerr(a_gpu - a0, a_ref - a0) < 1e-3


def test_full_size_slice_profile_sampled_voxels(mr):
    """224 x 224, 1120 TRs, 32 isochromats x 16 sub-steps: the time courses of sampled
    voxels against the oracle."""
    seq, ph = synth.config("brain224")
    alpha = f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                          ph.rho.imag.ravel()]))
    vox = np.sort(np.random.default_rng(21).choice(seq.nv, 12, replace=False))
    prof = sp.SliceProfile()
    with mr.Plan(seq) as plan:
        set_profile(plan, prof)
        plan.linearize(cuda(alpha))
        idx = torch.tensor(vox, device="cuda")
        tcs = [plan.timecourses(c)[:, idx].cpu().numpy() for c in range(3)]
    ref = sp.simulate(seq, np.exp(alpha[0, vox]), np.exp(alpha[1, vox]), prof)
    for c, key in enumerate(["m", "dm_dlnT1", "dm_dlnT2"]):
        assert metrics.relerr(tcs[c], ref[key].imag) < TOL, key
