"""Pins of the oracle's solver pieces: Steihaug CG against direct solves and the
trust-region geometry, CGLS against the exact rho, and Gauss-Newton against
quadratic local convergence and noiseless recovery of ground-truth maps."""
import numpy as np
import pytest

import synth
from oracle import model, solver, metrics


def _spd(n, seed, cond=100.0):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (q * np.geomspace(1, cond, n)) @ q.T


def test_steihaug_interior_solution_equals_direct_solve():
    B = _spd(12, 0)
    g = np.random.default_rng(1).standard_normal(12)
    p, mval, it, why = solver.steihaug_cg(lambda v: B @ v, g, 1e9, 100, rel_tol=1e-13)
    ref = np.linalg.solve(B, -g)
    assert np.allclose(p, ref, rtol=1e-9)
    assert np.isclose(mval, g @ ref + 0.5 * ref @ B @ ref, rtol=1e-9)
    assert why == "converged"


def test_steihaug_stops_on_the_trust_boundary():
    B = _spd(12, 2)
    g = np.random.default_rng(3).standard_normal(12)
    p, mval, it, why = solver.steihaug_cg(lambda v: B @ v, g, 0.05, 100)
    assert why == "boundary"
    assert np.isclose(np.linalg.norm(p), 0.05, rtol=1e-12)
    assert np.isclose(mval, g @ p + 0.5 * p @ B @ p, rtol=1e-10)
    assert mval < 0


def test_steihaug_negative_curvature_goes_to_the_boundary():
    B = np.diag([1.0, -2.0, 3.0])
    g = np.array([0.0, 1.0, 0.0])
    p, mval, it, why = solver.steihaug_cg(lambda v: B @ v, g, 2.0, 10)
    assert why == "negative_curvature"
    assert np.isclose(np.linalg.norm(p), 2.0)
    assert np.isclose(mval, g @ p + 0.5 * p @ B @ p)


def test_cgls_recovers_rho_at_the_true_relaxation_times():
    seq, ph = synth.config("quad16")
    alpha = np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel()])
    lin = model.linearize(seq, alpha)
    d = model.signal(lin)
    rho = solver.cgls_rho(lin, d, iters=60)
    assert metrics.nrmse(rho, ph.rho.ravel()) < 1e-8


def test_ls_rho_recovers_rho_at_the_true_relaxation_times():
    seq, ph = synth.config("quad16")
    alpha = np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel()])
    lin = model.linearize(seq, alpha)
    rho = solver.ls_rho(lin, model.signal(lin))
    assert metrics.nrmse(rho, ph.rho.ravel()) < 1e-10


def _initial_lin(seq):
    a0 = np.zeros((4, seq.nv))
    a0[0], a0[1] = np.log(1000.0), np.log(100.0)
    return model.linearize(seq, a0)


def test_ls_rho_solves_the_normal_equations_and_matches_converged_cgls():
    """At the paper's initial guess (uniform T1 = 1000 ms, T2 = 100 ms) and arbitrary
    data on a ragged grid (Ny = 12, extra TRs): the residual is orthogonal to the range
    of M, checked through the oracle's adjoint (encode_adjoint, not the dense M), and
    CGLS reaches the same rho.  With uniform relaxation times M^H M has one eigenvalue
    per sampled ky, so CGLS converges in at most Ny steps; 20 steps, not many more
    (past convergence the tiny residual only feeds rounding)."""
    seq = synth.make_sequence(16, 12, 3, 7.8, 3.9, seed=1, extra_trs=5)
    lin = _initial_lin(seq)
    d = synth.random_kspace(seq.ntr, seq.nkx, 3)
    rho = solver.ls_rho(lin, d)
    v = np.zeros((4, seq.nv))
    v[2], v[3] = rho.real, rho.imag
    g = model.jhw(lin, d - model.jvp(lin, v))[2:4]
    assert np.linalg.norm(g) < 1e-9 * np.linalg.norm(model.jhw(lin, d)[2:4])
    assert metrics.relerr(solver.cgls_rho(lin, d, iters=20), rho) < 1e-8


def test_ls_rho_is_minimum_norm_when_a_phase_encode_line_is_never_sampled():
    """With ky = 2 dropped from the sequence that component of rho is unobservable; the
    least-squares solution of minimum norm has none of it (E_2 rho = 0)."""
    full = synth.make_sequence(8, 8, 2, 7.8, 3.9, seed=2)
    keep = np.asarray(full.ky) != 2
    seq = synth.Sequence(nx=8, ny=8, nkx=8, tr_ms=full.tr_ms, te_ms=full.te_ms,
                         flip_rad=np.asarray(full.flip_rad)[keep], ky=np.asarray(full.ky)[keep],
                         inversion=full.inversion, alternate_phase=full.alternate_phase)
    lin = _initial_lin(seq)
    d = synth.random_kspace(seq.ntr, seq.nkx, 4)
    rho = solver.ls_rho(lin, d)
    from oracle import encoding
    assert np.linalg.norm(encoding.phase_matrix(seq, 2) @ rho) < 1e-9 * np.linalg.norm(rho)
    assert np.linalg.norm(encoding.phase_matrix(seq, 1) @ rho) > 1e-3 * np.linalg.norm(rho)


def test_gauss_newton_converges_quadratically_near_the_solution():
    seq, ph = synth.config("quad16")
    truth = np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel()])
    d = model.forward(seq, truth)
    a1 = truth + 0.1 * synth.random_params(seq.nv, 5)
    a, rep = solver.gauss_newton(seq, d, a1, opts=solver.GNOptions(outer_iters=6, inner_iters=40))
    assert all(np.diff(rep.f) < 0)
    assert rep.f_final < 1e-12 * rep.f[0]
    assert metrics.nrmse(np.exp(a[0]), ph.t1_ms.ravel()) < 1e-7


@pytest.mark.slow
@pytest.mark.parametrize("seed", [0, 2])
def test_noiseless_recovery_from_the_papers_initial_guess(seed):
    """Start at T1 = 1000 ms, T2 = 100 ms with CGLS rho and a drawn mask (Methods) on a
    16x16 four-region phantom scanned with 24 fills (384 TRs, 3 s)."""
    seq = synth.make_sequence(16, 16, 24, 7.8, 3.9, seed=seed)
    ph = synth.quadrant_phantom(16, seed)
    truth = np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel()])
    d = model.forward(seq, truth)
    a0, mask = solver.initial_alpha(seq, d, seq.nv)
    a, rep = solver.gauss_newton(seq, d, a0, mask=mask, opts=solver.GNOptions(outer_iters=10, inner_iters=20))
    assert rep.f_final < 1e-6 * rep.f[0]
    assert metrics.nrmse(np.exp(a[0]), ph.t1_ms.ravel()) < 1e-3
    assert metrics.nrmse(np.exp(a[1]), ph.t2_ms.ravel()) < 1e-3
    assert metrics.nrmse(a[2] + 1j * a[3], ph.rho.ravel()) < 1e-3


def test_noisy_fit_reaches_the_noise_floor():
    """With SNR 50 noise the final objective sits at about 1/2 ||noise||^2 (Results)."""
    seq = synth.make_sequence(16, 16, 24, 7.8, 3.9, seed=0)
    ph = synth.quadrant_phantom(16, 0)
    truth = np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel()])
    s = model.forward(seq, truth)
    d = synth.add_noise(s, 50.0, 9)
    floor = 0.5 * np.linalg.norm(d - s) ** 2
    a, rep = solver.gauss_newton(seq, d, truth, opts=solver.GNOptions(outer_iters=4, inner_iters=30))
    # the fit absorbs about N of the 2 Nt real noise components: f_final ~ floor * (1 - N / (2 Nt))
    expected = floor * (1 - truth.size / (2 * d.size))
    assert 0.8 * expected < rep.f_final < 1.05 * floor


@pytest.mark.slow
def test_noiseless_recovery_with_b1_estimated():
    """B1 as the fifth unknown (Methods, "Reconstructions"): from T1 = 1000 ms, T2 = 100 ms,
    B1 = 1 and the CGLS rho, the fit recovers a smooth B1 field in [0.8, 1.2] with the
    tissue maps on the 16x16 phantom scanned with 24 fills."""
    seq = synth.make_sequence(16, 16, 24, 7.8, 3.9, seed=0)
    ph = synth.quadrant_phantom(16, 0)
    b1 = synth.smooth_b1(16, 16, 3).ravel()
    truth = np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel(),
                      b1])
    d = model.forward(seq, truth)
    a0, mask = solver.initial_alpha(seq, d, seq.nv, estimate_b1=True)
    assert a0.shape[0] == 5 and np.all(a0[4] == 1.0)
    # B1 and T1 are partly confounded, so the Gauss-Newton systems are worse conditioned
    # than with B1 known: 60 CG steps per outer iteration instead of 20
    a, rep = solver.gauss_newton(seq, d, a0, mask=mask, opts=solver.GNOptions(outer_iters=15, inner_iters=60))
    assert rep.f_final < 1e-10 * rep.f[0]
    assert metrics.nrmse(np.exp(a[0]), ph.t1_ms.ravel()) < 1e-5
    assert metrics.nrmse(np.exp(a[1]), ph.t2_ms.ravel()) < 1e-5
    assert metrics.nrmse(a[4], b1) < 1e-5
