"""GPU Gauss-Newton (mrstat_gn_solve) against the oracle's trust-region solver.

Both run Algorithm 6 with the same Steihaug truncated CG and trust-region rules; the
GPU keeps vectors in float32 and scalars in float64, so trajectories agree closely
at first and drift slowly.  Bars: objective and gradient norm at the start 1e-5
(single products), CG exit reasons and step counts equal, the first step 1e-3
(ten float32 CG iterations), objective history 1e-3 over four outer iterations,
noiseless recovery NRMSE < 1e-3.
"""
import numpy as np
import pytest

import synth
from oracle import model, solver, metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import paper_1904_13244_gb300 as mr
    from paper_1904_13244_gb300 import build
    build.build()
    return mr


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def truth_of(ph):
    return f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                         ph.rho.imag.ravel()]))


def cuda(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


@pytest.fixture(scope="module")
def noisy_quad():
    seq, ph = synth.config("quad16")
    truth = truth_of(ph)
    d = synth.add_noise(model.forward(seq, truth), 50.0, 3)
    d = d.astype(np.complex64).astype(np.complex128)
    a0 = f32(truth + 0.05 * synth.random_params(seq.nv, 4))
    return seq, ph, truth, d, a0


def test_first_outer_iteration_matches_oracle(mr, noisy_quad):
    seq, ph, truth, d, a0 = noisy_quad
    opts = solver.GNOptions(outer_iters=1, inner_iters=10)
    a_ref, rep_ref = solver.gauss_newton(seq, d, a0, opts=opts)
    with mr.Plan(seq) as plan:
        a = cuda(a0)
        rep = plan.gn_solve(cuda(d, torch.complex64), a, outer_iters=1, inner_iters=10)
        a_gpu = a.cpu().numpy()
    assert abs(rep["f"][0] - rep_ref.f[0]) / rep_ref.f[0] < 1e-5
    assert abs(rep["gnorm"][0] - rep_ref.gnorm[0]) / rep_ref.gnorm[0] < 1e-5
    assert rep["cg_exit"][0] == rep_ref.exit[0]
    assert rep["cg_steps"][0] == rep_ref.cg_steps[0]
    assert abs(rep["delta"][0] - rep_ref.delta[0]) / rep_ref.delta[0] < 1e-6
    assert rep["accepted"][0] == rep_ref.accepted[0]
    assert metrics.relerr(a_gpu - a0, a_ref - a0) < 1e-3


def test_objective_history_matches_oracle(mr, noisy_quad):
    seq, ph, truth, d, a0 = noisy_quad
    opts = solver.GNOptions(outer_iters=4, inner_iters=20)
    a_ref, rep_ref = solver.gauss_newton(seq, d, a0, opts=opts)
    with mr.Plan(seq) as plan:
        a = cuda(a0)
        rep = plan.gn_solve(cuda(d, torch.complex64), a, outer_iters=4, inner_iters=20)
    assert rep["accepted"] == rep_ref.accepted
    assert np.allclose(rep["f"], rep_ref.f, rtol=1e-3)
    assert abs(rep["f_final"] - rep_ref.f_final) / rep_ref.f_final < 1e-3


def test_rho_initialisation_and_mask_match_oracle(mr):
    seq, ph = synth.config("ellipse64")
    truth = truth_of(ph)
    d = model.forward(seq, truth).astype(np.complex64).astype(np.complex128)
    a0_ref, mask_ref = solver.initial_alpha(seq, d, seq.nv, rho_iters=30)
    with mr.Plan(seq) as plan:
        a = cuda(np.zeros((4, seq.nv)))
        mask = torch.zeros(seq.nv, dtype=torch.uint8, device="cuda")
        rep = plan.gn_solve(cuda(d, torch.complex64), a, mask=mask, outer_iters=0, rho_init_iters=30,
                            mask_threshold=0.1)
        a_gpu = a.cpu().numpy()
        m_gpu = mask.cpu().numpy().astype(bool)
    # the masks may only differ where |rho| sits at the threshold
    rho_ref = a0_ref[2] + 1j * a0_ref[3]
    diff = m_gpu != mask_ref
    thr = 0.1 * np.abs(rho_ref).max()
    assert np.all(np.abs(np.abs(rho_ref[diff]) - thr) < 1e-3 * thr)
    assert rep["mask_voxels"] == int(m_gpu.sum())
    both = m_gpu & mask_ref
    assert metrics.relerr((a_gpu[2] + 1j * a_gpu[3])[both], rho_ref[both]) < 1e-4
    assert np.allclose(a_gpu[0], np.log(1000.0)) and np.allclose(a_gpu[1], np.log(100.0))


def _dropped_ky_sequence():
    full = synth.make_sequence(8, 8, 2, 7.8, 3.9, seed=2)
    keep = np.asarray(full.ky) != 2
    return synth.Sequence(nx=8, ny=8, nkx=8, tr_ms=full.tr_ms, te_ms=full.te_ms,
                          flip_rad=np.asarray(full.flip_rad)[keep], ky=np.asarray(full.ky)[keep],
                          inversion=full.inversion, alternate_phase=full.alternate_phase)


EXACT_RHO_CASES = {
    "quad16": lambda: synth.config("quad16")[0],
    "ragged_24x20": lambda: synth.make_sequence(24, 20, 2, 7.8, 3.9, seed=3, extra_trs=5),
    "one_ky_never_sampled": _dropped_ky_sequence,
    "ny_equals_ntr": lambda: synth.make_sequence(12, 12, 1, 7.8, 3.9, seed=4),
}


@pytest.mark.parametrize("name", list(EXACT_RHO_CASES))
def test_exact_rho_initialisation_matches_oracle_lstsq(mr, name):
    """rho_init_exact against the oracle's dense minimum-norm least squares at the paper's
    alpha_0 (T1 = 1000 ms, T2 = 100 ms), arbitrary data, no mask drawn."""
    seq = EXACT_RHO_CASES[name]()
    a0 = np.zeros((4, seq.nv))
    a0[0], a0[1] = np.log(1000.0), np.log(100.0)
    d = synth.random_kspace(seq.ntr, seq.nkx, 5).astype(np.complex64).astype(np.complex128)
    ref = solver.ls_rho(model.linearize(seq, a0), d)
    with mr.Plan(seq) as plan:
        a = cuda(np.zeros((4, seq.nv)))
        rep = plan.gn_solve(cuda(d, torch.complex64), a, outer_iters=0, rho_init_exact=1, mask_threshold=0.0)
        a_gpu = a.cpu().numpy().astype(np.float64)
    assert rep["mask_voxels"] == seq.nv
    assert metrics.relerr(a_gpu[2] + 1j * a_gpu[3], ref) < 1e-5
    assert np.allclose(a_gpu[0], np.log(1000.0)) and np.allclose(a_gpu[1], np.log(100.0))


def test_exact_rho_initialisation_and_mask_match_oracle(mr):
    seq, ph = synth.config("ellipse64")
    d = model.forward(seq, truth_of(ph)).astype(np.complex64).astype(np.complex128)
    a0 = np.zeros((4, seq.nv))
    a0[0], a0[1] = np.log(1000.0), np.log(100.0)
    lin0 = model.linearize(seq, a0)
    # the oracle's dense M is too large at 64 x 64: converged CGLS (one eigenvalue of M^H M
    # per sampled ky, so Ny steps reach the solution) stands in for lstsq here
    rho_ref = solver.cgls_rho(lin0, d, iters=seq.ny + 8)
    mask_ref = solver.draw_mask(rho_ref, 0.1)
    with mr.Plan(seq) as plan:
        a = cuda(np.zeros((4, seq.nv)))
        mask = torch.zeros(seq.nv, dtype=torch.uint8, device="cuda")
        rep = plan.gn_solve(cuda(d, torch.complex64), a, mask=mask, outer_iters=0, rho_init_exact=1,
                            mask_threshold=0.1)
        a_gpu = a.cpu().numpy()
        m_gpu = mask.cpu().numpy().astype(bool)
    diff = m_gpu != mask_ref
    thr = 0.1 * np.abs(rho_ref).max()
    assert np.all(np.abs(np.abs(rho_ref[diff]) - thr) < 1e-4 * thr)
    assert rep["mask_voxels"] == int(m_gpu.sum())
    both = m_gpu & mask_ref
    assert metrics.relerr((a_gpu[2] + 1j * a_gpu[3])[both], rho_ref[both]) < 1e-5


def test_exact_rho_initialisation_rejects_what_it_does_not_cover(mr):
    cases = [synth.make_sequence(16, 16, 2, 7.8, 3.9, seed=0, nkx=20),   # oversampled readout
             synth.make_sequence(16, 16, 0, 7.8, 3.9, seed=0, extra_trs=9)]  # fewer TRs than ky lines
    for seq in cases:
        with mr.Plan(seq) as plan:
            d = cuda(np.zeros((seq.ntr, seq.nkx)), torch.complex64)
            with pytest.raises(mr.MrstatError) as e:
                plan.gn_solve(d, cuda(np.zeros((4, seq.nv))), outer_iters=0, rho_init_exact=1, mask_threshold=0.0)
            assert e.value.status == 7
    seq = synth.make_sequence(16, 16, 2, 7.8, 3.9, seed=0)
    with mr.Plan(seq) as plan:
        d = cuda(np.zeros((seq.ntr, seq.nkx)), torch.complex64)
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(d, cuda(np.zeros((4, seq.nv))), b1=cuda(np.ones(seq.nv)), outer_iters=0,
                          rho_init_exact=1, mask_threshold=0.0)
        assert e.value.status == 7


def test_exact_rho_initialisation_full_size_normal_equations(mr):
    """224 x 224, 1120 TRs: the exact rho satisfies the normal equations of the rho block
    (checked with the plan's own J^H, itself pinned to the oracle) and the 50-step CGLS
    of the same problem lands close to it."""
    seq, ph = synth.config("brain224")
    truth = truth_of(ph)
    a0 = np.zeros((4, seq.nv), np.float32)
    a0[0], a0[1] = np.log(1000.0), np.log(100.0)
    with mr.Plan(seq) as plan:
        d = plan.forward(cuda(truth))
        d = d + 0.01 * torch.linalg.vector_norm(d) / np.sqrt(d.numel()) * torch.randn_like(d)
        a = cuda(np.zeros((4, seq.nv)))
        plan.gn_solve(d, a, outer_iters=0, rho_init_exact=1, mask_threshold=0.0)
        a_cg = cuda(np.zeros((4, seq.nv)))
        plan.gn_solve(d, a_cg, outer_iters=0, rho_init_iters=50, mask_threshold=0.0)
        plan.linearize(a)
        r = d - plan.forward(a)
        g = plan.jhw(r)[2:4]
        g0 = plan.jhw(d)[2:4]
        rel = float(torch.linalg.vector_norm(g) / torch.linalg.vector_norm(g0))
        drift = float(torch.linalg.vector_norm(a_cg[2:4] - a[2:4]) / torch.linalg.vector_norm(a[2:4]))
    assert rel < 1e-4
    assert drift < 1e-2


@pytest.mark.parametrize("seed", [0, 2])
def test_noiseless_recovery_from_the_papers_initial_guess(mr, seed):
    seq = synth.make_sequence(16, 16, 24, 7.8, 3.9, seed=seed)
    ph = synth.quadrant_phantom(16, seed)
    truth = truth_of(ph)
    d = model.forward(seq, truth)
    with mr.Plan(seq) as plan:
        a = cuda(np.zeros((4, seq.nv)))
        mask = torch.zeros(seq.nv, dtype=torch.uint8, device="cuda")
        rep = plan.gn_solve(cuda(d, torch.complex64), a, mask=mask, outer_iters=10, inner_iters=20,
                            rho_init_iters=50, mask_threshold=0.1)
        a_gpu = a.cpu().numpy().astype(np.float64)
    assert rep["mask_voxels"] == seq.nv
    assert rep["f_final"] < 1e-5 * rep["f"][0]
    assert metrics.nrmse(np.exp(a_gpu[0]), ph.t1_ms.ravel()) < 1e-3
    assert metrics.nrmse(np.exp(a_gpu[1]), ph.t2_ms.ravel()) < 1e-3
    assert metrics.nrmse(a_gpu[2] + 1j * a_gpu[3], ph.rho.ravel()) < 1e-3


def test_plan_holds_the_final_linearisation(mr, noisy_quad):
    seq, ph, truth, d, a0 = noisy_quad
    with mr.Plan(seq) as plan:
        a = cuda(a0)
        plan.gn_solve(cuda(d, torch.complex64), a, outer_iters=2, inner_iters=5)
        lin = model.linearize(seq, a.cpu().numpy().astype(np.float64))
        tc = plan.timecourses(0).cpu().numpy()
    assert metrics.relerr(tc, lin.m.imag) < 1e-5


def test_invalid_options_are_rejected(mr, noisy_quad):
    seq, ph, truth, d, a0 = noisy_quad
    with mr.Plan(seq) as plan:
        for bad in [dict(outer_iters=-1), dict(outer_iters=65), dict(inner_iters=0),
                    dict(t1_min_ms=0.0), dict(t2_max_ms=1.0), dict(rho_init_iters=5, mask_threshold=0.1)]:
            with pytest.raises(mr.MrstatError) as e:
                plan.gn_solve(cuda(d, torch.complex64), cuda(a0), **bad)
            assert e.value.status == 1, bad


def _basis(plan, rank=16, n=1024, seed=3):
    rng = np.random.default_rng(seed)
    train = np.stack([rng.uniform(np.log(100), np.log(6000), n), rng.uniform(np.log(10), np.log(3000), n)])
    U, _ = plan.lowrank_basis(cuda(train), rank)
    return U


def test_lowrank_hessian_reaches_the_exact_minimiser(mr, noisy_quad):
    """Low-rank Gauss-Newton matrix in the CG, exact gradient and objective: the iteration
    converges to the same point as the exact-Hessian solve."""
    seq, ph, truth, d, a0 = noisy_quad
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(_basis(plan, 32))
        a_ex = cuda(a0)
        rep_ex = plan.gn_solve(cuda(d, torch.complex64), a_ex, outer_iters=12, inner_iters=20)
        a_lr = cuda(a0)
        rep_lr = plan.gn_solve(cuda(d, torch.complex64), a_lr, outer_iters=12, inner_iters=20, hessian=1)
        plan.check()
    assert abs(rep_lr["f_final"] - rep_ex["f_final"]) / rep_ex["f_final"] < 1e-3
    assert metrics.relerr(a_lr.cpu().numpy(), a_ex.cpu().numpy()) < 1e-2


def test_lowrank_hessian_noiseless_recovery(mr):
    seq = synth.make_sequence(16, 16, 24, 7.8, 3.9, seed=0)
    ph = synth.quadrant_phantom(16, 0)
    truth = truth_of(ph)
    d = model.forward(seq, truth)
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(_basis(plan, 32))
        a = cuda(np.zeros((4, seq.nv)))
        mask = torch.zeros(seq.nv, dtype=torch.uint8, device="cuda")
        rep = plan.gn_solve(cuda(d, torch.complex64), a, mask=mask, outer_iters=15, inner_iters=20,
                            rho_init_iters=50, mask_threshold=0.1, hessian=1)
        a_gpu = a.cpu().numpy().astype(np.float64)
    assert metrics.nrmse(np.exp(a_gpu[0]), ph.t1_ms.ravel()) < 1e-3
    assert metrics.nrmse(np.exp(a_gpu[1]), ph.t2_ms.ravel()) < 1e-3


def _trained_surrogate(mr, plan, rank, hidden=128, steps=2500, seed=0):
    """A surrogate fitted to the plan's projected Bloch model (exact sample projections)."""
    rng = np.random.default_rng(seed)
    n = 32768
    x = cuda(np.stack([rng.uniform(np.log(100), np.log(6000), n), rng.uniform(np.log(10), np.log(3000), n)]))
    tgt = plan.lowrank_project_samples(x)
    scale = tgt[0].abs().amax(dim=1).clamp_min(1e-6).cpu().numpy()
    net = mr.Surrogate(hidden, rank, (np.log(1000.0), 1.0, np.log(100.0), 1.2, 1.0, 0.2), 0.5, seed=seed)
    net.set_output_scale(scale)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    for it in range(steps):
        idx = torch.randint(0, n, (1024,), device="cuda", generator=gen)
        net.train_step(x[:, idx].contiguous(), tgt[:, :, idx].contiguous(), 3e-3 if it < 1800 else 1e-3)
    return net


def test_surrogate_phase_then_exact_reaches_the_exact_minimiser(mr, noisy_quad):
    """The first iterations on the learned surrogate's low-rank model, the rest exact: the
    solve ends at the exact-model solution, and the surrogate phase lowers the exact
    objective on its own."""
    seq, ph, truth, d, a0 = noisy_quad
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(_basis(plan, 16))
        net = _trained_surrogate(mr, plan, 16)
        a_ex = cuda(a0)
        rep_ex = plan.gn_solve(cuda(d, torch.complex64), a_ex, outer_iters=12, inner_iters=20)
        a_s = cuda(a0)
        rep_s = plan.gn_solve(cuda(d, torch.complex64), a_s, outer_iters=12, inner_iters=20, surrogate_iters=6,
                              surrogate=net)
        # objective of the point the surrogate phase alone reaches, under the exact model
        a_p = cuda(a0)
        plan.gn_solve(cuda(d, torch.complex64), a_p, outer_iters=6, inner_iters=20, surrogate_iters=6, surrogate=net)
        f_p = plan.gn_solve(cuda(d, torch.complex64), a_p.clone(), outer_iters=0)["f_final"]
        plan.check()
        net.close()
    assert rep_s["iterations"] == 12
    assert f_p < 0.5 * rep_ex["f"][0]
    assert abs(rep_s["f_final"] - rep_ex["f_final"]) / rep_ex["f_final"] < 1e-3
    assert metrics.relerr(a_s.cpu().numpy(), a_ex.cpu().numpy()) < 1e-2


def test_surrogate_options_are_checked(mr, noisy_quad):
    seq, ph, truth, d, a0 = noisy_quad
    with mr.Plan(seq) as plan:
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(cuda(d, torch.complex64), cuda(a0), outer_iters=2, surrogate_iters=1)
        assert e.value.status == 1
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(cuda(d, torch.complex64), cuda(a0), outer_iters=2, surrogate_iters=-1)
        assert e.value.status == 1
        with mr.Surrogate(64, 8, (7.0, 1.0, 4.5, 1.2, 1.0, 0.2)) as net:
            with pytest.raises(mr.MrstatError) as e:  # no basis yet
                plan.gn_solve(cuda(d, torch.complex64), cuda(a0), outer_iters=2, surrogate_iters=1, surrogate=net)
            assert e.value.status == 3
            plan.lowrank_set_basis(_basis(plan, 16))
            with pytest.raises(mr.MrstatError) as e:  # rank 8 net, rank 16 basis
                plan.gn_solve(cuda(d, torch.complex64), cuda(a0), outer_iters=2, surrogate_iters=1, surrogate=net)
            assert e.value.status == 1


@pytest.mark.parametrize("inner,delta_scale", [(8, 1.0), (40, 0.02)])
def test_lowrank_hessian_steihaug_on_the_column_path_matches_oracle(mr, inner, delta_scale):
    """64 x 64 with a fully sampled readout: the low-rank Gauss-Newton matrix takes the
    column form, and Steihaug's CG runs in one persistent launch.  Its first outer
    iteration against the oracle's Steihaug CG with the projected model's B and the exact
    gradient: the same exit and step count, and the same step.  The small trust region of
    the second case ends CG on the boundary."""
    seq = synth.make_sequence(64, 64, 5, 7.8, 3.9, seed=2)
    ph = synth.ellipse_phantom(64, 1)
    truth = truth_of(ph)
    d = synth.add_noise(model.forward(seq, truth), 50.0, 5).astype(np.complex64).astype(np.complex128)
    a0 = f32(truth + 0.05 * synth.random_params(seq.nv, 6))
    delta = delta_scale * 0.1 * float(np.linalg.norm(a0))
    with mr.Plan(seq) as plan:
        U = _basis(plan, 32)
        plan.lowrank_set_basis(U)
        plan.profile_start(kernels=("jhw_dot",))
        a = cuda(a0)
        rep = plan.gn_solve(cuda(d, torch.complex64), a, outer_iters=1, inner_iters=inner, hessian=1,
                            delta0=delta)
        prof = plan.profile_stop()
        plan.check()
        a_gpu = a.cpu().numpy()
        Uh = U.cpu().numpy().astype(np.float64)
    # one persistent launch for the whole inner solve (plus the gradient's product)
    assert prof["jhw_dot"]["launches"] <= 2
    lin = model.linearize(seq, a0)
    g = -model.jhw(lin, d - model.signal(lin))
    lin_p = model.project_onto_basis(lin, Uh)
    z, mchange, steps, why = solver.steihaug_cg(lambda v: model.gauss_newton_product(lin_p, v), g, delta, inner)
    assert rep["cg_exit"][0] == why
    assert rep["cg_steps"][0] == steps
    assert rep["accepted"][0]
    assert metrics.relerr(a_gpu - a0, solver.apply_bounds(a0 + z, solver.GNOptions()) - a0) < 1e-3


def test_lowrank_hessian_steihaug_column_path_converges_under_a_mask(mr):
    """The persistent Steihaug launch on a 48 x 64 grid with rank 24, whole image
    columns outside the mask, and a relative tolerance that ends CG early (exit
    'converged'): against the oracle's Steihaug CG on the projected model."""
    seq = synth.make_sequence(48, 64, 5, 7.8, 3.9, seed=4)
    rng = np.random.default_rng(14)
    t1 = np.exp(rng.uniform(np.log(300), np.log(2500), (64, 48)))
    t2 = np.exp(rng.uniform(np.log(30), np.log(250), (64, 48)))
    rho = rng.uniform(0.6, 1.0, (64, 48)) * np.exp(1j * rng.uniform(0, 0.5, (64, 48)))
    truth = f32(np.stack([np.log(t1.ravel()), np.log(t2.ravel()), rho.real.ravel(), rho.imag.ravel()]))
    mask = rng.random((64, 48)) > 0.1
    mask[:, :6] = False
    mask[:, 30:33] = False
    mask = mask.ravel()
    d = synth.add_noise(model.forward(seq, truth), 50.0, 8).astype(np.complex64).astype(np.complex128)
    a0 = f32(truth + 0.03 * synth.random_params(seq.nv, 9))
    delta = 0.1 * float(np.linalg.norm(a0 * mask[None]))
    with mr.Plan(seq) as plan:
        U = _basis(plan, 24)
        plan.lowrank_set_basis(U)
        plan.profile_start(kernels=("jhw_dot",))
        a = cuda(a0)
        rep = plan.gn_solve(cuda(d, torch.complex64), a, mask=cuda(mask.astype(np.uint8), torch.uint8),
                            outer_iters=1, inner_iters=40, hessian=1, cg_rel_tol=0.1)
        prof = plan.profile_stop()
        plan.check()
        a_gpu = a.cpu().numpy()
        Uh = U.cpu().numpy().astype(np.float64)
    assert prof["jhw_dot"]["launches"] <= 2
    lin = model.linearize(seq, a0, mask=mask)
    g = -model.jhw(lin, d - model.signal(lin))
    lin_p = model.project_onto_basis(lin, Uh)
    z, mchange, steps, why = solver.steihaug_cg(lambda v: model.gauss_newton_product(lin_p, v), g, delta, 40, 0.1)
    assert why == "converged"
    assert rep["cg_exit"][0] == why
    assert rep["cg_steps"][0] == steps
    assert rep["accepted"][0]
    trial = np.where(mask[None], solver.apply_bounds(a0 + z, solver.GNOptions()), a0)
    assert metrics.relerr(a_gpu - a0, trial - a0) < 1e-3
    assert np.array_equal(a_gpu[:, ~mask], a0[:, ~mask].astype(np.float32))


def test_resumed_solve_continues_where_it_stopped(mr, noisy_quad):
    """Checkpoint and resume on the host: 3 + 3 outer iterations (the second call starts
    from the first's alpha, its mask, report delta_final and iteration_offset = 3) follow
    the same trajectory as 6 iterations in one call, also with a surrogate phase of 4
    iterations that straddles the break."""
    seq, ph, truth, d, a0 = noisy_quad
    mask = torch.ones(seq.nv, dtype=torch.uint8, device="cuda")
    mask[::7] = 0
    dd = cuda(d, torch.complex64)
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(_basis(plan, 16))
        net = _trained_surrogate(mr, plan, 16)
        for kw in (dict(), dict(hessian=1, surrogate_iters=4, surrogate=net)):
            a_one = cuda(a0)
            rep = plan.gn_solve(dd, a_one, mask=mask.clone(), outer_iters=6, inner_iters=15, **kw)
            a_two = cuda(a0)
            r1 = plan.gn_solve(dd, a_two, mask=mask.clone(), outer_iters=3, inner_iters=15, **kw)
            r2 = plan.gn_solve(dd, a_two, mask=mask.clone(), outer_iters=3, inner_iters=15,
                               delta0=r1["delta_final"], iteration_offset=3, **kw)
            f_two = r1["f"] + r2["f"]
            assert np.allclose(f_two, rep["f"], rtol=1e-6), (kw, f_two, rep["f"])
            assert r1["delta"] + r2["delta"] == pytest.approx(rep["delta"], rel=1e-9)
            assert r2["delta_final"] == pytest.approx(rep["delta_final"], rel=1e-9)
            assert r2["f_final"] == pytest.approx(rep["f_final"], rel=1e-6)
            assert metrics.relerr(a_two.cpu().numpy(), a_one.cpu().numpy()) < 1e-6
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(dd, cuda(a0), outer_iters=2, iteration_offset=-1)
        assert e.value.status == 1
        plan.check()
        net.close()
