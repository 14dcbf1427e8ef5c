"""Low-rank (compressed) form on the GPU against the oracle's projected model.

The low-rank model replaces every time course by its projection onto a real time
basis U (oracle.model.project_onto_basis); given the same U, the GPU products must
equal the oracle's products of the projected model.  The DFTs run as split-BF16
tcgen05 products, so the bar is the split form's 3e-5 normwise.  The basis itself is
checked against numpy's SVD of the same simulated training time courses.
"""
import numpy as np
import pytest

import synth
from oracle import bloch, encoding, model, metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 3e-5


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


def training_set(n, seed):
    rng = np.random.default_rng(seed)
    return f32(np.stack([rng.uniform(np.log(100), np.log(6000), n), rng.uniform(np.log(10), np.log(3000), n)]))


def random_phantom(nx, ny, seed):
    rng = np.random.default_rng(seed)
    t1 = np.exp(rng.uniform(np.log(200), np.log(3000), (ny, nx)))
    t2 = np.exp(rng.uniform(np.log(20), np.log(300), (ny, nx)))
    rho = rng.uniform(0.5, 1.0, (ny, nx)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (ny, nx)))
    return f32(np.stack([np.log(t1.ravel()), np.log(t2.ravel()), rho.real.ravel(), rho.imag.ravel()]))


def test_time_basis_matches_numpy_svd(mr):
    seq = synth.make_sequence(40, 24, 5, 7.8, 3.9, seed=3, extra_trs=6)
    train = training_set(600, 1)
    U_ref, s_ref = model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), 16)
    with mr.Plan(seq) as plan:
        U, sv = plan.lowrank_basis(cuda(train), 16)
        U = U.cpu().numpy().astype(np.float64)
    assert np.allclose(U.T @ U, np.eye(16), atol=1e-6)
    assert np.allclose(sv, s_ref, rtol=1e-4)
    # the well-separated leading directions span the same subspace, and the whole basis
    # compresses the training time courses as well as the exact SVD basis does
    assert np.linalg.norm(U[:, :8] @ U[:, :8].T - U_ref[:, :8] @ U_ref[:, :8].T, 2) < 1e-3
    sim = bloch.simulate(seq, np.exp(train[0]), np.exp(train[1]))
    Y = np.concatenate([sim["m"].imag, sim["dm_dlnT1"].imag, sim["dm_dlnT2"].imag], axis=1)
    res_gpu = np.linalg.norm(Y - U @ (U.T @ Y))
    res_ref = np.linalg.norm(Y - U_ref @ (U_ref.T @ Y))
    assert res_gpu < 1.01 * res_ref


# nkx == nx from the third case on: J^H J v takes the path without the readout DFT pair;
# ny = 32 N1 for every N1 = 1 .. 8 (32, 64, 96, 128, 160, 192, 224, 256) takes the
# factorised phase-encode DFT on top (a 2 N1-point DFT from two N1-point DFTs, then a
# 16-point FFT), the whole product in one kernel per image column (the 32-row case has
# 10 TRs per ky)
@pytest.mark.parametrize("case", [(40, 24, 5, 6, 48, 16), (33, 17, 3, 3, 30, 8), (64, 64, 5, 0, 64, 32),
                                  (36, 20, 3, 2, 36, 24), (1, 12, 2, 1, 1, 8), (24, 96, 2, 3, 24, 16),
                                  (8, 224, 1, 0, 8, 8), (13, 256, 1, 1, 13, 24), (16, 32, 10, 0, 16, 8),
                                  (6, 128, 1, 0, 6, 8), (5, 160, 1, 1, 5, 16), (4, 192, 1, 2, 4, 24)])
def test_lowrank_products_match_projected_oracle(mr, case):
    nx, ny, fills, extra, nkx, R = case
    seq = synth.make_sequence(nx, ny, fills, 7.8, 3.9, seed=5, nkx=nkx, extra_trs=extra)
    alpha = random_phantom(nx, ny, 7)
    train = training_set(400, 2)
    U, _ = model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), R)
    U = f32(U)
    lin = model.project_onto_basis(model.linearize(seq, alpha), U)
    v = synth.random_params(seq.nv, 11)
    w = synth.random_kspace(seq.ntr, seq.nkx, 12)
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha))
        coef = plan.lowrank_coefficients().cpu().numpy()
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        h = plan.jhjv(cuda(v)).cpu().numpy()
        h2 = plan.jhw(plan.jvp(cuda(v))).cpu().numpy()
        plan.check()
    raw = model.linearize(seq, alpha)
    assert metrics.relerr(coef[0], U.T @ raw.m.imag) < 1e-5
    assert metrics.relerr(coef[1], U.T @ raw.dm1.imag) < 1e-5
    assert metrics.relerr(coef[2], U.T @ raw.dm2.imag) < 1e-5
    assert metrics.relerr(jv, model.jvp(lin, v)) < TOL
    assert metrics.relerr(g, model.jhw(lin, w)) < TOL
    ref_h = model.gauss_newton_product(lin, v)
    assert metrics.relerr(h, ref_h) < TOL
    assert metrics.relerr(h2, ref_h) < TOL


def test_lowrank_masked_columns_match_projected_oracle(mr):
    """A mask that leaves whole image columns empty (the column kernel skips them) and
    random holes elsewhere: the low-rank products against the projected oracle model."""
    seq = synth.make_sequence(64, 64, 5, 7.8, 3.9, seed=6)
    alpha = random_phantom(64, 64, 8)
    train = training_set(400, 2)
    U = f32(model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), 16)[0])
    mask = np.random.default_rng(9).random((64, 64)) > 0.3
    mask[:, :10] = False
    mask[:, 40:44] = False
    mask = mask.ravel()
    lin = model.project_onto_basis(model.linearize(seq, alpha, mask=mask), U)
    v = synth.random_params(seq.nv, 13)
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha), mask=cuda(mask.astype(np.uint8), torch.uint8))
        h = plan.jhjv(cuda(v)).cpu().numpy()
        h2 = plan.jhw(plan.jvp(cuda(v))).cpu().numpy()
        plan.check()
    ref = model.gauss_newton_product(lin, v)
    assert metrics.relerr(h, ref) < TOL
    assert metrics.relerr(h2, ref) < TOL
    assert np.all(h[:, ~mask] == 0)


@pytest.mark.parametrize("iters", [1, 4])
def test_lowrank_cg_fixed_matches_oracle_cg(mr, iters):
    """Fixed-count CG on the low-rank Re(J^H J) through the column kernel, which also takes
    each direction update p <- r + beta p into its first pass from the second iteration
    on.  Against textbook CG in float64 on the projected oracle model; the bar after
    several iterations is 1e-4, as for the exact form."""
    seq = synth.make_sequence(64, 64, 5, 7.8, 3.9, seed=5)
    alpha = random_phantom(64, 64, 7)
    train = training_set(400, 2)
    U = f32(model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), 16)[0])
    lin = model.project_onto_basis(model.linearize(seq, alpha), U)
    b = model.jhw(lin, synth.random_kspace(seq.ntr, seq.nkx, 40))
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    for _ in range(iters):
        q = model.gauss_newton_product(lin, p)
        a = rr / float(np.sum(p * q))
        x = x + a * p
        r = r - a * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha))
        xg = plan.cg_fixed(cuda(b), iters).cpu().numpy()
        plan.check()
    assert metrics.relerr(xg, x) < (1e-5 if iters == 1 else 1e-4)


def test_lowrank_full_size_sampled_jhw(mr):
    seq, ph = synth.config("brain224")
    alpha = f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                          ph.rho.imag.ravel()]))
    w = synth.random_kspace(seq.ntr, seq.nkx, 52)
    vox = np.sort(np.random.default_rng(5).choice(seq.nv, 64, replace=False))
    with mr.Plan(seq) as plan:
        train = cuda(training_set(2048, 3))
        U, sv = plan.lowrank_basis(train, 32)
        plan.lowrank_set_basis(U)
        plan.lowrank_linearize(cuda(alpha))
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()[:, vox]
        Uh = U.cpu().numpy().astype(np.float64)
        plan.check()
    sim = bloch.simulate(seq, np.exp(alpha[0, vox]), np.exp(alpha[1, vox]))
    W = encoding.encode_adjoint(seq, w, vox)
    rho = alpha[2, vox] + 1j * alpha[3, vox]
    P = lambda x: 1j * (Uh @ (Uh.T @ x.imag))
    m, d1, d2 = P(sim["m"]), P(sim["dm_dlnT1"]), P(sim["dm_dlnT2"])
    ref = np.stack([np.real(np.sum(np.conj(rho[None] * d1) * W, 0)), np.real(np.sum(np.conj(rho[None] * d2) * W, 0)),
                    np.real(np.sum(np.conj(m) * W, 0)), np.real(np.sum(np.conj(1j * m) * W, 0))])
    assert metrics.relerr(g, ref) < TOL
    # the rank-32 model is close to the exact one on these voxels (projection error ~1e-3)
    exact = np.stack([np.real(np.sum(np.conj(rho[None] * sim["dm_dlnT1"]) * W, 0)),
                      np.real(np.sum(np.conj(rho[None] * sim["dm_dlnT2"]) * W, 0)),
                      np.real(np.sum(np.conj(sim["m"]) * W, 0)), np.real(np.sum(np.conj(1j * sim["m"]) * W, 0))])
    assert metrics.relerr(g, exact) < 1e-2


@pytest.mark.parametrize("nx,ny,rank,holes,fills", [(40, 96, 24, True, 4), (33, 32, 8, False, 4),
                                                     (24, 224, 32, True, 8)])
def test_persistent_cg_shapes_match_oracle_cg(mr, nx, ny, rank, holes, fills):
    """The persistent CG launch on other column shapes: 96 = 3 x 32 rows with rank 24
    (twelve basis functions per block of a cluster), whole image columns and
    random voxels outside the mask; and 32 rows (one 32-point FFT, half-columns of 16)
    with an odd number of columns; and 224 rows with eight TRs per phase-encode line (the
    largest shared-memory layout: two blocks per SM, enough for these 24 columns).  Six
    iterations against textbook CG in float64 on the projected oracle model; one launch
    carries all products."""
    seq = synth.make_sequence(nx, ny, fills, 7.8, 3.9, seed=11)
    alpha = random_phantom(nx, ny, 12)
    train = training_set(400, 3)
    U = f32(model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), rank)[0])
    mask = np.ones((ny, nx), bool)
    if holes:
        mask = np.random.default_rng(13).random((ny, nx)) > 0.2
        mask[:, :5] = False
        mask[:, 20:23] = False
    mask = mask.ravel()
    lin = model.project_onto_basis(model.linearize(seq, alpha, mask=mask), U)
    b = model.jhw(lin, synth.random_kspace(seq.ntr, seq.nkx, 41))
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    for _ in range(6):
        q = model.gauss_newton_product(lin, p)
        a = rr / float(np.sum(p * q))
        x = x + a * p
        r = r - a * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha), mask=cuda(mask.astype(np.uint8), torch.uint8))
        plan.profile_start(kernels=("jhw_dot", "vector"))
        xg = plan.cg_fixed(cuda(b), 6).cpu().numpy()
        prof = plan.profile_stop()
        plan.check()
    # one persistent launch (counted as six products) and no per-iteration vector launches
    assert prof["jhw_dot"]["launches"] == 6
    assert prof["vector"]["launches"] <= 1
    assert metrics.relerr(xg, x) < 1e-4
    assert np.all(xg[:, ~mask] == 0)


def test_persistent_launch_wait_runs_out_and_the_plan_recovers(mr):
    """Failure path of the persistent launches, without a fault: with the test hook one
    block withholds its first arrival at the grid counter, every block's bounded wait runs
    out (2 s), the CG launch ends and mrstat_plan_check reports TIMEOUT (and clears the
    flag); the Gauss-Newton solve reports TIMEOUT from its Steihaug launch.  With the hook
    off the same plan then solves correctly."""
    import time
    seq = synth.make_sequence(64, 64, 5, 7.8, 3.9, seed=5)
    alpha = random_phantom(64, 64, 7)
    train = training_set(400, 2)
    U = f32(model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), 16)[0])
    lin = model.project_onto_basis(model.linearize(seq, alpha), U)
    b = model.jhw(lin, synth.random_kspace(seq.ntr, seq.nkx, 40))
    q = model.gauss_newton_product(lin, b)
    x1 = (float(np.sum(b * b)) / float(np.sum(b * q))) * b  # one CG iteration from zero
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha))
        plan.inject_grid_stall(5)
        t0 = time.perf_counter()
        plan.cg_fixed(cuda(b), 3)
        with pytest.raises(mr.MrstatError) as e:
            plan.check()
        assert e.value.status == 6  # MRSTAT_ERR_TIMEOUT
        assert time.perf_counter() - t0 > 1.5
        d = synth.add_noise(model.forward(seq, alpha), 50.0, 3).astype(np.complex64)
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(cuda(d, torch.complex64), cuda(alpha), outer_iters=1, inner_iters=5, hessian=1)
        assert e.value.status == 6
        plan.inject_grid_stall(-1)
        # a block outside the persistent grid (two blocks per image column) is refused
        with pytest.raises(mr.MrstatError) as e:
            plan.inject_grid_stall(2 * seq.nx)
        assert e.value.status == 1
        plan.check()
        plan.lowrank_linearize(cuda(alpha))
        xg = plan.cg_fixed(cuda(b), 1).cpu().numpy()
        plan.check()
        assert plan.cg_applied() == 1
    assert metrics.relerr(xg, x1) < 1e-5
