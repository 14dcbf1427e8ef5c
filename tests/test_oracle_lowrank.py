"""Pins of the oracle's low-rank model (the time-course compression of Methods, "Numerical
Brain Simulation", applied to the signal model) and of the bound handling of its
Gauss-Newton solver (Methods, "Reconstructions": reflection at the feasible boundaries).

None of these compares the oracle with a retyped copy of itself:

* project_onto_basis against the identity (a complete basis), a least-squares fit by
  numpy's solver, and the algebra of orthogonal projectors (idempotent, residual
  orthogonal to the basis, span kept exactly);
* time_basis against Eckart-Young (the captured energy and the residual follow from the
  eigenvalues of the Gram matrix, and no other rank-R basis captures more), against exact
  reproduction of one sample's three time courses, and against the bSSFP steady state
  (Freeman-Hill): for a constant flip train the tail of every time course, and so of every
  basis vector, is the sign-alternating steady-state pattern;
* reflect_into_bounds / apply_bounds against hand-computed reflections at both ends of the
  T1, T2 and B1 boxes, including steps that overshoot by more than the box width.
"""
import numpy as np
import pytest

import synth
from oracle import bloch, metrics, model, solver


def _alpha(ph):
    return np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                     ph.rho.imag.ravel()])


@pytest.fixture(scope="module")
def lin():
    seq = synth.make_sequence(8, 6, 3, 7.8, 3.9, seed=5, extra_trs=3)  # 21 TRs, ragged
    ph = synth.quadrant_phantom(8, 2)
    ph.t1_ms, ph.t2_ms, ph.rho = ph.t1_ms[:6], ph.t2_ms[:6], ph.rho[:6]
    return model.linearize(seq, _alpha(ph))


def _orthonormal(rows, cols, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((rows, cols)))
    return q


def test_projection_on_a_complete_basis_is_the_identity(lin):
    """rank = ntr: U U^T = I, so the projected model is the exact one (and so are its
    products)."""
    U = _orthonormal(lin.seq.ntr, lin.seq.ntr, 0)
    p = model.project_onto_basis(lin, U)
    for a, b in ((p.m, lin.m), (p.dm1, lin.dm1), (p.dm2, lin.dm2)):
        assert metrics.relerr(a, b) < 1e-12
    v = synth.random_params(lin.seq.nv, 3)
    w = synth.random_kspace(lin.seq.ntr, lin.seq.nkx, 4)
    assert metrics.relerr(model.jvp(p, v), model.jvp(lin, v)) < 1e-12
    assert metrics.relerr(model.jhw(p, w), model.jhw(lin, w)) < 1e-12


def test_projection_is_the_least_squares_fit_in_the_basis(lin):
    """Each projected time course is U c with c the least-squares coefficients of the
    exact one (numpy's lstsq, an SVD solver that never forms U U^T); real and imaginary
    parts separately, because the basis is real."""
    U = _orthonormal(lin.seq.ntr, 5, 1)
    p = model.project_onto_basis(lin, U)
    for exact, proj in ((lin.m, p.m), (lin.dm1, p.dm1), (lin.dm2, p.dm2)):
        for part in (np.real, np.imag):
            c = np.linalg.lstsq(U, part(exact), rcond=None)[0]
            assert np.allclose(part(proj), U @ c, rtol=0, atol=1e-13 * np.abs(exact).max())


def test_projection_is_an_orthogonal_projector(lin):
    """Idempotent, residual orthogonal to every basis vector, and the span of the basis kept:
    a basis built from three voxels' time courses reproduces those voxels exactly and
    changes the others."""
    U = _orthonormal(lin.seq.ntr, 4, 2)
    p = model.project_onto_basis(lin, U)
    pp = model.project_onto_basis(p, U)
    assert metrics.relerr(pp.m, p.m) < 1e-13
    assert np.abs(U.T @ (lin.m - p.m)).max() < 1e-13 * np.abs(lin.m).max()
    assert np.abs(U.T @ (lin.dm2 - p.dm2)).max() < 1e-13 * np.abs(lin.dm2).max()
    keep = [0, 17, 40]
    Y = np.concatenate([lin.m[:, keep].imag, lin.dm1[:, keep].imag, lin.dm2[:, keep].imag], axis=1)
    V = np.linalg.qr(Y)[0]
    q = model.project_onto_basis(lin, V)
    for a, b in ((q.m, lin.m), (q.dm1, lin.dm1), (q.dm2, lin.dm2)):
        assert metrics.relerr(a[:, keep], b[:, keep]) < 1e-12
    others = np.setdiff1d(np.arange(lin.seq.nv), keep)
    assert metrics.relerr(q.m[:, others], lin.m[:, others]) > 1e-3


def _train(n, seed):
    rng = np.random.default_rng(seed)
    return (np.exp(rng.uniform(np.log(200), np.log(3000), n)), np.exp(rng.uniform(np.log(20), np.log(300), n)))


def test_time_basis_is_optimal_by_eckart_young():
    """The basis is orthonormal, the singular values are the square roots of the largest
    eigenvalues of Y^T Y (numpy's symmetric eigensolver), the residual energy of the
    training set is the sum of the remaining eigenvalues, and neither a random basis nor
    one spanned by the first training columns captures more energy."""
    seq = synth.make_sequence(4, 8, 4, 7.8, 3.9, seed=2)  # 32 TRs
    t1, t2 = _train(12, 0)
    R = 6
    U, s = model.time_basis(seq, t1, t2, R)
    assert U.shape == (seq.ntr, R)
    assert np.allclose(U.T @ U, np.eye(R), atol=1e-13)
    sim = bloch.simulate(seq, t1, t2)
    Y = np.concatenate([sim["m"].imag, sim["dm_dlnT1"].imag, sim["dm_dlnT2"].imag], axis=1)
    ev = np.sort(np.linalg.eigvalsh(Y.T @ Y))[::-1]
    assert np.allclose(s, np.sqrt(ev[:R]), rtol=1e-9)
    assert np.all(np.diff(s) <= 0)
    resid = np.linalg.norm(Y - U @ (U.T @ Y)) ** 2
    assert np.isclose(resid, ev[R:].clip(min=0).sum(), rtol=1e-6, atol=1e-12 * ev[0])
    captured = np.linalg.norm(U.T @ Y) ** 2
    for k in range(5):
        assert np.linalg.norm(_orthonormal(seq.ntr, R, 10 + k).T @ Y) ** 2 < captured
    assert np.linalg.norm(np.linalg.qr(Y[:, :R])[0].T @ Y) ** 2 <= captured * (1 + 1e-12)


def test_time_basis_of_one_sample_reproduces_its_time_courses():
    """One training voxel and rank 3: its m_y, dm_y/dlnT1, dm_y/dlnT2 lie in the span, so
    the low-rank model of that voxel is exact."""
    seq = synth.make_sequence(4, 8, 3, 7.8, 3.9, seed=4)
    t1, t2 = np.array([900.0]), np.array([70.0])
    U, _ = model.time_basis(seq, t1, t2, 3)
    alpha = np.array([[np.log(900.0)], [np.log(70.0)], [0.8], [-0.3]])
    one = synth.Sequence(nx=1, ny=1, nkx=1, tr_ms=seq.tr_ms, te_ms=seq.te_ms, flip_rad=seq.flip_rad,
                         ky=np.zeros(seq.ntr, np.int32), inversion=seq.inversion,
                         alternate_phase=seq.alternate_phase)
    lin1 = model.linearize(one, alpha)
    p = model.project_onto_basis(lin1, U)
    for a, b in ((p.m, lin1.m), (p.dm1, lin1.dm1), (p.dm2, lin1.dm2)):
        assert metrics.relerr(a, b) < 1e-12


def test_time_basis_tail_is_the_steady_state_pattern():
    """Constant flip angle, RF phase alternating, no inversion: every voxel reaches the
    bSSFP steady state, whose echo has the Freeman-Hill amplitude with alternating sign, so
    in the tail every training time course and every tangent is a multiple of
    (-1)^n -- and so is the tail of every basis vector.  The leading singular vector is
    dominated by that pattern over the whole train."""
    N = 1500
    seq = synth.Sequence(nx=1, ny=1, nkx=1, tr_ms=10.0, te_ms=5.0, flip_rad=np.full(N, np.deg2rad(50.0)),
                         ky=np.zeros(N, np.int32), inversion=False, alternate_phase=True)
    rng = np.random.default_rng(0)
    t1 = np.exp(rng.uniform(np.log(100), np.log(300), 40))
    t2 = np.exp(rng.uniform(np.log(30), np.log(80), 40))
    # the closed form itself, checked on the simulated tail first
    a = np.deg2rad(50.0)
    e1, e2 = np.exp(-10.0 / t1), np.exp(-10.0 / t2)
    ss = (1 - e1) * np.sin(a) / (1 - (e1 - e2) * np.cos(a) - e1 * e2) * np.exp(-5.0 / t2)
    m_last = bloch.simulate(seq, t1, t2, tangents=False)["m"][-1]
    assert np.allclose(np.abs(m_last), ss, rtol=1e-10)
    U, s = model.time_basis(seq, t1, t2, 3)
    tail = slice(N // 2, N)
    alt = (-1.0) ** np.arange(N)
    for k in range(3):
        u = U[tail, k]
        assert abs(u @ alt[tail]) / (np.linalg.norm(u) * np.linalg.norm(alt[tail])) > 1 - 1e-10
    assert abs(U[:, 0] @ alt) / np.sqrt(N) > 0.99
    assert s[0] > 10 * s[1]


# ---------------------------------------------------------------------------
# bounds: reflect a component that leaves [lo, hi] back inside, then clip
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("x,expect", [
    (2.0, 2.0),        # inside: unchanged
    (1.0, 1.0),        # on the bounds: unchanged
    (3.0, 3.0),
    (3.5, 2.5),        # 0.5 past hi -> 0.5 inside hi
    (0.2, 1.8),        # 0.8 past lo -> 0.8 inside lo
    (4.9, 1.1),        # 1.9 past hi (the box is 2 wide) -> 1.1
    (5.5, 1.5),        # 2.5 past hi: 2 hi - x = 0.5 < lo, reflected at lo -> 1.5
    (-2.0, 3.0),       # 3 past lo: 2 lo - x = 4 > hi, clipped -> 3
    (9.0, 3.0),        # 6 past hi: -3, reflected at lo -> 5, clipped -> 3
])
def test_reflect_into_bounds_hand_values(x, expect):
    """Box [1, 3]: one reflection at hi, then one at lo, then a clip (the simplified
    Coleman-Li reflection)."""
    got = solver.reflect_into_bounds(np.array([x]), 1.0, 3.0)[0]
    assert got == pytest.approx(expect, abs=1e-15)


def test_apply_bounds_on_every_box():
    """T1 in [50, 6000] ms and T2 in [5, 3000] ms on the ln scale, B1 in [0.5, 1.5]; the rho
    rows are never touched, and a 4-row alpha has no B1 row to bound.  Expected values
    worked out by hand from the bounds."""
    opts = solver.GNOptions()
    l1a, l1b = np.log(50.0), np.log(6000.0)
    l2a, l2b = np.log(5.0), np.log(3000.0)
    w1, w2 = l1b - l1a, l2b - l2a
    a = np.zeros((5, 6))
    a[0] = [l1b + 0.3, l1a - 0.2, np.log(1000.0), l1b + w1 + 0.1, l1a, l1b]
    a[1] = [l2a - 0.4, l2b + 0.7, np.log(80.0), l2a - w2 - 0.5, l2b, l2a]
    a[2] = [5.0, -5.0, 1e3, -1e3, 0.0, 2.0]
    a[3] = [-7.0, 7.0, 0.5, 1e-9, 3.0, -3.0]
    a[4] = [1.7, 0.2, 1.0, 3.6, 0.5, -1.0]
    before = a.copy()
    out = solver.apply_bounds(a, opts)
    # T1: 2 hi - (hi + w1 + 0.1) = lo - 0.1, reflected at lo -> lo + 0.1
    assert np.allclose(out[0], [l1b - 0.3, l1a + 0.2, np.log(1000.0), l1a + 0.1, l1a, l1b], rtol=0, atol=1e-12)
    # T2: 2 lo - (lo - w2 - 0.5) = hi + 0.5, clipped -> hi
    assert np.allclose(out[1], [l2a + 0.4, l2b - 0.7, np.log(80.0), l2b, l2b, l2a], rtol=0, atol=1e-12)
    # B1: 3.6 -> -0.6 -> 1.6 -> 1.5; -1.0 -> 2.0 -> 1.5
    assert np.allclose(out[4], [1.3, 0.8, 1.0, 1.5, 0.5, 1.5], rtol=0, atol=1e-12)
    assert np.array_equal(out[2:4], before[2:4])
    assert np.array_equal(a, before)  # the input is not modified
    out4 = solver.apply_bounds(a[:4], opts)
    assert np.array_equal(out4, out[:4])
