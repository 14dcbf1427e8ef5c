"""Pins of the oracle's signal and Jacobian products (Theory; Algorithms 2 and 4;
Eq. 4): finite differences of the signal, exact linearity in rho, the adjoint
identity, the gradient of f and the mask."""
import numpy as np
import pytest

import synth
from oracle import model, metrics


def _alpha(ph, b1=False):
    rows = [np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(), ph.rho.imag.ravel()]
    if b1:
        rows.append(ph.b1.ravel())
    return np.stack(rows)


@pytest.fixture(scope="module")
def case():
    seq = synth.make_sequence(12, 10, 3, 7.8, 3.9, seed=3, extra_trs=5)
    ph = synth.quadrant_phantom(12, 1)
    ph.t1_ms = ph.t1_ms[:10]; ph.t2_ms = ph.t2_ms[:10]; ph.rho = ph.rho[:10]; ph.b1 = ph.b1[:10]
    return seq, ph


@pytest.mark.parametrize("b1", [False, True])
def test_jvp_matches_central_differences(case, b1):
    seq, ph = case
    alpha = _alpha(ph, b1)
    if b1:
        alpha[4] = synth.smooth_b1(12, 10, 4).ravel()
    lin = model.linearize(seq, alpha)
    v = synth.random_params(seq.nv, 7, alpha.shape[0])
    h = 1e-5
    fd = (model.forward(seq, alpha + h * v) - model.forward(seq, alpha - h * v)) / (2 * h)
    assert metrics.relerr(model.jvp(lin, v), fd) < 1e-8


def test_rho_block_is_exactly_linear(case):
    """s = M rho (Eq. s = M rho): J_s applied to (0, 0, Re rho, Im rho) reproduces s."""
    seq, ph = case
    alpha = _alpha(ph)
    lin = model.linearize(seq, alpha)
    v = np.zeros_like(alpha)
    v[2:4] = alpha[2:4]
    assert metrics.relerr(model.jvp(lin, v), model.signal(lin)) < 1e-14
    # and the Im rho column is i times the Re rho column
    e = np.zeros_like(alpha); e[2, 17] = 1.0
    f = np.zeros_like(alpha); f[3, 17] = 1.0
    assert np.allclose(model.jvp(lin, f), 1j * model.jvp(lin, e), atol=1e-14)


@pytest.mark.parametrize("b1", [False, True])
def test_adjoint_identity(case, b1):
    """Re<J_s v, w> = <v, Re(J_s^H w)>."""
    seq, ph = case
    alpha = _alpha(ph, b1)
    lin = model.linearize(seq, alpha)
    v = synth.random_params(seq.nv, 1, alpha.shape[0])
    w = synth.random_kspace(seq.ntr, seq.nkx, 2)
    lhs = np.vdot(model.jvp(lin, v), w).real
    rhs = np.sum(v * model.jhw(lin, w))
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_gradient_matches_objective_differences(case):
    seq, ph = case
    alpha = _alpha(ph)
    d = synth.random_kspace(seq.ntr, seq.nkx, 11) * 0.05 + model.forward(seq, alpha)
    a = alpha + 0.05 * synth.random_params(seq.nv, 12)
    g = model.gradient(model.linearize(seq, a), d)
    v = synth.random_params(seq.nv, 13)
    h = 1e-6
    fd = (model.objective(d, model.forward(seq, a + h * v)) - model.objective(d, model.forward(seq, a - h * v))) / (2 * h)
    assert abs(np.sum(g * v) - fd) / abs(fd) < 1e-6


def test_mask_removes_voxels(case):
    seq, ph = case
    alpha = _alpha(ph)
    mask = np.zeros(seq.nv, bool)
    mask[::3] = True
    lin = model.linearize(seq, alpha, mask=mask)
    w = synth.random_kspace(seq.ntr, seq.nkx, 2)
    g = model.jhw(lin, w)
    assert np.all(g[:, ~mask] == 0)
    a2 = alpha.copy()
    a2[2:4, ~mask] = 0.0
    assert metrics.relerr(model.signal(lin), model.forward(seq, a2)) < 1e-14
