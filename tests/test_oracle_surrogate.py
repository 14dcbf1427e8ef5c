"""Pins of the oracle's surrogate MLP: forward-mode tangents against central
differences of the network output, and the hand-written loss gradient against central
differences of the Sobolev loss."""
import numpy as np

from oracle import surrogate

H, R = 8, 4
NORM = (6.5, 1.0, 4.0, 1.2, 1.0, 0.2)
SCALE = np.array([2.0, 1.0, 0.5, 0.25])


def _setup(seed=0, B=7):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(surrogate.num_params(H, R)) * 0.5
    x = np.stack([rng.uniform(5, 8, B), rng.uniform(3, 7, B), rng.uniform(0.8, 1.2, B)])
    target = tuple(rng.standard_normal((R, B)) for _ in range(3))
    return theta, x, target


def test_tangents_match_central_differences_of_the_output():
    theta, x, _ = _setup()
    c, d1, d2, _ = surrogate.forward(theta, x, NORM, SCALE, H, R)
    h = 1e-6
    for k, dk in ((0, d1), (1, d2)):
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        fd = (surrogate.forward(theta, xp, NORM, SCALE, H, R)[0] - surrogate.forward(theta, xm, NORM, SCALE, H, R)[0]) / (2 * h)
        assert np.allclose(dk, fd, rtol=1e-6, atol=1e-8)


def test_loss_gradient_matches_central_differences():
    theta, x, target = _setup(1)
    L, g = surrogate.loss_grad(theta, x, target, NORM, SCALE, H, R, lam=0.3)
    assert np.isclose(L, surrogate.loss(theta, x, target, NORM, SCALE, H, R, 0.3))
    rng = np.random.default_rng(2)
    idx = rng.choice(theta.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (surrogate.loss(tp, x, target, NORM, SCALE, H, R, 0.3) - surrogate.loss(tm, x, target, NORM, SCALE, H, R, 0.3)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
