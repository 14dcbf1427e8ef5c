"""Pins of the oracle's small helpers against values worked out by hand: the error metrics
(NRMSE read as the normwise relative error over the masked voxels, MAPE in percent) and the
mask drawn from the initial proton density (|rho| > threshold * max |rho|, Methods,
"Reconstructions")."""
import numpy as np
import pytest

from oracle import metrics, solver


def test_nrmse_and_relerr_hand_values():
    ref = np.array([3.0, 4.0, 0.0, 12.0])
    est = np.array([3.0, 5.0, 7.0, 12.0])
    # ||(0, 1, 7, 0)|| / ||(3, 4, 0, 12)|| = sqrt(50) / 13
    assert metrics.nrmse(est, ref) == pytest.approx(np.sqrt(50.0) / 13.0, rel=1e-15)
    assert metrics.relerr(est, ref) == pytest.approx(np.sqrt(50.0) / 13.0, rel=1e-15)
    # the mask drops the third entry: ||(0, 1, 0)|| / ||(3, 4, 12)|| = 1 / 13
    mask = np.array([True, True, False, True])
    assert metrics.nrmse(est, ref, mask) == pytest.approx(1.0 / 13.0, rel=1e-15)
    # complex maps: |(1 + 1j) - 1| / |1| = 1
    assert metrics.nrmse(np.array([1 + 1j]), np.array([1.0])) == pytest.approx(1.0, rel=1e-15)
    # a zero reference gives the absolute error
    assert metrics.relerr(np.array([3.0, 4.0]), np.zeros(2)) == pytest.approx(5.0, rel=1e-15)


def test_mape_hand_values():
    ref = np.array([2.0, -4.0, 10.0])
    est = np.array([3.0, -3.0, 10.0])
    # mean(1/2, 1/4, 0) * 100 = 25
    assert metrics.mape(est, ref) == pytest.approx(25.0, rel=1e-15)
    assert metrics.mape(est, ref, np.array([False, True, True])) == pytest.approx(12.5, rel=1e-15)


def test_draw_mask_hand_values():
    rho = np.array([0.0, 0.05 + 0.0j, 0.3j, -1.0, 0.1, 0.1000001])
    # max |rho| = 1, threshold 0.1: strictly above 0.1
    assert np.array_equal(solver.draw_mask(rho, 0.1), [False, False, True, True, False, True])
    assert np.array_equal(solver.draw_mask(rho, 0.5), [False, False, False, True, False, False])
    assert solver.draw_mask(np.zeros(0), 0.1).shape == (0,)
