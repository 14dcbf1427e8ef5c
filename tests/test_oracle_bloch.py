"""Pins of the oracle's Bloch recursion (Supporting Information S2) to results
that do not come from the oracle itself: closed forms, a library rotation,
complex-step and finite-difference derivatives."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from oracle import bloch


def _seq(flips, tr=10.0, te=5.0, inversion=False, alternate=True):
    flips = np.asarray(flips, np.float64)
    return synth.Sequence(nx=1, ny=1, nkx=1, tr_ms=tr, te_ms=te, flip_rad=flips,
                          ky=np.zeros(flips.shape[0], np.int32), inversion=inversion,
                          alternate_phase=alternate)


@pytest.mark.parametrize("t1,t2,deg", [(500.0, 50.0, 60.0), (1000.0, 100.0, 30.0),
                                       (800.0, 70.0, 45.0), (2000.0, 1500.0, 20.0)])
def test_freeman_hill_steady_state(t1, t2, deg):
    """Constant flip, RF phase alternating 0/180, on resonance, TE = TR/2: the echo
    amplitude converges to the bSSFP steady state (Freeman-Hill), a closed form
    that shares nothing with the recursion."""
    tr, te = 10.0, 5.0
    a = np.deg2rad(deg)
    seq = _seq(np.full(6000, a), tr, te)
    m = bloch.simulate(seq, np.array([t1]), np.array([t2]), tangents=False)["m"][:, 0]
    e1, e2 = np.exp(-tr / t1), np.exp(-tr / t2)
    ss = (1 - e1) * np.sin(a) / (1 - (e1 - e2) * np.cos(a) - e1 * e2) * np.exp(-te / t2)
    assert abs(abs(m[-1]) - ss) / ss < 1e-10
    # the alternating RF phase makes the steady-state echo alternate in sign
    assert np.sign(m[-1].imag) == -np.sign(m[-2].imag)


def test_inversion_recovery_without_rf():
    """Zero flips after an ideal inversion: m_z(t) = 1 - 2 exp(-t/T1), m_xy = 0."""
    tr, te = 7.8, 3.9
    seq = _seq(np.zeros(200), tr, te, inversion=True)
    t1 = np.array([300.0, 1200.0])
    r = bloch.simulate(seq, t1, np.array([40.0, 90.0]))
    t = np.arange(200) * tr + te
    mz = r["mxyz"][:, 2, :]
    assert np.allclose(mz, 1 - 2 * np.exp(-t[:, None] / t1[None, :]), rtol=0, atol=1e-13)
    assert np.all(r["m"] == 0)
    assert np.all(r["dm_dlnT1"] == 0) and np.all(r["dm_dlnT2"] == 0)


def test_free_induction_decay_after_single_pulse():
    """One pulse of angle a from equilibrium, then nothing: |m_xy(t)| = sin(a) exp(-t/T2)
    at the echoes, and its ln T2 derivative is (t/T2) sin(a) exp(-t/T2)."""
    tr, te = 8.0, 4.0
    a = np.deg2rad(35.0)
    flips = np.zeros(50)
    flips[0] = a
    seq = _seq(flips, tr, te)
    t2 = np.array([50.0, 250.0])
    r = bloch.simulate(seq, np.array([900.0, 900.0]), t2)
    t = np.arange(50) * tr + te
    amp = np.sin(a) * np.exp(-t[:, None] / t2[None, :])
    assert np.allclose(np.abs(r["m"]), amp, rtol=1e-13, atol=0)
    assert np.allclose(np.abs(r["dm_dlnT2"]), (t[:, None] / t2[None, :]) * amp, rtol=1e-12, atol=0)


def test_rodrigues_matches_library_rotation():
    """S2's Rodrigues formula equals scipy's rotation by the rotation vector a."""
    rng = np.random.default_rng(3)
    m = rng.standard_normal((3, 7))
    for _ in range(5):
        a = rng.standard_normal(3)
        theta = np.linalg.norm(a)
        mine = bloch.rodrigues(m, a / theta, theta)
        ref = Rotation.from_rotvec(a).apply(m.T).T
        assert np.allclose(mine, ref, atol=1e-14)


def test_rf_axis_convention_positive_flip_gives_positive_my():
    """RF phase 0 rotates about -x (S2: a = [-|B1| Re RF, ...]): m_0 = z goes to +y."""
    seq = _seq([0.3], 10.0, 5.0)
    r = bloch.simulate(seq, np.array([1e12]), np.array([1e12]), tangents=False)
    assert np.isclose(r["mxyz"][0, 1, 0], np.sin(0.3), atol=1e-12)
    assert np.isclose(r["mxyz"][0, 2, 0], np.cos(0.3), atol=1e-12)


def test_transverse_x_stays_zero_for_0_180_phases():
    """With RF phases in {0, 180} degrees the rotation axis is +-x, so m_x never leaves 0:
    the echo signal is i * m_y (the GPU path stores only m_y)."""
    seq, ph = synth.config("quad16")
    r = bloch.simulate(seq, ph.t1_ms.ravel(), ph.t2_ms.ravel())
    assert np.abs(r["mxyz"][:, 0, :]).max() < 1e-14
    assert np.abs(r["m"].real).max() < 1e-14


@pytest.mark.parametrize("which", ["t1", "t2", "b1"])
def test_tangents_match_complex_step(which):
    """Forward-mode tangents equal complex-step derivatives (Squire & Trapp) to ~1e-13."""
    seq = synth.make_sequence(4, 4, 5, 7.8, 3.9, seed=2)
    rng = np.random.default_rng(1)
    t1 = np.exp(rng.uniform(np.log(200), np.log(3000), 16))
    t2 = np.exp(rng.uniform(np.log(20), np.log(300), 16))
    b1 = rng.uniform(0.8, 1.2, 16)
    ref = bloch.simulate(seq, t1, t2, b1, tangents=True, b1_tangent=True)
    h = 1e-30
    if which == "t1":
        rc = bloch.simulate(seq, np.exp(np.log(t1) + 1j * h), t2, b1, tangents=False)
        key = "dm_dlnT1"
    elif which == "t2":
        rc = bloch.simulate(seq, t1, np.exp(np.log(t2) + 1j * h), b1, tangents=False)
        key = "dm_dlnT2"
    else:
        rc = bloch.simulate(seq, t1, t2, b1 + 1j * h, tangents=False)
        key = "dm_dB1"
    cs = (rc["mxyz"][:, 0, :].imag + 1j * rc["mxyz"][:, 1, :].imag) / h
    err = np.linalg.norm(cs - ref[key]) / np.linalg.norm(cs)
    assert err < 1e-12, err


def test_tangents_match_central_differences():
    """Central differences with a relative step h = 1e-3 (the paper's FD alternative)."""
    seq = synth.make_sequence(4, 4, 5, 7.8, 3.9, seed=4)
    rng = np.random.default_rng(2)
    t1 = np.exp(rng.uniform(np.log(200), np.log(3000), 16))
    t2 = np.exp(rng.uniform(np.log(20), np.log(300), 16))
    ref = bloch.simulate(seq, t1, t2)
    h = 1e-3
    for key, fp, fm in [("dm_dlnT1", (t1 * np.exp(h), t2), (t1 * np.exp(-h), t2)),
                        ("dm_dlnT2", (t1, t2 * np.exp(h)), (t1, t2 * np.exp(-h)))]:
        mp = bloch.simulate(seq, *fp, tangents=False)["m"]
        mm = bloch.simulate(seq, *fm, tangents=False)["m"]
        fd = (mp - mm) / (2 * h)
        assert np.linalg.norm(fd - ref[key]) / np.linalg.norm(ref[key]) < 1e-5
