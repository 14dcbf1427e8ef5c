"""Pins of the slice-profile oracle (oracle/slice_profile.py) to facts that do not come
from its own code: the hard-pulse model it must reduce to, the mirror symmetry of the
slice, the small-tip slice profile (the Fourier transform of the RF envelope), and
finite differences for its tangents."""
import numpy as np

import synth
from oracle import bloch, model, metrics, slice_profile as sp


def _seq(seed=1, ntr_fills=3, ny=8, inversion=True):
    return synth.make_sequence(6, ny, ntr_fills, 7.8, 3.9, seed=seed, extra_trs=3, inversion=inversion)


def _tissue(nv, seed):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(200), np.log(3000), nv)), np.exp(rng.uniform(np.log(20), np.log(300), nv))


def test_one_isochromat_is_the_hard_pulse_model():
    """At the slice centre (one isochromat, no gradient phase) the sub-pulses compose to
    one rotation by the nominal flip: the hard-pulse recursion, for any sub-step count."""
    seq = _seq()
    t1, t2 = _tissue(5, 2)
    ref = bloch.simulate(seq, t1, t2)
    for n_sub in (1, 4, 16):
        got = sp.simulate(seq, t1, t2, sp.SliceProfile(n_iso=1, n_sub=n_sub))
        for key in ("m", "dm_dlnT1", "dm_dlnT2"):
            assert metrics.relerr(got[key], ref[key]) < 1e-12, (n_sub, key)


def test_mean_x_component_vanishes():
    seq = _seq(seed=3)
    t1, t2 = _tissue(4, 5)
    got = sp.simulate(seq, t1, t2, sp.SliceProfile(n_iso=16, n_sub=12, tbw=3.0))
    assert np.abs(got["mx_mean"]).max() < 1e-12 * np.abs(got["m"]).max()
    assert np.abs(got["m"].real).max() < 1e-12 * np.abs(got["m"]).max()


def test_small_tip_profile_is_the_envelope_fourier_transform():
    """One 0.5 degree pulse from equilibrium, relaxation switched off: to first order in
    the flip, isochromat u ends with i alpha sum_s w_s exp(i beta_u (n_sub/2 - s)) --
    the Fourier transform of the Gaussian envelope (the small-tip approximation)."""
    alpha = np.deg2rad(0.5)
    seq = synth.Sequence(nx=1, ny=1, nkx=1, tr_ms=7.8, te_ms=3.9, flip_rad=np.array([alpha]),
                         ky=np.array([0]), inversion=False, alternate_phase=False)
    p = sp.SliceProfile(n_iso=24, n_sub=20, sigma=0.18, tbw=5.0, extent=2.5)
    got = sp.simulate(seq, np.array([1e12]), np.array([1e12]), p, per_iso=True)["m_iso"][0, :, 0]
    w, beta = sp.weights(p), sp.gradient_phase(p)
    s = np.arange(p.n_sub)
    pred = 1j * alpha * (w[None, :] * np.exp(1j * beta[:, None] * (p.n_sub / 2 - s[None, :]))).sum(1)
    assert metrics.relerr(got, pred) < 1e-3
    # the centre of the slice sees the full flip, the edges (|u| ~ 1.2 slices) much less
    assert abs(got[p.n_iso // 2]) > 0.95 * alpha and abs(got[0]) < 0.2 * alpha


def test_tangents_match_central_differences():
    seq = _seq(seed=4)
    t1, t2 = _tissue(3, 6)
    p = sp.SliceProfile(n_iso=8, n_sub=6)
    got = sp.simulate(seq, t1, t2, p)
    h = 1e-6
    for key, (a, b) in (("dm_dlnT1", (t1 * np.exp(h), t1 * np.exp(-h))), ("dm_dlnT2", (t2 * np.exp(h), t2 * np.exp(-h)))):
        if key == "dm_dlnT1":
            fd = (sp.simulate(seq, a, t2, p)["m"] - sp.simulate(seq, b, t2, p)["m"]) / (2 * h)
        else:
            fd = (sp.simulate(seq, t1, a, p)["m"] - sp.simulate(seq, t1, b, p)["m"]) / (2 * h)
        assert metrics.relerr(got[key], fd) < 1e-6, key


def test_slice_profile_lowers_the_signal_and_linearize_uses_it():
    """Off-centre isochromats see smaller flips, so the slice average differs from the
    hard-pulse signal; model.linearize(profile=...) carries the slice model through."""
    seq = _seq(seed=5)
    t1, t2 = _tissue(4, 7)
    alpha = np.stack([np.log(t1), np.log(t2), np.ones(4), np.zeros(4)])
    p = sp.SliceProfile()
    lin = model.linearize(seq, alpha, profile=p)
    ref = sp.simulate(seq, t1, t2, p)
    assert metrics.relerr(lin.m, ref["m"]) == 0.0
    hard = bloch.simulate(seq, t1, t2)["m"]
    assert metrics.relerr(lin.m, hard) > 0.05
