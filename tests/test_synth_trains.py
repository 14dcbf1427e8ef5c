"""The seeded flip-angle trains of the supporting information (host logic, no GPU).

* constant per k-space fill (S3): one value per fill, different between fills, inside
  the requested range;
* connected sine-squared waves (S1): zero at the start of every fill, the peak where the
  fill samples the central line ky = 0, peaks inside [lo_frac, 1] x max.
"""
import numpy as np

import synth


def test_constant_flip_train():
    ny, fills = 12, 6
    f = np.rad2deg(synth.constant_flip_train(fills * ny + 5, ny, seed=3, lo_deg=10, hi_deg=60))
    assert f.shape == (fills * ny + 5,)
    per = f[: fills * ny].reshape(fills, ny)
    assert np.all(per == per[:, :1])
    assert len(np.unique(per[:, 0])) == fills
    assert np.all((f >= 10) & (f <= 60))
    assert np.all(f[fills * ny:] == f[fills * ny])  # the partial last fill keeps one value


def test_sine_squared_train_peaks_at_the_central_line():
    ny, fills = 16, 5
    seq = synth.make_sequence(8, ny, fills, 7.8, 3.9, seed=4, train="sine2", max_deg=60)
    f = np.rad2deg(np.asarray(seq.flip_rad)).reshape(fills, ny)
    ky = np.asarray(seq.ky).reshape(fills, ny)
    assert np.all(f[:, 0] == 0)
    peak = np.argmax(f, axis=1)
    assert np.all(ky[np.arange(fills), peak] == 0)
    assert np.all((f.max(1) >= 0.3 * 60 - 1e-4) & (f.max(1) <= 60 + 1e-4))
    # sin^2 shape: alpha_n / peak = sin^2(pi n / ny) within a fill (float32 rounding)
    ratio = f / f.max(1, keepdims=True)
    assert np.allclose(ratio, np.sin(np.pi * np.arange(ny) / ny)[None] ** 2, atol=1e-5)


def test_named_shapes():
    s, ph = synth.config("const112x88")
    assert (s.nx, s.ny, s.ntr, s.tr_ms, s.te_ms) == (112, 88, 1408, 5.6, 2.8)
    assert ph.t1_ms.shape == (88, 112) and 0.3 < ph.support.mean() < 0.7
    s, ph = synth.config("brain224_1792")
    assert (s.nx, s.ny, s.ntr) == (224, 224, 1792)
    # the default workload is unchanged by the new options
    s0, _ = synth.config("brain224")
    assert s0.ntr == 1120 and np.isclose(np.rad2deg(np.asarray(s0.flip_rad)).max(), 60.0, atol=1e-4)
