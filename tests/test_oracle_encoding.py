"""Pins of the oracle's volumetric encoding (Theory, Eqs. 1-2) to numpy.fft,
to an explicit quadruple loop, and to Parseval's identity."""
import numpy as np

import synth
from oracle import encoding


def test_encode_equals_shifted_fft2_for_time_constant_images():
    """If q does not change within a fill, the fill's k-space is fftshift(fft2(q))."""
    nx, ny = 8, 6
    seq = synth.make_sequence(nx, ny, 2, 7.8, 3.9, seed=1)
    rng = np.random.default_rng(0)
    img = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    q = np.tile(img.ravel(), (seq.ntr, 1))
    s = encoding.encode(seq, q)
    ref = np.fft.fftshift(np.fft.fft2(img))
    for n in range(seq.ntr):
        assert np.allclose(s[n], ref[seq.ky[n] + ny // 2], atol=1e-12)


def test_encode_equals_explicit_sum_on_a_tiny_grid():
    """Odd sizes, nkx != nx, arbitrary ky order, time-varying q: direct loops."""
    nx, ny, nkx = 3, 2, 4
    ky = np.array([0, -1, 0, -1, -1], np.int32)
    seq = synth.Sequence(nx=nx, ny=ny, nkx=nkx, tr_ms=5, te_ms=2.5,
                         flip_rad=np.zeros(5), ky=ky)
    rng = np.random.default_rng(5)
    q = rng.standard_normal((5, nx * ny)) + 1j * rng.standard_normal((5, nx * ny))
    s = encoding.encode(seq, q)
    for n in range(5):
        for k in range(nkx):
            kx = k - nkx // 2
            acc = 0j
            for iy in range(ny):
                for ix in range(nx):
                    acc += q[n, iy * nx + ix] * np.exp(-2j * np.pi * (kx * ix / nx + ky[n] * iy / ny))
            assert abs(s[n, k] - acc) < 1e-13


def test_adjoint_identity_and_parseval():
    nx, ny = 10, 7
    seq = synth.make_sequence(nx, ny, 3, 7.8, 3.9, seed=2, extra_trs=3)
    rng = np.random.default_rng(9)
    q = rng.standard_normal((seq.ntr, seq.nv)) + 1j * rng.standard_normal((seq.ntr, seq.nv))
    w = rng.standard_normal((seq.ntr, seq.nkx)) + 1j * rng.standard_normal((seq.ntr, seq.nkx))
    lhs = np.vdot(encoding.encode(seq, q), w)
    rhs = np.vdot(q, encoding.encode_adjoint(seq, w))
    assert abs(lhs - rhs) / abs(lhs) < 1e-13
    # Parseval along the readout (nkx = nx): each TR's energy is nx * ||sum_iy ...||^2;
    # for q supported on one row iy, |s[n]|^2 summed over kx equals nx * ||q[n]||^2.
    qr = np.zeros_like(q)
    qr[:, 3 * nx:4 * nx] = q[:, 3 * nx:4 * nx]
    s = encoding.encode(seq, qr)
    assert np.allclose((np.abs(s) ** 2).sum(1), nx * (np.abs(qr) ** 2).sum(1), rtol=1e-12)


def test_table1_memory_formulas():
    from oracle import metrics
    path = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                      "table1_matrix_sizes.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for side, nv, m_gb, j_gb, h_gb in rows:
        assert int(side) ** 2 == int(nv)
        m, j, h = metrics.stored_matrix_bytes(int(nv))
        assert (m, j, h) == (int(m_gb) << 30, int(j_gb) << 30, int(h_gb) << 30)
