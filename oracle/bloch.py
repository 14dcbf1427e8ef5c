"""Hard-pulse Bloch recursion with forward-mode derivatives (Supporting Information S2).

Per TR n of the balanced gradient-echo sequence (Methods, "Pulse Sequence"):

1. RF rotation.  The rotation vector is a = alpha_n * B1 * (-cos psi_n, sin psi_n, 0)
   (S2: a = gamma dt [-|B1| Re RF, |B1| Im RF, GR.r + dB0/gamma] with the RF of
   amplitude alpha_n/(gamma dt) and phase psi_n; the gradient and off-resonance
   terms vanish because the encoding phase is applied at the echo (Eq. 1-2 with
   e^{-i k.r}) and dB0 = 0 (Methods, "Reconstructions")).  k = a/|a|,
   theta = |a|, and m_rot follows Rodrigues' formula (S2, Eq. m_rot).
2. Decay and regrowth over TE (S2, Eq. m_decay): m <- m o [E2, E2, E1] + [0, 0, 1-E1].
3. Sample m_x + i m_y (the transverse magnetisation at the echo, Theory Eq. 1).
4. Decay and regrowth over TR - TE.

m_0 = [0, 0, 1] (S2), followed by an ideal non-selective inversion when the
sequence has one (Methods, "Pulse Sequence"): m_0 = [0, 0, -1].

Derivatives follow S2's forward-mode recipe: the rotation does not depend on T1
or T2, so d m_rot = R d m (S2, Eq. dm_rot); differentiating the decay step gives
the extra source terms.  We differentiate with respect to ln T1 and ln T2 (the
paper's log scaling, Methods) -- i.e. T1 times S2's d/dT1 form -- and with
respect to B1, for which the rotation contributes (dR/dtheta) m * alpha_n.

Everything is float64, or complex128 when a caller runs the complex-step check.
"""
from __future__ import annotations

import numpy as np


def rf_phase(seq) -> np.ndarray:
    """RF phase psi_n per TR: 0, pi, 0, pi, ... when the phase alternates, else 0."""
    n = np.arange(seq.ntr)
    return np.pi * (n % 2) if seq.alternate_phase else np.zeros(seq.ntr)


def _cross(k, m):
    """k x m for a fixed 3-vector k and a [3, nv] array m."""
    return np.stack([k[1] * m[2] - k[2] * m[1],
                     k[2] * m[0] - k[0] * m[2],
                     k[0] * m[1] - k[1] * m[0]])


def _dot(k, m):
    return k[0] * m[0] + k[1] * m[1] + k[2] * m[2]


def rodrigues(m, k, theta):
    """m_rot = cos(theta) m + sin(theta) (k x m) + (1 - cos(theta)) (k.m) k   (S2)."""
    c, s = np.cos(theta), np.sin(theta)
    kd = _dot(k, m)
    return c * m + s * _cross(k, m) + (1.0 - c) * kd * k[:, None]


def rodrigues_dtheta(m, k, theta):
    """d m_rot / d theta for fixed axis k."""
    c, s = np.cos(theta), np.sin(theta)
    kd = _dot(k, m)
    return -s * m + c * _cross(k, m) + s * kd * k[:, None]


def relax(m, e1, e2):
    """S2 decay/regrowth: m o [E2, E2, E1] + [0, 0, 1 - E1]."""
    return np.stack([m[0] * e2, m[1] * e2, m[2] * e1 + (1.0 - e1)])


def scale(dm, e1, e2):
    """The linear part of the decay step, dm o [E2, E2, E1], which carries a tangent."""
    return np.stack([dm[0] * e2, dm[1] * e2, dm[2] * e1])


def simulate(seq, t1_ms, t2_ms, b1=None, tangents=True, b1_tangent=False, rows=None):
    """Simulate the transverse magnetisation at every echo.

    Parameters are flat arrays over voxels (length nv).  ``t1_ms``/``t2_ms`` may
    be complex (complex-step checks).  Returns a dict with ``m`` [ntr, nv] and,
    when requested, ``dm_dlnT1``, ``dm_dlnT2`` and ``dm_dB1`` of the same shape,
    plus the full 3-component state ``mxyz`` at every echo [ntr, 3, nv].  With
    ``rows`` (sorted TR indices) only those echoes are kept, in that order.
    """
    t1 = np.asarray(t1_ms)
    t2 = np.asarray(t2_ms)
    nv = t1.shape[0]
    dtype = np.result_type(t1.dtype, t2.dtype, np.float64)
    if b1 is None:
        b1 = np.ones(nv)
    b1 = np.asarray(b1)
    dtype = np.result_type(dtype, b1.dtype)
    te, tr = float(seq.te_ms), float(seq.tr_ms)

    # per-voxel relaxation factors over TE and over TR - TE
    e1a, e2a = np.exp(-te / t1), np.exp(-te / t2)
    e1b, e2b = np.exp(-(tr - te) / t1), np.exp(-(tr - te) / t2)

    m = np.zeros((3, nv), dtype)
    m[2] = -1.0 if seq.inversion else 1.0
    d1 = np.zeros((3, nv), dtype)
    d2 = np.zeros((3, nv), dtype)
    db = np.zeros((3, nv), dtype)

    keep = np.arange(seq.ntr) if rows is None else np.asarray(rows)
    slot = np.full(seq.ntr, -1)
    slot[keep] = np.arange(keep.shape[0])
    out_m = np.zeros((keep.shape[0], nv), np.result_type(dtype, np.complex128))
    out_xyz = np.zeros((keep.shape[0], 3, nv), dtype)
    if tangents:
        out_d1 = np.zeros_like(out_m)
        out_d2 = np.zeros_like(out_m)
    if b1_tangent:
        out_db = np.zeros_like(out_m)

    psi = rf_phase(seq)

    def decay(m, d1, d2, db, e1, e2, dt):
        # d/dlnT1 of [0,0,E1 m_z + 1 - E1] is (dt/T1) E1 (m_z - 1); d/dlnT2 of E2 m_xy is (dt/T2) E2 m_xy
        n1 = scale(d1, e1, e2)
        n1[2] = n1[2] + (dt / t1) * e1 * (m[2] - 1.0)
        n2 = scale(d2, e1, e2)
        n2[0] = n2[0] + (dt / t2) * e2 * m[0]
        n2[1] = n2[1] + (dt / t2) * e2 * m[1]
        return relax(m, e1, e2), n1, n2, scale(db, e1, e2)

    for n in range(seq.ntr):
        amp = float(seq.flip_rad[n])
        if amp != 0.0:
            k = np.array([-np.cos(psi[n]), np.sin(psi[n]), 0.0])
            theta = amp * b1
            if b1_tangent:
                db = rodrigues(db, k, theta) + amp * rodrigues_dtheta(m, k, theta)
            d1 = rodrigues(d1, k, theta)
            d2 = rodrigues(d2, k, theta)
            m = rodrigues(m, k, theta)
        m, d1, d2, db = decay(m, d1, d2, db, e1a, e2a, te)
        i = slot[n]
        if i >= 0:
            out_m[i] = m[0] + 1j * m[1]
            out_xyz[i] = m
            if tangents:
                out_d1[i] = d1[0] + 1j * d1[1]
                out_d2[i] = d2[0] + 1j * d2[1]
            if b1_tangent:
                out_db[i] = db[0] + 1j * db[1]
        m, d1, d2, db = decay(m, d1, d2, db, e1b, e2b, tr - te)

    res = {"m": out_m, "mxyz": out_xyz}
    if tangents:
        res["dm_dlnT1"] = out_d1
        res["dm_dlnT2"] = out_d2
    if b1_tangent:
        res["dm_dB1"] = out_db
    return res
