"""Slice-profile Bloch recursion (Methods, "Pulse Sequence": every RF pulse has a Gaussian
envelope; "Reconstructions": the Bloch solver takes the slice profile into account).

Test infrastructure: only tests, the smoke check and the benchmark's CPU baseline use
this module; the product path never does.

The paper names the effect but gives no pulse parameters.  Readings (all stated, all
options of SliceProfile):

* Across the slice, n_iso isochromats sit at u_k = extent * ((k + 1/2)/n_iso - 1/2),
  k < n_iso, in units of the nominal slice thickness (symmetric about the slice centre).
* The RF pulse is n_sub hard sub-pulses with Gaussian weights
  w_s = exp(-((s + 1/2)/n_sub - 1/2)^2 / (2 sigma^2)) normalised to sum to 1, so the
  slice centre turns by the nominal flip alpha_n B1.
* The slice-select gradient advances the phase of isochromat k by
  beta_k = 2 pi tbw u_k / n_sub per sub-step (tbw: the envelope's time-bandwidth
  product; a unit slice spans the pulse's bandwidth).  The sequence is balanced: a
  pre-winder (-n_sub/2 beta_k) before and a rewinder (-n_sub/2 beta_k) after the pulse,
  so the net gradient phase over a TR is zero and a zero flip changes nothing.
* No relaxation during the pulse (short against TR).
* Sub-step s: the RF rotation of the hard-pulse model (Rodrigues about the TR's RF axis)
  by theta_s = alpha_n B1 w_s, then precession about z by beta_k.
* The rest of the TR as in the hard-pulse model, per isochromat; the echo of the voxel
  is the mean of m_x + i m_y over the isochromats (the volume integral over the slice).

Mirror symmetry (u -> -u flips the precession, and the x-flip commutes with rotations
about the x axis) makes the mean m_x vanish: the voxel signal stays i * mean(m_y).

With n_iso = 1 (u = 0) the sub-steps compose to one rotation by alpha_n B1: the
hard-pulse model.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import bloch


@dataclass
class SliceProfile:
    n_iso: int = 32        # isochromats across the slice
    n_sub: int = 16        # RF sub-steps
    sigma: float = 0.2     # Gaussian width as a fraction of the pulse length
    tbw: float = 4.0       # time-bandwidth product
    extent: float = 2.0    # isochromats span this many slice thicknesses


def positions(p: SliceProfile) -> np.ndarray:
    k = np.arange(p.n_iso)
    return p.extent * ((k + 0.5) / p.n_iso - 0.5)


def weights(p: SliceProfile) -> np.ndarray:
    s = np.arange(p.n_sub)
    w = np.exp(-(((s + 0.5) / p.n_sub - 0.5) ** 2) / (2.0 * p.sigma ** 2))
    return w / w.sum()


def gradient_phase(p: SliceProfile) -> np.ndarray:
    """beta_k, the phase one sub-step of the slice-select gradient adds to isochromat k."""
    return 2.0 * np.pi * p.tbw * positions(p) / p.n_sub


def precess(m, beta):
    """Rotation about z by beta (per column): m_x + i m_y -> e^{i beta} (m_x + i m_y)."""
    c, s = np.cos(beta), np.sin(beta)
    return np.stack([c * m[0] - s * m[1], s * m[0] + c * m[1], m[2]])


def simulate(seq, t1_ms, t2_ms, profile: SliceProfile, b1=None, rows=None, per_iso=False):
    """Echo magnetisation averaged over the slice and its ln T1 / ln T2 tangents.

    Returns ``m``, ``dm_dlnT1``, ``dm_dlnT2`` ([ntr, nv] complex) and ``mx_mean`` (the mean
    x component, [ntr, nv], zero by symmetry); with ``per_iso`` also ``m_iso``
    ([ntr, n_iso, nv] complex, every isochromat's echo).  Every isochromat runs the hard-pulse
    recursion of oracle.bloch with the RF step replaced by the sub-stepped pulse.
    """
    t1 = np.asarray(t1_ms, np.float64)
    t2 = np.asarray(t2_ms, np.float64)
    nv = t1.shape[0]
    K = profile.n_iso
    b1v = np.ones(nv) if b1 is None else np.asarray(b1, np.float64)
    # isochromat-major columns: column k * nv + j is isochromat k of voxel j
    T1 = np.tile(t1, K)
    T2 = np.tile(t2, K)
    B1 = np.tile(b1v, K)
    beta = np.repeat(gradient_phase(profile), nv)
    w = weights(profile)
    half = profile.n_sub / 2.0
    te, tr = float(seq.te_ms), float(seq.tr_ms)
    e1a, e2a = np.exp(-te / T1), np.exp(-te / T2)
    e1b, e2b = np.exp(-(tr - te) / T1), np.exp(-(tr - te) / T2)

    m = np.zeros((3, K * nv))
    m[2] = -1.0 if seq.inversion else 1.0
    d1 = np.zeros((3, K * nv))
    d2 = np.zeros((3, K * nv))

    keep = np.arange(seq.ntr) if rows is None else np.asarray(rows)
    slot = np.full(seq.ntr, -1)
    slot[keep] = np.arange(keep.shape[0])
    out_m = np.zeros((keep.shape[0], nv), np.complex128)
    out_d1 = np.zeros_like(out_m)
    out_d2 = np.zeros_like(out_m)
    out_mx = np.zeros((keep.shape[0], nv))
    out_iso = np.zeros((keep.shape[0], K, nv), np.complex128) if per_iso else None
    psi = bloch.rf_phase(seq)

    def decay(m, d1, d2, e1, e2, dt):
        n1 = bloch.scale(d1, e1, e2)
        n1[2] = n1[2] + (dt / T1) * e1 * (m[2] - 1.0)
        n2 = bloch.scale(d2, e1, e2)
        n2[0] = n2[0] + (dt / T2) * e2 * m[0]
        n2[1] = n2[1] + (dt / T2) * e2 * m[1]
        return bloch.relax(m, e1, e2), n1, n2

    def mean(x):
        return x.reshape(K, nv).mean(axis=0)

    for n in range(seq.ntr):
        amp = float(seq.flip_rad[n])
        if amp != 0.0:
            k = np.array([-np.cos(psi[n]), np.sin(psi[n]), 0.0])
            # balanced slice-select gradient around the sub-stepped pulse
            m, d1, d2 = precess(m, -half * beta), precess(d1, -half * beta), precess(d2, -half * beta)
            for s in range(profile.n_sub):
                theta = amp * w[s] * B1
                m, d1, d2 = bloch.rodrigues(m, k, theta), bloch.rodrigues(d1, k, theta), bloch.rodrigues(d2, k, theta)
                m, d1, d2 = precess(m, beta), precess(d1, beta), precess(d2, beta)
            m, d1, d2 = precess(m, -half * beta), precess(d1, -half * beta), precess(d2, -half * beta)
        m, d1, d2 = decay(m, d1, d2, e1a, e2a, te)
        i = slot[n]
        if i >= 0:
            out_m[i] = mean(m[0]) + 1j * mean(m[1])
            out_d1[i] = mean(d1[0]) + 1j * mean(d1[1])
            out_d2[i] = mean(d2[0]) + 1j * mean(d2[1])
            out_mx[i] = mean(m[0])
            if per_iso:
                out_iso[i] = (m[0] + 1j * m[1]).reshape(K, nv)
        m, d1, d2 = decay(m, d1, d2, e1b, e2b, tr - te)
    res = {"m": out_m, "dm_dlnT1": out_d1, "dm_dlnT2": out_d2, "mx_mean": out_mx}
    if per_iso:
        res["m_iso"] = out_iso
    return res
