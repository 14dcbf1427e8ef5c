"""Volumetric signal sum with Cartesian gradient encoding (Theory, Eqs. 1-2, s = M rho).

The demodulated signal of TR n, readout sample kx, is the discretised volume
integral of rho * m weighted by the encoding phase of the voxel position:

    s[n, kx] = sum_j q_j[n] * exp(-2 pi i (kx * ix_j / nx + ky(n) * iy_j / ny)),

with q_j[n] = rho_j m_j[n] (Delta_V = 1), voxel j = iy * nx + ix, and the
magnetisation held at its echo value across the readout (the separable reading
of the model; no decay or off-resonance phase during the readout).  kx runs over
k - nkx//2 for k = 0..nkx-1.  The adjoint maps k-space back to per-voxel time
courses: W[n, j] = sum_kx conj(exp(-i k.r_j)) w[n, kx].

This is the definition written out: one dense [nkx, nv] phase matrix per distinct
ky value, applied to every TR that samples that ky.  No FFT and no separable
x/y factorisation.
"""
from __future__ import annotations

import numpy as np


def kx_values(nkx: int) -> np.ndarray:
    return np.arange(nkx) - nkx // 2


def voxel_coords(nx: int, ny: int):
    j = np.arange(nx * ny)
    return j % nx, j // nx  # ix, iy


def phase_matrix(seq, ky: int, voxels=None) -> np.ndarray:
    """E[kx, j] = exp(-2 pi i (kx ix_j / nx + ky iy_j / ny)), shape [nkx, nv] (or only the
    columns of the listed voxels)."""
    ix, iy = voxel_coords(seq.nx, seq.ny)
    if voxels is not None:
        ix, iy = ix[voxels], iy[voxels]
    kx = kx_values(seq.nkx)
    ph = kx[:, None] * ix[None, :] / seq.nx + ky * iy[None, :] / seq.ny
    return np.exp(-2j * np.pi * ph)


def encode(seq, q: np.ndarray, rows=None) -> np.ndarray:
    """s[n] = E_{ky(n)} q[n] for every TR n.  With ``rows``, only those TRs are encoded
    and q[i] holds the voxel values of TR rows[i]."""
    rows = np.arange(seq.ntr) if rows is None else np.asarray(rows)
    s = np.zeros((rows.shape[0], seq.nkx), np.complex128)
    ky = np.asarray(seq.ky)[rows]
    for u in np.unique(ky):
        sel = np.nonzero(ky == u)[0]
        e = phase_matrix(seq, int(u))
        s[sel] = q[sel] @ e.T
    return s


def encode_adjoint(seq, w: np.ndarray, voxels=None) -> np.ndarray:
    """W[n] = E_{ky(n)}^H w[n], shape [ntr, nv] (or [ntr, len(voxels)])."""
    nv = seq.nv if voxels is None else len(voxels)
    out = np.zeros((seq.ntr, nv), np.complex128)
    ky = np.asarray(seq.ky)
    for u in np.unique(ky):
        sel = np.nonzero(ky == u)[0]
        e = phase_matrix(seq, int(u), voxels)
        out[sel] = w[sel] @ np.conj(e)
    return out
