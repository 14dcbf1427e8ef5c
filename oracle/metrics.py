"""Error metrics (Results, "Numerical Brain Phantom"; Table 3).

The paper reports NRMSE without a formula; the reading used here is the
normwise relative error over the masked voxels of one map:
NRMSE(x, x*) = ||x - x*||_2 / ||x*||_2.  MAPE is the mean of |x - x*| / |x*|.
"""
from __future__ import annotations

import numpy as np


def nrmse(est, ref, mask=None) -> float:
    est = np.asarray(est).ravel()
    ref = np.asarray(ref).ravel()
    if mask is not None:
        m = np.asarray(mask, bool).ravel()
        est, ref = est[m], ref[m]
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(est - ref) / den) if den > 0 else float(np.linalg.norm(est - ref))


def mape(est, ref, mask=None) -> float:
    est = np.asarray(est).ravel()
    ref = np.asarray(ref).ravel()
    if mask is not None:
        m = np.asarray(mask, bool).ravel()
        est, ref = est[m], ref[m]
    return float(100.0 * np.mean(np.abs(est - ref) / np.abs(ref)))


def relerr(x, ref) -> float:
    """Normwise relative error ||x - ref|| / ||ref|| over a whole output array."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / den) if den > 0 else float(np.linalg.norm(x - ref))


def stored_matrix_bytes(nv: int, npar: int = 4, nt: int | None = None):
    """Bytes needed to store M (Nt x Nv complex), J (Nt x N complex) and H (N x N real)
    in float64 (Theory, "Computational Challenges"; Table 1), with N = npar * nv and,
    by default, Nt = N."""
    n = npar * nv
    nt = n if nt is None else nt
    return 2 * nv * nt * 8, 2 * n * nt * 8, n * n * 8
