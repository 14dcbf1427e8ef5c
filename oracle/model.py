"""Signal, residual, gradient and Jacobian products (Theory, Algorithms 2 and 4, Eq. 4).

Parameter vector (Theory, "MR-STAT Framework"): alpha in R^N with N = Np * Nv,
parameter-major, so alpha[k, j] belongs to voxel j:

    k = 0: ln(T1 / ms), k = 1: ln(T2 / ms)   (log scaling, Methods "Reconstructions")
    k = 2: Re rho,      k = 3: Im rho         (complex proton density, Theory)
    k = 4: B1 (only when the transmit field is estimated)

The signal Jacobian is J_s = ds/dalpha.  The paper's J = dr/dalpha = -J_s
(Theory, "Computing the gradient g"), so the gradient of f = 1/2 ||d - s||^2 is
g = Re(J^H r) = -Re(J_s^H r).  Because voxels evolve independently, the column
of J_s for a parameter of voxel j only involves q_j = rho_j m_j (Theory,
"Computing the gradient g"):

    d q_j / d lnT1 = rho_j dm_j/dlnT1,  d q_j / d lnT2 = rho_j dm_j/dlnT2,
    d q_j / d Re rho = m_j,             d q_j / d Im rho = i m_j,
    d q_j / d B1 = rho_j dm_j/dB1.

So J_s v = encode(sum_k v_k dq/dalpha_k) and Re(J_s^H w)_k,j =
Re sum_n conj(dq_j[n]/dalpha_k) W[n, j] with W = encode_adjoint(w) (Algorithm 4:
one inner product of each partial-derivative vector with the k-space vector).
A mask (Methods: voxels without significant proton density are excluded) removes
voxels from every product: their q and their gradient entries are zero.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import bloch, encoding, slice_profile


@dataclass
class Linearization:
    seq: object
    alpha: np.ndarray       # [Np, nv]
    b1: np.ndarray          # [nv]
    mask: np.ndarray        # [nv] bool
    m: np.ndarray           # [ntr, nv]
    dm1: np.ndarray         # dm/dlnT1
    dm2: np.ndarray         # dm/dlnT2
    dmb: np.ndarray | None  # dm/dB1 when B1 is a parameter

    @property
    def rho(self):
        return self.alpha[2] + 1j * self.alpha[3]

    @property
    def npar(self):
        return self.alpha.shape[0]


def linearize(seq, alpha, b1=None, mask=None, profile=None) -> Linearization:
    """Simulate m and its tangents at alpha (Algorithm 2 step 1 plus S2 derivatives);
    with a slice profile (oracle.slice_profile.SliceProfile) the slice-averaged model."""
    alpha = np.asarray(alpha, np.float64)
    nv = alpha.shape[1]
    estimate_b1 = alpha.shape[0] == 5
    if estimate_b1:
        b1 = alpha[4]
    elif b1 is None:
        b1 = np.ones(nv)
    mask = np.ones(nv, bool) if mask is None else np.asarray(mask, bool)
    if profile is not None:
        if estimate_b1:
            raise ValueError("the slice-profile model has no B1 tangent")
        sim = slice_profile.simulate(seq, np.exp(alpha[0]), np.exp(alpha[1]), profile, b1)
    else:
        sim = bloch.simulate(seq, np.exp(alpha[0]), np.exp(alpha[1]), b1, tangents=True,
                             b1_tangent=estimate_b1)
    return Linearization(seq, alpha, np.asarray(b1, np.float64), mask, sim["m"],
                         sim["dm_dlnT1"], sim["dm_dlnT2"], sim.get("dm_dB1"))


def signal(lin: Linearization) -> np.ndarray:
    """s = M rho = sum_j rho_j m_j, encoded (Algorithm 2)."""
    q = lin.m * (lin.rho * lin.mask)[None, :]
    return encoding.encode(lin.seq, q)


def forward(seq, alpha, b1=None, mask=None, profile=None) -> np.ndarray:
    return signal(linearize(seq, alpha, b1, mask, profile))


def objective(d, s) -> float:
    """f = 1/2 ||d - s||_2^2 (Theory)."""
    r = d - s
    return 0.5 * float(np.vdot(r, r).real)


def jvp(lin: Linearization, v) -> np.ndarray:
    """J_s v: encode(rho (v1 dm1 + v2 dm2 [+ v5 dmb]) + (v3 + i v4) m)."""
    v = np.asarray(v, np.float64)
    rho = lin.rho
    q = rho[None, :] * (v[0][None, :] * lin.dm1 + v[1][None, :] * lin.dm2)
    q = q + (v[2] + 1j * v[3])[None, :] * lin.m
    if lin.npar == 5:
        q = q + rho[None, :] * v[4][None, :] * lin.dmb
    q = q * lin.mask[None, :]
    return encoding.encode(lin.seq, q)


def jhw(lin: Linearization, w) -> np.ndarray:
    """Re(J_s^H w), shape [Np, nv] (Algorithm 4 with the sign of J_s)."""
    W = encoding.encode_adjoint(lin.seq, np.asarray(w, np.complex128))
    rho = lin.rho
    g = np.zeros((lin.npar, lin.alpha.shape[1]))
    g[0] = np.real(np.sum(np.conj(rho[None, :] * lin.dm1) * W, axis=0))
    g[1] = np.real(np.sum(np.conj(rho[None, :] * lin.dm2) * W, axis=0))
    g[2] = np.real(np.sum(np.conj(lin.m) * W, axis=0))
    g[3] = np.real(np.sum(np.conj(1j * lin.m) * W, axis=0))
    if lin.npar == 5:
        g[4] = np.real(np.sum(np.conj(rho[None, :] * lin.dmb) * W, axis=0))
    return g * lin.mask[None, :]


def gradient(lin: Linearization, d) -> np.ndarray:
    """g = grad f = Re(J^H r) with J = -J_s and r = d - s."""
    return -jhw(lin, d - signal(lin))


def gauss_newton_product(lin: Linearization, v) -> np.ndarray:
    """Re(J^H J) v = Re(J_s^H (J_s v)) (Eq. 4: first y = J v, then Re(J^H y))."""
    return jhw(lin, jvp(lin, v))


def project_onto_basis(lin: Linearization, U) -> Linearization:
    """Low-rank model: every time course replaced by its orthogonal projection onto the
    columns of the real time basis U [ntr, R] (m_j ~ U U^T m_j, and the same for each
    tangent).  The basis comes from an SVD of simulated time courses, the compression the
    paper's comparison pipeline applies to its dictionary (Methods, "Numerical Brain
    Simulation": rank-5 SVD compression); here it compresses the model itself."""
    U = np.asarray(U, np.float64)

    def proj(x):
        return U @ (U.T @ x)

    return Linearization(lin.seq, lin.alpha, lin.b1, lin.mask, proj(lin.m), proj(lin.dm1), proj(lin.dm2),
                         None if lin.dmb is None else proj(lin.dmb))


def time_basis(seq, t1_ms, t2_ms, rank, b1=None):
    """Leading left singular vectors of the simulated training time courses [m_y, dm_y/dlnT1,
    dm_y/dlnT2] (columns over the training samples); returns (U [ntr, rank], singular values)."""
    from . import bloch
    sim = bloch.simulate(seq, np.asarray(t1_ms), np.asarray(t2_ms), b1)
    Y = np.concatenate([sim["m"].imag, sim["dm_dlnT1"].imag, sim["dm_dlnT2"].imag], axis=1)
    u, s, _ = np.linalg.svd(Y, full_matrices=False)
    return u[:, :rank], s[:rank]
