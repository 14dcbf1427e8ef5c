"""Inexact Gauss-Newton reconstruction (Algorithm 6) with a trust region.

Pieces, in the order the paper uses them (Methods, "Reconstructions"):

* ``cgls_rho``: the initial proton density solves M(alpha_0) rho = d in the
  least-squares sense with a Krylov solver (the paper uses LSQR; CGLS is the
  algebraically equivalent normal-equations form).  T1 = 1000 ms, T2 = 100 ms,
  B1 = 1 for alpha_0.  The unknowns are (Re rho, Im rho) and the operator is the
  rho-block of J_s, which is exactly linear in rho.
* ``ls_rho``: the same least-squares solution computed exactly (minimum norm) from the
  dense matrix M(alpha_0) by an SVD-based solver -- the plain definition of what the
  Krylov solver approximates.
* ``draw_mask``: voxels whose initial |rho| exceeds a fraction of the maximum.
* ``steihaug_cg``: truncated CG on the Gauss-Newton model
  m(p) = f + g.p + 1/2 p.B p with B = Re(J^H J) (Eq. 4) inside ||p|| <= Delta,
  following Steihaug / Nocedal & Wright Algorithm 7.2: stop on negative
  curvature or on the trust boundary (then move to the boundary along the
  current direction), on a relative residual tolerance, or after a fixed number
  of inner iterations (the "inexact" limit of Algorithm 6).
* ``gauss_newton``: the outer loop of Algorithm 6 with the trust-region radius
  update of Nocedal & Wright Algorithm 4.1, and bound constraints handled by
  reflecting a step that leaves the feasible box back inside it (Methods; a
  simplified form of the Coleman-Li reflection).

Readings where the paper is silent: Delta_0 = 0.1 ||alpha_0|| over masked
parameters; shrink by 1/4 when the ratio < 1/4, double (up to Delta_max) when
the ratio > 3/4 and the step reached the boundary; accept when ratio > eta =
1e-4; the predicted reduction is the CG model's; bounds T1 in [50, 6000] ms,
T2 in [5, 3000] ms, B1 in [0.5, 1.5]; rho unbounded.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import encoding, model


# ----------------------------------------------------------------------------
# Initial proton density and mask
# ----------------------------------------------------------------------------
def cgls_rho(lin: model.Linearization, d, iters: int = 50):
    """Least-squares rho for fixed (T1, T2, B1): min ||d - J_rho x|| by CGLS.

    x = (Re rho, Im rho); J_rho x = J_s [0, 0, Re rho, Im rho] and its adjoint is
    the rho rows of Re(J_s^H .).  Returns complex rho [nv].
    """
    nv = lin.alpha.shape[1]
    npar = lin.npar

    def A(x):
        v = np.zeros((npar, nv))
        v[2:4] = x
        return model.jvp(lin, v)

    def AH(w):
        return model.jhw(lin, w)[2:4]

    x = np.zeros((2, nv))
    r = np.array(d, np.complex128)
    s = AH(r)
    p = s.copy()
    gamma = float(np.sum(s * s))
    for _ in range(iters):
        if gamma == 0.0:
            break
        q = A(p)
        qq = float(np.vdot(q, q).real)
        if qq == 0.0:
            break
        a = gamma / qq
        x = x + a * p
        r = r - a * q
        s = AH(r)
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    return x[0] + 1j * x[1]


def ls_rho(lin: model.Linearization, d):
    """Minimum-norm least-squares rho for fixed (T1, T2, B1): argmin ||d - M rho||, with
    M[(n, kx), j] = m_j[n] E_{ky(n)}[kx, j] built densely (small cases only) and solved
    by numpy's SVD-based lstsq.  Returns complex rho [nv]."""
    seq = lin.seq
    nv = lin.m.shape[1]
    M = np.zeros((seq.ntr, seq.nkx, nv), np.complex128)
    ky = np.asarray(seq.ky)
    for u in np.unique(ky):
        sel = np.nonzero(ky == u)[0]
        e = encoding.phase_matrix(seq, int(u))
        M[sel] = lin.m[sel][:, None, :] * e[None, :, :]
    rho, *_ = np.linalg.lstsq(M.reshape(seq.ntr * seq.nkx, nv), np.asarray(d).reshape(-1), rcond=None)
    return rho


def draw_mask(rho, threshold: float = 0.1):
    """Voxels with |rho| > threshold * max |rho|."""
    a = np.abs(rho)
    return a > threshold * a.max() if a.size else np.zeros(0, bool)


# ----------------------------------------------------------------------------
# Steihaug truncated CG
# ----------------------------------------------------------------------------
def _to_boundary(z, d, delta):
    """tau >= 0 with ||z + tau d|| = delta."""
    zd = float(np.sum(z * d))
    dd = float(np.sum(d * d))
    zz = float(np.sum(z * z))
    disc = zd * zd + dd * (delta * delta - zz)
    return (-zd + np.sqrt(max(disc, 0.0))) / dd


def steihaug_cg(apply_B, g, delta, max_iter, rel_tol=0.0):
    """Approximately minimise g.p + 1/2 p.B p subject to ||p|| <= delta.

    Returns (p, model_change, iterations, exit_reason) where model_change =
    g.p + 1/2 p.B p (negative for a decrease).  The model value is tracked along
    the iteration from m(z + t d) = m(z) + t r.d + t^2/2 d.B d with r the model
    gradient at z.
    """
    z = np.zeros_like(g)
    r = g.copy()
    d = -r
    rr = float(np.sum(r * r))
    gnorm = np.sqrt(rr)
    mval = 0.0
    if gnorm == 0.0:
        return z, 0.0, 0, "zero_gradient"
    for it in range(max_iter):
        Bd = apply_B(d)
        dBd = float(np.sum(d * Bd))
        rd = float(np.sum(r * d))
        if dBd <= 0.0:
            tau = _to_boundary(z, d, delta)
            return z + tau * d, mval + tau * rd + 0.5 * tau * tau * dBd, it + 1, "negative_curvature"
        a = rr / dBd
        z_new = z + a * d
        if np.sqrt(float(np.sum(z_new * z_new))) >= delta:
            tau = _to_boundary(z, d, delta)
            return z + tau * d, mval + tau * rd + 0.5 * tau * tau * dBd, it + 1, "boundary"
        mval = mval + a * rd + 0.5 * a * a * dBd
        z = z_new
        r = r + a * Bd
        rr_new = float(np.sum(r * r))
        if np.sqrt(rr_new) <= rel_tol * gnorm:
            return z, mval, it + 1, "converged"
        d = -r + (rr_new / rr) * d
        rr = rr_new
    return z, mval, max_iter, "max_iter"


# ----------------------------------------------------------------------------
# Trust-region inexact Gauss-Newton
# ----------------------------------------------------------------------------
@dataclass
class GNOptions:
    outer_iters: int = 10
    inner_iters: int = 20
    delta0: float = 0.0            # <= 0: 0.1 * ||alpha_0|| over masked parameters
    delta_max: float = 1e30
    eta: float = 1e-4
    cg_rel_tol: float = 0.0
    t1_bounds_ms: tuple = (50.0, 6000.0)
    t2_bounds_ms: tuple = (5.0, 3000.0)
    b1_bounds: tuple = (0.5, 1.5)


@dataclass
class GNReport:
    f: list = field(default_factory=list)         # objective at the start of each iteration
    gnorm: list = field(default_factory=list)
    delta: list = field(default_factory=list)
    cg_steps: list = field(default_factory=list)
    ratio: list = field(default_factory=list)
    accepted: list = field(default_factory=list)
    exit: list = field(default_factory=list)
    f_final: float = 0.0


def reflect_into_bounds(x, lo, hi):
    """Reflect components outside [lo, hi] back inside, then clip (simplified Coleman-Li)."""
    x = np.where(x > hi, 2 * hi - x, x)
    x = np.where(x < lo, 2 * lo - x, x)
    return np.clip(x, lo, hi)


def apply_bounds(alpha, opts: GNOptions):
    a = alpha.copy()
    a[0] = reflect_into_bounds(a[0], np.log(opts.t1_bounds_ms[0]), np.log(opts.t1_bounds_ms[1]))
    a[1] = reflect_into_bounds(a[1], np.log(opts.t2_bounds_ms[0]), np.log(opts.t2_bounds_ms[1]))
    if a.shape[0] == 5:
        a[4] = reflect_into_bounds(a[4], opts.b1_bounds[0], opts.b1_bounds[1])
    return a


def gauss_newton(seq, d, alpha0, b1=None, mask=None, opts: GNOptions | None = None, profile=None):
    """Algorithm 6: outer GN iterations, each with one truncated-CG inner solve.

    Returns (alpha, report).  Parameters outside the mask stay at alpha0.  With a slice
    profile (oracle.slice_profile.SliceProfile) the model is the slice-averaged one.
    """
    opts = opts or GNOptions()
    alpha = np.array(alpha0, np.float64)
    nv = alpha.shape[1]
    mask = np.ones(nv, bool) if mask is None else np.asarray(mask, bool)
    mflt = mask[None, :].astype(np.float64)
    lin = model.linearize(seq, alpha, b1, mask, profile)
    s = model.signal(lin)
    f = model.objective(d, s)
    delta = opts.delta0 if opts.delta0 > 0 else 0.1 * np.linalg.norm(alpha * mflt)
    rep = GNReport()

    def apply_B(v):
        return model.gauss_newton_product(lin, v)

    for _ in range(opts.outer_iters):
        g = -model.jhw(lin, d - s)
        rep.f.append(f)
        rep.gnorm.append(float(np.linalg.norm(g)))
        rep.delta.append(delta)
        p, mchange, steps, why = steihaug_cg(apply_B, g, delta, opts.inner_iters, opts.cg_rel_tol)
        rep.cg_steps.append(steps)
        rep.exit.append(why)
        trial = apply_bounds(alpha + p, opts)
        trial = np.where(mask[None, :], trial, alpha)
        lin_t = model.linearize(seq, trial, b1, mask, profile)
        s_t = model.signal(lin_t)
        f_t = model.objective(d, s_t)
        pred = -mchange
        ratio = (f - f_t) / pred if pred > 0 else -np.inf
        rep.ratio.append(float(ratio))
        pnorm = float(np.linalg.norm(p))
        if ratio < 0.25:
            delta = 0.25 * delta
        elif ratio > 0.75 and pnorm >= 0.99 * delta:
            delta = min(2.0 * delta, opts.delta_max)
        acc = ratio > opts.eta
        rep.accepted.append(bool(acc))
        if acc:
            alpha, lin, s, f = trial, lin_t, s_t, f_t
    rep.f_final = f
    return alpha, rep


def initial_alpha(seq, d, nv, rho_iters=50, t1_ms=1000.0, t2_ms=100.0, b1=None,
                  mask_threshold=0.1, estimate_b1=False, exact=False):
    """alpha_0 of the paper (T1 = 1000 ms, T2 = 100 ms, B1 = 1, rho the least-squares
    solution: rho_iters CGLS steps, or with exact=True the exact solution) and its mask."""
    npar = 5 if estimate_b1 else 4
    a0 = np.zeros((npar, nv))
    a0[0] = np.log(t1_ms)
    a0[1] = np.log(t2_ms)
    if estimate_b1:
        a0[4] = 1.0
    lin = model.linearize(seq, a0, b1)
    rho = ls_rho(lin, d) if exact else cgls_rho(lin, d, rho_iters)
    mask = draw_mask(rho, mask_threshold)
    a0[2] = np.where(mask, rho.real, 0.0)
    a0[3] = np.where(mask, rho.imag, 0.0)
    return a0, mask
