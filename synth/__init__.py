"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the reconstruction method itself: it only draws
the inputs the method is applied to -- a pulse-sequence description (flip-angle
train and phase-encode order), tissue-parameter phantoms, random direction vectors
and complex Gaussian noise.  Everything is drawn from ``numpy.random.default_rng``
with an explicit seed, so both sides see bit-identical inputs.

Workload recipe (the paper's datasets are not available, so these stand in):

* Sequence (Methods "Pulse Sequence"; Supporting Information S1): balanced
  gradient-echo, fixed TR, TE = TR/2, RF phase alternating 0/180 degrees, linear
  Cartesian order (each fill sweeps ky ascending), non-selective inversion at the
  start.  The smooth flip train is a seeded sum of three sinusoids rescaled to
  0..60 degrees (the paper's own train -- connected sin^2 lobes -- is only drawn
  in a figure that is not available).
* Phantoms: a 4-region quadrant phantom (16x16), a 6-class nested-ellipse phantom
  (64x64) and a brain-like phantom with WM/GM/CSF/fat classes (224x224 and
  256x256) whose T1/T2 values follow the in-vivo tissue classes of the paper's
  brain experiments; background has rho = 0 and covers about half the FOV, which
  matches the ~25 000 masked voxels of a 224x224 slice.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Sequence", "Phantom", "flip_train", "constant_flip_train", "sine_squared_train", "cartesian_ky",
    "make_sequence",
    "quadrant_phantom", "ellipse_phantom", "brain_phantom", "smooth_field",
    "smooth_b1", "random_params", "random_kspace", "complex_noise", "add_noise",
    "CONFIGS", "config",
]


# ----------------------------------------------------------------------------
# Sequence description
# ----------------------------------------------------------------------------
@dataclass
class Sequence:
    """Pulse-sequence description consumed by both the oracle and the C ABI.

    ``flip_rad[n]`` is the nominal flip-angle amplitude of TR n (radians, >= 0);
    ``ky[n]`` is the phase-encode index sampled in TR n, in [-ny//2, ny - ny//2);
    the nkx readout samples of every TR have kx = k - nkx//2, k = 0..nkx-1.
    ``alternate_phase`` selects RF phase 0, 180, 0, 180, ... degrees per TR.
    """
    nx: int
    ny: int
    nkx: int
    tr_ms: float
    te_ms: float
    flip_rad: np.ndarray
    ky: np.ndarray
    inversion: bool = True
    alternate_phase: bool = True

    @property
    def ntr(self) -> int:
        return int(self.flip_rad.shape[0])

    @property
    def nv(self) -> int:
        return self.nx * self.ny


def flip_train(ntr: int, fills: float, seed: int = 0, max_deg: float = 60.0) -> np.ndarray:
    """Smooth flip-angle amplitudes (radians) in [0, max_deg] degrees.

    raw(n) = sum_{i=1..3} a_i sin(2 pi f_i n / ntr + psi_i), with a_i ~ U(0.5, 1),
    f_i ~ U(1, 2*fills) cycles per scan and psi_i ~ U(0, 2 pi); the train is raw
    rescaled affinely so that its minimum is 0 and its maximum is max_deg.
    """
    if ntr <= 0:
        return np.zeros(0)
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.5, 1.0, 3)
    f = rng.uniform(1.0, max(2.0 * fills, 1.0 + 1e-9), 3)
    psi = rng.uniform(0.0, 2.0 * np.pi, 3)
    n = np.arange(ntr, dtype=np.float64)
    raw = (a[:, None] * np.sin(2.0 * np.pi * f[:, None] * n[None, :] / ntr + psi[:, None])).sum(0)
    lo, hi = raw.min(), raw.max()
    if hi - lo <= 0:
        return np.full(ntr, np.deg2rad(max_deg) * 0.5)
    return np.deg2rad(max_deg) * (raw - lo) / (hi - lo)


def constant_flip_train(ntr: int, ny: int, seed: int = 0, lo_deg: float = 10.0,
                        hi_deg: float = 60.0) -> np.ndarray:
    """One flip angle per k-space fill (TRs f*ny .. f*ny + ny - 1), different between fills
    (the sequence of Supporting Information S3): alpha_f ~ U(lo_deg, hi_deg) degrees,
    seeded; radians."""
    if ntr <= 0:
        return np.zeros(0)
    nf = (ntr + ny - 1) // ny
    a = np.random.default_rng(seed).uniform(lo_deg, hi_deg, nf)
    return np.deg2rad(a[np.arange(ntr) // ny])


def sine_squared_train(ntr: int, ny: int, seed: int = 0, max_deg: float = 60.0,
                       lo_frac: float = 0.3) -> np.ndarray:
    """Connected sine-squared waves, one per k-space fill, starting at zero, each peaking
    where the fill samples the central line ky = 0 (Supporting Information S1):
    alpha_n = A_f sin^2(pi (n mod ny) / ny) with peak A_f ~ U(lo_frac, 1) * max_deg, seeded;
    radians."""
    if ntr <= 0:
        return np.zeros(0)
    nf = (ntr + ny - 1) // ny
    peak = np.random.default_rng(seed).uniform(lo_frac, 1.0, nf) * max_deg
    n = np.arange(ntr)
    return np.deg2rad(peak[n // ny] * np.sin(np.pi * (n % ny) / ny) ** 2)


def cartesian_ky(ntr: int, ny: int) -> np.ndarray:
    """Linear Cartesian order: TR n samples ky = (n mod ny) - ny//2."""
    return (np.arange(ntr) % ny - ny // 2).astype(np.int32)


def make_sequence(nx: int, ny: int, fills: int, tr_ms: float, te_ms: float, seed: int = 0,
                  nkx: int | None = None, extra_trs: int = 0, inversion: bool = True,
                  alternate_phase: bool = True, max_deg: float = 60.0, train: str = "smooth") -> Sequence:
    """train: "smooth" (flip_train), "constant" (constant_flip_train) or "sine2"
    (sine_squared_train)."""
    ntr = fills * ny + extra_trs
    if train == "smooth":
        flips = flip_train(ntr, fills + extra_trs / max(ny, 1), seed, max_deg)
    elif train == "constant":
        flips = constant_flip_train(ntr, ny, seed, hi_deg=max_deg)
    elif train == "sine2":
        flips = sine_squared_train(ntr, ny, seed, max_deg)
    else:
        raise ValueError(f"unknown flip train {train!r}")
    # flips are rounded to float32 so that a float32 consumer sees exactly these values
    flips = flips.astype(np.float32)
    return Sequence(nx=nx, ny=ny, nkx=nx if nkx is None else nkx, tr_ms=tr_ms, te_ms=te_ms,
                    flip_rad=flips.astype(np.float64),
                    ky=cartesian_ky(ntr, ny), inversion=inversion,
                    alternate_phase=alternate_phase)


# ----------------------------------------------------------------------------
# Phantoms
# ----------------------------------------------------------------------------
@dataclass
class Phantom:
    """Tissue maps on an [ny, nx] grid (row iy, column ix)."""
    t1_ms: np.ndarray
    t2_ms: np.ndarray
    rho: np.ndarray              # complex
    b1: np.ndarray               # relative transmit field
    support: np.ndarray          # bool: rho != 0
    labels: np.ndarray = field(default=None)

    @property
    def shape(self):
        return self.t1_ms.shape


def _grid(nx: int, ny: int):
    u = (np.arange(nx) - nx / 2 + 0.5) / (nx / 2)
    v = (np.arange(ny) - ny / 2 + 0.5) / (ny / 2)
    return np.meshgrid(u, v)  # U[iy, ix], V[iy, ix]


def smooth_field(nx: int, ny: int, seed: int, sigma_px: float) -> np.ndarray:
    """Zero-mean, unit-std Gaussian random field smoothed by a Gaussian of sigma_px."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((ny, nx))
    fy = np.fft.fftfreq(ny)[:, None]
    fx = np.fft.fftfreq(nx)[None, :]
    kern = np.exp(-2.0 * (np.pi * sigma_px) ** 2 * (fx ** 2 + fy ** 2))
    f = np.real(np.fft.ifft2(np.fft.fft2(w) * kern))
    f -= f.mean()
    sd = f.std()
    return f / sd if sd > 0 else f


def _poly_phase(nx: int, ny: int, rng) -> np.ndarray:
    u, v = _grid(nx, ny)
    c = rng.uniform(-np.pi / 2, np.pi / 2, 6)
    return c[0] + c[1] * u + c[2] * v + c[3] * u * v + 0.5 * c[4] * u * u + 0.5 * c[5] * v * v


def quadrant_phantom(n: int = 16, seed: int = 0) -> Phantom:
    """Four rectangular quadrants, piecewise-constant tissue values.

    T1 ~ log-U(200, 3000) ms, T2 ~ log-U(20, 300) ms, rho = U(0.5, 1) e^{i U(0, 2 pi)}.
    """
    rng = np.random.default_rng(seed)
    t1 = np.exp(rng.uniform(np.log(200.0), np.log(3000.0), 4))
    t2 = np.exp(rng.uniform(np.log(20.0), np.log(300.0), 4))
    rho = rng.uniform(0.5, 1.0, 4) * np.exp(1j * rng.uniform(0.0, 2 * np.pi, 4))
    lab = np.zeros((n, n), dtype=np.int32)
    h = n // 2
    lab[:h, h:] = 1
    lab[h:, :h] = 2
    lab[h:, h:] = 3
    return Phantom(t1_ms=t1[lab], t2_ms=t2[lab], rho=rho[lab], b1=np.ones((n, n)),
                   support=np.ones((n, n), bool), labels=lab)


# (cx, cy, a, b, angle_deg, class) in normalised [-1, 1] coordinates; painted in order.
_ELLIPSES64 = [
    (0.00, 0.00, 0.86, 0.94, 0.0, 0),     # outer shell
    (0.00, -0.02, 0.76, 0.84, 0.0, 1),    # bulk tissue
    (0.20, 0.05, 0.12, 0.30, -18.0, 2),   # right ventricle-like
    (-0.20, 0.05, 0.14, 0.32, 18.0, 2),   # left ventricle-like
    (0.00, 0.45, 0.20, 0.16, 0.0, 3),     # upper blob
    (0.00, -0.50, 0.22, 0.12, 0.0, 4),    # lower blob
    (-0.45, -0.20, 0.10, 0.10, 0.0, 5),   # small spot
    (0.45, -0.20, 0.08, 0.12, 30.0, 5),   # small spot
]


def _paint(nx, ny, ellipses):
    u, v = _grid(nx, ny)
    lab = np.full((ny, nx), -1, dtype=np.int32)
    for cx, cy, a, b, ang, cls in ellipses:
        t = np.deg2rad(ang)
        x = (u - cx) * np.cos(t) + (v - cy) * np.sin(t)
        y = -(u - cx) * np.sin(t) + (v - cy) * np.cos(t)
        lab[(x / a) ** 2 + (y / b) ** 2 <= 1.0] = cls
    return lab


def ellipse_phantom(n: int = 64, seed: int = 0) -> Phantom:
    """Six-class nested-ellipse phantom (Shepp-Logan-like, own ellipse set).

    Per class: T1 ~ log-U(300, 2500) ms, T2 ~ log-U(30, 250) ms, |rho| ~ U(0.5, 1);
    rho carries one smooth random phase (low-order polynomial).  Background: rho = 0.
    """
    rng = np.random.default_rng(seed)
    t1c = np.exp(rng.uniform(np.log(300.0), np.log(2500.0), 6))
    t2c = np.exp(rng.uniform(np.log(30.0), np.log(250.0), 6))
    mag = rng.uniform(0.5, 1.0, 6)
    lab = _paint(n, n, _ELLIPSES64)
    inside = lab >= 0
    li = np.where(inside, lab, 0)
    t1 = np.where(inside, t1c[li], 1000.0)
    t2 = np.where(inside, t2c[li], 100.0)
    rho = np.where(inside, mag[li], 0.0) * np.exp(1j * _poly_phase(n, n, rng))
    return Phantom(t1_ms=t1, t2_ms=t2, rho=rho, b1=np.ones((n, n)), support=inside, labels=lab)


# Tissue classes of the brain-like phantom: 0 WM, 1 GM, 2 CSF, 3 fat.
BRAIN_T1 = np.array([800.0, 1300.0, 4000.0, 350.0])
BRAIN_T2 = np.array([70.0, 90.0, 2000.0, 80.0])
BRAIN_PD = np.array([0.65, 0.80, 1.00, 0.90])


def _brain_labels(n: int, ny: int | None = None) -> np.ndarray:
    ell = [
        (0.0, 0.0, 0.760, 0.840, 0.0, 3),   # fat (scalp) ring: outer boundary
        (0.0, 0.0, 0.700, 0.780, 0.0, 1),   # cortex (GM)
        (0.0, 0.0, 0.570, 0.650, 0.0, 0),   # white-matter core
        (0.0, 0.02, 0.300, 0.340, 0.0, 1),  # deep GM (basal ganglia-like)
        (0.0, 0.02, 0.240, 0.280, 0.0, 0),  # WM inside deep GM
        (0.13, 0.05, 0.060, 0.200, -15.0, 2),  # ventricles
        (-0.13, 0.05, 0.060, 0.200, 15.0, 2),
        (0.0, -0.30, 0.040, 0.080, 0.0, 2),    # small third-ventricle-like spot
    ]
    # sulci: thin radial CSF ellipses through the cortical ring
    for k in range(12):
        t = 2 * np.pi * (k + 0.37) / 12
        r = 0.64
        ell.append((r * np.cos(t) * 0.76 / 0.76, r * np.sin(t) * 0.84 / 0.76 * 0.9,
                    0.085, 0.018, np.rad2deg(t), 2))
    return _paint(n, n if ny is None else ny, ell)


def brain_phantom(n: int = 224, seed: int = 0, b1_map: bool = False, ny: int | None = None) -> Phantom:
    """Brain-like phantom: fat ring, GM cortex, WM core, deep GM, CSF ventricles/sulci.

    T1 = 800/1300/4000/350 ms and T2 = 70/90/2000/80 ms for WM/GM/CSF/fat, each
    multiplied by (1 + 0.1 g) with g a smooth unit-std Gaussian field (independent
    for T1 and T2); |rho| = 0.65/0.8/1.0/0.9 with a smooth polynomial phase; about
    half of the FOV lies inside the head.  With ``b1_map`` the relative transmit
    field is 1 + 0.2 * smooth field, clipped to [0.8, 1.2]; else B1 = 1.  With ``ny`` the
    grid is n (x) by ny (y) and the head an ellipse filling that field of view.
    """
    rng = np.random.default_rng(seed)
    nx, ny = n, (n if ny is None else ny)
    lab = _brain_labels(nx, ny)
    inside = lab >= 0
    li = np.where(inside, lab, 0)
    g1 = smooth_field(nx, ny, seed + 101, nx / 32)
    g2 = smooth_field(nx, ny, seed + 202, nx / 32)
    t1 = np.where(inside, BRAIN_T1[li] * (1 + 0.1 * g1), 1000.0)
    t2 = np.where(inside, BRAIN_T2[li] * (1 + 0.1 * g2), 100.0)
    rho = np.where(inside, BRAIN_PD[li], 0.0) * np.exp(1j * _poly_phase(nx, ny, rng))
    b1 = smooth_b1(nx, ny, seed + 303) if b1_map else np.ones((ny, nx))
    return Phantom(t1_ms=t1, t2_ms=t2, rho=rho, b1=b1, support=inside, labels=lab)


def smooth_b1(nx: int, ny: int, seed: int) -> np.ndarray:
    return np.clip(1.0 + 0.2 * smooth_field(nx, ny, seed, max(nx, ny) / 8), 0.8, 1.2)


# ----------------------------------------------------------------------------
# Random vectors and noise
# ----------------------------------------------------------------------------
def random_params(nv: int, seed: int, npar: int = 4) -> np.ndarray:
    """Standard-normal direction vector in parameter space, shape [npar, nv]."""
    return np.random.default_rng(seed).standard_normal((npar, nv))


def random_kspace(ntr: int, nkx: int, seed: int) -> np.ndarray:
    """Complex standard-normal k-space vector, shape [ntr, nkx]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ntr, nkx)) + 1j * rng.standard_normal((ntr, nkx))


def complex_noise(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def add_noise(s: np.ndarray, snr: float, seed: int) -> np.ndarray:
    """d = s + e with complex i.i.d. Gaussian e scaled so that ||s||_2 / ||e||_2 = snr."""
    e = complex_noise(s.shape, seed)
    return s + e * (np.linalg.norm(s) / (snr * np.linalg.norm(e)))


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------
CONFIGS = {
    # name: (grid, fills, TR ms, TE ms, phantom)
    "quad16": dict(n=16, fills=4, tr=7.8, te=3.9, phantom="quadrant"),
    "ellipse64": dict(n=64, fills=5, tr=7.8, te=3.9, phantom="ellipse"),
    "brain224": dict(n=224, fills=5, tr=7.6, te=3.8, phantom="brain"),
    "brain256": dict(n=256, fills=5, tr=7.6, te=3.8, phantom="brain"),
    # the in-vivo shape: 224 x 224 with 8 fills (1792 TRs), sine-squared train (S1)
    "brain224_1792": dict(n=224, fills=8, tr=7.6, te=3.8, phantom="brain", train="sine2"),
    # Supporting Information S3: 1.8 mm over 201.5 x 158 mm (112 x 88), TR 5.6 ms, TE 2.8 ms,
    # 16 k-spaces with a constant flip angle each (1408 TRs, 7.9 s)
    "const112x88": dict(n=112, ny=88, fills=16, tr=5.6, te=2.8, phantom="brain", train="constant"),
}


def config(name: str, seed: int = 0, b1_map: bool = False):
    """Return (Sequence, Phantom) of a named workload."""
    c = CONFIGS[name]
    n = c["n"]
    ny = c.get("ny", n)
    seq = make_sequence(n, ny, c["fills"], c["tr"], c["te"], seed=seed, train=c.get("train", "smooth"))
    if c["phantom"] == "quadrant":
        ph = quadrant_phantom(n, seed)
    elif c["phantom"] == "ellipse":
        ph = ellipse_phantom(n, seed)
    else:
        ph = brain_phantom(n, seed, b1_map=b1_map, ny=ny)
    return seq, ph
