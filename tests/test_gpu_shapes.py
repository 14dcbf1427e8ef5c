"""The other sequence shapes of the paper at full size, on the GPU against the oracle.

* brain224_1792: 224 x 224 with eight k-space fills (1792 TRs, the in-vivo shape) and
  the sine-squared flip train; eight TRs per ky line, so the low-rank product runs in
  the column kernel at its largest TR count per ky.
* const112x88: the constant-flip-per-k-space scan (112 x 88 at 1.8 mm, 16 fills, 1408
  TRs, TR 5.6 ms); Ny = 88 is not a multiple of 32, so the low-rank product takes the
  tensor-core DFT path.

Exact products are checked on sampled TRs and voxels the oracle computes one by one
(1e-5 normwise); the low-rank J^H J v at full size is checked against the low-rank
J^H (J v) of the separate jvp and jhw (each of them pinned to the oracle) at 1e-4.
"""
import numpy as np
import pytest

import synth
from oracle import bloch, encoding, metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def mr():
    import paper_1904_13244_gb300 as mr
    from paper_1904_13244_gb300 import build
    build.build()
    return mr


def cuda(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def alpha_of(ph):
    return f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                         ph.rho.imag.ravel()]))


SHAPES = ["brain224_1792", "const112x88"]


@pytest.fixture(scope="module", params=SHAPES)
def shape(request, mr):
    name = request.param
    seq, ph = synth.config(name)
    alpha = alpha_of(ph)
    v = synth.random_params(seq.nv, 61)
    w = synth.random_kspace(seq.ntr, seq.nkx, 62)
    rng = np.random.default_rng(63)
    rows = np.sort(rng.choice(seq.ntr, 10, replace=False))
    vox = np.sort(rng.choice(seq.nv, 48, replace=False))
    rng2 = np.random.default_rng(64)
    train = f32(np.stack([rng2.uniform(np.log(100), np.log(6000), 2048), rng2.uniform(np.log(10), np.log(3000), 2048)]))
    with mr.Plan(seq) as plan:
        a = cuda(alpha)
        plan.linearize(a)
        out = dict(tc=[plan.timecourses(c)[:, torch.tensor(vox, device="cuda")].cpu().numpy() for c in range(3)],
                   s=plan.forward(a).cpu().numpy()[rows], jv=plan.jvp(cuda(v)).cpu().numpy()[rows],
                   g=plan.jhw(cuda(w, torch.complex64)).cpu().numpy()[:, vox])
        U, _ = plan.lowrank_basis(cuda(train), 32)
        plan.lowrank_set_basis(U)
        plan.lowrank_linearize(a)
        vd = cuda(v)
        out["lr_h"] = plan.jhjv(vd).cpu().numpy()
        out["lr_h2"] = plan.jhw(plan.jvp(vd)).cpu().numpy()
        out["column_path"] = seq.ny % 32 == 0
        plan.check()
    return name, seq, alpha, v, w, rows, vox, out


def test_sequence_shapes(shape):
    name, seq, *_ = shape
    fl = np.asarray(seq.flip_rad)
    if name == "const112x88":
        assert (seq.nx, seq.ny, seq.ntr) == (112, 88, 1408)
        per_fill = fl.reshape(16, 88)
        assert np.all(per_fill == per_fill[:, :1]) and len(np.unique(per_fill[:, 0])) == 16
    else:
        assert (seq.nx, seq.ny, seq.ntr) == (224, 224, 1792)
        per_fill = fl.reshape(8, 224)
        assert np.all(per_fill[:, 0] == 0)
        assert np.all(np.argmax(per_fill, axis=1) == 112)  # the peak samples ky = 0
        assert np.asarray(seq.ky)[112] == 0


def test_timecourses_sampled_voxels(shape):
    name, seq, alpha, v, w, rows, vox, out = shape
    sim = bloch.simulate(seq, np.exp(alpha[0, vox]), np.exp(alpha[1, vox]))
    for c, key in enumerate(["m", "dm_dlnT1", "dm_dlnT2"]):
        assert metrics.relerr(out["tc"][c], sim[key].imag) < TOL, key


def test_signal_and_jvp_sampled_trs(shape):
    name, seq, alpha, v, w, rows, vox, out = shape
    sim = bloch.simulate(seq, np.exp(alpha[0]), np.exp(alpha[1]), rows=rows)
    rho = alpha[2] + 1j * alpha[3]
    q_s = rho[None, :] * sim["m"]
    q_j = rho[None, :] * (v[0][None, :] * sim["dm_dlnT1"] + v[1][None, :] * sim["dm_dlnT2"]) \
        + (v[2] + 1j * v[3])[None, :] * sim["m"]
    assert metrics.relerr(out["s"], encoding.encode(seq, q_s, rows)) < TOL
    assert metrics.relerr(out["jv"], encoding.encode(seq, q_j, rows)) < TOL


def test_jhw_sampled_voxels(shape):
    name, seq, alpha, v, w, rows, vox, out = shape
    sim = bloch.simulate(seq, np.exp(alpha[0, vox]), np.exp(alpha[1, vox]))
    W = encoding.encode_adjoint(seq, w, vox)
    rho = alpha[2, vox] + 1j * alpha[3, vox]
    ref = np.stack([
        np.real(np.sum(np.conj(rho[None] * sim["dm_dlnT1"]) * W, 0)),
        np.real(np.sum(np.conj(rho[None] * sim["dm_dlnT2"]) * W, 0)),
        np.real(np.sum(np.conj(sim["m"]) * W, 0)),
        np.real(np.sum(np.conj(1j * sim["m"]) * W, 0))])
    assert metrics.relerr(out["g"], ref) < TOL


def test_lowrank_jhjv_full_size_consistent(shape):
    name, seq, alpha, v, w, rows, vox, out = shape
    for k in range(4):
        assert metrics.relerr(out["lr_h"][k], out["lr_h2"][k]) < 1e-4, k
