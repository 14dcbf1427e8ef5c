"""GPU parity: every C-ABI product against the FP64 oracle on the same seeded inputs.

Tolerance: 1e-5 normwise relative error, ||x_gpu - x_oracle|| / ||x_oracle||, per
output array (FP32 signals and Jacobian products).  Cases span several tiles of
every kernel and ragged tails: TR counts that are not a multiple of 4 (TR quads),
grids that are not multiples of 32 columns (warp tiles), nkx != nx, odd and
one-line grids, arbitrary phase-encode order, masks, B1 maps, no inversion and a
constant RF phase.  The 224x224 / 1120-TR workload (the benchmark's launch
configuration) is checked on sampled outputs the oracle computes one by one.
"""
import numpy as np
import pytest

import synth
from oracle import bloch, encoding, model, metrics

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def mr():
    import paper_1904_13244_gb300 as mr
    from paper_1904_13244_gb300 import build
    build.build()
    assert torch.cuda.is_available()
    return mr


def alpha_of(ph):
    """Parameter maps rounded to float32 (the ABI's input type), held in float64 for the oracle."""
    return np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                     ph.rho.imag.ravel()]).astype(np.float32).astype(np.float64)


def random_phantom(nx, ny, seed):
    rng = np.random.default_rng(seed)
    t1 = np.exp(rng.uniform(np.log(200), np.log(3000), (ny, nx)))
    t2 = np.exp(rng.uniform(np.log(20), np.log(300), (ny, nx)))
    rho = rng.uniform(0.5, 1.0, (ny, nx)) * np.exp(1j * rng.uniform(0, 2 * np.pi, (ny, nx)))
    return synth.Phantom(t1_ms=t1, t2_ms=t2, rho=rho, b1=np.ones((ny, nx)), support=np.ones((ny, nx), bool))


def cuda(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


CASES = {
    # name: (nx, ny, fills, extra_trs, nkx, kwargs)
    "quad16": (16, 16, 4, 0, 16, {}),
    "ragged_40x24": (40, 24, 3, 5, 48, {}),
    "odd_33x7": (33, 7, 2, 3, 30, {}),
    "one_line": (64, 1, 9, 2, 64, {}),
    "one_column": (1, 20, 2, 1, 1, {}),
    "single_voxel_single_tr": (1, 1, 1, 0, 1, {}),
    "no_inversion_const_phase": (24, 16, 3, 1, 24, {"inversion": False, "alternate_phase": False}),
    "ellipse64": (64, 64, 5, 0, 64, {}),
    # the flip trains of the supporting information: constant per k-space fill (S3) and
    # connected sine-squared waves peaking at the central line (S1)
    "constant_flip_12x16": (12, 16, 4, 0, 12, {"train": "constant"}),
    "sine2_ragged_20x12": (20, 12, 3, 5, 24, {"train": "sine2"}),
}


def make_case(name, seed=0):
    nx, ny, fills, extra, nkx, kw = CASES[name]
    seq = synth.make_sequence(nx, ny, fills, 7.8, 3.9, seed=seed, nkx=nkx, extra_trs=extra, **kw)
    if name == "ellipse64":
        ph = synth.ellipse_phantom(64, seed)
        ph.rho = ph.rho + 0.3 * (~ph.support)  # keep background voxels active for this case
    elif name == "quad16":
        ph = synth.quadrant_phantom(16, seed)
    else:
        ph = random_phantom(nx, ny, seed + 7)
    return seq, ph


@pytest.mark.parametrize("name", list(CASES))
def test_products_match_oracle(mr, name):
    seq, ph = make_case(name)
    alpha = alpha_of(ph)
    lin = model.linearize(seq, alpha)
    v = synth.random_params(seq.nv, 11)
    w = synth.random_kspace(seq.ntr, seq.nkx, 12)
    with mr.Plan(seq) as plan:
        a = cuda(alpha)
        plan.linearize(a)
        for c, ref in enumerate([lin.m, lin.dm1, lin.dm2]):
            tc = plan.timecourses(c).cpu().numpy()
            assert metrics.relerr(tc, ref.imag) < TOL, (c, metrics.relerr(tc, ref.imag))
        s = plan.forward(a).cpu().numpy()
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        # J^H J v: with nkx == nx the readout DFT pair cancels and is skipped
        h = plan.jhjv(cuda(v)).cpu().numpy()
    assert metrics.relerr(s, model.signal(lin)) < TOL
    assert metrics.relerr(jv, model.jvp(lin, v)) < TOL
    gref = model.jhw(lin, w)
    assert metrics.relerr(g, gref) < TOL
    # every parameter row on its own as well (rows differ in scale)
    for k in range(4):
        assert metrics.relerr(g[k], gref[k]) < TOL, k
    href = model.gauss_newton_product(lin, v)
    assert metrics.relerr(h, href) < TOL
    for k in range(4):
        assert metrics.relerr(h[k], href[k]) < TOL, k


def test_mask_b1_and_shuffled_ky(mr):
    nx, ny = 36, 20
    seq = synth.make_sequence(nx, ny, 3, 7.6, 3.8, seed=4, extra_trs=6)
    seq.ky = np.random.default_rng(3).permutation(seq.ky).astype(np.int32)
    ph = random_phantom(nx, ny, 9)
    b1 = synth.smooth_b1(nx, ny, 5).ravel().astype(np.float32).astype(np.float64)
    mask = np.random.default_rng(1).random(seq.nv) > 0.3
    alpha = alpha_of(ph)
    lin = model.linearize(seq, alpha, b1=b1, mask=mask)
    v = synth.random_params(seq.nv, 21)
    w = synth.random_kspace(seq.ntr, seq.nkx, 22)
    with mr.Plan(seq) as plan:
        a = cuda(alpha)
        b = cuda(b1)
        mk = cuda(mask.astype(np.uint8), torch.uint8)
        plan.linearize(a, b, mk)
        s = plan.forward(a, b, mk).cpu().numpy()
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        h = plan.jhjv(cuda(v)).cpu().numpy()
        tc = plan.timecourses(0).cpu().numpy()
    assert metrics.relerr(h, model.gauss_newton_product(lin, v)) < TOL
    assert np.all(tc[:, ~mask] == 0)
    assert metrics.relerr(tc[:, mask], lin.m.imag[:, mask]) < TOL
    assert metrics.relerr(s, model.signal(lin)) < TOL
    assert metrics.relerr(jv, model.jvp(lin, v)) < TOL
    assert metrics.relerr(g, model.jhw(lin, w)) < TOL
    assert np.all(g[:, ~mask] == 0)


def test_zero_flip_train_gives_zero_signal(mr):
    seq = synth.make_sequence(16, 8, 2, 7.8, 3.9, seed=0)
    seq.flip_rad = np.zeros(seq.ntr)
    ph = random_phantom(16, 8, 1)
    with mr.Plan(seq) as plan:
        a = cuda(alpha_of(ph))
        plan.linearize(a)
        assert torch.count_nonzero(plan.forward(a)).item() == 0
        assert torch.count_nonzero(plan.jvp(cuda(synth.random_params(seq.nv, 1)))).item() == 0
        assert torch.count_nonzero(plan.jhw(cuda(synth.random_kspace(seq.ntr, seq.nkx, 2),
                                                 torch.complex64))).item() == 0


def test_adjoint_identity_on_gpu(mr):
    seq, ph = make_case("ragged_40x24")
    v = synth.random_params(seq.nv, 31)
    w = synth.random_kspace(seq.ntr, seq.nkx, 32)
    with mr.Plan(seq) as plan:
        plan.linearize(cuda(alpha_of(ph)))
        jv = plan.jvp(cuda(v)).cpu().numpy().astype(np.complex128)
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy().astype(np.float64)
    lhs = np.vdot(jv, w).real
    rhs = float(np.sum(v * g))
    assert abs(lhs - rhs) / abs(lhs) < TOL


def test_dot_float64(mr):
    rng = np.random.default_rng(0)
    seq, _ = make_case("quad16")
    with mr.Plan(seq) as plan:
        for n in [0, 1, 1000, 1 << 20]:
            a = rng.standard_normal(n).astype(np.float32)
            b = rng.standard_normal(n).astype(np.float32)
            out = plan.dot(cuda(a), cuda(b)).item()
            ref = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
            # per-thread float32 products of a handful of elements, float64 beyond
            assert abs(out - ref) <= 2e-7 * max(1.0, np.abs(a.astype(np.float64) * b).sum())


def _oracle_cg(lin, b, iters):
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.sum(r * r))
    for _ in range(iters):
        q = model.gauss_newton_product(lin, p)
        pq = float(np.sum(p * q))
        a = rr / pq
        x = x + a * p
        r = r - a * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


@pytest.mark.parametrize("iters", [0, 1, 3])
def test_cg_fixed_matches_oracle_cg(mr, iters):
    """Fixed-count CG on Re(J^H J) x = b.  CG multiplies rounding differences between
    the float32 and float64 runs by roughly the condition number seen so far, so the
    bar after a few iterations is 1e-4 instead of the single-product 1e-5."""
    seq, ph = make_case("quad16")
    alpha = alpha_of(ph)
    lin = model.linearize(seq, alpha)
    b = model.jhw(lin, synth.random_kspace(seq.ntr, seq.nkx, 40))
    with mr.Plan(seq) as plan:
        plan.linearize(cuda(alpha))
        x = plan.cg_fixed(cuda(b), iters).cpu().numpy()
    ref = _oracle_cg(lin, b, iters)
    if iters == 0:
        assert np.all(x == 0)
    else:
        assert metrics.relerr(x, ref) < (TOL if iters == 1 else 1e-4)


def test_jvp_before_linearize_is_an_error(mr):
    seq, _ = make_case("quad16")
    with mr.Plan(seq) as plan:
        with pytest.raises(mr.MrstatError) as e:
            plan.jvp(cuda(synth.random_params(seq.nv, 1)))
        assert e.value.status == 3


# ---------------------------------------------------------------------------
# full-size workload (224 x 224, 1120 TRs): sampled outputs
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def brain(mr):
    seq, ph = synth.config("brain224")
    alpha = alpha_of(ph)
    v = synth.random_params(seq.nv, 51)
    w = synth.random_kspace(seq.ntr, seq.nkx, 52)
    rng = np.random.default_rng(53)
    rows = np.sort(rng.choice(seq.ntr, 12, replace=False))
    vox = np.sort(rng.choice(seq.nv, 64, replace=False))
    with mr.Plan(seq) as plan:
        a = cuda(alpha)
        plan.linearize(a)
        out = dict(
            tc=[plan.timecourses(c)[:, torch.tensor(vox, device="cuda")].cpu().numpy() for c in range(3)],
            s=plan.forward(a).cpu().numpy()[rows],
            jv=plan.jvp(cuda(v)).cpu().numpy()[rows],
            g=plan.jhw(cuda(w, torch.complex64)).cpu().numpy()[:, vox])
    return seq, ph, alpha, v, w, rows, vox, out


@pytest.fixture(scope="module")
def brain_oracle(brain):
    """The oracle's s and J.v on the sampled TRs and Re(J^H w) on the sampled voxels of
    the full 224 x 224 / 1120-TR workload."""
    seq, ph, alpha, v, w, rows, vox, out = brain
    sim = bloch.simulate(seq, np.exp(alpha[0]), np.exp(alpha[1]), rows=rows)
    rho = alpha[2] + 1j * alpha[3]
    q_s = rho[None, :] * sim["m"]
    q_j = rho[None, :] * (v[0][None, :] * sim["dm_dlnT1"] + v[1][None, :] * sim["dm_dlnT2"]) \
        + (v[2] + 1j * v[3])[None, :] * sim["m"]
    simv = bloch.simulate(seq, np.exp(alpha[0, vox]), np.exp(alpha[1, vox]))
    W = encoding.encode_adjoint(seq, w, vox)
    rv = alpha[2, vox] + 1j * alpha[3, vox]
    g = np.stack([
        np.real(np.sum(np.conj(rv[None] * simv["dm_dlnT1"]) * W, 0)),
        np.real(np.sum(np.conj(rv[None] * simv["dm_dlnT2"]) * W, 0)),
        np.real(np.sum(np.conj(simv["m"]) * W, 0)),
        np.real(np.sum(np.conj(1j * simv["m"]) * W, 0))])
    return dict(s=encoding.encode(seq, q_s, rows), jv=encoding.encode(seq, q_j, rows), g=g)


def test_full_size_timecourses_sampled_voxels(brain):
    seq, ph, alpha, v, w, rows, vox, out = brain
    sim = bloch.simulate(seq, np.exp(alpha[0, vox]), np.exp(alpha[1, vox]))
    for c, key in enumerate(["m", "dm_dlnT1", "dm_dlnT2"]):
        assert metrics.relerr(out["tc"][c], sim[key].imag) < TOL, key


def test_full_size_signal_and_jvp_sampled_trs(brain, brain_oracle):
    out = brain[-1]
    assert metrics.relerr(out["s"], brain_oracle["s"]) < TOL
    assert metrics.relerr(out["jv"], brain_oracle["jv"]) < TOL


def test_full_size_jhw_sampled_voxels(brain, brain_oracle):
    out = brain[-1]
    assert metrics.relerr(out["g"], brain_oracle["g"]) < TOL


# ---------------------------------------------------------------------------
# split-BF16 form: readout DFT on tcgen05 tensor cores
# ---------------------------------------------------------------------------
# Each operand keeps ~16 significant bits (hi + lo), the dropped lo*lo term is
# ~2^-18 relative per product; summed over the 2*nx (or 2*nkx) real terms of a
# DFT row the normwise error stays near 1e-5.  Bar: 3e-5 normwise per output.
SPLIT_TOL = 3e-5


@pytest.mark.parametrize("name", ["quad16", "ragged_40x24", "odd_33x7", "ellipse64", "one_line"])
def test_split_bf16_products_match_oracle(mr, name):
    seq, ph = make_case(name)
    alpha = alpha_of(ph)
    lin = model.linearize(seq, alpha)
    v = synth.random_params(seq.nv, 11)
    w = synth.random_kspace(seq.ntr, seq.nkx, 12)
    with mr.Plan(seq, form=mr.MRSTAT_FORM_SPLIT_BF16) as plan:
        a = cuda(alpha)
        plan.linearize(a)
        s = plan.forward(a).cpu().numpy()
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        plan.check()
    e = [metrics.relerr(s, model.signal(lin)), metrics.relerr(jv, model.jvp(lin, v)),
         metrics.relerr(g, model.jhw(lin, w))]
    assert max(e) < SPLIT_TOL, e


def test_split_bf16_full_size_sampled(mr, brain, brain_oracle):
    """The split-BF16 form at 224 x 224 / 1120 TRs against the FP64 oracle on the sampled
    TRs (s, J.v) and voxels (Re(J^H w)), and against the plain FP32 form."""
    seq, ph, alpha, v, w, rows, vox, out = brain
    with mr.Plan(seq, form=mr.MRSTAT_FORM_SPLIT_BF16) as plan:
        a = cuda(alpha)
        plan.linearize(a)
        s = plan.forward(a).cpu().numpy()[rows]
        jv = plan.jvp(cuda(v)).cpu().numpy()[rows]
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()[:, vox]
        plan.check()
    e = [metrics.relerr(s, brain_oracle["s"]), metrics.relerr(jv, brain_oracle["jv"]),
         metrics.relerr(g, brain_oracle["g"])]
    assert max(e) < SPLIT_TOL, e
    assert metrics.relerr(jv, out["jv"]) < SPLIT_TOL
    assert metrics.relerr(g, out["g"]) < SPLIT_TOL
