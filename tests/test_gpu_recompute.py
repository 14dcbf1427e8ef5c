"""Recompute form of the exact model (mrstat_set_recompute): the Bloch recursion re-run
inside every product from segment states, fused with the phase-encode sums (Algorithms
2 and 4 evaluate the simulation inside every product).  Parity against the FP64 oracle
at the float32 bar 1e-5 normwise, on ragged cases: rows that are not a whole number of
warps, TR counts that are not a multiple of the segment or of the 8-TR chunk, segments
of 1 TR and longer than the train, nkx != nx (the general J^H J v path), masks, a B1 map,
shuffled phase-encode order and no inversion.  At the 224 x 224 / 1120-TR workload the
recompute products and fixed-count CG match the cached form."""
import numpy as np
import pytest

import synth
from oracle import metrics, model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def mr():
    import paper_1904_13244_gb300 as mr
    from paper_1904_13244_gb300 import build
    build.build()
    return mr


def f32(x):
    return np.asarray(x).astype(np.float32).astype(np.float64)


def cuda(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def random_alpha(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return f32(np.stack([rng.uniform(np.log(200), np.log(3000), nx * ny), rng.uniform(np.log(20), np.log(300), nx * ny),
                         rng.uniform(0.5, 1.0, nx * ny) * np.cos(rng.uniform(0, 6.3, nx * ny)),
                         rng.uniform(0.5, 1.0, nx * ny) * np.sin(rng.uniform(0, 6.3, nx * ny))]))


CASES = {
    # name: (nx, ny, fills, extra_trs, nkx, segment, options)
    "quad16_seg16": (16, 16, 4, 0, 16, 16, {}),
    "ragged_40x24_seg7": (40, 24, 3, 5, 48, 7, {}),
    "odd_33x7_seg1": (33, 7, 2, 3, 33, 1, {}),
    "rows_37_seg100": (9, 37, 3, 2, 9, 100, {}),
    "one_column_long_segment": (1, 20, 2, 1, 1, 1000, {}),
    "one_line_seg12": (64, 1, 9, 2, 64, 12, {}),
    "no_inversion_seg20": (24, 16, 3, 1, 24, 20, {"inversion": False, "alternate_phase": False}),
    "rows_224_seg64": (6, 224, 2, 3, 6, 64, {}),
    "rows_256_seg128": (5, 256, 1, 0, 5, 128, {}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_recompute_products_match_oracle(mr, name):
    nx, ny, fills, extra, nkx, seg, kw = CASES[name]
    seq = synth.make_sequence(nx, ny, fills, 7.8, 3.9, seed=2, nkx=nkx, extra_trs=extra, **kw)
    alpha = random_alpha(nx, ny, 3)
    lin = model.linearize(seq, alpha)
    v = synth.random_params(seq.nv, 11)
    w = synth.random_kspace(seq.ntr, seq.nkx, 12)
    with mr.Plan(seq) as plan:
        plan.set_recompute(seg)
        plan.linearize(cuda(alpha))
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        h = plan.jhjv(cuda(v)).cpu().numpy()
        plan.check()
    assert metrics.relerr(jv, model.jvp(lin, v)) < TOL
    gref = model.jhw(lin, w)
    href = model.gauss_newton_product(lin, v)
    for k in range(4):
        assert metrics.relerr(g[k], gref[k]) < TOL, k
        assert metrics.relerr(h[k], href[k]) < TOL, k


def test_recompute_mask_b1_and_shuffled_ky(mr):
    nx, ny = 36, 20
    seq = synth.make_sequence(nx, ny, 3, 7.6, 3.8, seed=4, extra_trs=6)
    seq.ky = np.random.default_rng(3).permutation(seq.ky).astype(np.int32)
    alpha = random_alpha(nx, ny, 9)
    b1 = f32(synth.smooth_b1(nx, ny, 5).ravel())
    mask = np.random.default_rng(1).random(seq.nv) > 0.3
    lin = model.linearize(seq, alpha, b1=b1, mask=mask)
    v = synth.random_params(seq.nv, 21)
    w = synth.random_kspace(seq.ntr, seq.nkx, 22)
    with mr.Plan(seq) as plan:
        plan.set_recompute(16)
        plan.linearize(cuda(alpha), b1=cuda(b1), mask=cuda(mask.astype(np.uint8), torch.uint8))
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        h = plan.jhjv(cuda(v)).cpu().numpy()
        plan.check()
    assert metrics.relerr(jv, model.jvp(lin, v)) < TOL
    assert metrics.relerr(g, model.jhw(lin, w)) < TOL
    assert metrics.relerr(h, model.gauss_newton_product(lin, v)) < TOL
    assert np.all(g[:, ~mask] == 0) and np.all(h[:, ~mask] == 0)


def test_recompute_full_size_matches_cached_form(mr):
    """224 x 224 / 1120 TRs: products and a 30-iteration CG of the recompute form against
    the cached form (itself pinned to the oracle on sampled outputs), and the switch back."""
    seq, ph = synth.config("brain224")
    alpha = f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                          ph.rho.imag.ravel()]))
    v = cuda(synth.random_params(seq.nv, 5))
    w = cuda(synth.random_kspace(seq.ntr, seq.nkx, 6), torch.complex64)
    with mr.Plan(seq) as plan:
        a = cuda(alpha)
        plan.linearize(a)
        ref = [plan.jvp(v), plan.jhw(w), plan.jhjv(v)]
        g = plan.jhw(w)
        b = (g / torch.sqrt(torch.mean(g * g))).contiguous()
        x_ref = plan.cg_fixed(b, 30).clone()
        plan.set_recompute(192)
        with pytest.raises(mr.MrstatError):
            plan.jvp(v)  # the switch drops the linearisation
        plan.linearize(a)
        got = [plan.jvp(v), plan.jhw(w), plan.jhjv(v)]
        x = plan.cg_fixed(b, 30)
        assert plan.cg_applied() == 30
        with pytest.raises(mr.MrstatError) as e:
            plan.timecourses(0)
        assert e.value.status == 7
        with pytest.raises(mr.MrstatError) as e:
            plan.gn_solve(w, a.clone(), outer_iters=1)
        assert e.value.status == 7
        plan.set_recompute(0)
        plan.linearize(a)
        back = plan.jhjv(v)
        plan.check()
    for r, o in zip(ref, got):
        assert float(torch.linalg.vector_norm(o - r) / torch.linalg.vector_norm(r)) < 2e-6
    assert float(torch.linalg.vector_norm(back - ref[2]) / torch.linalg.vector_norm(ref[2])) < 1e-6
    assert float(torch.linalg.vector_norm(x - x_ref) / torch.linalg.vector_norm(x_ref)) < 5e-3


def test_recompute_rejects_what_it_does_not_cover(mr):
    seq = synth.make_sequence(4, 300, 1, 7.8, 3.9)
    with mr.Plan(seq) as plan:
        with pytest.raises(mr.MrstatError) as e:
            plan.set_recompute(64)
        assert e.value.status == 7
        with pytest.raises(mr.MrstatError) as e:
            plan.set_recompute(-1)
        assert e.value.status == 1
    seq = synth.make_sequence(8, 8, 2, 7.8, 3.9)
    with mr.Plan(seq, estimate_b1=True) as plan:
        with pytest.raises(mr.MrstatError) as e:
            plan.set_recompute(16)
        assert e.value.status == 7
