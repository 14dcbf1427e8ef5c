"""Learned surrogate (mrstat_mlp_*) against the FP64 oracle MLP, and its use as the
source of the low-rank coefficients.

The GPU network runs its GEMMs in BF16 (float32 accumulation) with BF16 activations,
weights and gradient rows; each layer rounds its inputs and weights to 8 significant
bits (relative 2^-9), so four layers give a few 1e-3 normwise.  Bars: outputs 1e-2,
tangents 2e-2, loss 2e-2 and gradient 5e-2 normwise against oracle.surrogate at the
same float32 parameters.  Sample projections (the training targets) are the exact
projected Bloch model and must match the oracle at the float32 bar 1e-5.
"""
import numpy as np
import pytest

import synth
from oracle import bloch, model, metrics, surrogate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NORM = (np.log(1000.0), 1.0, np.log(100.0), 1.2, 1.0, 0.2)


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


def glorot(hidden, rank, seed):
    rng = np.random.default_rng(seed)
    th = []
    for o, i in surrogate.layer_shapes(hidden, rank):
        lim = np.sqrt(6.0 / (o + i))
        th.append(rng.uniform(-lim, lim, o * i))
        th.append(rng.uniform(-0.1, 0.1, o))
    return f32(np.concatenate(th))


def samples(n, seed, b1=True):
    rng = np.random.default_rng(seed)
    x = np.stack([rng.uniform(np.log(100), np.log(6000), n), rng.uniform(np.log(10), np.log(3000), n),
                  rng.uniform(0.8, 1.2, n) if b1 else np.ones(n)])
    return f32(x)


@pytest.mark.parametrize("hidden,rank,n", [(64, 16, 1000), (128, 8, 77), (256, 32, 4099)])
def test_forward_matches_oracle(mr, hidden, rank, n):
    theta = glorot(hidden, rank, 1)
    scale = f32(np.linspace(2.0, 0.1, rank))
    x = samples(n, 2)
    with mr.Surrogate(hidden, rank, NORM, 0.5, seed=3) as net:
        assert net.num_params == surrogate.num_params(hidden, rank)
        net.set_params(theta)
        net.set_output_scale(scale)
        assert np.array_equal(net.get_params(), theta.astype(np.float32))
        out = net.infer(cuda(x[:2]), cuda(x[2])).cpu().numpy().astype(np.float64)
    c, d1, d2, _ = surrogate.forward(theta, x, NORM, scale, hidden, rank)
    assert metrics.relerr(out[0], c) < 1e-2
    assert metrics.relerr(out[1], d1) < 2e-2
    assert metrics.relerr(out[2], d2) < 2e-2


def test_loss_and_gradient_match_oracle(mr):
    hidden, rank, B = 64, 16, 1500
    theta = glorot(hidden, rank, 4)
    scale = f32(np.linspace(1.0, 0.2, rank))
    x = samples(B, 5)
    rng = np.random.default_rng(6)
    target = f32(rng.standard_normal((3, rank, B)) * scale[None, :, None])
    with mr.Surrogate(hidden, rank, NORM, 0.3, seed=0) as net:
        net.set_params(theta)
        net.set_output_scale(scale)
        grad = torch.zeros(net.num_params, dtype=torch.float32, device="cuda")
        L = net.loss_grad(cuda(x[:2]), cuda(target), b1=cuda(x[2]), grad=grad)
        g = grad.cpu().numpy().astype(np.float64)
    L_ref, g_ref = surrogate.loss_grad(theta, x, tuple(target), NORM, scale, hidden, rank, 0.3)
    assert abs(L - L_ref) / L_ref < 2e-2
    assert metrics.relerr(g, g_ref) < 5e-2


def test_project_samples_match_linearize_and_oracle(mr):
    seq = synth.make_sequence(20, 12, 3, 7.8, 3.9, seed=1, extra_trs=2)
    rng = np.random.default_rng(7)
    train = f32(np.stack([rng.uniform(np.log(100), np.log(6000), 500), rng.uniform(np.log(10), np.log(3000), 500)]))
    U, _ = model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), 16)
    U = f32(U)
    alpha = f32(np.stack([rng.uniform(np.log(200), np.log(3000), seq.nv), rng.uniform(np.log(20), np.log(300), seq.nv),
                          rng.uniform(0.5, 1, seq.nv), rng.uniform(-0.5, 0.5, seq.nv)]))
    b1 = f32(rng.uniform(0.8, 1.2, seq.nv))
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(cuda(U))
        plan.lowrank_linearize(cuda(alpha), b1=cuda(b1))
        c_lin = plan.lowrank_coefficients().cpu().numpy()
        c_smp = plan.lowrank_project_samples(cuda(alpha[:2]), b1=cuda(b1)).cpu().numpy()
        plan.check()
    assert np.array_equal(c_lin, c_smp)
    sim = bloch.simulate(seq, np.exp(alpha[0]), np.exp(alpha[1]), b1)
    assert metrics.relerr(c_smp[0], U.T @ sim["m"].imag) < 1e-5
    assert metrics.relerr(c_smp[1], U.T @ sim["dm_dlnT1"].imag) < 1e-5
    assert metrics.relerr(c_smp[2], U.T @ sim["dm_dlnT2"].imag) < 1e-5


def test_surrogate_coefficients_drive_the_lowrank_products(mr):
    """lowrank_linearize with caller coefficients: the products are those of the model
    m_j = i U c_j built from exactly those coefficients."""
    seq = synth.make_sequence(24, 16, 3, 7.8, 3.9, seed=2, extra_trs=3)
    R, hidden = 16, 64
    rng = np.random.default_rng(8)
    train = f32(np.stack([rng.uniform(np.log(100), np.log(6000), 500), rng.uniform(np.log(10), np.log(3000), 500)]))
    U = f32(model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), R)[0])
    alpha = f32(np.stack([rng.uniform(np.log(200), np.log(3000), seq.nv), rng.uniform(np.log(20), np.log(300), seq.nv),
                          rng.uniform(0.5, 1, seq.nv), rng.uniform(-0.5, 0.5, seq.nv)]))
    v = synth.random_params(seq.nv, 9)
    w = synth.random_kspace(seq.ntr, seq.nkx, 10)
    with mr.Plan(seq) as plan, mr.Surrogate(hidden, R, NORM, 1.0, seed=5) as net:
        plan.lowrank_set_basis(cuda(U))
        coef = net.infer(cuda(alpha[:2]))
        plan.lowrank_linearize(cuda(alpha), coef=coef)
        C = coef.cpu().numpy().astype(np.float64)
        jv = plan.jvp(cuda(v)).cpu().numpy()
        g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
        plan.check()
    lin = model.Linearization(seq, alpha, np.ones(seq.nv), np.ones(seq.nv, bool), 1j * (U @ C[0]), 1j * (U @ C[1]),
                              1j * (U @ C[2]), None)
    assert metrics.relerr(jv, model.jvp(lin, v)) < 3e-5
    assert metrics.relerr(g, model.jhw(lin, w)) < 3e-5


def test_training_fits_the_projected_model(mr):
    seq = synth.make_sequence(40, 24, 5, 7.8, 3.9, seed=3, extra_trs=6)
    R, hidden, B = 16, 128, 1024
    with mr.Plan(seq) as plan:
        train = cuda(samples(4096, 11, b1=False)[:2])
        U, _ = plan.lowrank_basis(train, R)
        plan.lowrank_set_basis(U)
        x = cuda(samples(32768, 12))
        tgt = plan.lowrank_project_samples(x[:2].contiguous(), b1=x[2].contiguous())
        xt = cuda(samples(4096, 13))
        tgt_test = plan.lowrank_project_samples(xt[:2].contiguous(), b1=xt[2].contiguous())
        scale = tgt[0].abs().amax(dim=1).clamp_min(1e-6).cpu().numpy()
        with mr.Surrogate(hidden, R, NORM, 0.5, seed=1) as net:
            net.set_output_scale(scale)
            L0 = net.loss_grad(xt[:2].contiguous(), tgt_test, b1=xt[2].contiguous())
            gen = torch.Generator(device="cuda").manual_seed(0)
            for it in range(3000):
                idx = torch.randint(0, x.shape[1], (B,), device="cuda", generator=gen)
                lr = 3e-3 if it < 2000 else 1e-3
                net.train_step(x[:2, idx].contiguous(), tgt[:, :, idx].contiguous(), lr, b1=x[2, idx].contiguous())
            L1 = net.loss_grad(xt[:2].contiguous(), tgt_test, b1=xt[2].contiguous())
            pred = net.infer(xt[:2].contiguous(), xt[2].contiguous())
            err = [float(torch.linalg.norm(pred[k] - tgt_test[k]) / torch.linalg.norm(tgt_test[k])) for k in range(3)]
    print(f"surrogate held-out loss {L0:.3e} -> {L1:.3e}; relative errors c {err[0]:.2e} dc1 {err[1]:.2e} dc2 {err[2]:.2e}")
    assert L1 < 0.02 * L0
    assert err[0] < 5e-2


def test_b1_map_surrogate_products_match_projected_oracle(mr):
    """The learned-part form with a known, smooth B1 map (0.8..1.2): a surrogate trained on
    the device on B1-varied samples gives the coefficients; the low-rank products are those
    of the oracle model m_j = i U c_j built from exactly those coefficients (3e-5), the
    compressed-exact products with the same map are the oracle's projected model (3e-5), and
    the trained surrogate's Gauss-Newton product stays within 10 % of the projected exact
    one."""
    seq = synth.make_sequence(24, 64, 5, 7.8, 3.9, seed=4)  # ny = 64: the column path
    R, hidden, B = 16, 128, 1024
    train = samples(2000, 21)
    U = f32(model.time_basis(seq, np.exp(train[0]), np.exp(train[1]), R, b1=train[2])[0])
    rng = np.random.default_rng(22)
    alpha = f32(np.stack([rng.uniform(np.log(300), np.log(2500), seq.nv), rng.uniform(np.log(30), np.log(250), seq.nv),
                          rng.uniform(0.5, 1, seq.nv), rng.uniform(-0.5, 0.5, seq.nv)]))
    b1 = f32(synth.smooth_b1(seq.nx, seq.ny, 5).ravel())
    v = synth.random_params(seq.nv, 23)
    w = synth.random_kspace(seq.ntr, seq.nkx, 24)
    with mr.Plan(seq) as plan:
        plan.lowrank_set_basis(cuda(U))
        x = cuda(samples(32768, 25))
        tgt = plan.lowrank_project_samples(x[:2].contiguous(), b1=x[2].contiguous())
        scale = tgt[0].abs().amax(dim=1).clamp_min(1e-6).cpu().numpy()
        with mr.Surrogate(hidden, R, NORM, 0.5, seed=3) as net:
            net.set_output_scale(scale)
            gen = torch.Generator(device="cuda").manual_seed(1)
            for it in range(3000):
                idx = torch.randint(0, x.shape[1], (B,), device="cuda", generator=gen)
                net.train_step(x[:2, idx].contiguous(), tgt[:, :, idx].contiguous(), 3e-3 if it < 2000 else 1e-3,
                               b1=x[2, idx].contiguous())
            a, bm = cuda(alpha), cuda(b1)
            coef = net.infer(a[:2].contiguous(), b1=bm)
            plan.lowrank_linearize(a, b1=bm, coef=coef)
            C = coef.cpu().numpy().astype(np.float64)
            jv = plan.jvp(cuda(v)).cpu().numpy()
            g = plan.jhw(cuda(w, torch.complex64)).cpu().numpy()
            h_sur = plan.jhjv(cuda(v)).cpu().numpy()
            plan.lowrank_linearize(a, b1=bm)
            h_lr = plan.jhjv(cuda(v)).cpu().numpy()
            plan.check()
    lin_net = model.Linearization(seq, alpha, b1, np.ones(seq.nv, bool), 1j * (U @ C[0]), 1j * (U @ C[1]),
                                  1j * (U @ C[2]), None)
    assert metrics.relerr(jv, model.jvp(lin_net, v)) < 3e-5
    assert metrics.relerr(g, model.jhw(lin_net, w)) < 3e-5
    assert metrics.relerr(h_sur, model.gauss_newton_product(lin_net, v)) < 3e-5
    lin_proj = model.project_onto_basis(model.linearize(seq, alpha, b1=b1), U)
    ref = model.gauss_newton_product(lin_proj, v)
    assert metrics.relerr(h_lr, ref) < 3e-5
    e_sur = metrics.relerr(h_sur, ref)
    # the same product with the B1 map ignored (B1 = 1 in the projected model): the map
    # matters by far more than the surrogate's error
    e_nob1 = metrics.relerr(model.gauss_newton_product(model.project_onto_basis(model.linearize(seq, alpha), U), v), ref)
    print(f"surrogate J^H J v vs projected exact with the B1 map: {e_sur:.2e} (B1 map ignored: {e_nob1:.2e})")
    assert e_sur < 0.1
    assert e_sur < 0.5 * e_nob1


def test_surrogate_linearisation_beats_the_exact_projection(mr):
    """What the network buys per linearisation at 224 x 224 / 1120 TRs, rank 32: one MLP
    inference (tcgen05) plus adopting its coefficients against projecting the exact Bloch
    recursion onto the basis; the products afterwards cost the same.  CUDA-event times of
    20 back-to-back linearisations each, after a warm-up."""
    seq, ph = synth.config("brain224")
    alpha = f32(np.stack([np.log(ph.t1_ms.ravel()), np.log(ph.t2_ms.ravel()), ph.rho.real.ravel(),
                          ph.rho.imag.ravel()]))
    R = 32
    U = np.linalg.qr(np.random.default_rng(3).standard_normal((seq.ntr, R)))[0]
    with mr.Plan(seq) as plan, mr.Surrogate(256, R, NORM, 0.5, seed=1) as net:
        plan.lowrank_set_basis(cuda(f32(U)))
        a = cuda(alpha)
        coef = torch.empty((3, R, seq.nv), dtype=torch.float32, device="cuda")

        def surrogate():
            net.infer(a[:2], out=coef)
            plan.lowrank_linearize(a, coef=coef)

        def exact():
            plan.lowrank_linearize(a)

        def ms(fn):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 20
        t_sur, t_exact = ms(surrogate), ms(exact)
        plan.check()
    print(f"linearisation: surrogate {t_sur:.3f} ms, exact projection {t_exact:.3f} ms ({t_exact / t_sur:.1f}x)")
    assert t_sur < t_exact / 1.5
