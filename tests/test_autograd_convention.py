"""Host-side check of the differentiation form's contract: for a real input alpha
and a complex output s = J alpha, PyTorch passes the backward the conjugate
Wirtinger gradient grad_s, and the correct input gradient is Re(J^H grad_s) -- the
quantity mrstat_jhw returns.  Checked against PyTorch's own autograd on a dense J."""
import torch


class _Dense(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, J):
        ctx.J = J
        return J @ x.to(J.dtype)

    @staticmethod
    def backward(ctx, g):
        return (ctx.J.conj().T @ g).real, None


def test_backward_is_real_part_of_adjoint():
    gen = torch.Generator().manual_seed(0)
    J = torch.randn(9, 5, dtype=torch.complex128, generator=gen)
    w = torch.randn(9, dtype=torch.complex128, generator=gen)
    x0 = torch.randn(5, dtype=torch.float64, generator=gen)
    for loss in [lambda s: (s.abs() ** 2).sum(), lambda s: torch.real(torch.vdot(s, w)),
                 lambda s: (s * s.conj()).real.sum() + s.real.sum() - 2 * s.imag.sum()]:
        x1 = x0.clone().requires_grad_(True)
        loss(J @ x1.to(J.dtype)).backward()
        x2 = x0.clone().requires_grad_(True)
        loss(_Dense.apply(x2, J)).backward()
        assert torch.allclose(x1.grad, x2.grad, rtol=1e-12, atol=1e-12)
