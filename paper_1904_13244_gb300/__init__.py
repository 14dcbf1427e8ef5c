"""GB300-native MR-STAT hot path: the signal model and its Jacobian products.

MR-STAT (van der Heide et al., arXiv 1904.13244) reconstructs T1, T2 and complex
proton density maps by an inexact Gauss-Newton method whose inner CG solve only
needs s(alpha), J.v and Re(J^H w) (Theory, Eq. 4; Algorithms 2, 4 and 6).  These
run in libmrstat.so (hand-written sm_103a CUDA behind a C ABI, include/mrstat.h);
this package only marshals torch tensors into that ABI.

    plan = Plan(seq)                 # seq: nx, ny, nkx, tr_ms, te_ms, flip_rad, ky, ...
    plan.linearize(alpha)            # alpha: cuda float32 [4, nv]
    jv = plan.jvp(v)                 # cuda complex64 [ntr, nkx]
    g = plan.jhw(w)                  # cuda float32 [4, nv]
"""
from __future__ import annotations

import torch

from . import _binding as _b
from ._binding import (MrstatError, MRSTAT_FORM_PLAIN_FP32, MRSTAT_FORM_SPLIT_BF16, MRSTAT_ESTIMATE_B1,  # noqa: F401
                       mrstat_plan_create, mrstat_plan_destroy, mrstat_plan_info, mrstat_linearize,
                       mrstat_plan_inject_grid_stall,
                       mrstat_forward, mrstat_jvp, mrstat_jhw, mrstat_timecourses, mrstat_dot,
                       mrstat_cg_fixed, mrstat_cg_applied, mrstat_set_recompute, mrstat_status_string, mrstat_last_error,
                       mrstat_profile_start, mrstat_profile_stop, mrstat_gn_default_opts,
                       mrstat_gn_solve, mrstat_plan_check, mrstat_forward_ckpt, mrstat_jhw_ckpt,
                       mrstat_jhjv, mrstat_lowrank_basis, mrstat_lowrank_set_basis, mrstat_lowrank_linearize,
                       mrstat_lowrank_coefficients, mrstat_lowrank_rank, mrstat_lowrank_project_samples,
                       mrstat_mlp_create, mrstat_mlp_destroy, mrstat_mlp_num_params, mrstat_mlp_set_output_scale,
                       mrstat_mlp_get_params, mrstat_mlp_set_params, mrstat_mlp_train_step, mrstat_mlp_loss_grad,
                       mrstat_mlp_infer, mrstat_set_slice_profile)

__all__ = ["Plan", "Surrogate", "MrstatError", "load", "Signal", "signal"]


def load():
    """Load libmrstat.so; raises if it has not been built."""
    return _b.load()


class Plan:
    """Owns one mrstat_plan (device tables and the cached linearisation)."""

    def __init__(self, seq, form: int = MRSTAT_FORM_PLAIN_FP32, estimate_b1: bool = False):
        """estimate_b1: B1 is the fifth unknown (alpha, v, g and the GN vectors get 5 rows)."""
        self.nx, self.ny, self.nkx = int(seq.nx), int(seq.ny), int(seq.nkx)
        self.ntr = int(len(seq.flip_rad))
        self.nv = self.nx * self.ny
        self.npar = 5 if estimate_b1 else 4
        self._h = mrstat_plan_create(seq, form | (MRSTAT_ESTIMATE_B1 if estimate_b1 else 0))

    # -- life cycle --
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value is not None:
            mrstat_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        return mrstat_plan_info(self._h)

    def check(self):
        """Synchronise and raise if a device-side bounded wait gave up."""
        mrstat_plan_check(self._h)

    def inject_grid_stall(self, block=-1):
        """Test hook: block `block` of the persistent CG / Steihaug launches withholds its
        first grid arrival, so their bounded waits run out (TIMEOUT); -1 turns it off."""
        mrstat_plan_inject_grid_stall(self._h, block)

    # -- products --
    def _kspace(self, out):
        if out is None:
            out = torch.empty((self.ntr, self.nkx), dtype=torch.complex64, device="cuda")
        return out

    def _params(self, out):
        if out is None:
            out = torch.empty((self.npar, self.nv), dtype=torch.float32, device="cuda")
        return out

    def linearize(self, alpha, b1=None, mask=None, stream=None):
        mrstat_linearize(self._h, alpha, b1, mask, stream)

    def forward(self, alpha, b1=None, mask=None, out=None, stream=None):
        out = self._kspace(out)
        mrstat_forward(self._h, alpha, b1, mask, out, stream)
        return out

    def forward_ckpt(self, alpha, b1=None, mask=None, interval: int = 64, out=None, stream=None):
        out = self._kspace(out)
        mrstat_forward_ckpt(self._h, alpha, b1, mask, interval, out, stream)
        return out

    def jhw_ckpt(self, w, out=None, stream=None):
        out = self._params(out)
        mrstat_jhw_ckpt(self._h, w, out, stream)
        return out

    def jhjv(self, v, out=None, stream=None):
        out = self._params(out)
        mrstat_jhjv(self._h, v, out, stream)
        return out

    # -- low-rank form --
    def lowrank_basis(self, train, rank: int, train_b1=None, stream=None):
        """Time basis U [ntr, rank] from training parameters train [2, ns] (ln T1, ln T2)."""
        U = torch.empty((self.ntr, rank), dtype=torch.float32, device="cuda")
        sv = mrstat_lowrank_basis(self._h, train, train_b1, rank, U, stream)
        return U, sv

    def lowrank_set_basis(self, U, stream=None):
        mrstat_lowrank_set_basis(self._h, U, stream)

    def lowrank_linearize(self, alpha, b1=None, mask=None, coef=None, stream=None):
        mrstat_lowrank_linearize(self._h, alpha, b1, mask, coef, stream)

    def lowrank_coefficients(self, out=None, stream=None):
        R = mrstat_lowrank_rank(self._h)
        if out is None:
            out = torch.empty((3, R, self.nv), dtype=torch.float32, device="cuda")
        mrstat_lowrank_coefficients(self._h, out, stream)
        return out

    def lowrank_project_samples(self, params, b1=None, out=None, stream=None):
        """Exact coefficients [3, R, ns] of sample time courses (ln T1, ln T2 in params [2, ns])."""
        R = mrstat_lowrank_rank(self._h)
        if out is None:
            out = torch.empty((3, R, int(params.shape[1])), dtype=torch.float32, device="cuda")
        mrstat_lowrank_project_samples(self._h, params, b1, out, stream)
        return out

    def jvp(self, v, out=None, stream=None):
        out = self._kspace(out)
        mrstat_jvp(self._h, v, out, stream)
        return out

    def jhw(self, w, out=None, stream=None):
        out = self._params(out)
        mrstat_jhw(self._h, w, out, stream)
        return out

    def timecourses(self, channel: int, out=None, stream=None):
        if out is None:
            out = torch.empty((self.ntr, self.nv), dtype=torch.float32, device="cuda")
        mrstat_timecourses(self._h, channel, out, stream)
        return out

    def dot(self, a, b, out=None, stream=None):
        if out is None:
            out = torch.empty((), dtype=torch.float64, device="cuda")
        mrstat_dot(self._h, a, b, a.numel(), out, stream)
        return out

    def gn_solve(self, d, alpha, b1=None, mask=None, stream=None, **opts) -> dict:
        """Algorithm 6 on the device; alpha (cuda float32 [4, nv]) is updated in place."""
        return mrstat_gn_solve(self._h, d, alpha, b1, mask, mrstat_gn_default_opts(**opts), stream)

    def profile_start(self, kernels=("ycontract", "jhw_dot")):
        mrstat_profile_start(self._h, kernels)

    def profile_stop(self) -> dict:
        return mrstat_profile_stop(self._h)

    def set_slice_profile(self, n_iso=None, n_sub=16, sigma=0.2, tbw=4.0, extent=2.0):
        """Slice-profile Bloch model (n_iso isochromats, n_sub Gaussian RF sub-steps);
        n_iso=None restores hard pulses.  Drops the cached linearisation."""
        mrstat_set_slice_profile(self._h, n_iso, n_sub, sigma, tbw, extent)

    def cg_fixed(self, rhs, iters: int, out=None, stream=None):
        out = self._params(out)
        mrstat_cg_fixed(self._h, rhs, out, iters, stream)
        return out

    def set_recompute(self, segment: int):
        """segment > 0: re-run the Bloch recursion inside every product from states kept
        every `segment` TRs (no cached time courses); 0: cached time courses.  Drops the
        cached linearisation."""
        mrstat_set_recompute(self._h, segment)

    def cg_applied(self) -> int:
        """Iterations the last cg_fixed applied (its iters unless the solve froze);
        synchronises."""
        return mrstat_cg_applied(self._h)



class Surrogate:
    """Learned surrogate (mrstat_mlp): (ln T1, ln T2, B1) -> time-basis coefficients and
    their ln T1 / ln T2 derivatives, an MLP trained on device with a Sobolev loss."""

    def __init__(self, hidden: int, rank: int, norm, sobolev_weight: float = 1.0, seed: int = 0):
        self.hidden, self.rank = int(hidden), int(rank)
        self._h = mrstat_mlp_create(hidden, rank, norm, sobolev_weight, seed)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value is not None:
            mrstat_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    @property
    def num_params(self) -> int:
        return mrstat_mlp_num_params(self._h)

    def set_output_scale(self, scale):
        mrstat_mlp_set_output_scale(self._h, scale)

    def get_params(self):
        return mrstat_mlp_get_params(self._h)

    def set_params(self, params):
        mrstat_mlp_set_params(self._h, params)

    def train_step(self, lnT, target, lr: float, b1=None, loss=None, stream=None):
        mrstat_mlp_train_step(self._h, lnT, b1, target, lr, loss, stream)

    def loss_grad(self, lnT, target, b1=None, grad=None, stream=None) -> float:
        return mrstat_mlp_loss_grad(self._h, lnT, b1, target, grad, stream)

    def infer(self, lnT, b1=None, out=None, stream=None):
        if out is None:
            out = torch.empty((3, self.rank, int(lnT.shape[1])), dtype=torch.float32, device="cuda")
        mrstat_mlp_infer(self._h, lnT, b1, out, stream)
        return out


from .autograd import Signal, signal  # noqa: E402
