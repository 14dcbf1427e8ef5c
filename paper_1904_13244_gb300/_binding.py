"""ctypes binding of libmrstat.so: argument marshalling only.

Every function here has the name of the C entry point it wraps (include/mrstat.h)
and forwards raw device pointers taken from torch tensors plus the current CUDA
stream; all arithmetic runs in the library's kernels.  Loading fails loudly if the
library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmrstat.so")

MRSTAT_OK = 0
MRSTAT_FORM_PLAIN_FP32 = 0
MRSTAT_FORM_SPLIT_BF16 = 1
MRSTAT_ESTIMATE_B1 = 0x100


class MrstatError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {message} (status {status})")
        self.status = status


class mrstat_seq(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nkx", ctypes.c_int32),
                ("ntr", ctypes.c_int32), ("tr_ms", ctypes.c_double), ("te_ms", ctypes.c_double),
                ("inversion", ctypes.c_int32), ("alternate_phase", ctypes.c_int32),
                ("flip_rad", ctypes.POINTER(ctypes.c_float)), ("ky", ctypes.POINTER(ctypes.c_int32))]


class mrstat_plan_info_t(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nkx", ctypes.c_int32),
                ("ntr", ctypes.c_int32), ("nv", ctypes.c_int32), ("form", ctypes.c_int32),
                ("ntr_padded", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("timecourse_bytes", ctypes.c_int64), ("npar", ctypes.c_int32)]


class mrstat_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("ms", ctypes.c_double * 8), ("timed", ctypes.c_int64 * 8),
                ("kernels", ctypes.c_int64 * 8)]


GN_MAX_OUTER = 64
CG_EXIT = {0: "max_iter", 1: "boundary", 2: "negative_curvature", 3: "converged", 4: "zero_gradient"}


class mrstat_gn_opts(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("delta0", ctypes.c_double), ("delta_max", ctypes.c_double), ("eta", ctypes.c_double),
                ("cg_rel_tol", ctypes.c_double), ("t1_min_ms", ctypes.c_double), ("t1_max_ms", ctypes.c_double),
                ("t2_min_ms", ctypes.c_double), ("t2_max_ms", ctypes.c_double),
                ("rho_init_iters", ctypes.c_int32), ("t1_init_ms", ctypes.c_double),
                ("t2_init_ms", ctypes.c_double), ("mask_threshold", ctypes.c_double),
                ("hessian", ctypes.c_int32), ("surrogate_iters", ctypes.c_int32),
                ("surrogate", ctypes.c_void_p), ("b1_min", ctypes.c_double), ("b1_max", ctypes.c_double),
                ("rho_init_exact", ctypes.c_int32), ("iteration_offset", ctypes.c_int32)]


class mrstat_slice_profile(ctypes.Structure):
    _fields_ = [("n_iso", ctypes.c_int32), ("n_sub", ctypes.c_int32), ("sigma", ctypes.c_double),
                ("tbw", ctypes.c_double), ("extent", ctypes.c_double)]


class mrstat_gn_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("mask_voxels", ctypes.c_int32),
                ("cg_steps", ctypes.c_int32 * GN_MAX_OUTER), ("cg_exit", ctypes.c_int32 * GN_MAX_OUTER),
                ("accepted", ctypes.c_int32 * GN_MAX_OUTER), ("f", ctypes.c_double * GN_MAX_OUTER),
                ("gnorm", ctypes.c_double * GN_MAX_OUTER), ("delta", ctypes.c_double * GN_MAX_OUTER),
                ("ratio", ctypes.c_double * GN_MAX_OUTER), ("f_final", ctypes.c_double),
                ("seconds", ctypes.c_double), ("delta_final", ctypes.c_double)]


class mrstat_mlp_config(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("rank", ctypes.c_int32), ("norm", ctypes.c_float * 6),
                ("sobolev_weight", ctypes.c_float), ("seed", ctypes.c_uint64)]


KERNEL_IDS = {"bloch": 0, "ycontract": 1, "xdft": 2, "xdft_adj": 3, "jhw_dot": 4, "vector": 5}

_lib = None

_SIGS = {
    "mrstat_plan_create": [ctypes.POINTER(mrstat_seq), ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
    "mrstat_plan_destroy": [ctypes.c_void_p],
    "mrstat_plan_info": [ctypes.c_void_p, ctypes.POINTER(mrstat_plan_info_t)],
    "mrstat_plan_check": [ctypes.c_void_p],
    "mrstat_plan_inject_grid_stall": [ctypes.c_void_p, ctypes.c_int32],
    "mrstat_set_slice_profile": [ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_linearize": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_forward": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                       ctypes.c_void_p],
    "mrstat_jvp": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_jhw": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_timecourses": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_forward_ckpt": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                            ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_jhw_ckpt": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_jhjv": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_lowrank_basis": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p],
    "mrstat_lowrank_set_basis": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "mrstat_lowrank_linearize": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_lowrank_coefficients": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_lowrank_rank": [ctypes.c_void_p],
    "mrstat_lowrank_project_samples": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_mlp_create": [ctypes.POINTER(mrstat_mlp_config), ctypes.POINTER(ctypes.c_void_p)],
    "mrstat_mlp_destroy": [ctypes.c_void_p],
    "mrstat_mlp_num_params": [ctypes.c_void_p],
    "mrstat_mlp_set_output_scale": [ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_mlp_get_params": [ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_mlp_set_params": [ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_mlp_train_step": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                              ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_mlp_loss_grad": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                             ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_mlp_infer": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                         ctypes.c_void_p],
    "mrstat_dot_static": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p],
    "mrstat_dot": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_void_p],
    "mrstat_cg_fixed": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p],
    "mrstat_cg_applied": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)],
    "mrstat_set_recompute": [ctypes.c_void_p, ctypes.c_int32],
    "mrstat_gn_default_opts": [ctypes.POINTER(mrstat_gn_opts)],
    "mrstat_gn_solve": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.POINTER(mrstat_gn_opts), ctypes.POINTER(mrstat_gn_report), ctypes.c_void_p],
    "mrstat_profile_start": [ctypes.c_void_p, ctypes.c_uint32],
    "mrstat_profile_stop": [ctypes.c_void_p, ctypes.POINTER(mrstat_kernel_stats)],
    "mrstat_status_string": [ctypes.c_int],
    "mrstat_last_error": [],
}


def load(path: str = LIB_PATH):
    """Load libmrstat.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libmrstat.so not built ({path}); run paper_1904_13244_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            if name in ("mrstat_status_string", "mrstat_last_error"):
                f.restype = ctypes.c_char_p
            elif name == "mrstat_gn_default_opts":
                f.restype = None
            elif name == "mrstat_mlp_num_params":
                f.restype = ctypes.c_int64
            else:
                f.restype = ctypes.c_int
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(status: int, where: str):
    if status != MRSTAT_OK:
        lib = load()
        raise MrstatError(status, where, lib.mrstat_last_error().decode() or
                          lib.mrstat_status_string(status).decode())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


_dims_cache = {}


def _npar(plan) -> int:
    """Unknowns per voxel of a plan (4, or 5 with B1 estimated)."""
    key = ("npar", plan.value if isinstance(plan, ctypes.c_void_p) else plan)
    if key not in _dims_cache:
        _dims_cache[key] = mrstat_plan_info(plan)["npar"]
    return _dims_cache[key]


def _dims(plan):
    """(nv, ntr, nkx) of a plan, from mrstat_plan_info (cached per handle)."""
    key = plan.value if isinstance(plan, ctypes.c_void_p) else plan
    if key not in _dims_cache:
        info = mrstat_plan_info(plan)
        _dims_cache[key] = (info["nv"], info["ntr"], info["nkx"])
    return _dims_cache[key]


def _ptr(t, dtype, shape=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# same-name wrappers of the C entry points
# ---------------------------------------------------------------------------
def mrstat_plan_create(seq, form: int = MRSTAT_FORM_PLAIN_FP32) -> ctypes.c_void_p:
    lib = load()
    import numpy as np
    flips = np.ascontiguousarray(np.asarray(seq.flip_rad, dtype=np.float32))
    ky = np.ascontiguousarray(np.asarray(seq.ky, dtype=np.int32))
    s = mrstat_seq(int(seq.nx), int(seq.ny), int(seq.nkx), int(flips.shape[0]), float(seq.tr_ms),
                   float(seq.te_ms), int(bool(seq.inversion)), int(bool(seq.alternate_phase)),
                   flips.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                   ky.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    h = ctypes.c_void_p()
    _check(lib.mrstat_plan_create(ctypes.byref(s), int(form), ctypes.byref(h)), "mrstat_plan_create")
    return h


def mrstat_plan_destroy(plan):
    key = plan.value if isinstance(plan, ctypes.c_void_p) else plan
    _dims_cache.pop(key, None)
    _dims_cache.pop(("npar", key), None)
    _check(load().mrstat_plan_destroy(plan), "mrstat_plan_destroy")


def mrstat_plan_info(plan) -> dict:
    info = mrstat_plan_info_t()
    _check(load().mrstat_plan_info(plan, ctypes.byref(info)), "mrstat_plan_info")
    return {f: getattr(info, f) for f, _ in mrstat_plan_info_t._fields_}


def mrstat_plan_check(plan):
    _check(load().mrstat_plan_check(plan), "mrstat_plan_check")


def mrstat_plan_inject_grid_stall(plan, block):
    _check(load().mrstat_plan_inject_grid_stall(plan, int(block)), "mrstat_plan_inject_grid_stall")


def mrstat_linearize(plan, alpha, b1=None, mask=None, stream=None):
    nv, _, _ = _dims(plan)
    npar = _npar(plan)
    _check(load().mrstat_linearize(plan, _ptr(alpha, torch.float32, (npar, nv), "alpha"),
                                   _ptr(b1, torch.float32, (nv,), "b1"),
                                   _ptr(mask, torch.uint8, (nv,), "mask"), _stream(stream)),
           "mrstat_linearize")


def mrstat_forward(plan, alpha, b1, mask, s, stream=None):
    nv, ntr, nkx = _dims(plan)
    npar = _npar(plan)
    _check(load().mrstat_forward(plan, _ptr(alpha, torch.float32, (npar, nv), "alpha"),
                                 _ptr(b1, torch.float32, (nv,), "b1"), _ptr(mask, torch.uint8, (nv,), "mask"),
                                 _ptr(s, torch.complex64, (ntr, nkx), "s"), _stream(stream)), "mrstat_forward")


def mrstat_jvp(plan, v, jv, stream=None):
    nv, ntr, nkx = _dims(plan)
    npar = _npar(plan)
    _check(load().mrstat_jvp(plan, _ptr(v, torch.float32, (npar, nv), "v"),
                             _ptr(jv, torch.complex64, (ntr, nkx), "jv"), _stream(stream)), "mrstat_jvp")


def mrstat_jhw(plan, w, g, stream=None):
    nv, ntr, nkx = _dims(plan)
    npar = _npar(plan)
    _check(load().mrstat_jhw(plan, _ptr(w, torch.complex64, (ntr, nkx), "w"),
                             _ptr(g, torch.float32, (npar, nv), "g"), _stream(stream)), "mrstat_jhw")


def mrstat_forward_ckpt(plan, alpha, b1, mask, interval, s, stream=None):
    nv, ntr, nkx = _dims(plan)
    _check(load().mrstat_forward_ckpt(plan, _ptr(alpha, torch.float32, (4, nv), "alpha"),
                                      _ptr(b1, torch.float32, (nv,), "b1"), _ptr(mask, torch.uint8, (nv,), "mask"),
                                      int(interval), _ptr(s, torch.complex64, (ntr, nkx), "s"), _stream(stream)),
           "mrstat_forward_ckpt")


def mrstat_jhw_ckpt(plan, w, g, stream=None):
    nv, ntr, nkx = _dims(plan)
    _check(load().mrstat_jhw_ckpt(plan, _ptr(w, torch.complex64, (ntr, nkx), "w"),
                                  _ptr(g, torch.float32, (4, nv), "g"), _stream(stream)), "mrstat_jhw_ckpt")


def mrstat_jhjv(plan, v, out, stream=None):
    nv, _, _ = _dims(plan)
    npar = _npar(plan)
    _check(load().mrstat_jhjv(plan, _ptr(v, torch.float32, (npar, nv), "v"), _ptr(out, torch.float32, (npar, nv), "out"),
                              _stream(stream)), "mrstat_jhjv")


def mrstat_lowrank_basis(plan, train, train_b1, rank, U_out, stream=None):
    ns = int(train.shape[1])
    nv, ntr, _ = _dims(plan)
    sv = (ctypes.c_double * rank)()
    _check(load().mrstat_lowrank_basis(plan, _ptr(train, torch.float32, (2, ns), "train"),
                                       _ptr(train_b1, torch.float32, (ns,), "train_b1"), ns, int(rank),
                                       _ptr(U_out, torch.float32, (ntr, rank), "U"), sv, _stream(stream)),
           "mrstat_lowrank_basis")
    return list(sv)


def mrstat_lowrank_set_basis(plan, U, stream=None):
    nv, ntr, _ = _dims(plan)
    rank = int(U.shape[1])
    _check(load().mrstat_lowrank_set_basis(plan, _ptr(U, torch.float32, (ntr, rank), "U"), rank, _stream(stream)),
           "mrstat_lowrank_set_basis")


def mrstat_lowrank_linearize(plan, alpha, b1=None, mask=None, coef=None, stream=None):
    nv, _, _ = _dims(plan)
    R = load().mrstat_lowrank_rank(plan)
    _check(load().mrstat_lowrank_linearize(plan, _ptr(alpha, torch.float32, (4, nv), "alpha"),
                                           _ptr(b1, torch.float32, (nv,), "b1"), _ptr(mask, torch.uint8, (nv,), "mask"),
                                           _ptr(coef, torch.float32, (3, R, nv), "coef"), _stream(stream)),
           "mrstat_lowrank_linearize")


def mrstat_lowrank_coefficients(plan, out, stream=None):
    nv, _, _ = _dims(plan)
    R = load().mrstat_lowrank_rank(plan)
    _check(load().mrstat_lowrank_coefficients(plan, _ptr(out, torch.float32, (3, R, nv), "coef"), _stream(stream)),
           "mrstat_lowrank_coefficients")


def mrstat_lowrank_rank(plan) -> int:
    return int(load().mrstat_lowrank_rank(plan))


def mrstat_timecourses(plan, channel, out, stream=None):
    nv, ntr, _ = _dims(plan)
    _check(load().mrstat_timecourses(plan, int(channel), _ptr(out, torch.float32, (ntr, nv), "out"),
                                     _stream(stream)), "mrstat_timecourses")


def mrstat_dot(plan, a, b, n, out, stream=None):
    if a.numel() < n or b.numel() < n:
        raise ValueError("a and b must hold at least n elements")
    _check(load().mrstat_dot(plan, _ptr(a, torch.float32, name="a"), _ptr(b, torch.float32, name="b"),
                             int(n), _ptr(out, torch.float64, (), "out"), _stream(stream)), "mrstat_dot")


def mrstat_cg_fixed(plan, rhs, x, iters, stream=None):
    nv, _, _ = _dims(plan)
    npar = _npar(plan)
    _check(load().mrstat_cg_fixed(plan, _ptr(rhs, torch.float32, (npar, nv), "rhs"),
                                  _ptr(x, torch.float32, (npar, nv), "x"), int(iters), _stream(stream)),
           "mrstat_cg_fixed")


def mrstat_set_recompute(plan, segment):
    _check(load().mrstat_set_recompute(plan, int(segment)), "mrstat_set_recompute")


def mrstat_cg_applied(plan) -> int:
    n = ctypes.c_int32(0)
    _check(load().mrstat_cg_applied(plan, ctypes.byref(n)), "mrstat_cg_applied")
    return int(n.value)


def mrstat_set_slice_profile(plan, n_iso=None, n_sub=16, sigma=0.2, tbw=4.0, extent=2.0):
    """n_iso = None: hard pulses; else the slice-profile model with these pulse readings."""
    if n_iso is None:
        _check(load().mrstat_set_slice_profile(plan, None), "mrstat_set_slice_profile")
        return
    prof = mrstat_slice_profile(int(n_iso), int(n_sub), float(sigma), float(tbw), float(extent))
    _check(load().mrstat_set_slice_profile(plan, ctypes.byref(prof)), "mrstat_set_slice_profile")


def mrstat_gn_default_opts(**overrides) -> mrstat_gn_opts:
    o = mrstat_gn_opts()
    load().mrstat_gn_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(f"unknown Gauss-Newton option {k}")
        if k == "surrogate" and v is not None and not isinstance(v, (int, ctypes.c_void_p)):
            v = v.handle  # a Surrogate object
        if isinstance(v, ctypes.c_void_p):
            v = v.value
        setattr(o, k, v)
    return o


def mrstat_gn_solve(plan, d, alpha, b1=None, mask=None, opts=None, stream=None) -> dict:
    nv, ntr, nkx = _dims(plan)
    npar = _npar(plan)
    opts = opts if opts is not None else mrstat_gn_default_opts()
    rep = mrstat_gn_report()
    _check(load().mrstat_gn_solve(plan, _ptr(d, torch.complex64, (ntr, nkx), "d"),
                                  _ptr(alpha, torch.float32, (npar, nv), "alpha"), _ptr(b1, torch.float32, (nv,), "b1"),
                                  _ptr(mask, torch.uint8, (nv,), "mask"), ctypes.byref(opts), ctypes.byref(rep),
                                  _stream(stream)), "mrstat_gn_solve")
    k = rep.iterations
    return {"iterations": k, "mask_voxels": rep.mask_voxels, "f": list(rep.f[:k]), "gnorm": list(rep.gnorm[:k]),
            "delta": list(rep.delta[:k]), "ratio": list(rep.ratio[:k]), "cg_steps": list(rep.cg_steps[:k]),
            "cg_exit": [CG_EXIT.get(x, str(x)) for x in rep.cg_exit[:k]],
            "accepted": [bool(x) for x in rep.accepted[:k]], "f_final": rep.f_final, "seconds": rep.seconds,
            "delta_final": rep.delta_final}


def mrstat_profile_start(plan, kernels=("ycontract", "jhw_dot")):
    mask = 0
    for k in kernels:
        mask |= 1 << KERNEL_IDS[k]
    _check(load().mrstat_profile_start(plan, mask), "mrstat_profile_start")


def mrstat_profile_stop(plan) -> dict:
    st = mrstat_kernel_stats()
    _check(load().mrstat_profile_stop(plan, ctypes.byref(st)), "mrstat_profile_stop")
    return {name: {"launches": st.launches[i], "ms": st.ms[i], "timed": st.timed[i], "kernels": st.kernels[i]}
            for name, i in KERNEL_IDS.items()}


def mrstat_status_string(status: int) -> str:
    return load().mrstat_status_string(int(status)).decode()


def mrstat_last_error() -> str:
    return load().mrstat_last_error().decode()


# ---------------------------------------------------------------------------
# learned surrogate
# ---------------------------------------------------------------------------
def mrstat_lowrank_project_samples(plan, params, b1, coef, stream=None):
    ns = int(params.shape[1])
    R = load().mrstat_lowrank_rank(plan)
    _check(load().mrstat_lowrank_project_samples(plan, _ptr(params, torch.float32, (2, ns), "params"),
                                                 _ptr(b1, torch.float32, (ns,), "b1"), ns,
                                                 _ptr(coef, torch.float32, (3, R, ns), "coef"), _stream(stream)),
           "mrstat_lowrank_project_samples")


def mrstat_mlp_create(hidden, rank, norm, sobolev_weight=1.0, seed=0):
    cfg = mrstat_mlp_config(int(hidden), int(rank), (ctypes.c_float * 6)(*[float(x) for x in norm]),
                            float(sobolev_weight), int(seed))
    h = ctypes.c_void_p()
    _check(load().mrstat_mlp_create(ctypes.byref(cfg), ctypes.byref(h)), "mrstat_mlp_create")
    return h


def mrstat_mlp_destroy(mlp):
    _check(load().mrstat_mlp_destroy(mlp), "mrstat_mlp_destroy")


def mrstat_mlp_num_params(mlp) -> int:
    return int(load().mrstat_mlp_num_params(mlp))


def mrstat_mlp_set_output_scale(mlp, scale):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(scale, np.float32))
    _check(load().mrstat_mlp_set_output_scale(mlp, a.ctypes.data_as(ctypes.c_void_p)), "mrstat_mlp_set_output_scale")


def mrstat_mlp_get_params(mlp):
    import numpy as np
    out = np.empty(mrstat_mlp_num_params(mlp), np.float32)
    _check(load().mrstat_mlp_get_params(mlp, out.ctypes.data_as(ctypes.c_void_p)), "mrstat_mlp_get_params")
    return out


def mrstat_mlp_set_params(mlp, params):
    import numpy as np
    a = np.ascontiguousarray(np.asarray(params, np.float32))
    if a.size != mrstat_mlp_num_params(mlp):
        raise ValueError("parameter vector has the wrong length")
    _check(load().mrstat_mlp_set_params(mlp, a.ctypes.data_as(ctypes.c_void_p)), "mrstat_mlp_set_params")


def mrstat_mlp_train_step(mlp, lnT, b1, target, lr, loss=None, stream=None):
    B = int(lnT.shape[1])
    _check(load().mrstat_mlp_train_step(mlp, _ptr(lnT, torch.float32, (2, B), "lnT"),
                                        _ptr(b1, torch.float32, (B,), "b1"),
                                        _ptr(target, torch.float32, (3, target.shape[1], B), "target"), B, float(lr),
                                        _ptr(loss, torch.float64, (), "loss"), _stream(stream)), "mrstat_mlp_train_step")


def mrstat_mlp_loss_grad(mlp, lnT, b1, target, grad=None, stream=None) -> float:
    B = int(lnT.shape[1])
    L = ctypes.c_double()
    _check(load().mrstat_mlp_loss_grad(mlp, _ptr(lnT, torch.float32, (2, B), "lnT"), _ptr(b1, torch.float32, (B,), "b1"),
                                       _ptr(target, torch.float32, (3, target.shape[1], B), "target"), B,
                                       ctypes.byref(L), _ptr(grad, torch.float32, None, "grad"), _stream(stream)),
           "mrstat_mlp_loss_grad")
    return L.value


def mrstat_mlp_infer(mlp, lnT, b1, coef, stream=None):
    n = int(lnT.shape[1])
    _check(load().mrstat_mlp_infer(mlp, _ptr(lnT, torch.float32, (2, n), "lnT"), _ptr(b1, torch.float32, (n,), "b1"), n,
                                   _ptr(coef, torch.float32, (3, coef.shape[1], n), "coef"), _stream(stream)),
           "mrstat_mlp_infer")


def mrstat_dot_static(a, b, out, stream=None):
    """Allocation-free inner product (no plan); out: cuda float64 scalar tensor."""
    n = int(a.numel())
    _check(load().mrstat_dot_static(_ptr(a, torch.float32, (n,), "a"), _ptr(b, torch.float32, (n,), "b"), n,
                                    _ptr(out, torch.float64, None, "out"), _stream(stream)), "mrstat_dot_static")
    return out
