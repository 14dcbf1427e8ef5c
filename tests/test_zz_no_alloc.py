"""mrstat_dot_static, the allocation-free inner product, against mrstat_dot.

Collected last on purpose: it must pass both alone in a fresh process (the first call
on the device performs the scratch-address look-up) and after every other test.  The
GPU test calls the C entry point directly and compares two calls in a row with the
plan-based mrstat_dot, at the dot-product bar of the parity tests (2e-7 of sum |a b|).
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

MAX_N = 4096 * 256 * 16


def _lib():
    from paper_1904_13244_gb300 import _binding
    return _binding.load()


def test_sizes_beyond_the_static_scratch_are_rejected():
    lib = _lib()
    dummy = ctypes.c_void_p(256)  # never dereferenced: the size check comes first
    for n in (MAX_N + 1, -1):
        assert lib.mrstat_dot_static(dummy, dummy, n, dummy, None) == 1
        assert "mrstat_dot_static" in lib.mrstat_last_error().decode()


@pytest.mark.gpu
def test_two_calls_in_a_row_match_mrstat_dot():
    from paper_1904_13244_gb300 import build
    import paper_1904_13244_gb300 as mr
    build.build()
    lib = _lib()
    seq, _ = synth.config("quad16")
    rng = np.random.default_rng(11)
    with mr.Plan(seq) as plan:
        for n in (1_000_003, MAX_N):
            a = torch.tensor(rng.standard_normal(n), dtype=torch.float32, device="cuda")
            b = torch.tensor(rng.standard_normal(n), dtype=torch.float32, device="cuda")
            got = torch.full((), np.nan, dtype=torch.float64, device="cuda")
            ref = torch.full((), np.nan, dtype=torch.float64, device="cuda")
            st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            status = lib.mrstat_dot_static(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), n,
                                           ctypes.c_void_p(got.data_ptr()), st)
            assert status == 0, lib.mrstat_last_error().decode()
            status = lib.mrstat_dot(plan.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), n,
                                    ctypes.c_void_p(ref.data_ptr()), st)
            assert status == 0, lib.mrstat_last_error().decode()
            torch.cuda.synchronize()
            scale = float(torch.sum(torch.abs(a.double() * b.double())))
            assert abs(float(got) - float(ref)) <= 2e-7 * scale, (n, float(got), float(ref))
            exact = float(torch.dot(a.double(), b.double()))
            assert abs(float(got) - exact) <= 2e-7 * scale
