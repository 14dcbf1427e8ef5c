"""mrstat_dot_static, the allocation-free inner product, against mrstat_dot.

Collected last on purpose: it must pass both alone in a fresh process (the first call
on the device performs the scratch-address look-up) and after every other test.  The
GPU test calls the C entry point directly and compares two calls in a row of the same
size with the plan-based mrstat_dot, at the dot-product bar of the parity tests (2e-7 of
sum |a b|), and checks that those calls take no device memory.
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
    """For each size: two back-to-back static calls of the same n (the second reuses the
    shared scratch and ticket the first left behind) both match mrstat_dot and the float64
    dot product; the device's free memory (cudaMemGetInfo) is the same before and after
    those calls, which follow a warm-up call of the same size."""
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
            got = [torch.full((), np.nan, dtype=torch.float64, device="cuda") for _ in range(3)]
            ref = torch.full((), np.nan, dtype=torch.float64, device="cuda")
            st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

            def static_dot(out):
                status = lib.mrstat_dot_static(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), n,
                                               ctypes.c_void_p(out.data_ptr()), st)
                assert status == 0, lib.mrstat_last_error().decode()

            static_dot(got[0])  # warm-up (the first call on a device looks up the scratch)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            static_dot(got[1])
            static_dot(got[2])
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            assert free1 == free0, (n, free0, free1)
            status = lib.mrstat_dot(plan.handle, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), n,
                                    ctypes.c_void_p(ref.data_ptr()), st)
            assert status == 0, lib.mrstat_last_error().decode()
            torch.cuda.synchronize()
            scale = float(torch.sum(torch.abs(a.double() * b.double())))
            exact = float(torch.dot(a.double(), b.double()))
            for g in got:
                assert abs(float(g) - float(ref)) <= 2e-7 * scale, (n, float(g), float(ref))
                assert abs(float(g) - exact) <= 2e-7 * scale
            # the same arithmetic in the same order: the repeated calls agree exactly
            assert float(got[1]) == float(got[2]) == float(got[0])
