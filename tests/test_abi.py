"""Host-side checks of the C ABI that need no GPU: the library builds and loads, it
exports every entry point include/mrstat.h declares, and argument validation in
mrstat_plan_create rejects bad sequences before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_13244_gb300 import build as b
    b.build()
    from paper_1904_13244_gb300 import _binding
    return _binding.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mrstat.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrstat_\w+)\s*\(", text)))


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert "mrstat_jvp" in names and "mrstat_jhw" in names and "mrstat_forward" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_1904_13244_gb300 import _binding
    assert sorted(_binding.exported_symbols()) == names


def test_status_strings(lib):
    lib.mrstat_status_string.restype = ctypes.c_char_p
    assert lib.mrstat_status_string(0) == b"ok"
    assert lib.mrstat_status_string(3) == b"plan not linearised"
    assert lib.mrstat_status_string(99) == b"unknown status"


def _create(seq_kwargs, form=0):
    from paper_1904_13244_gb300 import _binding as b
    seq = synth.make_sequence(8, 8, 1, 7.8, 3.9)
    for k, v in seq_kwargs.items():
        setattr(seq, k, v)
    with pytest.raises(b.MrstatError) as e:
        b.mrstat_plan_create(seq, form)
    return e.value.status


def test_plan_create_validates_before_touching_the_gpu(lib):
    assert _create({"nx": 0}) == 2
    assert _create({"ny": 5000}) == 2
    assert _create({"nkx": 0}) == 2
    assert _create({"flip_rad": np.zeros(0), "ky": np.zeros(0, np.int32)}) == 2   # empty train
    assert _create({"te_ms": 9.0}) == 1                                            # te >= tr
    assert _create({"te_ms": -1.0}) == 1
    assert _create({"flip_rad": np.full(8, np.nan)}) == 1
    assert _create({"flip_rad": -np.ones(8)}) == 1
    assert _create({"ky": np.full(8, 4, np.int32)}) == 2                           # ky >= ny/2
    assert _create({"ky": np.full(8, -5, np.int32)}) == 2
    assert _create({}, form=7) == 1


def test_null_arguments_are_rejected(lib):
    lib.mrstat_plan_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    assert lib.mrstat_plan_create(None, 0, ctypes.byref(h)) == 1
    assert lib.mrstat_jvp(None, None, None, None) == 1
    assert lib.mrstat_jhw(None, None, None, None) == 1
    assert lib.mrstat_linearize(None, None, None, None, None) == 1
    assert lib.mrstat_plan_destroy(None) == 0
    assert lib.mrstat_cg_applied(None, None) == 1
    n = ctypes.c_int32(-1)
    assert lib.mrstat_cg_applied(None, ctypes.byref(n)) == 1 and n.value == -1
    assert lib.mrstat_plan_inject_grid_stall(None, 0) == 1
