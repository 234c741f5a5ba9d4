"""The C-ABI library builds, loads, and exports every declared symbol.

No GPU needed: only argument validation that runs before any CUDA call is
exercised here.
"""
import ctypes as C
import os
import re

import pytest

from paper_0907_3390_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gamer_hydro.h")).read()
    return sorted(set(re.findall(r"\b(gamer_(?:hydro|poisson|gravity)_\w+)\s*\(", src)))


def test_header_matches_binding_exports():
    assert declared_functions() == sorted(B.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = B.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_create_rejects_bad_arguments_before_touching_the_device():
    lib = B.load()
    h = C.c_void_p()
    assert lib.gamer_hydro_create(5 / 3, 0, 4, 0, C.byref(h)) == B.GAMER_ERR_UNSUPPORTED
    assert b"ghost_width" in lib.gamer_hydro_last_error(None)
    assert lib.gamer_hydro_create(1.0, 0, 3, 0, C.byref(h)) == B.GAMER_ERR_ARG
    assert lib.gamer_hydro_create(5 / 3, 7, 3, 0, C.byref(h)) == B.GAMER_ERR_ARG
    assert lib.gamer_hydro_create(5 / 3, 0, 3, 9, C.byref(h)) == B.GAMER_ERR_ARG
    assert lib.gamer_hydro_create(5 / 3, 0, 3, 0, None) == B.GAMER_ERR_ARG


def test_null_handle_is_rejected():
    lib = B.load()
    assert lib.gamer_hydro_destroy(None) == B.GAMER_OK
    assert lib.gamer_hydro_advance(None, None, 0, 0.1) == B.GAMER_ERR_ARG
    assert lib.gamer_hydro_cfl_dt(None, None, 0.5, None) == B.GAMER_ERR_ARG
    assert lib.gamer_hydro_set_launch_groups(None, 1) == B.GAMER_ERR_ARG


def test_struct_layouts_match_header():
    # gamer_level_t: 2 int32 + double + 6 pointers; gamer_hierarchy_t: 2 int32 + ptr + u64
    assert C.sizeof(B.gamer_level_t) == 8 + 8 + 6 * 8
    assert C.sizeof(B.gamer_hierarchy_t) == 8 + 8 + 8


def test_gravity_update_validates_before_any_cuda_call():
    lib = B.load()
    assert lib.gamer_gravity_update(7, 1, None, None, 0.1, 0.01, None) == B.GAMER_ERR_ARG
    assert lib.gamer_gravity_update(B.GAMER_FP32, -1, None, None, 0.1, 0.01, None) == B.GAMER_ERR_ARG
    assert lib.gamer_gravity_update(B.GAMER_FP32, 1, None, None, 0.0, 0.01, None) == B.GAMER_ERR_ARG
    assert lib.gamer_gravity_update(B.GAMER_FP32, 1, None, None, 0.1, -1.0, None) == B.GAMER_ERR_ARG
    assert lib.gamer_gravity_update(B.GAMER_FP64, 1, None, None, 0.1, float("nan"), None) == B.GAMER_ERR_ARG
    assert lib.gamer_gravity_update(B.GAMER_FP32, 1, None, None, 0.1, 0.01, None) == B.GAMER_ERR_ARG
    assert lib.gamer_gravity_update(B.GAMER_FP32, 0, None, None, 0.1, 0.01, None) == B.GAMER_OK


def test_poisson_sor_validates_before_any_cuda_call():
    lib = B.load()
    assert lib.gamer_poisson_sor(B.GAMER_FP32, 1, None, None, 1.0, 2.5, 10, 0.0, None, None) == B.GAMER_ERR_ARG
    assert lib.gamer_poisson_sor(7, 1, None, None, 1.0, 1.5, 10, 0.0, None, None) == B.GAMER_ERR_ARG
    assert lib.gamer_poisson_sor(B.GAMER_FP32, 1, None, None, 1.0, 1.5, 10, -1.0, None, None) == B.GAMER_ERR_ARG
    assert lib.gamer_poisson_sor(B.GAMER_FP32, 1, None, None, 1.0, 1.5, 10, 0.0, None, None) == B.GAMER_ERR_ARG
    assert lib.gamer_poisson_sor(B.GAMER_FP32, 0, None, None, 1.0, 1.5, 10, 0.0, None, None) == B.GAMER_OK

