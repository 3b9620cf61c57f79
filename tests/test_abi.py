"""C ABI: the library builds, loads without a GPU, exports every entry point
declared in include/hz.h, and rejects bad arguments on the host before any
device work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1510_01831_gb300 import hz

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hz_[a-zA-Z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = hz.load()
    names = _declared()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(hz.EXPORTS) == names


def test_default_opts():
    o = hz.hz_default_opts()
    assert o.precision == hz.HZ_FP64 and o.precond == hz.HZ_PGS
    assert o.restart == 30 and o.max_it == 200 and o.refine_tol == 1e-8
    assert o.wait_ms == 1000.0
    assert o.compress == -1.0  # automatic: compressed inner factors in mixed precision


def test_struct_layouts_match_header():
    # field order and sizes of hz_opts / hz_stats as declared in include/hz.h
    src = open(os.path.join(ROOT, "include", "hz.h")).read()
    body = src[src.index("typedef struct {\n    int precision;"):src.index("} hz_opts;")]
    fields = re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*;", body, flags=re.M)
    assert fields == [f for f, _ in hz.HzOpts._fields_]
    body = src[src.index("typedef struct {\n    int iterations;"):src.index("} hz_stats;")]
    fields = re.findall(r"^\s*\w+\s+(\w+)\s*(?:\[\d+\])?\s*;", body, flags=re.M)
    assert fields == [f for f, _ in hz.HzStats._fields_]


@pytest.mark.parametrize("args,frag", [
    (dict(n_x=0), "n_x"),
    (dict(L=1), "L"),
    (dict(C=0), "C"),
    (dict(n_pml=0), "n_pml"),
    (dict(omega=float("nan")), "omega"),
    (dict(h=-1.0), "omega and h"),
])
def test_setup_rejects_bad_sizes(args, frag):
    base = dict(n_x=8, n_z=8, omega=10.0, h=0.1, n_pml=2, L=2, C=2)
    base.update(args)
    NX, NZ = max(base["n_x"], 0) + 2 * max(base["n_pml"], 0), base["n_z"] + 2 * max(base["n_pml"], 0)
    m = np.ones((max(NZ, 1), max(NX, 1)))
    lib = hz.load()
    h_ = ctypes.c_void_p()
    o = hz.hz_default_opts()
    st = lib.hz_setup(ctypes.byref(h_), m.ctypes.data, base["n_x"], base["n_z"], base["omega"], base["h"],
                      base["n_pml"], base["L"], base["C"], ctypes.byref(o))
    assert st == hz.HZ_EINVAL
    assert h_.value is None
    assert lib.hz_last_error(None)


def test_setup_rejects_bad_medium_and_partition():
    lib = hz.load()
    m = np.ones((12, 12))
    m[3, 4] = np.nan
    h_ = ctypes.c_void_p()
    o = hz.hz_default_opts()
    assert lib.hz_setup(ctypes.byref(h_), m.ctypes.data, 8, 8, 10.0, 0.1, 2, 2, 2, ctypes.byref(o)) == hz.HZ_EINVAL
    assert b"m must be" in lib.hz_last_error(None)
    m = np.ones((12, 12))
    rows = (ctypes.c_int * 2)(3, 4)  # sums to 7, not 8
    o.layer_rows = ctypes.cast(rows, ctypes.POINTER(ctypes.c_int))
    assert lib.hz_setup(ctypes.byref(h_), m.ctypes.data, 8, 8, 10.0, 0.1, 2, 2, 2, ctypes.byref(o)) == hz.HZ_EINVAL
    assert b"layer_rows" in lib.hz_last_error(None)
    o = hz.hz_default_opts()
    o.precision = 7
    assert lib.hz_setup(ctypes.byref(h_), m.ctypes.data, 8, 8, 10.0, 0.1, 2, 2, 2, ctypes.byref(o)) == hz.HZ_EINVAL


def test_null_context_calls_fail_cleanly():
    lib = hz.load()
    assert lib.hz_factor(None) == hz.HZ_EINVAL
    assert lib.hz_solve(None, None, 1, None, None) == hz.HZ_EINVAL
    assert lib.hz_update_model(None, None, None) == hz.HZ_EINVAL
    assert lib.hz_device_bytes(None) == 0
    lib.hz_destroy(None)
    assert lib.hz_solve_group(None, 1, None, 1, None, None) == hz.HZ_EINVAL
    G = 2
    hs = (ctypes.c_void_p * G)(None, None)
    assert lib.hz_solve_group(hs, G, None, 1, None, None) == hz.HZ_EINVAL
    assert lib.hz_solve_group(hs, 0, None, 1, None, None) == hz.HZ_EINVAL


def test_setup_rejects_unknown_krylov():
    lib = hz.load()
    m = np.ones((12, 12))
    o = hz.hz_default_opts()
    o.krylov = 7
    h_ = ctypes.c_void_p()
    assert lib.hz_setup(ctypes.byref(h_), m.ctypes.data, 8, 8, 10.0, 0.1, 2, 2, 2, ctypes.byref(o)) == hz.HZ_EINVAL
    assert b"krylov" in lib.hz_last_error(None)


def test_setup_rejects_unknown_tensor_core_mode():
    lib = hz.load()
    m = np.ones((12, 12))
    o = hz.hz_default_opts()
    o.tensor_cores = 3
    h_ = ctypes.c_void_p()
    assert lib.hz_setup(ctypes.byref(h_), m.ctypes.data, 8, 8, 10.0, 0.1, 2, 2, 2, ctypes.byref(o)) == hz.HZ_EINVAL
    assert b"tensor_cores" in lib.hz_last_error(None)


def test_setup_rejects_bad_lane_count():
    lib = hz.load()
    m = np.ones((12, 12))
    o = hz.hz_default_opts()
    assert o.rhs_lanes == 1
    o.rhs_lanes = 0
    h_ = ctypes.c_void_p()
    assert lib.hz_setup(ctypes.byref(h_), m.ctypes.data, 8, 8, 10.0, 0.1, 2, 2, 2, ctypes.byref(o)) == hz.HZ_EINVAL
    assert b"rhs_lanes" in lib.hz_last_error(None)


@pytest.mark.parametrize("C,krylov,lanes,inner", [(1, 0, 1, 1), (2, 1, 1, 1), (2, 0, 2, 1), (2, 0, 1, 5)])
def test_setup_rejects_unsupported_nested_inner_level(C, krylov, lanes, inner):
    # the nested inner level needs cells to sweep over, a flexible outer solver and one lane
    lib = hz.load()
    m = np.ones((12, 12))
    o = hz.hz_default_opts()
    o.inner, o.krylov, o.rhs_lanes = inner, krylov, lanes
    h_ = ctypes.c_void_p()
    assert lib.hz_setup(ctypes.byref(h_), m.ctypes.data, 8, 8, 10.0, 0.1, 2, 2, C, ctypes.byref(o)) == hz.HZ_EINVAL
    assert b"inner" in lib.hz_last_error(None)
