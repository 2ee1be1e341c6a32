"""The C-ABI library loads and exports every entry point include/of.h
declares; host-side logic of the binding and the partition prior (no GPU
compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "of.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(of_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_02977_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("of_create", "of_setup_grid", "of_set_frames", "of_set_alpha", "of_solve", "of_adjoint",
              "of_adapt_alpha", "of_destroy", "of_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_wraps_every_export(lib):
    from paper_1508_02977_gb300 import ofsolve
    assert set(ofsolve.EXPORTS) == set(declared_symbols())
    for s in ofsolve.EXPORTS:
        assert callable(getattr(ofsolve, s))


def test_struct_layouts_match_header():
    from paper_1508_02977_gb300 import ofsolve as S
    # of_grid_opts: 4 ints, enum, (pad), double, enum, (pad), double, double, enum, int, double, int, (pad),
    # double, int (+ pad);
    # of_solve_opts: double, 3 ints, (pad), double, int (+ pad)
    assert ctypes.sizeof(S.GridOpts) == 96
    assert [getattr(S.GridOpts, f).offset for f in
            ("tile_x", "sweeps", "precision", "lam", "preconditioner", "omega", "sigma", "model", "coarse",
             "rho", "schwarz", "lambda_min", "half_sweeps")] == [0, 12, 16, 24, 32, 40, 48, 56, 60, 64, 72, 80, 88]
    assert ctypes.sizeof(S.SolveOpts) == 48
    assert [getattr(S.SolveOpts, f).offset for f in
            ("rtol", "max_outer", "max_inner", "warm_start", "inner_rtol", "host_loop", "pass_frac")] == \
        [0, 8, 12, 16, 24, 32, 40]
    assert ctypes.sizeof(S.SolveInfo) == 32


def test_create_without_gpu_reports_an_error(lib):
    """On a machine without a GPU of_create must return a status (not
    abort) and leave a message."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    lib.of_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]
    lib.of_last_error.restype = ctypes.c_char_p
    lib.of_last_error.argtypes = [ctypes.c_void_p]
    st = lib.of_create(ctypes.byref(h), 0, None)
    assert st == 2  # OF_ERR_CUDA
    assert len(lib.of_last_error(None)) > 0


def test_null_handle_calls_return_arg_error(lib):
    lib.of_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.of_solve(None, None, None, 0, None) == 1  # OF_ERR_ARG
    lib.of_set_alloc_limit.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.of_set_alloc_limit(None, 0) == 1
    lib.of_destroy.argtypes = [ctypes.c_void_p]
    assert lib.of_destroy(None) == 0
