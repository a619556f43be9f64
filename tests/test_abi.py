"""Host-side checks of the C ABI: the library loads, exports every entry point include/rmge.h declares,
sizes its buffers, and rejects bad arguments before touching the GPU (no CUDA call is made here)."""
import ctypes as C
import os
import re

import pytest

from paper_1406_5802_gb300 import build as B
from paper_1406_5802_gb300 import rmge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return rmge.load_library()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rmge_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert set(rmge.EXPORTED) <= declared


def test_workspace_and_multiplier_sizes(lib):
    assert rmge.workspace_size(4096, 16, "gaussian", "f64") > 3 * 4096 * 16 * 8
    assert rmge.workspace_size(4096, 16, "circulant", "f64") > rmge.workspace_size(4096, 16, "gaussian", "f64")
    assert rmge.workspace_size(0, 1, "gaussian", "f64") == 0
    assert rmge.workspace_size(100, 1, "circulant", "f64") == 0  # circulant needs n = 2^p
    assert rmge.multiplier_bytes("gaussian", 256, "f64") == 256 * 256 * 8
    assert rmge.multiplier_bytes("gaussian", 256, "f32") == 256 * 256 * 4
    assert rmge.multiplier_bytes("circulant", 256, "f64") == 3 * 256 * 8
    # one real transform of length 4 .. 16384 per CTA
    assert rmge.multiplier_bytes("circulant", 16384, "f64") == 3 * 16384 * 8
    assert rmge.multiplier_bytes("circulant", 32768, "f64") == 0
    assert rmge.multiplier_bytes("circulant", 2, "f64") == 0
    # the unitary circulant stores like the others; a Toeplitz multiplier stores its 2n circulant
    assert rmge.multiplier_bytes("circulant_unitary", 16384, "f64") == 3 * 16384 * 8
    assert rmge.multiplier_bytes("toeplitz", 4096, "f64") == 6 * 4096 * 8
    assert rmge.multiplier_bytes("toeplitz_uniform", 64, "f32") == 6 * 64 * 8
    assert rmge.multiplier_bytes("toeplitz", 8192, "f64") == 6 * 8192 * 8
    assert rmge.multiplier_bytes("toeplitz", 16384, "f64") == 0  # its 32768-point transform is too long
    assert rmge.multiplier_bytes("toeplitz", 2, "f64") == 6 * 2 * 8
    assert rmge.multiplier_bytes("toeplitz", 1000, "f64") == 0  # not a power of two
    assert rmge.workspace_size(1000, 1, "toeplitz", "f64") == 0


def test_bad_arguments_are_rejected_without_gpu_work(lib):
    INVALID, WORKSPACE = 1, 7
    # n = 0, NULL matrix, ld < n
    assert lib.rmge_factor(0, None, 1, 0, None, None, None, 0, None) == INVALID
    assert lib.rmge_factor(8, None, 8, 0, None, None, None, 0, None) == INVALID
    assert lib.rmge_factor(8, C.c_void_p(256), 4, 0, None, None, None, 0, None) == INVALID
    # valid shape, missing / misaligned / short workspace
    assert lib.rmge_factor(8, C.c_void_p(256), 8, 0, None, None, None, 0, None) == WORKSPACE
    assert lib.rmge_factor(8, C.c_void_p(256), 8, 0, None, None, C.c_void_p(256 + 8), 1 << 20, None) == WORKSPACE
    assert lib.rmge_factor(8, C.c_void_p(256), 8, 0, None, None, C.c_void_p(512), 16, None) == WORKSPACE
    # unknown enum values and too many refinement sweeps
    assert lib.rmge_make_multiplier(7, 8, 1, 1, 0, C.c_void_p(256), None) == INVALID
    p = C.c_void_p(256)
    assert lib.rmge_refine(0, 8, 1, p, 8, p, 8, p, p, 1, p, 1, 0, 99, 1e-13, None, None, p, 1 << 20, None) == INVALID
    assert lib.rmge_refine(0, 8, 1, p, 8, p, 8, p, p, 1, p, 1, 0, 3, -1.0, None, None, p, 1 << 20, None) == INVALID
    assert lib.rmge_status_string(6) == b"bounded device wait expired"
    # empty inputs: no right-hand sides, an empty batch
    assert lib.rmge_solve(0, 8, 0, p, 8, p, p, 1, p, 1, 0, p, 1 << 20, None) == INVALID
    assert lib.rmge_workspace_size(8, 0, 0, 0) == 0
    lib.rmge_solve_batched.restype = C.c_int
    lib.rmge_solve_batched.argtypes = [C.c_int64] + [C.c_void_p] * 10 + [C.c_uint64, C.c_int32, C.c_double,
                                                                          C.c_int64, C.c_int32, C.c_int32,
                                                                          C.c_void_p, C.c_size_t, C.c_void_p]
    assert lib.rmge_solve_batched(0, p, p, p, p, p, p, p, p, p, p, 1, 10, 1e-13, 8, 1, 152, p, 1 << 20,
                                  None) == INVALID


def test_options_defaults_and_validation(lib):
    INVALID = 1
    o = rmge.options()
    assert o.growth_tol == 0.0 and o.gmres_m == 16 and o.spin_limit == 1 << 22 and o.sync == 0 and not o.status
    assert o.apply_digits == 7 and o.factor_digits == 7
    assert rmge.workspace_size_ex(64, 1, "gaussian", "f64x", rmge.options(factor_digits=3)) == 0
    assert rmge.workspace_size_ex(64, 1, "gaussian", "f64x", rmge.options(factor_digits=8)) == 0
    assert rmge.workspace_size_ex(64, 1, "gaussian", "f64x", rmge.options(factor_digits=4)) > 0
    assert rmge.workspace_size_ex(64, 1, "gaussian", "f64x", rmge.options(apply_digits=0)) == 0
    assert rmge.workspace_size_ex(64, 1, "gaussian", "f64x", rmge.options(apply_digits=8)) == 0
    # the FGMRES basis grows with the restart length; out-of-range options make every size request invalid
    base = rmge.workspace_size_ex(4096, 8, "gaussian", "bf16x3", o)
    assert base == rmge.workspace_size(4096, 8, "gaussian", "bf16x3")
    assert rmge.workspace_size_ex(4096, 8, "gaussian", "bf16x3", rmge.options(gmres_m=64)) > base
    assert rmge.workspace_size_ex(4096, 8, "gaussian", "f64", rmge.options(gmres_m=64)) == \
        rmge.workspace_size(4096, 8, "gaussian", "f64")  # FP64 factors refine classically: no basis
    assert rmge.workspace_size_ex(4096, 8, "gaussian", "bf16x3", rmge.options(gmres_m=257)) == 0
    assert rmge.workspace_size_ex(4096, 8, "gaussian", "bf16x3", rmge.options(gmres_m=0)) == 0
    assert rmge.workspace_size_ex(64, 1, "gaussian", "f64", rmge.options(growth_tol=-1.0)) == 0
    assert rmge.workspace_size_ex(64, 1, "gaussian", "f64", rmge.options(spin_limit=-1)) == 0
    p = C.c_void_p(256)
    bad = rmge.options(gmres_m=1000)
    assert lib.rmge_factor_ex(8, p, 8, 0, None, None, C.byref(bad), p, 1 << 20, None) == INVALID
    assert lib.rmge_solve_ex(0, 8, 1, p, 8, p, p, 1, p, 1, 0, C.byref(bad), p, 1 << 20, None) == INVALID
    assert lib.rmge_refine_ex(0, 8, 1, p, 8, p, 8, p, p, 1, p, 1, 0, 3, 1e-13, None, None, C.byref(bad), p, 1 << 20,
                              None) == INVALID
    assert lib.rmge_solve_batched_ex(4, p, p, p, p, p, p, p, p, p, p, 1, 10, 1e-13, 8, 1, 152, C.byref(bad), p,
                                     1 << 20, None) == INVALID
    assert lib.rmge_status_string(9) == b"non-finite values in the result"
    assert lib.rmge_status_string(3) == b"growth above threshold"


def test_uniform_batch_sizes_and_argument_checks(lib):
    INVALID, WORKSPACE, UNSUPPORTED = 1, 7, 8
    assert lib.rmge_batched_uniform_workspace_size(64, 2048, 6) > 2 * 64 * 7 * 2048 * 2048 * 2
    assert lib.rmge_batched_uniform_workspace_size(64, 2048, 0) == 0  # emulated FP64 only
    assert lib.rmge_batched_uniform_workspace_size(0, 2048, 6) == 0
    assert lib.rmge_batched_uniform_workspace_size(70000, 64, 6) == 0
    p = C.c_void_p(256)
    # overlapping systems (stride below (n - 1) ld + n) are refused before any GPU work
    assert lib.rmge_factor_batched(2, 8, p, 8, 10, 6, p, None, None, p, 1 << 20, None) == INVALID
    assert lib.rmge_factor_batched(2, 8, p, 8, 64, 0, p, None, None, p, 1 << 20, None) == UNSUPPORTED
    assert lib.rmge_factor_batched(2, 8, p, 8, 64, 6, p, None, None, p, 16, None) == WORKSPACE
    bad = rmge.options(factor_digits=3)
    assert lib.rmge_factor_batched(2, 8, p, 8, 64, 6, p, None, C.byref(bad), p, 1 << 20, None) == INVALID
    assert lib.rmge_apply_multiplier_batched(2, 8, p, 8, 64, p, 64, p, 8, 63, 6, None, p, 1 << 20, None) == INVALID


def test_launch_timing_arguments_and_empty_records(lib):
    """rmge_launch_timing rejects flags other than 0 and 1, rmge_launch_timing_read unknown launch classes
    and null outputs; with nothing launched the records are empty (no CUDA call is made)."""
    INVALID = rmge.CODES["RMGE_ERR_INVALID_ARG"]
    assert lib.rmge_launch_timing(2) == INVALID
    n, ms, fl = C.c_int64(-1), C.c_double(-1.0), C.c_double(-1.0)
    assert lib.rmge_launch_timing_read(2, C.byref(n), C.byref(ms), C.byref(fl)) == INVALID
    assert lib.rmge_launch_timing_read(-1, C.byref(n), C.byref(ms), C.byref(fl)) == INVALID
    assert lib.rmge_launch_timing_read(0, None, C.byref(ms), C.byref(fl)) == INVALID
    rmge.launch_timing(True)
    assert rmge.launch_timing_read(rmge.TIMED_UPDATE128) == (0, 0.0, 0.0)
    assert rmge.launch_timing_read(rmge.TIMED_UPDATE) == (0, 0.0, 0.0)
    rmge.launch_timing(False)
