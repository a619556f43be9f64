"""Thin Python binding of librmge (argument marshalling only).

Every function here has the name of the C entry point it wraps (``include/rmge.h``) without the
``rmge_`` prefix, takes torch tensors, passes their device pointers and the current CUDA stream
to the library, and raises ``RmgeError`` on a non-OK status.  All arithmetic runs in the
library's CUDA kernels; PyTorch only provides device memory and streams.  There is no fallback:
if the library is not built or no CUDA device is present, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librmge.so")

# enums (include/rmge.h)
GAUSSIAN, CIRCULANT_GAUSSIAN, CIRCULANT_UNIFORM = 0, 1, 2
F64, F32, BF16_TC, F16_TC = 0, 1, 2, 3
KINDS = {"gaussian": GAUSSIAN, "circulant": CIRCULANT_GAUSSIAN, "circulant_uniform": CIRCULANT_UNIFORM,
         "circulant_unitary": 3, "toeplitz": 4, "toeplitz_uniform": 5}
PRECS = {"f64": F64, "f32": F32, "bf16": BF16_TC, "f16": F16_TC, "bf16x3": 4, "f16x3": 5, "f64x": 6}
STATUS = {0: "RMGE_OK", 1: "RMGE_ERR_INVALID_ARG", 2: "RMGE_ERR_BREAKDOWN", 3: "RMGE_ERR_GROWTH",
          4: "RMGE_ERR_NOT_CONVERGED", 5: "RMGE_ERR_CUDA", 6: "RMGE_ERR_TIMEOUT", 7: "RMGE_ERR_WORKSPACE",
          8: "RMGE_ERR_UNSUPPORTED", 9: "RMGE_ERR_NONFINITE"}
CODES = {v: k for k, v in STATUS.items()}
# outcomes a synchronising _ex call returns (numerical results, not errors of the call)
OUTCOMES = {0, 2, 3, 4, 6, 9}

EXPORTED = ["rmge_multiplier_bytes", "rmge_workspace_size", "rmge_make_multiplier", "rmge_apply_multiplier",
            "rmge_factor", "rmge_solve", "rmge_refine", "rmge_solve_backward", "rmge_status_string",
            "rmge_kernel_launches", "rmge_solve_workspace_size", "rmge_solve_noalloc", "rmge_noalloc_capacity",
            "rmge_workspace_size_two_sided", "rmge_apply_two_sided", "rmge_solve_two_sided", "rmge_refine_two_sided",
            "rmge_lowrank_workspace_size", "rmge_lowrank_multiplier", "rmge_lowrank_basis", "rmge_lowrank_project",
            "rmge_options_init", "rmge_workspace_size_ex", "rmge_factor_ex", "rmge_solve_ex", "rmge_refine_ex",
            "rmge_apply_multiplier_ex", "rmge_batched_uniform_workspace_size", "rmge_apply_multiplier_batched",
            "rmge_factor_batched", "rmge_uniform_solve_workspace_size", "rmge_solve_uniform_batched",
            "rmge_refine_uniform_batched", "rmge_solve_backward_uniform_batched",
            "rmge_solve_batched", "rmge_solve_batched_ex", "rmge_batched_workspace_size", "rmge_launch_timing",
            "rmge_launch_timing_read"]


class Options(C.Structure):
    """rmge_options (include/rmge.h)."""
    _fields_ = [("growth_tol", C.c_double), ("spin_limit", C.c_int64), ("status", C.c_void_p), ("gmres_m", C.c_int32),
                ("apply_digits", C.c_int32), ("sync", C.c_int32), ("factor_digits", C.c_int32)]


class RmgeError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {STATUS.get(code, code)}")
        self.code = code


_lib = None
_i64, _u64, _vp, _sz = C.c_int64, C.c_uint64, C.c_void_p, C.c_size_t


def load_library(path: str = LIB_PATH):
    """Load librmge and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librmge is not built ({path} missing): run __graft_entry__.build()")
    L = C.CDLL(path)
    sig = {
        "rmge_multiplier_bytes": (_sz, [C.c_int, _i64, C.c_int]),
        "rmge_workspace_size": (_sz, [_i64, _i64, C.c_int, C.c_int]),
        "rmge_make_multiplier": (C.c_int, [C.c_int, _i64, _u64, _u64, C.c_int, _vp, _vp]),
        "rmge_apply_multiplier": (C.c_int, [C.c_int, _i64, _vp, _i64, _vp, _vp, _i64, C.c_int, _vp, _sz, _vp]),
        "rmge_factor": (C.c_int, [_i64, _vp, _i64, C.c_int, _vp, _vp, _vp, _sz, _vp]),
        "rmge_solve": (C.c_int, [C.c_int, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, C.c_int, _vp, _sz, _vp]),
        "rmge_refine": (C.c_int, [C.c_int, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, C.c_int,
                                  C.c_int32, C.c_double, _vp, _vp, _vp, _sz, _vp]),
        "rmge_solve_backward": (C.c_int, [C.c_int, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, _vp,
                                          _i64, _vp, _i64, C.c_int, C.c_int32, C.c_double, _vp, _vp, _vp, _sz, _vp]),
        "rmge_status_string": (C.c_char_p, [C.c_int]),
        "rmge_kernel_launches": (C.c_ulonglong, []),
        "rmge_launch_timing": (C.c_int, [C.c_int32]),
        "rmge_launch_timing_read": (C.c_int, [C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                              C.POINTER(C.c_double)]),
        "rmge_solve_workspace_size": (_sz, [_i64, _i64, C.c_int, C.c_int]),
        "rmge_solve_noalloc": (C.c_int, [C.c_int, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, C.c_int, _vp]),
        "rmge_noalloc_capacity": (_sz, []),
        "rmge_workspace_size_two_sided": (_sz, [_i64, _i64, C.c_int, C.c_int, C.c_int]),
        "rmge_apply_two_sided": (C.c_int, [C.c_int, _vp, C.c_int, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                                           C.c_int, _vp, _sz, _vp]),
        "rmge_solve_two_sided": (C.c_int, [C.c_int, _vp, C.c_int, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                                           C.c_int, _vp, _sz, _vp]),
        "rmge_refine_two_sided": (C.c_int, [C.c_int, _vp, C.c_int, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp,
                                            _i64, _vp, _i64, C.c_int, C.c_int32, C.c_double, _vp, _vp, _vp, _sz,
                                            _vp]),
        "rmge_lowrank_workspace_size": (_sz, [C.c_int, _i64, _i64, C.c_int32]),
        "rmge_lowrank_multiplier": (C.c_int, [C.c_int, _i64, C.c_int32, _u64, _u64, _vp, _vp]),
        "rmge_lowrank_basis": (C.c_int, [C.c_int, _i64, _i64, C.c_int32, _vp, _i64, _vp, _vp, _i64, _vp, _vp, _sz,
                                         _vp]),
        "rmge_lowrank_project": (C.c_int, [_i64, _i64, C.c_int32, _vp, _i64, _vp, _i64, _vp, _i64, _vp]),
        "rmge_options_init": (None, [C.POINTER(Options)]),
        "rmge_workspace_size_ex": (_sz, [_i64, _i64, C.c_int, C.c_int, C.POINTER(Options)]),
        "rmge_factor_ex": (C.c_int, [_i64, _vp, _i64, C.c_int, _vp, _vp, C.POINTER(Options), _vp, _sz, _vp]),
        "rmge_apply_multiplier_ex": (C.c_int, [C.c_int, _i64, _vp, _i64, _vp, _vp, _i64, C.c_int, C.POINTER(Options),
                                               _vp, _sz, _vp]),
        "rmge_solve_ex": (C.c_int, [C.c_int, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, C.c_int,
                                    C.POINTER(Options), _vp, _sz, _vp]),
        "rmge_refine_ex": (C.c_int, [C.c_int, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, C.c_int,
                                     C.c_int32, C.c_double, _vp, _vp, C.POINTER(Options), _vp, _sz, _vp]),
        "rmge_batched_workspace_size": (_sz, [_i64, C.c_int32]),
        "rmge_batched_uniform_workspace_size": (_sz, [_i64, _i64, C.c_int]),
        "rmge_apply_multiplier_batched": (C.c_int, [_i64, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _i64, C.c_int,
                                                    C.POINTER(Options), _vp, _sz, _vp]),
        "rmge_factor_batched": (C.c_int, [_i64, _i64, _vp, _i64, _i64, C.c_int, _vp, _vp, _vp, _vp, _sz, _vp]),
        "rmge_uniform_solve_workspace_size": (_sz, [_i64, _i64, _i64, C.c_int]),
        "rmge_solve_uniform_batched": (C.c_int, [_i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _i64, _vp,
                                                 _i64, _i64, C.c_int, _vp, _sz, _vp]),
        "rmge_refine_uniform_batched": (C.c_int, [_i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _vp,
                                                  _i64, _i64, _vp, _i64, _i64, C.c_int, C.c_int32, C.c_double, _vp,
                                                  _vp, _vp, _sz, _vp]),
        "rmge_solve_backward_uniform_batched": (C.c_int, [_i64, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64, _vp,
                                                          _i64, _vp, _i64, _i64, _vp, _i64, _i64, _vp, _i64, _i64,
                                                          _vp, _i64, _i64, C.c_int, C.c_int32, C.c_double, _vp, _vp,
                                                          _vp, _sz, _vp]),
        "rmge_solve_batched": (C.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _u64, C.c_int32,
                                         C.c_double, _i64, C.c_int32, C.c_int32, _vp, _sz, _vp]),
        "rmge_solve_batched_ex": (C.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _u64, C.c_int32,
                                            C.c_double, _i64, C.c_int32, C.c_int32, C.POINTER(Options), _vp, _sz,
                                            _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _cuda_lib():
    if not torch.cuda.is_available():
        raise RuntimeError("librmge needs a CUDA device; none is available")
    return load_library()


def _check(fn, code):
    if code != 0:
        raise RmgeError(fn, code)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _ld(t):
    return t.stride(0) if t.dim() == 2 else 1


def _kind(k):
    return KINDS[k] if isinstance(k, str) else int(k)


def _prec(p):
    return PRECS[p] if isinstance(p, str) else int(p)


def _need(t, dtype, name):
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() == 2 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major with unit column stride")


def kernel_launches() -> int:
    """Kernel launches enqueued through the library by this process so far."""
    return int(load_library().rmge_kernel_launches())


# launch classes of rmge_launch_timing (rmge_timed_kernel)
TIMED_UPDATE128, TIMED_UPDATE = 0, 1


def launch_timing(enable: bool) -> None:
    """rmge_launch_timing: True clears the records and starts recording event pairs around the emulated Schur
    updates (no CUDA call until a launch is recorded); False stops recording."""
    _check("rmge_launch_timing", load_library().rmge_launch_timing(1 if enable else 0))


def launch_timing_read(kernel: int):
    """rmge_launch_timing_read: (launches, summed device ms, summed BF16 MMA flops) of one launch class."""
    n, ms, fl = C.c_int64(0), C.c_double(0.0), C.c_double(0.0)
    _check("rmge_launch_timing_read",
           load_library().rmge_launch_timing_read(int(kernel), C.byref(n), C.byref(ms), C.byref(fl)))
    return int(n.value), float(ms.value), float(fl.value)


def factor_dtype(prec) -> torch.dtype:
    return torch.float64 if _prec(prec) in (F64, PRECS["f64x"]) else torch.float32


def multiplier_bytes(kind, n, prec) -> int:
    return int(load_library().rmge_multiplier_bytes(_kind(kind), int(n), _prec(prec)))


def workspace_size(n, nrhs, kind, prec) -> int:
    return int(load_library().rmge_workspace_size(int(n), int(nrhs), _kind(kind), _prec(prec)))


def workspace(n, nrhs, kind, prec, device="cuda") -> torch.Tensor:
    """A scratch buffer of rmge_workspace_size bytes (torch allocations are 256-byte aligned)."""
    nb = workspace_size(n, nrhs, kind, prec)
    if nb == 0:
        raise ValueError("invalid workspace request")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def empty_multiplier(kind, n, prec, device="cuda") -> torch.Tensor:
    kind, prec = _kind(kind), _prec(prec)
    if kind == GAUSSIAN:
        return torch.empty(n, n, dtype=factor_dtype(prec), device=device)
    return torch.empty((6 if kind >= 4 else 3) * n, dtype=torch.float64, device=device)


def make_multiplier(kind, n, seed, subsequence=1, prec="f64", G=None) -> torch.Tensor:
    L = _cuda_lib()
    if G is None:
        G = empty_multiplier(kind, n, prec)
    if G.numel() * G.element_size() < multiplier_bytes(kind, n, prec):
        raise ValueError("G too small")
    _check("rmge_make_multiplier", L.rmge_make_multiplier(_kind(kind), int(n), int(seed), int(subsequence),
                                                          _prec(prec), _p(G), _stream()))
    return G


def apply_multiplier(kind, A, G, prec="f64", M=None, ws=None) -> torch.Tensor:
    L = _cuda_lib()
    _need(A, torch.float64, "A")
    n = A.shape[0]
    if M is None:
        M = torch.empty(n, n, dtype=factor_dtype(prec), device=A.device)
    _need(M, factor_dtype(prec), "M")
    if ws is None:
        ws = workspace(n, 1, kind, prec)
    _check("rmge_apply_multiplier", L.rmge_apply_multiplier(_kind(kind), n, _p(A), _ld(A), _p(G), _p(M), _ld(M),
                                                            _prec(prec), _p(ws), ws.numel(), _stream()))
    return M


def factor(M, prec="f64", ws=None):
    """In-place GENP of M; returns (info, growth) device tensors (int32, float64)."""
    L = _cuda_lib()
    _need(M, factor_dtype(prec), "M")
    n = M.shape[0]
    info = torch.empty(1, dtype=torch.int32, device=M.device)
    growth = torch.empty(1, dtype=torch.float64, device=M.device)
    if ws is None:
        ws = workspace(n, 1, GAUSSIAN, prec)
    _check("rmge_factor", L.rmge_factor(n, _p(M), _ld(M), _prec(prec), _p(info), _p(growth), _p(ws), ws.numel(),
                                        _stream()))
    return info, growth


def solve(kind, LU, G, B, prec="f64", X=None, ws=None) -> torch.Tensor:
    L = _cuda_lib()
    _need(B, torch.float64, "B")
    n, k = B.shape
    if X is None:
        X = torch.empty(n, k, dtype=torch.float64, device=B.device)
    _need(X, torch.float64, "X")
    if ws is None:
        ws = workspace(n, k, kind, prec)
    _check("rmge_solve", L.rmge_solve(_kind(kind), n, k, _p(LU), _ld(LU), _p(G), _p(B), _ld(B), _p(X), _ld(X),
                                      _prec(prec), _p(ws), ws.numel(), _stream()))
    return X


def options(growth_tol=0.0, spin_limit=None, gmres_m=None, sync=False, status=None, apply_digits=None,
            factor_digits=None) -> Options:
    """rmge_options with the library's defaults (rmge_options_init) and the given fields replaced; status is
    a device int32 tensor or None."""
    o = Options()
    load_library().rmge_options_init(C.byref(o))
    o.growth_tol = float(growth_tol)
    if spin_limit is not None:
        o.spin_limit = int(spin_limit)
    if gmres_m is not None:
        o.gmres_m = int(gmres_m)
    if apply_digits is not None:
        o.apply_digits = int(apply_digits)
    if factor_digits is not None:
        o.factor_digits = int(factor_digits)
    o.sync = 1 if sync else 0
    o.status = None if status is None else status.data_ptr()
    return o


def _check_ex(fn, code, opts):
    # a synchronising call returns its numerical outcome, which is not an error of the call
    if opts is not None and opts.sync and code in OUTCOMES:
        return code
    _check(fn, code)
    return code


def workspace_size_ex(n, nrhs, kind, prec, opts) -> int:
    return int(load_library().rmge_workspace_size_ex(int(n), int(nrhs), _kind(kind), _prec(prec), C.byref(opts)))


def workspace_ex(n, nrhs, kind, prec, opts, device="cuda") -> torch.Tensor:
    nb = workspace_size_ex(n, nrhs, kind, prec, opts)
    if nb == 0:
        raise ValueError("invalid workspace request")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def apply_multiplier_ex(kind, A, G, prec, opts, M=None, ws=None) -> torch.Tensor:
    """rmge_apply_multiplier_ex: M = A G with options (apply_digits for the emulated FP64 product)."""
    L = _cuda_lib()
    _need(A, torch.float64, "A")
    n = A.shape[0]
    if M is None:
        M = torch.empty(n, n, dtype=factor_dtype(prec), device=A.device)
    _need(M, factor_dtype(prec), "M")
    if ws is None:
        ws = workspace_ex(n, 1, kind, prec, opts)
    _check("rmge_apply_multiplier_ex", L.rmge_apply_multiplier_ex(_kind(kind), n, _p(A), _ld(A), _p(G), _p(M), _ld(M),
                                                                  _prec(prec), C.byref(opts), _p(ws), ws.numel(),
                                                                  _stream()))
    return M


def uniform_workspace(count, n, prec, device="cuda") -> torch.Tensor:
    """Scratch for rmge_apply_multiplier_batched / rmge_factor_batched (count systems of order n)."""
    nb = int(load_library().rmge_batched_uniform_workspace_size(int(count), int(n), _prec(prec)))
    if nb == 0:
        raise ValueError("invalid uniform-batch workspace request")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def _need3(t, name):
    if t.device.type != "cuda" or t.dtype != torch.float64 or t.dim() != 3 or t.stride(2) != 1:
        raise ValueError(f"{name} must be a (count, n, n) row-major float64 CUDA tensor")


def apply_multiplier_batched(A, G, prec="f64x", opts=None, M=None, ws=None) -> torch.Tensor:
    """rmge_apply_multiplier_batched: M[i] = A[i] G[i] for (count, n, n) tensors, one launch per kernel."""
    L = _cuda_lib()
    _need3(A, "A")
    _need3(G, "G")
    count, n, _ = A.shape
    if M is None:
        M = torch.empty(count, n, n, dtype=torch.float64, device=A.device)
    _need3(M, "M")
    if ws is None:
        ws = uniform_workspace(count, n, prec)
    o = options() if opts is None else opts
    _check("rmge_apply_multiplier_batched", L.rmge_apply_multiplier_batched(
        count, n, _p(A), A.stride(1), A.stride(0), _p(G), G.stride(0), _p(M), M.stride(1), M.stride(0), _prec(prec),
        C.byref(o), _p(ws), ws.numel(), _stream()))
    return M


def factor_batched(M, prec="f64x", ws=None, opts=None):
    """rmge_factor_batched: in-place GENP of every M[i]; returns (info, growth) device tensors of count entries."""
    L = _cuda_lib()
    _need3(M, "M")
    count, n, _ = M.shape
    info = torch.empty(count, dtype=torch.int32, device=M.device)
    growth = torch.empty(count, dtype=torch.float64, device=M.device)
    if ws is None:
        ws = uniform_workspace(count, n, prec)
    o = options() if opts is None else opts
    _check("rmge_factor_batched", L.rmge_factor_batched(count, n, _p(M), M.stride(1), M.stride(0), _prec(prec),
                                                        _p(info), _p(growth), C.byref(o), _p(ws), ws.numel(),
                                                        _stream()))
    return info, growth


def uniform_solve_workspace(count, n, nrhs, prec, device="cuda") -> torch.Tensor:
    nb = int(load_library().rmge_uniform_solve_workspace_size(int(count), int(n), int(nrhs), _prec(prec)))
    if nb == 0:
        raise ValueError("invalid uniform-batch solve workspace request")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def _b3(t, name):
    if t.device.type != "cuda" or t.dtype != torch.float64 or t.dim() != 3 or t.stride(2) != 1:
        raise ValueError(f"{name} must be a (count, rows, cols) row-major float64 CUDA tensor")
    return t.stride(1), t.stride(0)


def solve_uniform_batched(LU, G, B, prec="f64x", X=None, ws=None) -> torch.Tensor:
    """rmge_solve_uniform_batched: X[i] = G[i] U_i^{-1} L_i^{-1} B[i] for (count, n, .) tensors."""
    L = _cuda_lib()
    count, n, k = B.shape
    if X is None:
        X = torch.empty(count, n, k, dtype=torch.float64, device=B.device)
    (ldlu, slu), (_, sg), (ldb, sb), (ldx, sx) = _b3(LU, "LU"), _b3(G, "G"), _b3(B, "B"), _b3(X, "X")
    if ws is None:
        ws = uniform_solve_workspace(count, n, k, prec)
    _check("rmge_solve_uniform_batched", L.rmge_solve_uniform_batched(
        count, n, k, _p(LU), ldlu, slu, _p(G), sg, _p(B), ldb, sb, _p(X), ldx, sx, _prec(prec), _p(ws), ws.numel(),
        _stream()))
    return X


def refine_uniform_batched(A, LU, G, B, X, prec="f64x", max_iters=10, be_tol=1e-13, ws=None):
    """rmge_refine_uniform_batched: in-place refinement of every X[i]; returns (berr (count, max_iters + 1),
    iters (count,))."""
    L = _cuda_lib()
    count, n, k = B.shape
    (lda, sa), (ldlu, slu), (_, sg), (ldb, sb), (ldx, sx) = (_b3(A, "A"), _b3(LU, "LU"), _b3(G, "G"), _b3(B, "B"),
                                                            _b3(X, "X"))
    berr = torch.empty(count, max_iters + 1, dtype=torch.float64, device=B.device)
    iters = torch.empty(count, dtype=torch.int32, device=B.device)
    if ws is None:
        ws = uniform_solve_workspace(count, n, k, prec)
    _check("rmge_refine_uniform_batched", L.rmge_refine_uniform_batched(
        count, n, k, _p(A), lda, sa, _p(LU), ldlu, slu, _p(G), sg, _p(B), ldb, sb, _p(X), ldx, sx, _prec(prec),
        int(max_iters), float(be_tol), _p(berr), _p(iters), _p(ws), ws.numel(), _stream()))
    return berr, iters


def solve_backward_uniform_batched(A, LU, G, X, dX, prec="f64x", want_dA=True, max_iters=0, be_tol=1e-13, ws=None):
    """rmge_solve_backward_uniform_batched: (dB, dA, berr, iters) for every system (dA None without want_dA)."""
    L = _cuda_lib()
    count, n, k = dX.shape
    dB = torch.empty(count, n, k, dtype=torch.float64, device=dX.device)
    dA = torch.empty(count, n, n, dtype=torch.float64, device=dX.device) if want_dA else None
    (lda, sa), (ldlu, slu), (_, sg), (ldx, sx), (lddx, sdx), (lddb, sdb) = (
        _b3(A, "A"), _b3(LU, "LU"), _b3(G, "G"), _b3(X, "X"), _b3(dX, "dX"), _b3(dB, "dB"))
    ldda, sda = _b3(dA, "dA") if dA is not None else (n, n * n)
    berr = torch.empty(count, max_iters + 1, dtype=torch.float64, device=dX.device)
    iters = torch.zeros(count, dtype=torch.int32, device=dX.device)
    if ws is None:
        ws = uniform_solve_workspace(count, n, k, prec)
    _check("rmge_solve_backward_uniform_batched", L.rmge_solve_backward_uniform_batched(
        count, n, k, _p(A), lda, sa, _p(LU), ldlu, slu, _p(G), sg, _p(X), ldx, sx, _p(dX), lddx, sdx, _p(dB), lddb,
        sdb, _p(dA), ldda, sda, _prec(prec), int(max_iters), float(be_tol), _p(berr) if max_iters > 0 else None,
        _p(iters) if max_iters > 0 else None, _p(ws), ws.numel(), _stream()))
    return dB, dA, berr, iters


def factor_ex(M, prec, opts, ws=None):
    """rmge_factor_ex: (info, growth, code); code is the call's return value (its outcome when opts.sync)."""
    L = _cuda_lib()
    _need(M, factor_dtype(prec), "M")
    n = M.shape[0]
    info = torch.empty(1, dtype=torch.int32, device=M.device)
    growth = torch.empty(1, dtype=torch.float64, device=M.device)
    if ws is None:
        ws = workspace_ex(n, 1, GAUSSIAN, prec, opts)
    code = L.rmge_factor_ex(n, _p(M), _ld(M), _prec(prec), _p(info), _p(growth), C.byref(opts), _p(ws), ws.numel(),
                            _stream())
    return info, growth, _check_ex("rmge_factor_ex", code, opts)


def solve_ex(kind, LU, G, B, prec, opts, X=None, ws=None):
    """rmge_solve_ex: (X, code)."""
    L = _cuda_lib()
    _need(B, torch.float64, "B")
    n, k = B.shape
    if X is None:
        X = torch.empty(n, k, dtype=torch.float64, device=B.device)
    _need(X, torch.float64, "X")
    if ws is None:
        ws = workspace_ex(n, k, kind, prec, opts)
    code = L.rmge_solve_ex(_kind(kind), n, k, _p(LU), _ld(LU), _p(G), _p(B), _ld(B), _p(X), _ld(X), _prec(prec),
                           C.byref(opts), _p(ws), ws.numel(), _stream())
    return X, _check_ex("rmge_solve_ex", code, opts)


def refine_ex(kind, A, LU, G, B, X, prec, max_iters, be_tol, opts, ws=None):
    """rmge_refine_ex: (berr, iters, code)."""
    L = _cuda_lib()
    n, k = B.shape
    berr = torch.empty(max_iters + 1, dtype=torch.float64, device=B.device)
    iters = torch.empty(1, dtype=torch.int32, device=B.device)
    if ws is None:
        ws = workspace_ex(n, k, kind, prec, opts)
    code = L.rmge_refine_ex(_kind(kind), n, k, _p(A), _ld(A), _p(LU), _ld(LU), _p(G), _p(B), _ld(B), _p(X), _ld(X),
                            _prec(prec), int(max_iters), float(be_tol), _p(berr), _p(iters), C.byref(opts), _p(ws),
                            ws.numel(), _stream())
    return berr, iters, _check_ex("rmge_refine_ex", code, opts)


def solve_noalloc(kind, LU, G, B, prec="f64", X=None) -> torch.Tensor:
    """rmge_solve with the library's fixed device scratch array instead of a workspace argument."""
    L = _cuda_lib()
    _need(B, torch.float64, "B")
    n, k = B.shape
    if X is None:
        X = torch.empty(n, k, dtype=torch.float64, device=B.device)
    _need(X, torch.float64, "X")
    _check("rmge_solve_noalloc", L.rmge_solve_noalloc(_kind(kind), n, k, _p(LU), _ld(LU), _p(G), _p(B), _ld(B),
                                                      _p(X), _ld(X), _prec(prec), _stream()))
    return X


def refine(kind, A, LU, G, B, X, prec="f64", max_iters=10, be_tol=1e-13, ws=None):
    """In-place refinement of X; returns (berr[max_iters+1], iters) device tensors."""
    L = _cuda_lib()
    n, k = B.shape
    berr = torch.empty(max_iters + 1, dtype=torch.float64, device=B.device)
    iters = torch.empty(1, dtype=torch.int32, device=B.device)
    if ws is None:
        ws = workspace(n, k, kind, prec)
    _check("rmge_refine", L.rmge_refine(_kind(kind), n, k, _p(A), _ld(A), _p(LU), _ld(LU), _p(G), _p(B), _ld(B),
                                        _p(X), _ld(X), _prec(prec), int(max_iters), float(be_tol), _p(berr),
                                        _p(iters), _p(ws), ws.numel(), _stream()))
    return berr, iters


def solve_backward(kind, LU, G, X, dX, prec="f64", want_dA=True, A=None, max_iters=0, be_tol=1e-13, ws=None):
    """(dB, dA, berr, iters) for X = A^{-1} B given dX; dA is None when want_dA is False.  With A and
    max_iters > 0, dB is refined on A^T dB = dX (berr/iters then describe that refinement)."""
    L = _cuda_lib()
    n, k = dX.shape
    dB = torch.empty(n, k, dtype=torch.float64, device=dX.device)
    dA = torch.empty(n, n, dtype=torch.float64, device=dX.device) if want_dA else None
    refine_it = int(max_iters) if A is not None else 0
    berr = torch.empty(refine_it + 1, dtype=torch.float64, device=dX.device)
    iters = torch.zeros(1, dtype=torch.int32, device=dX.device)
    if ws is None:
        ws = workspace(n, k, kind, prec)
    _check("rmge_solve_backward", L.rmge_solve_backward(
        _kind(kind), n, k, _p(A), _ld(A) if A is not None else 0, _p(LU), _ld(LU), _p(G), _p(X),
        _ld(X) if X is not None else 0, _p(dX), _ld(dX), _p(dB), _ld(dB), _p(dA), _ld(dA) if dA is not None else 0,
        _prec(prec), refine_it, float(be_tol), _p(berr) if refine_it > 0 else None, _p(iters) if refine_it > 0 else None,
        _p(ws), ws.numel(), _stream()))
    return dB, dA, berr, iters


def _side(kind):
    return GAUSSIAN if kind is None else _kind(kind)


def workspace_two_sided(n, nrhs, kindF, kindH, prec, device="cuda") -> torch.Tensor:
    nb = int(load_library().rmge_workspace_size_two_sided(int(n), int(nrhs), _side(kindF), _side(kindH), _prec(prec)))
    if nb == 0:
        raise ValueError("invalid workspace request")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def apply_two_sided(kindF, F, kindH, H, A, prec="f64", M=None, ws=None, T=None) -> torch.Tensor:
    """M = F A H (F or H None for the identity); T: n x n FP64 scratch for A H when both are given."""
    L = _cuda_lib()
    n = A.shape[0]
    if M is None:
        M = torch.empty(n, n, dtype=torch.float64, device=A.device)
    if F is None or H is None:
        T = None
    elif T is None:
        T = torch.empty(n, n, dtype=torch.float64, device=A.device)
    if ws is None:
        ws = workspace_two_sided(n, 1, kindF, kindH, prec)
    _check("rmge_apply_two_sided", L.rmge_apply_two_sided(
        _side(kindF), _p(F), _side(kindH), _p(H), n, _p(A), _ld(A), _p(M), _ld(M), _p(T), n if T is not None else 0,
        _prec(prec), _p(ws), ws.numel(), _stream()))
    return M


def solve_two_sided(kindF, F, kindH, H, LU, B, prec="f64", X=None, ws=None) -> torch.Tensor:
    L = _cuda_lib()
    n, k = B.shape
    if X is None:
        X = torch.empty(n, k, dtype=torch.float64, device=B.device)
    if ws is None:
        ws = workspace_two_sided(n, k, kindF, kindH, prec)
    _check("rmge_solve_two_sided", L.rmge_solve_two_sided(
        _side(kindF), _p(F), _side(kindH), _p(H), n, k, _p(LU), _ld(LU), _p(B), _ld(B), _p(X), _ld(X), _prec(prec),
        _p(ws), ws.numel(), _stream()))
    return X


def refine_two_sided(kindF, F, kindH, H, A, LU, B, X, prec="f64", max_iters=10, be_tol=1e-13, ws=None):
    L = _cuda_lib()
    n, k = B.shape
    berr = torch.empty(max_iters + 1, dtype=torch.float64, device=B.device)
    iters = torch.zeros(1, dtype=torch.int32, device=B.device)
    if ws is None:
        ws = workspace_two_sided(n, k, kindF, kindH, prec)
    _check("rmge_refine_two_sided", L.rmge_refine_two_sided(
        _side(kindF), _p(F), _side(kindH), _p(H), n, k, _p(A), _ld(A), _p(LU), _ld(LU), _p(B), _ld(B), _p(X), _ld(X),
        _prec(prec), int(max_iters), float(be_tol), _p(berr), _p(iters), _p(ws), ws.numel(), _stream()))
    return berr, iters


def gesv_two_sided(kindF, kindH, A, B, seed, prec="f64", max_iters=10, be_tol=1e-13):
    """F A H y = F b, x = H y (Fact 4.1) with F drawn from subsequence 1 and H from subsequence 2 of the
    seed's stream; kindF / kindH None for the identity.  Returns dict(X, LU, F, H, info, growth, berr, iters)."""
    n, k = B.shape
    ws = workspace_two_sided(n, k, kindF, kindH, prec)
    F = make_multiplier(kindF, n, seed, 1, prec) if kindF is not None else None
    H = make_multiplier(kindH, n, seed, 2, prec) if kindH is not None else None
    M = apply_two_sided(kindF, F, kindH, H, A, prec, ws=ws)
    info, growth = factor(M, prec, ws=ws)
    X = solve_two_sided(kindF, F, kindH, H, M, B, prec, ws=ws)
    berr, iters = refine_two_sided(kindF, F, kindH, H, A, M, B, X, prec, max_iters, be_tol, ws=ws)
    return {"X": X, "LU": M, "F": F, "H": H, "info": info, "growth": growth, "berr": berr, "iters": iters}


def lowrank_multiplier(kind, n, l, seed, subsequence=1) -> torch.Tensor:
    """Algorithm 6.1's multiplier: an n x l Gaussian, or a circulant (3n storage) whose n x l leading block
    is used."""
    L = _cuda_lib()
    k = _kind(kind)
    H = torch.empty((n, l) if k == GAUSSIAN else (3 * n,), dtype=torch.float64, device="cuda")
    _check("rmge_lowrank_multiplier", L.rmge_lowrank_multiplier(k, int(n), int(l), int(seed), int(subsequence),
                                                                _p(H), _stream()))
    return H


def lowrank(kind, A, H, l, Q=None, Z=None, ws=None):
    """Algorithm 6.1 on a device matrix A (m x n): (Q, Z, info) with Q = Q(A H) (m x l) and Z = Q^T A."""
    L = _cuda_lib()
    m, n = A.shape
    k = _kind(kind)
    if Q is None:
        Q = torch.empty(m, l, dtype=torch.float64, device=A.device)
    if Z is None:
        Z = torch.empty(l, n, dtype=torch.float64, device=A.device)
    if ws is None:
        nb = int(L.rmge_lowrank_workspace_size(k, int(m), int(n), int(l)))
        if nb == 0:
            raise ValueError("invalid low-rank request")
        ws = torch.empty(nb, dtype=torch.uint8, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check("rmge_lowrank_basis", L.rmge_lowrank_basis(k, int(m), int(n), int(l), _p(A), _ld(A), _p(H), _p(Q), _ld(Q),
                                                      _p(info), _p(ws), ws.numel(), _stream()))
    _check("rmge_lowrank_project", L.rmge_lowrank_project(int(m), int(n), int(l), _p(Q), _ld(Q), _p(A), _ld(A), _p(Z),
                                                          _ld(Z), _stream()))
    return Q, Z, info


def gesv(kind, A, B, seed, prec="f64", max_iters=10, be_tol=1e-13, subsequence=1):
    """The whole method on device tensors: G, M = A G, GENP, X = G Y, refinement.
    Returns dict(X, LU, G, info, growth, berr, iters) (device tensors)."""
    n, k = B.shape
    ws = workspace(n, k, kind, prec)
    G = make_multiplier(kind, n, seed, subsequence, prec)
    M = apply_multiplier(kind, A, G, prec, ws=ws)
    info, growth = factor(M, prec, ws=ws)
    X = solve(kind, M, G, B, prec, ws=ws)
    berr, iters = refine(kind, A, M, G, B, X, prec, max_iters, be_tol, ws=ws)
    return {"X": X, "LU": M, "G": G, "info": info, "growth": growth, "berr": berr, "iters": iters}
