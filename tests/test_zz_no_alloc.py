"""rmge_solve_noalloc: the solve for callers that cannot allocate device memory (a latency-bound serving
loop, where cudaMalloc may synchronise the device, or a plugin that only receives its inputs and outputs).
It must give what rmge_solve gives with a caller workspace, call after call, through the C ABI.  This file
is collected last so that a run stopping at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

OK, WORKSPACE = 0, 7


@pytest.fixture(scope="module")
def lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    return rmge.load_library()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _noalloc(lib, prec_code, LU, G, B, X):
    n, k = B.shape
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.rmge_solve_noalloc(0, n, k, _ptr(LU), LU.stride(0), _ptr(G), _ptr(B), B.stride(0), _ptr(X),
                                  X.stride(0), prec_code, stream)


@pytest.mark.parametrize("prec,code,dtype", [("f64", 0, torch.float64), ("f32", 1, torch.float32)])
def test_noalloc_solve_matches_workspace_solve(orc, lib, prec, code, dtype):
    shapes = [(300, 5), (64, 1), (300, 5)]  # a second shape in between: no stale state is reused
    for n, k in shapes:
        A, B = W.gaussian_system(n, k, seed=500 + n + k)
        G = W.gaussian_multiplier(n, 501 + n).astype(np.float32 if dtype == torch.float32 else np.float64)
        LU, info = orc.genp(orc.matmul(A, G.astype(np.float64)))
        assert info == 0
        LUd, Gd, Bd = _dev(LU, dtype), _dev(G, dtype), _dev(B)
        ref = rmge.solve("gaussian", LUd, Gd, Bd, prec)
        torch.cuda.synchronize()
        ref_h = ref.cpu().numpy()
        for _ in range(2):  # two calls in a row reuse the same device array
            X = torch.full((n, k), float("nan"), dtype=torch.float64, device="cuda")
            assert _noalloc(lib, code, LUd, Gd, Bd, X) == OK
            torch.cuda.synchronize()
            Xh = X.cpu().numpy()
            assert np.all(np.isfinite(Xh))
            assert np.max(np.abs(Xh - ref_h)) <= 1e-9 * np.max(np.abs(ref_h))


@pytest.mark.parametrize("kind,prec", [("circulant", "f64"), ("circulant_unitary", "f64"), ("gaussian", "bf16")])
def test_noalloc_binding_matches_workspace_solve(orc, lib, kind, prec):
    """The Python binding of the entry point, with the multipliers whose FFT twiddle table sits in the shared
    array, and with a tensor-core precision (FP32 factors)."""
    n, k = 256, 3
    A, B = W.gaussian_system(n, k, seed=700 + len(kind))
    f32 = rmge.factor_dtype(prec) == torch.float32
    G = rmge.make_multiplier(kind, n, seed=701, subsequence=1, prec=prec)
    torch.cuda.synchronize()
    Gh = G.cpu().numpy().astype(np.float64)
    H = Gh.reshape(n, n) if kind == "gaussian" else orc.circulant_dense(Gh[:n])
    LU, info = orc.genp(orc.matmul(A, H))
    assert info == 0
    LUd, Bd = _dev(LU, torch.float32 if f32 else torch.float64), _dev(B)
    ref = rmge.solve(kind, LUd, G, Bd, prec)
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    for _ in range(2):
        X = rmge.solve_noalloc(kind, LUd, G, Bd, prec)
        torch.cuda.synchronize()
        Xh = X.cpu().numpy()
        assert np.all(np.isfinite(Xh))
        assert np.max(np.abs(Xh - ref_h)) <= 1e-9 * np.max(np.abs(ref_h))


def test_noalloc_rejects_requests_beyond_its_array(lib):
    n, k = 60000, 16
    assert lib.rmge_solve_workspace_size(n, k, 0, 0) > lib.rmge_noalloc_capacity()
    X = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # nothing is read or enqueued: the size check comes first
    assert lib.rmge_solve_noalloc(0, n, k, _ptr(X), n, _ptr(X), _ptr(X), k, _ptr(X), k, 0, stream) == WORKSPACE
