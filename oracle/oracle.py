"""numpy front end of the plain-C FP64 oracle (``oracle/rmge_oracle.c``).

Test infrastructure only: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``; never by the product package.  Every
function here is argument marshalling around the C routine it names; the
arithmetic and its citations live in the C source.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i64 = C.c_int64
_u64 = C.c_uint64

# multiplier kinds (same meaning as the library's, defined independently here)
GAUSSIAN = 0
CIRCULANT_GAUSSIAN = 1
CIRCULANT_UNIFORM = 2
CIRCULANT_UNITARY = 3
TOEPLITZ_GAUSSIAN = 4
TOEPLITZ_UNIFORM = 5


def lib():
    global _lib
    if _lib is None:
        # RMGE_ORACLE_LIB names another build of the same source: the planted-mistake tests load a copy
        # with one deliberate error there, to show that the pins catch it
        path = os.environ.get("RMGE_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        sig = {
            "orc_set_threads": (None, [C.c_int]),
            "orc_get_threads": (C.c_int, []),
            "orc_philox4x32_10": (None, [_up, _up, _up]),
            "orc_gaussian": (None, [_i64, _u64, _u64, _dp]),
            "orc_uniform_pm1": (None, [_i64, _u64, _u64, _dp]),
            "orc_uniform01": (None, [_i64, _u64, _u64, _dp]),
            "orc_unitary_spectrum": (None, [_i64, _u64, _u64, _dp, _dp]),
            "orc_toeplitz_dense": (None, [_i64, _dp, _dp]),
            "orc_unitary_circulant_column": (None, [_i64, _u64, _u64, _dp, _dp]),
            "orc_multiplier_dense": (None, [C.c_int, _i64, _dp, _dp]),
            "orc_gaussian_f32": (None, [_i64, _u64, _u64, np.ctypeslib.ndpointer(dtype=np.float32,
                                                                               flags="C_CONTIGUOUS")]),
            "orc_matmul": (None, [_i64, _i64, _i64, _dp, _dp, _dp]),
            "orc_circulant_dense": (None, [_i64, _dp, _dp]),
            "orc_circulant_rows": (None, [_i64, _i64, _i64, _dp, _dp, _dp]),
            "orc_dft": (None, [_i64, _dp, _dp, _dp, _dp, C.c_int]),
            "orc_genp": (C.c_int, [_i64, _dp]),
            "orc_genp_blocked": (C.c_int, [_i64, _i64, _dp]),
            "orc_gepp": (C.c_int, [_i64, _dp, _ip]),
            "orc_lu_solve": (None, [_i64, _i64, _dp, _dp]),
            "orc_lu_solve_transposed": (None, [_i64, _i64, _dp, _dp]),
            "orc_gepp_solve": (None, [_i64, _i64, _dp, _ip, _dp]),
            "orc_residual": (None, [_i64, _i64, _dp, _dp, _dp, _dp]),
            "orc_norm_inf": (C.c_double, [_i64, _i64, _dp]),
            "orc_backward_error": (C.c_double, [_i64, _i64, _dp, _dp, _dp]),
            "orc_relative_residual": (C.c_double, [_i64, _i64, _dp, _dp, _dp]),
            "orc_growth": (C.c_double, [_i64, _dp, _dp]),
            "orc_apply_multiplier": (None, [C.c_int, _i64, _dp, _dp, _dp]),
            "orc_refine_step": (None, [C.c_int, _i64, _i64, _dp, _dp, _dp, _dp, _dp]),
            "orc_rmge_solve": (C.c_int, [C.c_int, _i64, _i64, _dp, _dp, _dp, _dp, _dp, C.c_int,
                                         C.c_double, _dp, C.POINTER(C.c_int)]),
            "orc_solve_adjoint_gepp": (C.c_int, [_i64, _i64, _dp, _dp, _dp, _dp, _dp]),
            "orc_rmge_solve_two_sided": (C.c_int, [C.c_int, _dp, C.c_int, _dp, _i64, _i64, _dp, _dp, _dp, _dp,
                                                   C.c_int, C.c_double, _dp, C.POINTER(C.c_int)]),
            "orc_qr": (None, [_i64, _i64, _dp, _dp, _dp]),
            "orc_lowrank_multiplier_dense": (None, [C.c_int, _i64, _i64, _dp, _dp]),
            "orc_lowrank": (None, [C.c_int, _i64, _i64, _i64, _dp, _dp, _dp, _dp]),
            "orc_genp_complex": (C.c_int, [_i64, _dp, _dp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        set_threads(int(os.environ.get("RMGE_ORACLE_THREADS", "1")))
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cols(b):
    b = _f64(b)
    return b.reshape(b.shape[0], -1)


def set_threads(t):
    lib().orc_set_threads(int(t))


def get_threads():
    return lib().orc_get_threads()


def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def gaussian(count, seed, subseq=0):
    out = np.empty(int(count), np.float64)
    lib().orc_gaussian(int(count), int(seed), int(subseq), out)
    return out


def gaussian_f32(count, seed, subseq=0):
    out = np.empty(int(count), np.float32)
    lib().orc_gaussian_f32(int(count), int(seed), int(subseq), out)
    return out


def uniform_pm1(count, seed, subseq=0):
    out = np.empty(int(count), np.float64)
    lib().orc_uniform_pm1(int(count), int(seed), int(subseq), out)
    return out


def uniform01(count, seed, subseq=0):
    out = np.empty(int(count), np.float64)
    lib().orc_uniform01(int(count), int(seed), int(subseq), out)
    return out


def unitary_spectrum(n, seed, subseq=1):
    """Hermitian-symmetric unit-modulus spectrum u (complex, length n) of a random unitary circulant."""
    ur = np.empty(int(n), np.float64)
    ui = np.empty(int(n), np.float64)
    lib().orc_unitary_spectrum(int(n), int(seed), int(subseq), ur, ui)
    return ur + 1j * ui


def unitary_circulant_column(n, seed, subseq=1):
    """First column c = Omega^{-1} u of the random unitary circulant (Ex. 5.2), by the naive inverse
    DFT (sign -1, divided by n); returns (c real part, imaginary part left by rounding)."""
    c = np.empty(int(n), np.float64)
    cim = np.empty(int(n), np.float64)
    lib().orc_unitary_circulant_column(int(n), int(seed), int(subseq), c, cim)
    return c, cim


def make_multiplier(kind, n, seed, subseq=1):
    """Dense Gaussian G (n x n) for GAUSSIAN; the first column c (n,) of the circulant kinds; the first
    column c2 (2n,) of the 2n x 2n circulant whose leading n x n block is the Toeplitz multiplier."""
    if kind == GAUSSIAN:
        return gaussian(n * n, seed, subseq).reshape(n, n)
    if kind in (CIRCULANT_GAUSSIAN, CIRCULANT_UNIFORM, CIRCULANT_UNITARY):
        base, m = kind, n
    elif kind in (TOEPLITZ_GAUSSIAN, TOEPLITZ_UNIFORM):
        base, m = kind - 3, 2 * n
    else:
        raise ValueError(kind)
    if base == CIRCULANT_GAUSSIAN:
        return gaussian(m, seed, subseq)
    if base == CIRCULANT_UNIFORM:
        return uniform_pm1(m, seed, subseq)
    return unitary_circulant_column(m, seed, subseq)[0]


def toeplitz_dense(n, c2):
    out = np.empty((int(n), int(n)), np.float64)
    lib().orc_toeplitz_dense(int(n), _f64(c2), out)
    return out


def multiplier_dense(kind, n, H):
    out = np.empty((int(n), int(n)), np.float64)
    lib().orc_multiplier_dense(int(kind), int(n), _f64(H), out)
    return out


def matmul(A, B):
    A, B = _f64(A), _f64(B)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    Cm = np.empty((m, n), np.float64)
    lib().orc_matmul(m, k, n, A, B, Cm)
    return Cm


def circulant_dense(c):
    c = _f64(c)
    n = c.shape[0]
    out = np.empty((n, n), np.float64)
    lib().orc_circulant_dense(n, c, out)
    return out


def circulant_rows(A_rows, c, N=None):
    """Rows of A H, H the leading n x n block of the N x N circulant with first column c (N = n by
    default), from the definition; A_rows is r x n."""
    A_rows, c = _f64(np.atleast_2d(A_rows)), _f64(c)
    r, n = A_rows.shape
    N = n if N is None else int(N)
    assert c.shape[0] >= N
    out = np.empty((r, n), np.float64)
    lib().orc_circulant_rows(n, N, r, A_rows, c, out)
    return out


def dft(x, sign=+1):
    x = np.asarray(x, np.complex128)
    n = x.shape[0]
    yr, yi = np.empty(n), np.empty(n)
    lib().orc_dft(n, _f64(x.real), _f64(x.imag), yr, yi, int(sign))
    return yr + 1j * yi


def genp(M):
    """Unblocked GENP; returns (packed L\\U, info)."""
    LU = _f64(M).copy()
    info = lib().orc_genp(LU.shape[0], LU)
    return LU, info


def genp_blocked(M, nb):
    LU = _f64(M).copy()
    info = lib().orc_genp_blocked(LU.shape[0], int(nb), LU)
    return LU, info


def gepp(M):
    LU = _f64(M).copy()
    piv = np.zeros(LU.shape[0], np.int64)
    info = lib().orc_gepp(LU.shape[0], LU, piv)
    return LU, piv, info


def lu_solve(LU, B):
    LU = _f64(LU)
    X = _cols(B).copy()
    lib().orc_lu_solve(LU.shape[0], X.shape[1], LU, X)
    return X


def lu_solve_transposed(LU, B):
    LU = _f64(LU)
    X = _cols(B).copy()
    lib().orc_lu_solve_transposed(LU.shape[0], X.shape[1], LU, X)
    return X


def gepp_solve(LU, piv, B):
    X = _cols(B).copy()
    lib().orc_gepp_solve(LU.shape[0], X.shape[1], _f64(LU), np.ascontiguousarray(piv, np.int64), X)
    return X


def residual(A, X, B):
    A, X, B = _f64(A), _cols(X), _cols(B)
    R = np.empty_like(B)
    lib().orc_residual(A.shape[0], B.shape[1], A, X, B, R)
    return R


def norm_inf(A):
    A = _f64(A)
    A2 = A.reshape(A.shape[0], -1)
    return lib().orc_norm_inf(A2.shape[0], A2.shape[1], A2)


def backward_error(A, X, B):
    A, X, B = _f64(A), _cols(X), _cols(B)
    return lib().orc_backward_error(A.shape[0], B.shape[1], A, X, B)


def relative_residual(A, X, B):
    A, X, B = _f64(A), _cols(X), _cols(B)
    return lib().orc_relative_residual(A.shape[0], B.shape[1], A, X, B)


def growth(M, LU):
    return lib().orc_growth(M.shape[0], _f64(M), _f64(LU))


def apply_multiplier(kind, A, H):
    A = _f64(A)
    out = np.empty_like(A)
    lib().orc_apply_multiplier(int(kind), A.shape[0], A, _f64(H), out)
    return out


def refine_step(kind, A, LU, H, B, X):
    X = _cols(X).copy()
    B = _cols(B)
    lib().orc_refine_step(int(kind), A.shape[0], B.shape[1], _f64(A), _f64(LU), _f64(H), B, X)
    return X


def rmge_solve(kind, A, H, B, max_iters=10, be_tol=1e-13):
    """Randomized GENP solve; returns dict(X, LU, info, iters, berr[list])."""
    A, B = _f64(A), _cols(B)
    n, k = B.shape
    X = np.zeros((n, k), np.float64)
    LU = np.empty((n, n), np.float64)
    berr = np.full(max_iters + 1, np.nan)
    iters = C.c_int(0)
    info = lib().orc_rmge_solve(int(kind), n, k, A, _f64(H), B, X, LU, int(max_iters), float(be_tol),
                                berr, C.byref(iters))
    return {"X": X, "LU": LU, "info": info, "iters": iters.value,
            "berr": [float(v) for v in berr[: iters.value + 1]] if info == 0 else []}


def rmge_solve_two_sided(kindF, F, kindH, H, A, B, max_iters=10, be_tol=1e-13):
    """Two-sided randomized GENP solve (F A H y = F b, x = H y); kind None (or < 0) for the identity.
    Returns dict(X, LU, info, iters, berr[list])."""
    A, B = _f64(A), _cols(B)
    n, k = B.shape
    kF = -1 if kindF is None else int(kindF)
    kH = -1 if kindH is None else int(kindH)
    dummy = np.zeros(1, np.float64)
    X = np.zeros((n, k), np.float64)
    LU = np.empty((n, n), np.float64)
    berr = np.full(max_iters + 1, np.nan)
    iters = C.c_int(0)
    info = lib().orc_rmge_solve_two_sided(kF, _f64(F) if kF >= 0 else dummy, kH, _f64(H) if kH >= 0 else dummy,
                                          n, k, A, B, X, LU, int(max_iters), float(be_tol), berr, C.byref(iters))
    return {"X": X, "LU": LU, "info": info, "iters": iters.value,
            "berr": [float(v) for v in berr[: iters.value + 1]] if info == 0 else []}


def qr(B):
    """Thin Householder QR with diag(R) >= 0: (Q, R)."""
    B = _f64(B)
    m, l = B.shape
    Q = np.empty((m, l), np.float64)
    R = np.empty((l, l), np.float64)
    lib().orc_qr(m, l, B, Q, R)
    return Q, R


def lowrank_multiplier(kind, n, l, seed, subseq=1):
    """Algorithm 6.1's multiplier: a dense n x l Gaussian for kind 0 (the first n*l entries of the Gaussian
    stream), else the first column c (n,) of the circulant whose n x l leading block is used."""
    if kind == GAUSSIAN:
        return gaussian(n * l, seed, subseq).reshape(n, l)
    return make_multiplier(kind, n, seed, subseq)


def lowrank_multiplier_dense(kind, n, l, H):
    out = np.empty((int(n), int(l)), np.float64)
    lib().orc_lowrank_multiplier_dense(int(kind), int(n), int(l), _f64(H), out)
    return out


def lowrank(kind, A, H, l):
    """Algorithm 6.1: (Q, Z) with Q = Q(A H) and Z = Q^T A."""
    A = _f64(A)
    m, n = A.shape
    Q = np.empty((m, int(l)), np.float64)
    Z = np.empty((int(l), n), np.float64)
    lib().orc_lowrank(int(kind), m, n, int(l), A, _f64(H), Q, Z)
    return Q, Z


def solve_adjoint_gepp(A, X, Wbar):
    A, X, Wbar = _f64(A), _cols(X), _cols(Wbar)
    n, k = X.shape
    dB = np.empty((n, k))
    dA = np.empty((n, n))
    info = lib().orc_solve_adjoint_gepp(n, k, A, X, Wbar, dB, dA)
    return dB, dA, info


def genp_complex(M):
    M = np.asarray(M, np.complex128)
    n = M.shape[0]
    re, im = _f64(M.real).copy(), _f64(M.imag).copy()
    pr, pi = np.zeros(n), np.zeros(n)
    info = lib().orc_genp_complex(n, re, im, pr, pi)
    return re + 1j * im, pr + 1j * pi, info
