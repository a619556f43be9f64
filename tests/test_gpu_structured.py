"""GPU-vs-oracle parity of the structured multipliers through the C ABI: the random unitary circulant of
Ex. 5.2 and the Toeplitz multipliers (leading n x n blocks of random 2n x 2n circulants, applied by
2n-point FFTs): the draw, A H, the whole solve in FP64 and in the mixed form, and the adjoint."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = 2.0**-53
KIND = {"circulant": 1, "circulant_uniform": 2, "circulant_unitary": 3, "toeplitz": 4, "toeplitz_uniform": 5}


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


def column_and_spectrum(G, N):
    u = G[N:3 * N].reshape(N, 2)
    return G[:N], u[:, 0] + 1j * u[:, 1]


@pytest.mark.parametrize("n", [4, 8, 256, 8192, 16384])
def test_unitary_circulant_matches_oracle(orc, n):
    G = host(rmge.make_multiplier("circulant_unitary", n, seed=31, subsequence=2, prec="f64"))
    assert G.shape == (3 * n,)
    c, u = column_and_spectrum(G, n)
    ref_u = orc.unitary_spectrum(n, 31, 2)
    # the oracle evaluates cos(2 pi phi) from the rounded product 2 pi phi, the kernel sincospi(2 phi)
    assert np.max(np.abs(u - ref_u)) <= 8 * np.pi * U64
    ref_c = orc.unitary_circulant_column(n, 31, 2)[0] if n <= 2048 else np.real(np.fft.fft(ref_u)) / n
    assert np.max(np.abs(c - ref_c)) <= 20 * np.log2(2 * n) * U64
    if n <= 256:  # the GPU's c defines a real orthogonal circulant
        C = orc.circulant_dense(c)
        assert np.max(np.abs(C.T @ C - np.eye(n))) <= 40 * n * U64


@pytest.mark.parametrize("kind", ["toeplitz", "toeplitz_uniform"])
@pytest.mark.parametrize("n", [2, 64, 4096, 8192])
def test_toeplitz_multiplier_matches_oracle(orc, kind, n):
    G = host(rmge.make_multiplier(kind, n, seed=8, subsequence=3, prec="f64"))
    assert G.shape == (6 * n,)
    c2, u2 = column_and_spectrum(G, 2 * n)
    ref = orc.make_multiplier(KIND[kind], n, 8, 3)
    if kind == "toeplitz_uniform":
        assert np.array_equal(c2, ref)
    else:
        assert np.max(np.abs(c2 - ref)) <= 8 * U64 * np.max(np.abs(ref))
    spec = orc.dft(ref, +1) if n <= 256 else np.fft.ifft(ref) * (2 * n)
    assert np.max(np.abs(u2 - spec)) <= 1e-12 * np.sqrt(2 * n) * np.max(np.abs(spec))


@pytest.mark.parametrize("kind", ["circulant_unitary", "toeplitz", "toeplitz_uniform"])
@pytest.mark.parametrize("n", [4, 64, 512, 4096])
def test_structured_apply_matches_dense_definition(orc, kind, n):
    A, _ = W.gaussian_system(n, 1, seed=5 * n + KIND[kind])
    Gd = rmge.make_multiplier(kind, n, seed=13, subsequence=1, prec="f64")
    M = host(rmge.apply_multiplier(kind, dev(A), Gd, "f64"))
    G = host(Gd)
    H = G[:n] if kind == "circulant_unitary" else G[:2 * n]
    D = orc.multiplier_dense(KIND[kind], n, H)
    ref = orc.matmul(A, D) if n <= 512 else A @ D
    scale = np.max(np.abs(A)) * np.max(np.sum(np.abs(D), axis=0))
    assert np.max(np.abs(M - ref)) <= 1e-14 * np.log2(4 * n) * np.sqrt(n) * scale


@pytest.mark.parametrize("kind,n", [("circulant", 16384), ("circulant_unitary", 16384), ("circulant_uniform", 8192),
                                    ("toeplitz", 8192)])
def test_structured_apply_at_the_largest_transforms(orc, kind, n):
    """A H by 16384-point real transforms (one per CTA, 192 KB of shared memory), against the oracle's rows of
    A H from the definition H_kj = c[(k - j) mod N]: the first and last rows, and rows in between."""
    A, _ = W.gaussian_system(n, 1, seed=11 * n + KIND.get(kind, 1))
    Gd = rmge.make_multiplier(kind, n, seed=17, subsequence=1, prec="f64")
    M = rmge.apply_multiplier(kind, dev(A), Gd, "f64")
    G = host(Gd)
    N = 2 * n if kind.startswith("toeplitz") else n
    rows = np.array([0, 1, 977, n // 2 + 3, n - 2, n - 1])
    got = host(M[torch.as_tensor(rows, device="cuda")])
    ref = orc.circulant_rows(A[rows], G[:N], N)
    scale = np.max(np.abs(A)) * np.sum(np.abs(G[:N]))
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.log2(4 * N) * np.sqrt(n) * scale
    # the FP32 working matrix of the reduced precisions is the same product rounded once
    M32 = host(rmge.apply_multiplier(kind, dev(A), Gd, "bf16x3")[torch.as_tensor(rows, device="cuda")])
    assert np.max(np.abs(M32 - ref)) <= 2.0**-24 * np.max(np.abs(ref)) + 1e-13 * scale


@pytest.mark.parametrize("kind", ["circulant_unitary", "toeplitz", "toeplitz_uniform"])
@pytest.mark.parametrize("prec", ["f64", "f64x"])
@pytest.mark.parametrize("n,k", [(64, 1), (1000, 3), (2048, 8)])
def test_structured_solve_reaches_fp64_target(orc, kind, prec, n, k):
    """Fact 4.1 with H structured: GENP of A H (A[0,0] = 0, so GENP of A itself breaks down), X = H Y,
    refinement; checked with the oracle's residual and against GEPP.  n = 1000 is not a power of two and
    must be refused."""
    A, B = W.gaussian_system(n, k, seed=W.SEED_BASE + 17 + n, zero_leading_pivot=True)
    if n & (n - 1):
        with pytest.raises((RuntimeError, ValueError)):
            rmge.gesv(kind, dev(A), dev(B), seed=4, prec=prec, max_iters=10, be_tol=1e-13)
        return
    out = rmge.gesv(kind, dev(A), dev(B), seed=4, prec=prec, max_iters=10, be_tol=1e-13)
    assert int(host(out["info"])[0]) == 0
    X = host(out["X"])
    be = orc.backward_error(A, X, B)
    assert be <= 1e-13
    LUp, piv, _ = orc.gepp(A)
    xr = orc.gepp_solve(LUp, piv, B)
    kappa = np.linalg.cond(A, np.inf)
    assert np.max(np.abs(X - xr)) <= 10 * kappa * 1e-13 * np.max(np.abs(xr))


@pytest.mark.parametrize("kind", ["circulant_unitary", "toeplitz"])
@pytest.mark.parametrize("n,k", [(16, 4), (256, 2)])
def test_structured_adjoint_matches_oracle_gradient(orc, kind, n, k):
    """The adjoint with H^T applied by FFT correlation: dB = A^-T W (refined), dA = -dB X^T, against the
    oracle's GEPP gradient."""
    A, B, Wt = W.grad_system(n, k, seed=W.SEED_BASE + 9 + n)
    out = rmge.gesv(kind, dev(A), dev(B), seed=3, prec="f64")
    X = out["X"]
    dB, dA, berr, it = rmge.solve_backward(kind, out["LU"], out["G"], X, dev(Wt), "f64", A=dev(A), max_iters=10,
                                           be_tol=1e-13)
    rdB, rdA, info = orc.solve_adjoint_gepp(A, host(X), Wt)
    assert info == 0
    assert orc.backward_error(A.T.copy(), host(dB), Wt) <= 1e-13
    kappa = np.linalg.cond(A, np.inf)
    assert np.max(np.abs(host(dB) - rdB)) <= 10 * kappa * 1e-13 * np.max(np.abs(rdB))
    assert np.max(np.abs(host(dA) - rdA)) <= 10 * kappa * 1e-13 * np.max(np.abs(rdA))
