"""GPU-vs-oracle parity of the FP64 path through the C ABI (multiplier draw, A G, blocked GENP, solve,
refinement, adjoint), at sizes that span several tiles with ragged tails, plus edge cases."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = 2.0**-53


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


# ----------------------------------------------------------------------------- multiplier draws

@pytest.mark.parametrize("n", [1, 3, 64, 257, 2048])
def test_gaussian_multiplier_matches_oracle(orc, n):
    """Philox + Box-Muller entries within a few ulps of the oracle's (libm log, cos, sin); n = 2048 draws
    4.2 million entries, among them uniforms within 1e-6 of 1, where ln u1 needs its full relative
    accuracy."""
    G = host(rmge.make_multiplier("gaussian", n, seed=W.SEED_BASE + 1, subsequence=1, prec="f64"))
    ref = orc.make_multiplier(orc.GAUSSIAN, n, seed=W.SEED_BASE + 1, subseq=1)
    assert np.max(np.abs(G - ref)) <= 8 * U64 * max(1.0, np.max(np.abs(ref)))


def test_uniform_circulant_column_is_bit_exact(orc):
    n = 1024
    G = host(rmge.make_multiplier("circulant_uniform", n, seed=99, subsequence=5, prec="f64"))
    assert np.array_equal(G[:n], orc.uniform_pm1(n, 99, 5))


@pytest.mark.parametrize("n", [4, 8, 512, 8192, 16384])
def test_circulant_spectrum_matches_dft(orc, n):
    G = host(rmge.make_multiplier("circulant", n, seed=7, subsequence=1, prec="f64"))
    c = orc.gaussian(n, 7, 1)
    assert np.max(np.abs(G[:n] - c)) <= 8 * U64 * np.max(np.abs(c))
    u = G[n:].reshape(n, 2)
    u = u[:, 0] + 1j * u[:, 1]
    ref = orc.dft(c, +1) if n <= 512 else np.fft.ifft(c) * n  # Omega c, w = exp(+2 pi i / n)
    assert np.max(np.abs(u - ref)) <= 1e-12 * np.sqrt(n) * np.max(np.abs(ref))


def test_f32_multiplier_matches_oracle(orc):
    n = 96
    G = host(rmge.make_multiplier("gaussian", n, seed=5, subsequence=2, prec="f32"))
    ref = orc.gaussian_f32(n * n, 5, 2).reshape(n, n)
    assert np.max(np.abs(G - ref)) <= 1e-5


# ----------------------------------------------------------------------------- A G

@pytest.mark.parametrize("n", [1, 7, 64, 65, 200, 600])
def test_dense_apply_matches_oracle(orc, n):
    A, _ = W.gaussian_system(n, 1, seed=n)
    G = W.gaussian_multiplier(n, n + 1)
    M = host(rmge.apply_multiplier("gaussian", dev(A), dev(G), "f64"))
    ref = orc.matmul(A, G)
    scale = np.abs(A) @ np.abs(G)
    assert np.all(np.abs(M - ref) <= 2 * n * U64 * scale + 1e-300)


@pytest.mark.parametrize("kind", ["circulant", "circulant_uniform"])
@pytest.mark.parametrize("n", [4, 16, 256, 2048])
def test_circulant_apply_matches_dense_definition(orc, kind, n):
    A, _ = W.gaussian_system(n, 1, seed=3 * n)
    Gd = rmge.make_multiplier(kind, n, seed=11, subsequence=1, prec="f64")
    M = host(rmge.apply_multiplier(kind, dev(A), Gd, "f64"))
    c = host(Gd)[:n]
    ref = orc.matmul(A, orc.circulant_dense(c)) if n <= 256 else A @ orc.circulant_dense(c)
    assert np.max(np.abs(M - ref)) <= 1e-13 * np.log2(n + 1) * np.sqrt(n) * np.max(np.abs(ref))


# ----------------------------------------------------------------------------- GENP

@pytest.mark.parametrize("n", [1, 5, 63, 64])
def test_factor_exact_on_exact_input(orc, n):
    """A single pivot block is plain GENP: on M = L0 U0 with exact arithmetic the factors come back bitwise."""
    r = W.rng(n)
    L0 = np.tril(r.integers(-3, 4, (n, n)), -1).astype(np.float64) + np.eye(n)
    U0 = np.triu(r.integers(-3, 4, (n, n)), 1).astype(np.float64) + np.diag(r.choice([-4.0, -2.0, -1.0, 1.0, 2.0, 4.0], n))
    M = dev(L0 @ U0)
    info, growth = rmge.factor(M, "f64")
    LU = host(M)
    assert int(host(info)[0]) == 0
    assert np.array_equal(np.tril(LU, -1) + np.eye(n), L0) and np.array_equal(np.triu(LU), U0)


@pytest.mark.parametrize("n", [65, 130, 257, 700])
def test_blocked_factor_matches_oracle(orc, n):
    A, _ = W.gaussian_system(n, 1, seed=17 + n)
    G = W.gaussian_multiplier(n, 18 + n)
    M = orc.matmul(A, G)
    Md = dev(M)
    info, growth = rmge.factor(Md, "f64")
    LU = host(Md)
    ref, rinfo = orc.genp(M)
    assert int(host(info)[0]) == rinfo == 0
    g = orc.growth(M, ref)
    assert abs(float(host(growth)[0]) - g) <= 1e-8 * g
    # same L and U to rounding x growth (Sec. 3: blockings share Schur complements)
    err = np.max(np.abs(LU - ref)) / np.max(np.abs(ref))
    assert err <= 1e3 * n * U64 * g, err


def test_breakdown_steps(orc):
    """Cor. 3.1: info = first step with a zero (or non-finite) pivot; later steps are skipped."""
    A, _ = W.gaussian_system(256, 1, seed=W.SEED_BASE + 1, zero_leading_pivot=True)
    info, growth = rmge.factor(dev(A), "f64")
    assert int(host(info)[0]) == 1 == orc.genp(A)[1]
    assert np.isnan(host(growth)[0])
    for n, step in [(200, 70), (130, 64), (130, 65), (300, 300)]:
        M = np.eye(n)
        M[step - 1, step - 1] = 0.0
        info, _ = rmge.factor(dev(M), "f64")
        assert int(host(info)[0]) == step == orc.genp(M)[1]
    M = np.eye(150)
    M[100, 100] = np.nan
    info, _ = rmge.factor(dev(M), "f64")
    assert int(host(info)[0]) == 101


# ----------------------------------------------------------------------------- solve / refine / end to end

@pytest.mark.parametrize("n,k", [(1, 1), (97, 2), (33, 3), (1000, 4), (100, 16), (256, 1), (300, 17)])
def test_solve_matches_oracle(orc, n, k):
    A, B = W.gaussian_system(n, k, seed=40 + n)
    G = W.gaussian_multiplier(n, 41 + n)
    LU, _ = orc.genp(orc.matmul(A, G))
    X = host(rmge.solve("gaussian", dev(LU), dev(G), dev(B), "f64"))
    ref = orc.matmul(G, orc.lu_solve(LU, B))
    # Two solves with the same factors that round in a different order differ by about kappa(A G) u
    # (the forward-error bound of a backward-stable solve); at n = 1000, kappa(A G) = 1.7e6 and the
    # oracle's own forward error is 2.4e-8.
    tol = max(1e-9, 64 * np.finfo(np.float64).eps * np.linalg.cond(orc.matmul(A, G)))
    assert np.max(np.abs(X - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("kind", ["gaussian", "circulant", "circulant_uniform"])
@pytest.mark.parametrize("n,k", [(64, 1), (256, 1), (512, 16)])
def test_end_to_end_backward_error(orc, kind, n, k):
    """The whole method on the GPU reaches the FP64 target, checked with the oracle's own residual."""
    A, B = W.gaussian_system(n, k, seed=W.SEED_BASE + n, zero_leading_pivot=True)
    out = rmge.gesv(kind, dev(A), dev(B), seed=W.SEED_BASE + 1, prec="f64", max_iters=10, be_tol=1e-13)
    assert int(host(out["info"])[0]) == 0
    X = host(out["X"])
    it = int(host(out["iters"])[0])
    berr = host(out["berr"])
    be = orc.backward_error(A, X, B)
    assert be <= 1e-13
    assert berr[it] <= 1e-13 and abs(berr[it] - be) <= 0.5 * be + 1e-16
    assert np.all(berr[it + 1:] == -1.0)
    # forward agreement with the oracle's GEPP solution, to kappa x backward error
    LUp, piv, _ = orc.gepp(A)
    xr = orc.gepp_solve(LUp, piv, B)
    kappa = np.linalg.cond(A, np.inf)
    assert np.max(np.abs(X - xr)) <= 10 * kappa * 1e-13 * np.max(np.abs(xr))


def test_refinement_sweep_matches_oracle(orc):
    """One sweep with the same factors from the same start: X1 = X0 + G U^-1 L^-1 (B - A X0)."""
    n, k = 192, 2
    A, B = W.orthogonal_factor_system(n, k, 1e-6, seed=12)
    G = W.gaussian_multiplier(n, 13)
    LU, _ = orc.genp(orc.matmul(A, G))
    X0 = orc.matmul(G, orc.lu_solve(LU, B))
    Xd = dev(X0)
    berr, iters = rmge.refine("gaussian", dev(A), dev(LU), dev(G), dev(B), Xd, "f64", max_iters=1, be_tol=0.0)
    X1 = host(Xd)
    ref = orc.refine_step(0, A, LU, G, B, X0)
    # the GPU residual is plain FP64, the oracle's compensated: they differ by ~n u ||A|| ||X||, which the
    # correction amplifies by up to kappa(A) = 1e6
    kappa = np.linalg.cond(A, np.inf)
    assert np.max(np.abs(X1 - ref)) <= kappa * n * U64 * np.max(np.abs(ref))
    e = host(berr)
    assert e[0] == pytest.approx(orc.backward_error(A, X0, B), rel=1e-3)
    assert e[1] == pytest.approx(orc.backward_error(A, X1, B), rel=0.5)


def test_dft_like_input_fails_without_gaussian_multiplier(orc):
    """Thm 5.2 (real analogue): the real Fourier matrix breaks GENP and circulant-GENP, not Gaussian-GENP."""
    n = 256
    F = W.real_fourier_matrix(n)
    b = W.rng(3).standard_normal((n, 1))
    out = rmge.gesv("gaussian", dev(F), dev(b), seed=5, prec="f64", max_iters=2, be_tol=0.0)
    assert orc.relative_residual(F, host(out["X"]), b) <= 1e-12
    out_c = rmge.gesv("circulant", dev(F), dev(b), seed=5, prec="f64", max_iters=0, be_tol=0.0)
    Xc = host(out_c["X"])
    assert not (orc.relative_residual(F, Xc, b) <= 1e-6)
    info, growth = rmge.factor(dev(F), "f64")
    assert int(host(info)[0]) != 0 or host(growth)[0] > 1e6


# ----------------------------------------------------------------------------- adjoint

@pytest.mark.parametrize("kind", ["gaussian", "circulant"])
@pytest.mark.parametrize("n,k", [(16, 4), (64, 1), (256, 9), (300, 2), (129, 3)])
def test_adjoint_matches_oracle_gradient(orc, kind, n, k):
    if kind == "circulant" and n & (n - 1):
        pytest.skip("the FFT multipliers take power-of-two orders")
    A, B, Wt = W.grad_system(n, k, seed=W.SEED_BASE + 5 + n)
    out = rmge.gesv(kind, dev(A), dev(B), seed=3, prec="f64")
    X = out["X"]
    dB, dA, _, _ = rmge.solve_backward(kind, out["LU"], out["G"], X, dev(Wt), "f64")
    rdB, rdA, info = orc.solve_adjoint_gepp(A, host(X), Wt)
    assert info == 0
    # the adjoint solve is unrefined: its error scales with kappa(A G) u (growth aside); the target for
    # gradients is 1e-6 relative
    tol = min(1e-6, max(1e-12, 100 * n * np.linalg.cond(orc.apply_multiplier(0 if kind == "gaussian" else 1, A,
                                                                            host(out["G"]) if kind == "gaussian"
                                                                            else host(out["G"])[:n])) * U64))
    assert np.max(np.abs(host(dB) - rdB)) <= tol * np.max(np.abs(rdB))
    assert np.max(np.abs(host(dA) - rdA)) <= tol * np.max(np.abs(rdA))
