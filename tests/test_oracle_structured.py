"""Pins of the oracle's structured multipliers: the random unitary circulant of Ex. 5.2 (drawn with
Hermitian-symmetric phases, so that it is real) and the Toeplitz multipliers, the leading n x n blocks
of random 2n x 2n circulants (Sec. 7.2)."""
import numpy as np
import pytest
from scipy import stats

U = np.finfo(np.float64).eps / 2


def test_uniform01_is_the_uniform_pm1_stream_rescaled(orc):
    """Both draws read the same Philox words: 2 phi - 1 reproduces the [-1, 1) entries exactly."""
    phi = orc.uniform01(1001, 77, 3)
    v = orc.uniform_pm1(1001, 77, 3)
    assert np.array_equal(2.0 * phi - 1.0, v)
    assert phi.min() >= 0.0 and phi.max() < 1.0


def test_phases_are_uniform(orc):
    phi = orc.uniform01(20000, 0x5EED, 1)
    assert stats.kstest(phi, "uniform").pvalue > 1e-3


@pytest.mark.parametrize("n", [2, 8, 64, 256])
def test_unitary_spectrum_has_unit_modulus_and_hermitian_symmetry(orc, n):
    u = orc.unitary_spectrum(n, 11, 1)
    assert np.max(np.abs(np.abs(u) - 1.0)) <= 4 * U
    # u_{n-j} = conj(u_j), so that c = Omega^{-1} u is real
    for j in range(1, n):
        assert u[n - j] == np.conj(u[j])
    assert u[0].imag == 0.0 and abs(u[0].real) == 1.0
    assert u[n // 2].imag == 0.0 and abs(u[n // 2].real) == 1.0


@pytest.mark.parametrize("n", [4, 32, 128, 512])
def test_unitary_circulant_is_real_orthogonal(orc, n):
    """Theorem 5.1: C = Omega^{-1} diag(u) Omega; with |u_j| = 1 it is unitary, and real because the
    spectrum is Hermitian-symmetric: C^T C = I, kappa(C) = 1."""
    c, cim = orc.unitary_circulant_column(n, 21 + n, 1)
    assert np.max(np.abs(cim)) <= 10 * n * U
    C = orc.circulant_dense(c)
    assert np.max(np.abs(C.T @ C - np.eye(n))) <= 20 * n * U
    s = np.linalg.svd(C, compute_uv=False)
    assert s.max() / s.min() <= 1 + 100 * n * U


@pytest.mark.parametrize("n", [8, 64, 256])
def test_unitary_column_transforms_back_to_its_spectrum(orc, n):
    """Omega c = u (Theorem 5.1, u = Omega c), by the oracle's plain forward DFT."""
    c, _ = orc.unitary_circulant_column(n, 5, 2)
    u = orc.unitary_spectrum(n, 5, 2)
    assert np.max(np.abs(orc.dft(c, sign=+1) - u)) <= 20 * n * U


@pytest.mark.parametrize("n", [1, 5, 16, 33])
def test_toeplitz_is_the_leading_block_of_the_2n_circulant(orc, n):
    c2 = orc.gaussian(2 * n, 9, 1)
    T = orc.toeplitz_dense(n, c2)
    C2 = orc.circulant_dense(c2)
    assert np.array_equal(T, C2[:n, :n])
    # constant diagonals: T_ij depends on i - j only
    for i in range(1, n):
        assert np.array_equal(T[i, 1:], T[i - 1, :-1])


@pytest.mark.parametrize("n", [8, 32, 64])
def test_leading_block_of_a_unitary_circulant_is_singular_when_its_real_eigenvalues_differ(orc, n):
    """Why no square Toeplitz multiplier is cut from a unitary circulant: the leading n x n block T of a
    real orthogonal 2n x 2n circulant (Hermitian-symmetric unit spectrum u) is singular exactly when
    u_0 u_n = -1, i.e. in half of the draws (checked on 40 draws per size), while the Gaussian and uniform
    Toeplitz blocks are well-conditioned."""
    for seed in range(40):
        c2, _ = orc.unitary_circulant_column(2 * n, seed, 1)
        u = orc.unitary_spectrum(2 * n, seed, 1)
        s = np.linalg.svd(orc.toeplitz_dense(n, c2), compute_uv=False)
        singular = s[-1] <= 1e-12 * s[0]
        assert singular == (u[0].real * u[n].real < 0)


@pytest.mark.parametrize("kind", [3, 4, 5])
def test_multiplier_kinds_generate_by_definition(orc, kind):
    n = 16
    h = orc.make_multiplier(kind, n, 40 + kind, 1)
    if kind == 3:
        assert h.shape == (n,)
        assert np.array_equal(h, orc.unitary_circulant_column(n, 40 + kind, 1)[0])
        D = orc.circulant_dense(h)
    else:
        assert h.shape == (2 * n,)
        base = {4: orc.gaussian(2 * n, 40 + kind, 1), 5: orc.uniform_pm1(2 * n, 40 + kind, 1)}[kind]
        assert np.array_equal(h, base)
        D = orc.toeplitz_dense(n, h)
    assert np.array_equal(orc.multiplier_dense(kind, n, h), D)


@pytest.mark.parametrize("kind", [3, 4, 5])
@pytest.mark.parametrize("n", [32, 128])
def test_structured_multiplier_solve(orc, kind, n):
    """Fact 4.1 with a structured H: GENP of A H, X = H Y and refinement reach the FP64 target and agree
    with the GEPP solution to kappa(A) times the backward errors."""
    r = np.random.default_rng(300 + n + kind)
    A = r.standard_normal((n, n))
    A[0, 0] = 0.0  # unmultiplied GENP breaks down at step 1
    B = r.standard_normal((n, 2))
    H = orc.make_multiplier(kind, n, 500 + kind, 1)
    out = orc.rmge_solve(kind, A, H, B, max_iters=10, be_tol=1e-13)
    assert out["info"] == 0
    be = orc.backward_error(A, out["X"], B)
    assert be <= 1e-13
    LU, piv, _ = orc.gepp(A)
    Xp = orc.gepp_solve(LU, piv, B)
    kappa = np.linalg.cond(A, np.inf)
    be_p = orc.backward_error(A, Xp, B)
    assert np.max(np.abs(out["X"] - Xp)) / np.max(np.abs(Xp)) <= 10 * kappa * (be + be_p)


@pytest.mark.parametrize("n,N", [(5, 5), (16, 16), (64, 128), (33, 66)])
def test_circulant_rows_is_the_product_with_the_dense_multiplier(orc, n, N):
    """orc_circulant_rows (rows of A H straight from H_kj = c[(k - j) mod N]) against the dense circulant or
    Toeplitz block times A by the plain product: same terms in the same order, so bit for bit."""
    rng = np.random.default_rng(n + N)
    A = rng.standard_normal((7, n))
    c = rng.standard_normal(N)
    D = orc.circulant_dense(c) if N == n else orc.toeplitz_dense(n, c)
    assert np.array_equal(orc.circulant_rows(A, c, N), orc.matmul(A, D))


def test_circulant_rows_exact_on_integers_and_by_the_dft(orc):
    """Integer inputs: the exact product by Python integers (brute force).  Real inputs: Theorem 5.1's
    diagonalisation, a row of A C is F^{-1}(F(a) conj(F(c))) for real c."""
    rng = np.random.default_rng(3)
    n = 12
    A = rng.integers(-9, 10, (3, n)).astype(np.float64)
    c = rng.integers(-9, 10, n).astype(np.float64)
    got = orc.circulant_rows(A, c)
    for i in range(3):
        for j in range(n):
            assert got[i, j] == sum(int(A[i, k]) * int(c[(k - j) % n]) for k in range(n))
    n = 1024
    A = rng.standard_normal((4, n))
    c = rng.standard_normal(n)
    ref = np.real(np.fft.ifft(np.fft.fft(A, axis=1) * np.conj(np.fft.fft(c))[None, :], axis=1))
    assert np.max(np.abs(orc.circulant_rows(A, c) - ref)) <= 1e-12 * np.max(np.abs(ref))
