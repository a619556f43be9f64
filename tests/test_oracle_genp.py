"""Pins for the oracle's GENP, blocked GENP, GEPP and triangular solves (Sec. 3, Cor. 3.1, Thm 3.2)."""
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from paper_1406_5802_gb300 import workloads as W


def _exact_factors(n, seed):
    """Integer unit-lower L0 and upper U0 with pivots in {+-1, +-2, +-4}: every GENP operation on
    M = L0 U0 is exact in FP64, so GENP must return L0 and U0 bit for bit."""
    r = W.rng(seed)
    L0 = np.tril(r.integers(-3, 4, (n, n)), -1).astype(np.float64) + np.eye(n)
    U0 = np.triu(r.integers(-3, 4, (n, n)), 1).astype(np.float64)
    U0 += np.diag(r.choice([-4.0, -2.0, -1.0, 1.0, 2.0, 4.0], n))
    return L0, U0


def _leading_minors(M_int):
    """Exact leading principal minors D_1..D_n of an integer matrix (fraction-free Gaussian elimination,
    done in exact rationals)."""
    n = len(M_int)
    A = [[Fraction(int(v)) for v in row] for row in M_int]
    D = []
    det = Fraction(1)
    for k in range(n):
        # D_{k+1} = det of the leading (k+1) block, by exact elimination with row pivoting inside it
        B = [row[: k + 1] for row in A[: k + 1]]
        det = Fraction(1)
        m = k + 1
        for s in range(m):
            p = next((i for i in range(s, m) if B[i][s] != 0), None)
            if p is None:
                det = Fraction(0)
                break
            if p != s:
                B[s], B[p] = B[p], B[s]
                det = -det
            det *= B[s][s]
            for i in range(s + 1, m):
                f = B[i][s] / B[s][s]
                for j in range(s, m):
                    B[i][j] -= f * B[s][j]
        D.append(det)
    return D


@pytest.mark.parametrize("n,seed", [(1, 1), (5, 2), (17, 3), (40, 4)])
def test_genp_exact_reconstruction(orc, n, seed):
    L0, U0 = _exact_factors(n, seed)
    M = L0 @ U0
    assert np.all(np.abs(M) < 2.0**50)
    LU, info = orc.genp(M)
    assert info == 0
    assert np.array_equal(np.tril(LU, -1) + np.eye(n), L0)
    assert np.array_equal(np.triu(LU), U0)


@pytest.mark.parametrize("seed", range(6))
def test_genp_pivots_are_ratios_of_leading_minors(orc, seed):
    """det A = det B det S (eq. (3.1)) gives pivot_k = D_k / D_{k-1}, with M = A G exact in integers."""
    r = W.rng(100 + seed)
    n = 3 + seed
    A = r.integers(-3, 4, (n, n))
    G = r.integers(-3, 4, (n, n))
    M = A @ G
    D = _leading_minors(M)
    if any(d == 0 for d in D):
        pytest.skip("a leading minor vanished for this draw")
    LU, info = orc.genp(M.astype(np.float64))
    assert info == 0
    prev = Fraction(1)
    for k in range(n):
        expect = float(D[k] / prev)
        assert LU[k, k] == pytest.approx(expect, rel=1e-12)
        prev = D[k]


def test_genp_breakdown_step_is_first_singular_leading_block(orc):
    """Cor. 3.1: GENP meets a zero pivot exactly when a leading block is singular."""
    A, _ = W.gaussian_system(32, 1, seed=5, zero_leading_pivot=True)
    _, info = orc.genp(A)
    assert info == 1
    # singular leading 2x2 (row 1 = 2 * row 0 on the first two columns), nonzero a00
    A2 = W.rng(6).integers(-3, 4, (6, 6)).astype(np.float64)
    A2[0, 0] = 3.0
    A2[1, :2] = 2.0 * A2[0, :2]
    assert _leading_minors(A2.astype(np.int64))[1] == 0
    _, info = orc.genp(A2)
    assert info == 2
    # NaN input: reported at the first pivot it reaches
    A3 = np.eye(4)
    A3[2, 2] = np.nan
    assert orc.genp(A3)[1] == 3


@pytest.mark.parametrize("n,nb", [(33, 1), (33, 8), (64, 16), (70, 32), (70, 70), (50, 64)])
def test_blocked_equals_unblocked(orc, n, nb):
    """Sec. 3: any blocking reaches the same Schur complements, hence the same L and U."""
    L0, U0 = _exact_factors(n, 31)
    M = L0 @ U0
    assert np.array_equal(orc.genp_blocked(M, nb)[0], orc.genp(M)[0])  # exact inputs: bitwise
    A = W.gaussian_multiplier(n, 7) + 4 * np.sqrt(n) * np.eye(n)
    Lb, ib = orc.genp_blocked(A, nb)
    Lu, iu = orc.genp(A)
    assert ib == iu == 0
    assert np.max(np.abs(Lb - Lu)) <= 1e-12 * np.max(np.abs(Lu))


def test_genp_matches_lapack_when_no_pivoting_is_needed(orc):
    """On a column diagonally dominant matrix partial pivoting never swaps, so GENP = LAPACK getrf."""
    n = 60
    A = W.gaussian_multiplier(n, 8)
    A += np.diag(np.sum(np.abs(A), axis=0) + 1.0)
    LU, info = orc.genp(A)
    lu, piv = sla.lu_factor(A)
    assert info == 0 and np.array_equal(piv, np.arange(n))
    assert np.max(np.abs(LU - lu)) <= 1e-13 * np.max(np.abs(lu))


def test_gepp_matches_lapack(orc):
    A = W.gaussian_multiplier(48, 9)
    LU, piv, info = orc.gepp(A)
    lu, lpiv = sla.lu_factor(A)
    assert info == 0 and np.array_equal(piv, lpiv)
    assert np.max(np.abs(LU - lu)) <= 1e-13 * np.max(np.abs(lu))
    b = W.rng(10).standard_normal((48, 3))
    x = orc.gepp_solve(LU, piv, b)
    assert np.max(np.abs(x - sla.lu_solve((lu, lpiv), b))) <= 1e-11 * np.max(np.abs(x))


def test_lu_solve_against_triangular_solves(orc):
    n, k = 45, 4
    L0, U0 = _exact_factors(n, 12)
    LU = np.tril(L0, -1) + U0
    b = W.rng(13).standard_normal((n, k))
    y = orc.lu_solve(LU, b)
    z = sla.solve_triangular(L0, b, lower=True, unit_diagonal=True)
    yy = sla.solve_triangular(U0, z, lower=False)
    assert np.allclose(y, yy, rtol=1e-10, atol=1e-10 * np.max(np.abs(yy)))
    # (L U)^T y = b  <=>  U^T p = b, L^T y = p
    yt = orc.lu_solve_transposed(LU, b)
    p = sla.solve_triangular(U0, b, lower=False, trans="T")
    yy = sla.solve_triangular(L0, p, lower=True, unit_diagonal=True, trans="T")
    assert np.allclose(yt, yy, rtol=1e-10, atol=1e-10 * np.max(np.abs(yy)))


@pytest.mark.parametrize("seed", range(4))
def test_pivot_magnitude_bounds(orc, seed):
    """Theorem 3.2: |pivot| <= N + N_- N^2 and 1/|pivot| <= N_-, N = ||A||, N_- = max_j ||(A^(j))^-1||."""
    n = 24
    A = W.rng(200 + seed).standard_normal((n, n))
    N = np.linalg.norm(A, 2)
    Nm = max(np.linalg.norm(np.linalg.inv(A[:j, :j]), 2) for j in range(1, n + 1))
    LU, info = orc.genp(A)
    assert info == 0
    piv = np.abs(np.diag(LU))
    assert np.all(piv <= (N + Nm * N * N) * (1 + 1e-12))
    assert np.all(1.0 / piv <= Nm * (1 + 1e-10))


def test_matmul_exact_on_integers(orc):
    r = W.rng(14)
    A = r.integers(-50, 51, (37, 53))
    B = r.integers(-50, 51, (53, 29))
    assert np.array_equal(orc.matmul(A.astype(float), B.astype(float)), (A @ B).astype(float))


def test_growth_definition_special_case(orc):
    M = np.array([[2.0, 1.0], [4.0, 1.0]])
    LU, _ = orc.genp(M)  # U = [[2, 1], [0, -1]]
    assert orc.growth(M, LU) == pytest.approx(2.0 / 4.0)
