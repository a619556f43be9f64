"""Pins for the oracle's multiplier application, circulants, solve, refinement, backward error and adjoint
(Fact 4.1, Thm 5.1, Thm 5.2, Sec. 7.1)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from paper_1406_5802_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def _paper_table():
    rows = {}
    with open(os.path.join(HERE, "golden", "paper_tables.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if len(t) == 5:
                rows[(t[0], int(t[1]), int(t[2]))] = float(t[3])
            else:
                rows[t[0]] = float(t[1])
    return rows


# ----------------------------------------------------------------------------- circulants, Thm 5.1

def test_circulant_dense_is_the_textbook_circulant(orc):
    c = W.gaussian_column(13, 1)
    assert np.array_equal(orc.circulant_dense(c), sla.circulant(c))


def test_dft_matches_fft(orc):
    x = W.rng(2).standard_normal(24) + 1j * W.rng(3).standard_normal(24)
    assert np.allclose(orc.dft(x, -1), np.fft.fft(x), atol=1e-12)
    assert np.allclose(orc.dft(x, +1), np.fft.ifft(x) * 24, atol=1e-12)


def test_circulant_diagonalised_by_dft(orc):
    """Theorem 5.1: C = Omega^{-1} diag(Omega c) Omega, Omega^{-1} = Omega^H / n."""
    n = 16
    c = W.gaussian_column(n, 4)
    Om = W.dft_matrix(n)
    u = orc.dft(c, +1)
    assert np.allclose(u, Om @ c, atol=1e-12)
    C = (Om.conj().T / n) @ np.diag(u) @ Om
    assert np.allclose(C, orc.circulant_dense(c), atol=1e-12)


def test_post_multiplication_by_circulant_is_circular_correlation(orc):
    """(A C)_{ij} = sum_k a_ik c_{(k-j) mod n}: each row of A C is the circular cross-correlation of the row
    with c, i.e. ifft(fft(a) * conj(fft(c))) for real c."""
    n = 32
    A = W.rng(5).standard_normal((6, n))
    c = W.gaussian_column(n, 6)
    M = orc.matmul(A, orc.circulant_dense(c))
    ref = np.real(np.fft.ifft(np.fft.fft(A, axis=1) * np.conj(np.fft.fft(c))[None, :], axis=1))
    assert np.allclose(M, ref, atol=1e-12)


# ----------------------------------------------------------------------------- residual / backward error

def test_residual_meets_the_dot2_error_bound(orc):
    """The compensated residual meets Ogita-Rump-Oishi's Dot2 bound |res - s| <= u|s| + gamma_n^2 sum|p_i|
    against the exact value s (rational arithmetic) on an ill-conditioned, cancellation-heavy dot product,
    far below what a plain FP64 dot product can reach."""
    r = W.rng(7)
    n = 40
    A = r.standard_normal((3, n)) * 2.0 ** r.integers(-30, 30, (3, n))
    X = r.standard_normal((n, 1))
    B = A @ X  # rounded: true residual is tiny and cancellation-heavy
    R = orc.residual(A if A.shape[0] == A.shape[1] else np.pad(A, ((0, n - 3), (0, 0))), X,
                     np.pad(B, ((0, n - 3), (0, 0))))
    for i in range(3):
        exact = Fraction(float(B[i, 0])) - sum(Fraction(float(A[i, t])) * Fraction(float(X[t, 0])) for t in range(n))
        u = 2.0**-53
        gam = (n + 1) * u / (1 - (n + 1) * u)
        bound = u * abs(float(exact)) + gam * gam * float(np.sum(np.abs(A[i] * X[:, 0]))) + abs(float(B[i, 0])) * gam * gam
        assert abs(R[i, 0] - float(exact)) <= bound
        plain = float(B[i, 0]) - float(np.dot(A[i], X[:, 0]))
        assert abs(R[i, 0] - float(exact)) <= abs(plain - float(exact)) + 1e-300


def test_backward_error_definition_and_invariance(orc):
    A = np.array([[2.0, 0.0], [0.0, 4.0]])
    X = np.array([[1.0], [1.0]])
    B = np.array([[2.0], [5.0]])  # residual (0, 1); ||A||_inf = 4, ||x|| = 1, ||b|| = 5
    assert orc.backward_error(A, X, B) == pytest.approx(1.0 / (4.0 + 5.0), rel=1e-15)
    r = W.rng(8)
    A = r.standard_normal((20, 20))
    X = r.standard_normal((20, 3))
    B = A @ X + 1e-9 * r.standard_normal((20, 3))
    e = orc.backward_error(A, X, B)
    assert orc.backward_error(8.0 * A, X, 8.0 * B) == pytest.approx(e, rel=1e-14)
    # the Rigal-Gaches value is the smallest relative perturbation: perturb A by dA = r x^T sign stuff and
    # check the perturbed system is solved exactly to rounding
    Xs = X[:, :1]
    R = orc.residual(A, Xs, B[:, :1])
    eta = orc.backward_error(A, Xs, B[:, :1])
    an, xn, bn = np.max(np.sum(np.abs(A), 1)), np.max(np.abs(Xs)), np.max(np.abs(B[:, :1]))
    j = int(np.argmax(np.abs(Xs)))
    dA = (an / (an * xn + bn)) * R @ (np.sign(Xs[j]) * np.eye(20)[j:j + 1])
    dB = -(bn / (an * xn + bn)) * R
    assert np.max(np.abs((A + dA) @ Xs - (B[:, :1] + dB))) <= 1e-12 * np.max(np.abs(B))
    assert np.max(np.sum(np.abs(dA), 1)) <= eta * an * (1 + 1e-9)


def test_relative_residual_definition(orc):
    """Sec. 7.1's relative residual ||A x - b||_2 / ||b||_2, the largest over the columns: closed forms
    with a residual of known length, and invariance under scaling of the whole system."""
    A = np.diag([2.0, 4.0, 1.0])
    X = np.array([[1.0, 0.0], [1.0, 0.0], [1.0, 0.0]])
    B = np.array([[2.0, 3.0], [7.0, 0.0], [1.0, 4.0]])  # residuals (0, 3, 0) and (3, 0, 4); ||b|| 7.348.., 5
    assert orc.relative_residual(A, X, B) == pytest.approx(1.0, rel=1e-15)  # column 2: ||(3, 0, 4)|| / 5
    assert orc.relative_residual(A, X[:, :1], B[:, :1]) == pytest.approx(3.0 / np.sqrt(54.0), rel=1e-15)
    r = W.rng(9)
    A = r.standard_normal((12, 12))
    X = r.standard_normal((12, 2))
    B = A @ X + 1e-6 * r.standard_normal((12, 2))
    e = orc.relative_residual(A, X, B)
    assert orc.relative_residual(3.0 * A, X, 3.0 * B) == pytest.approx(e, rel=1e-12)
    ref = max(np.linalg.norm(A @ X[:, c] - B[:, c]) / np.linalg.norm(B[:, c]) for c in range(2))
    assert e == pytest.approx(ref, rel=1e-6)


def test_backward_error_flags_nonfinite(orc):
    A = np.eye(3)
    X = np.array([[1.0], [np.nan], [0.0]])
    assert orc.backward_error(A, X, np.ones((3, 1))) == math.inf


# ----------------------------------------------------------------------------- the solve (Fact 4.1)

@pytest.mark.parametrize("kind", [0, 1, 2])
def test_solve_recovers_gepp_solution(orc, kind):
    """Fact 4.1: A^{-1} = H (A H)^{-1}, x = H y; the refined solution agrees with GEPP's."""
    n, k = 96, 3
    A, B = W.gaussian_system(n, k, seed=9, zero_leading_pivot=True)
    H = orc.make_multiplier(kind, n, seed=10)
    out = orc.rmge_solve(kind, A, H, B, max_iters=10, be_tol=1e-13)
    assert out["info"] == 0
    assert out["berr"][-1] <= 1e-13
    LU, piv, _ = orc.gepp(A)
    x_pp = orc.gepp_solve(LU, piv, B)
    kappa = np.linalg.cond(A, np.inf)
    assert np.max(np.abs(out["X"] - x_pp)) <= 10 * kappa * 1e-13 * np.max(np.abs(x_pp))
    # the returned factors are GENP of M = A H
    M = orc.apply_multiplier(kind, A, H)
    LU2, info = orc.genp(M)
    assert info == 0 and np.array_equal(LU2, out["LU"])


def test_unmultiplied_genp_breaks_down_and_multiplier_fixes_it(orc):
    n = 256
    A, B = W.gaussian_system(n, 1, seed=W.SEED_BASE + 1, zero_leading_pivot=True)
    assert orc.genp(A)[1] == 1
    G = orc.make_multiplier(0, n, seed=W.SEED_BASE + 1, subseq=1)
    out = orc.rmge_solve(0, A, G, B)
    assert out["info"] == 0 and out["berr"][-1] <= 1e-13


def test_refinement_sweep_contracts(orc):
    n = 128
    A, B = W.orthogonal_factor_system(n, 2, 1e-6, seed=11)
    G = W.gaussian_multiplier(n, 12)
    out = orc.rmge_solve(0, A, G, B, max_iters=4, be_tol=0.0)
    e = out["berr"]
    assert len(e) == 5
    assert e[1] < e[0] and e[1] <= 1e-14
    # one manual sweep reproduces the second backward error
    Y = orc.lu_solve(out["LU"], B)
    X0 = orc.matmul(G, Y)
    assert orc.backward_error(A, X0, B) == pytest.approx(e[0], rel=1e-12)
    X1 = orc.refine_step(0, A, out["LU"], G, B, X0)
    assert orc.backward_error(A, X1, B) == pytest.approx(e[1], rel=1e-6)


# ----------------------------------------------------------------------------- Theorem 5.2 (narrow class)

@pytest.mark.parametrize("n", [16, 64, 256])
def test_dft_second_pivot_closed_form(orc, n):
    """Thm 5.2(i): GENP on Omega has second pivot w - 1, |w - 1| = 2 sin(pi/n)."""
    _, piv, info = orc.genp_complex(W.dft_matrix(n)[:4, :4])
    w = np.exp(2j * np.pi / n)
    assert info == 0
    assert piv[0] == pytest.approx(1.0)
    assert abs(piv[1] - (w - 1)) <= 1e-13
    assert abs(piv[1]) == pytest.approx(2 * math.sin(math.pi / n), rel=1e-12)


def test_gaussian_circulant_keeps_the_dft_pivot_small(orc):
    """Thm 5.2(ii): Omega C = D Omega with D = diag(Omega c); GENP(D Omega) has pivots d_k pivot_k(Omega)."""
    n = 128
    c = W.gaussian_column(n, 13)
    Om = W.dft_matrix(n)
    C = orc.circulant_dense(c)
    OC = Om @ C
    d = Om @ c
    assert np.allclose(OC, d[:, None] * Om, atol=1e-9)
    _, piv, _ = orc.genp_complex(OC[:3, :3])
    w = np.exp(2j * np.pi / n)
    assert abs(piv[0] - d[0]) <= 1e-9 * abs(d[0])
    assert abs(piv[1] - d[1] * (w - 1)) <= 1e-8 * abs(d[1] * (w - 1))


def test_dft_like_input_defeats_genp_and_circulant_but_not_gaussian(orc):
    """Sec. 7.1 on DFT inputs (real orthogonal Fourier matrix as the real analogue): GENP and
    circulant-GENP fail numerically, Gaussian-GENP is fine after refinement."""
    n = 256
    F = W.real_fourier_matrix(n)
    assert np.allclose(F @ F.T, np.eye(n), atol=1e-12)
    b = W.rng(14).standard_normal((n, 1))
    LU, info = orc.genp(F)
    x = orc.lu_solve(LU, b) if info == 0 else np.full((n, 1), np.nan)
    assert not (orc.relative_residual(F, x, b) <= 1e-6)
    c = W.gaussian_column(n, 15)
    out_c = orc.rmge_solve(1, F, c, b, max_iters=0)
    assert not (orc.relative_residual(F, out_c["X"], b) <= 1e-6) if out_c["info"] == 0 else True
    G = W.gaussian_multiplier(n, 16)
    out_g = orc.rmge_solve(0, F, G, b, max_iters=1, be_tol=0.0)
    assert out_g["info"] == 0
    assert orc.relative_residual(F, out_g["X"], b) <= 1e-12


# ----------------------------------------------------------------------------- Sec. 7.1 statistics

@pytest.mark.slow
@pytest.mark.parametrize("n", [64, 256])
def test_paper_sec71_statistics(orc, n):
    """Order-of-magnitude agreement with Tables 7.2-7.4 on the Sec. 7.1 matrices (fewer runs than the
    paper's 1000; MATLAB's random stream is not reproducible, so only the levels are pinned)."""
    tab = _paper_table()
    runs = 12 if n == 256 else 40
    r = W.rng(W.SEED_BASE + 71 + n)
    res = {"nomult": [], "gauss0": [], "gauss1": [], "circ0": [], "circ1": [], "gepp": []}
    for t in range(runs):
        A = W.paper_sec71_matrix(n, r)
        b = r.standard_normal((n, 1))
        LU, info = orc.genp(A)
        x = orc.lu_solve(LU, b) if info == 0 else np.full((n, 1), np.nan)
        res["nomult"].append(orc.relative_residual(A, x, b))
        LUp, piv, _ = orc.gepp(A)
        res["gepp"].append(orc.relative_residual(A, orc.gepp_solve(LUp, piv, b), b))
        G = r.standard_normal((n, n))
        o = orc.rmge_solve(0, A, G, b, max_iters=1, be_tol=0.0)
        X0 = orc.matmul(G, orc.lu_solve(o["LU"], b))
        res["gauss0"].append(orc.relative_residual(A, X0, b))
        res["gauss1"].append(orc.relative_residual(A, o["X"], b))
        c = r.uniform(-1, 1, n)
        o = orc.rmge_solve(2, A, c, b, max_iters=1, be_tol=0.0)
        X0 = orc.matmul(orc.circulant_dense(c), orc.lu_solve(o["LU"], b))
        res["circ0"].append(orc.relative_residual(A, X0, b))
        res["circ1"].append(orc.relative_residual(A, o["X"], b))
    nm = np.array(res["nomult"])
    assert np.nanmin(nm) >= tab["nomult_range_lo"] / 10 or np.all(~np.isfinite(nm))
    for key, (table, it) in {"gauss0": ("gaussian", 0), "gauss1": ("gaussian", 1),
                             "circ0": ("circulant", 0), "circ1": ("circulant", 1),
                             "gepp": ("gepp", 0)}.items():
        ours = float(np.median(res[key]))
        paper = tab[(table, n, it)]
        # the paper's means are dominated by rare large draws; the median must not exceed the mean by
        # more than 10x and refinement must reach the paper's 1-step level within 100x
        assert ours <= 10 * paper, (key, ours, paper)
        assert ours >= paper / 1e4, (key, ours, paper)
    assert np.median(res["gauss1"]) < np.median(res["gauss0"]) / 100


# ----------------------------------------------------------------------------- adjoint reference

def test_adjoint_matches_central_differences(orc):
    """dL/dB = A^{-T} Wbar, dL/dA = -dL/dB X^T for L = sum(X * W), X = A^{-1} B; FP64 central FD, n = 16."""
    n, k = 16, 4
    A, B, Wt = W.grad_system(n, k, seed=W.SEED_BASE + 5)

    def loss(A_, B_):
        LU, piv, _ = orc.gepp(A_)
        return float(np.sum(orc.gepp_solve(LU, piv, B_) * Wt))

    LU, piv, _ = orc.gepp(A)
    X = orc.gepp_solve(LU, piv, B)
    dB, dA, info = orc.solve_adjoint_gepp(A, X, Wt)
    assert info == 0
    fdA = np.zeros_like(A)
    for i in range(n):
        for j in range(n):
            h = 1e-6 * max(1.0, abs(A[i, j]))
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h
            Am[i, j] -= h
            fdA[i, j] = (loss(Ap, B) - loss(Am, B)) / (2 * h)
    fdB = np.zeros_like(B)
    for i in range(n):
        for j in range(k):
            h = 1e-6 * max(1.0, abs(B[i, j]))
            Bp, Bm = B.copy(), B.copy()
            Bp[i, j] += h
            Bm[i, j] -= h
            fdB[i, j] = (loss(A, Bp) - loss(A, Bm)) / (2 * h)
    assert np.max(np.abs(dA - fdA)) <= 1e-6 * np.max(np.abs(fdA))
    assert np.max(np.abs(dB - fdB)) <= 1e-6 * np.max(np.abs(fdB))
    # and the GENP-factor route (A G = L U, A^{-T} = L^{-T} U^{-T} G^T) gives the same dB
    G = W.gaussian_multiplier(n, 17)
    LUg, info = orc.genp(orc.matmul(A, G))
    dB2 = orc.lu_solve_transposed(LUg, orc.matmul(G.T, Wt))
    assert np.max(np.abs(dB2 - dB)) <= 1e-10 * np.max(np.abs(dB))
