"""Pins of the oracle's pre-multiplied and two-sided randomized GENP solves (Fact 4.1: A^{-1} = (F A)^{-1} F
and A^{-1} = H (F A H)^{-1} F; Remark 5.1's simultaneous pre- and post-multipliers)."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1406_5802_gb300 import workloads as W
from test_oracle_genp import _leading_minors


def test_identity_multipliers_reduce_to_plain_genp(orc):
    """F = H = I: products with the identity are exact, so the result is the plain GENP solve bit for bit."""
    n, k = 40, 3
    r = W.rng(5)
    A = r.standard_normal((n, n)) + n * np.eye(n)
    B = r.standard_normal((n, k))
    out = orc.rmge_solve_two_sided(None, None, None, None, A, B, max_iters=0, be_tol=0.0)
    LU, info = orc.genp(A)
    assert out["info"] == info == 0
    assert np.array_equal(out["LU"], LU)
    assert np.array_equal(out["X"], orc.lu_solve(LU, B))


@pytest.mark.parametrize("kind", [0, 1])
def test_post_only_is_the_one_sided_solve(orc, kind):
    """F = I: the two-sided solve is exactly the post-multiplied solve of Fact 4.1 (same products, same
    sweeps), bit for bit."""
    n, k = 64, 2
    A, B = W.gaussian_system(n, k, seed=9, zero_leading_pivot=True)
    H = orc.make_multiplier(kind, n, 21, 1)
    two = orc.rmge_solve_two_sided(None, None, kind, H, A, B, max_iters=3, be_tol=1e-13)
    one = orc.rmge_solve(kind, A, H, B, max_iters=3, be_tol=1e-13)
    assert two["info"] == one["info"] == 0
    assert np.array_equal(two["LU"], one["LU"])
    assert np.array_equal(two["X"], one["X"])
    assert two["berr"] == one["berr"]


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("sides", ["pre", "both"])
def test_pivots_are_ratios_of_leading_minors_of_FAH(orc, seed, sides):
    """GENP runs on M = F A H (in this order): with small-integer F, A, H the product is exact and its
    pivots are ratios of the exact leading minors of F A H (det A = det B det S, eq. (3.1))."""
    r = W.rng(700 + seed)
    n = 4 + 2 * seed
    A = r.integers(-3, 4, (n, n))
    F = r.integers(-3, 4, (n, n))
    H = r.integers(-3, 4, (n, n)) if sides == "both" else np.eye(n, dtype=np.int64)
    M = F @ A @ H
    D = _leading_minors(M)
    if any(d == 0 for d in D):
        pytest.skip("a leading minor vanished for this draw")
    B = np.ones((n, 1))
    out = orc.rmge_solve_two_sided(0, F.astype(np.float64), 0 if sides == "both" else None,
                                   H.astype(np.float64) if sides == "both" else None, A.astype(np.float64), B,
                                   max_iters=0, be_tol=0.0)
    assert out["info"] == 0
    prev = Fraction(1)
    for kk in range(n):
        assert out["LU"][kk, kk] == pytest.approx(float(D[kk] / prev), rel=1e-12)
        prev = D[kk]


@pytest.mark.parametrize("kF,kH", [(0, None), (1, None), (0, 0), (1, 1), (1, 0)])
@pytest.mark.parametrize("n", [32, 200])
def test_pre_and_two_sided_solves_reach_the_fp64_target(orc, kF, kH, n):
    A, B = W.gaussian_system(n, 2, seed=40 + n, zero_leading_pivot=True)
    F = orc.make_multiplier(kF, n, 31, 1)
    H = orc.make_multiplier(kH, n, 31, 2) if kH is not None else None
    out = orc.rmge_solve_two_sided(kF, F, kH, H, A, B, max_iters=10, be_tol=1e-13)
    assert out["info"] == 0
    be = orc.backward_error(A, out["X"], B)
    assert be <= 1e-13
    LU, piv, _ = orc.gepp(A)
    Xp = orc.gepp_solve(LU, piv, B)
    kappa = np.linalg.cond(A, np.inf)
    assert np.max(np.abs(out["X"] - Xp)) / np.max(np.abs(Xp)) <= 10 * kappa * (be + orc.backward_error(A, Xp, B))


def test_pre_and_post_circulants_rescue_the_fourier_input(orc):
    """Theorem 5.2 (real analogue): on the orthogonal real Fourier matrix, a circulant post-multiplier leaves
    GENP failing; Remark 5.1 proposes random pre- and post-multipliers together, and with both circulants
    the unrefined solve is accurate again."""
    n = 256
    Fm = W.real_fourier_matrix(n)
    b = W.rng(3).standard_normal((n, 1))
    C1 = orc.make_multiplier(1, n, 11, 1)
    C2 = orc.make_multiplier(1, n, 12, 2)
    post = orc.rmge_solve_two_sided(None, None, 1, C2, Fm, b, max_iters=0, be_tol=0.0)
    both = orc.rmge_solve_two_sided(1, C1, 1, C2, Fm, b, max_iters=0, be_tol=0.0)
    assert post["info"] == 0 and both["info"] == 0
    assert orc.relative_residual(Fm, post["X"], b) > 1e-2
    assert orc.relative_residual(Fm, both["X"], b) <= 1e-10
