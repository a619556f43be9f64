"""Pins for the oracle's norm and growth helpers against closed forms (the infinity norm behind the
backward error of Sec. 7.1, and the growth factor of Thm 3.2 / Remark 3.2)."""
import numpy as np
import pytest


def test_norm_inf_closed_forms(orc):
    assert orc.norm_inf(np.ones((3, 5))) == 5.0  # every row sums to its length
    assert orc.norm_inf(np.diag([1.0, -7.0, 3.0])) == 7.0  # the largest |d_i|
    assert orc.norm_inf(np.zeros((4, 4))) == 0.0
    P = np.eye(6)[[3, 0, 5, 1, 4, 2]]
    assert orc.norm_inf(-2.5 * P) == 2.5  # a scaled permutation: one entry per row
    A = np.array([[1.0, -2.0, 3.0], [-4.0, 0.5, 0.25]])
    assert orc.norm_inf(A) == 6.0  # rows sum to 6 and 4.75
    # ||A||_inf = ||A^T||_1: the largest column sum of the transpose (a different traversal of A)
    r = np.random.default_rng(3).standard_normal((7, 9))
    assert orc.norm_inf(r) == pytest.approx(max(np.abs(r.T).sum(axis=0)), rel=1e-15)


def test_norm_inf_propagates_nan(orc):
    A = np.eye(3)
    A[1, 2] = np.nan
    assert np.isnan(orc.norm_inf(A))


def test_growth_closed_forms(orc):
    # an upper-triangular M is its own U: GENP leaves it unchanged and the growth is 1
    M = np.triu(np.random.default_rng(5).standard_normal((6, 6))) + 3 * np.eye(6)
    LU, info = orc.genp(M)
    assert info == 0
    assert orc.growth(M, LU) == 1.0
    # 2 x 2 with a small leading pivot: u_22 = d - c b / a = 1 - 1 / 1e-3 = -999, max |m_ij| = 1
    M = np.array([[1e-3, 1.0], [1.0, 1.0]])
    LU, info = orc.genp(M)
    assert info == 0
    assert orc.growth(M, LU) == pytest.approx(999.0, rel=1e-12)
    # scaling M scales U alike: the growth is scale-invariant
    LU2, _ = orc.genp(8.0 * M)
    assert orc.growth(8.0 * M, LU2) == pytest.approx(999.0, rel=1e-12)
