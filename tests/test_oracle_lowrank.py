"""Pins of the oracle's low-rank approximation (Sec. 6, Algorithm 6.1): the thin QR, the multipliers
(dense Gaussian n x l, or the n x l leading blocks of random circulants, Sec. 7.2), exactness on exactly
low-rank inputs, and the order of magnitude of the paper's Sec. 7.2 residual norms."""
import os

import numpy as np
import pytest

from paper_1406_5802_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
U = np.finfo(np.float64).eps / 2
MULT = {"gaussian": 0, "toeplitz_ex51": 2, "toeplitz_ex52": 3}


def golden():
    rows = []
    with open(os.path.join(HERE, "golden", "paper_lowrank_tables.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, mult, norm, r, n, mean, mx = line.split()
                rows.append((t, mult, norm, int(r), int(n), float(mean), float(mx)))
    return rows


@pytest.mark.parametrize("m,l", [(1, 1), (5, 1), (40, 7), (64, 64), (300, 32)])
def test_qr_against_lapack(orc, m, l):
    """Householder QR: Q^T Q = I, Q R = B, R upper with diag(R) >= 0, and equal to LAPACK's thin QR with
    the same sign convention (unique for full-rank B)."""
    B = W.rng(m + 17 * l).standard_normal((m, l))
    Q, R = orc.qr(B)
    assert np.max(np.abs(Q.T @ Q - np.eye(l))) <= 20 * m * U
    assert np.max(np.abs(Q @ R - B)) <= 20 * m * U * np.max(np.abs(B))
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) >= 0)
    Qn, Rn = np.linalg.qr(B)
    s = np.sign(np.diag(Rn))
    kappa = np.linalg.cond(B)
    assert np.max(np.abs(Q - Qn * s[None, :])) <= 100 * m * U * kappa
    assert np.max(np.abs(R - Rn * s[:, None])) <= 100 * m * U * kappa * np.max(np.abs(B))


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_multiplier_is_the_leading_block_of_the_circulant(orc, kind):
    n, l = 24, 5
    H = orc.lowrank_multiplier(kind, n, l, 9, 1)
    D = orc.lowrank_multiplier_dense(kind, n, l, H)
    if kind == 0:
        assert np.array_equal(D, H)
    else:
        assert np.array_equal(D, orc.circulant_dense(H)[:, :l])


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
@pytest.mark.parametrize("n,r", [(60, 3), (200, 16)])
def test_exact_on_exactly_low_rank_input(orc, kind, n, r):
    """For rank(A) = r and l = r, range(A H) = range(A) with probability 1, so Q Q^T A = A."""
    g = W.rng(1000 + n + kind)
    A = g.standard_normal((n, r)) @ g.standard_normal((r, n))
    H = orc.lowrank_multiplier(kind, n, r, 11 + kind, 1)
    Q, Z = orc.lowrank(kind, A, H, r)
    assert np.max(np.abs(Q.T @ Q - np.eye(r))) <= 50 * n * U
    assert np.linalg.norm(A - Q @ Z, 2) <= 1e-10 * np.linalg.norm(A, 2)
    # Q spans A H exactly (to rounding)
    B = A @ orc.lowrank_multiplier_dense(kind, n, r, H)
    assert np.linalg.norm(B - Q @ (Q.T @ B), 2) <= 1e-12 * np.linalg.norm(B, 2)


@pytest.mark.parametrize("row", [g for g in golden() if g[4] <= 128], ids=lambda g: f"{g[0]}-{g[2]}-r{g[3]}-n{g[4]}")
def test_residual_levels_match_the_paper(orc, row):
    """The order of magnitude of Sec. 7.2's mean residual norms over repeated draws (MATLAB's random stream
    cannot be reproduced, so only the level is pinned): the oracle's mean over 30 draws lies within two
    orders of magnitude of the printed mean, and far below the unapproximated norm 1/(r+1)."""
    _, mult, norm, r, n, mean, _ = row
    kind = MULT[mult]
    vals = []
    for t in range(30):
        A, Sr = W.lowrank_test_matrix(n, r, 5000 + 31 * t + n + r)
        H = orc.lowrank_multiplier(kind, n, r, 700 + t, 1)
        Q, Z = orc.lowrank(kind, A, H, r)
        vals.append(np.linalg.norm(Q @ (Q.T @ Sr) - Sr, 2) if norm == "rn1" else np.linalg.norm(A - Q @ Z, 2))
    m = float(np.mean(vals))
    assert mean / 100 <= m <= mean * 100, (m, mean)
