"""The seeded input generators draw what the input recipe states: the singular values of the
orthogonal-factor systems (Sec. 7.1) and low-rank matrices (Sec. 7.2), orthogonal factors, the uneven
batch's size range and scaled leading pivot, and reproducibility from the seed."""
import numpy as np

from paper_1406_5802_gb300 import workloads as W


def test_orthogonal_factor_system_has_the_graded_singular_values():
    A, B = W.orthogonal_factor_system(48, 3, 1e-6, seed=11)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, W.graded_sigma(48, 1e-6), rtol=1e-8, atol=1e-15)
    assert s[0] == np.max(s) and abs(s[0] - 1.0) < 1e-12 and abs(s[-1] / 1e-6 - 1.0) < 1e-6
    assert B.shape == (48, 3)


def test_haar_factor_is_orthogonal_with_positive_r_diagonal():
    Q = W.haar_orthogonal(32, W.rng(5))
    assert np.allclose(Q.T @ Q, np.eye(32), atol=1e-13)


def test_lowrank_matrix_has_rank_r_and_the_given_basis():
    A, S = W.lowrank_test_matrix(64, 5, seed=3, tail=1e-10)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s[:5], 1.0 / np.arange(1, 6), rtol=1e-10)
    assert np.all(s[5:] < 2e-10)
    # the returned columns span A's leading left singular space: projecting A onto it leaves the tail
    R = A - S @ (S.T @ A)
    assert np.linalg.norm(R, 2) < 2e-10


def test_uneven_batch_recipe():
    sizes = W.batch_sizes(500, 32, 512, seed=7)
    assert sizes.min() >= 32 and sizes.max() <= 512 and len(np.unique(sizes)) > 100
    systems = W.batch_systems(sizes[:4], seed=8)
    r = W.rng(8)
    for (A, b, G), n in zip(systems, sizes[:4]):
        ref = r.standard_normal((n, n))  # the same stream, in the same order
        assert A[0, 0] == ref[0, 0] * 1e-10 and np.array_equal(A.ravel()[1:], ref.ravel()[1:])
        assert np.array_equal(b, r.standard_normal((n, 1)))
        assert np.array_equal(G, r.standard_normal((n, n)))


def test_generators_are_reproducible_from_the_seed():
    a1, b1 = W.gaussian_system(20, 2, seed=99)
    a2, b2 = W.gaussian_system(20, 2, seed=99)
    a3, _ = W.gaussian_system(20, 2, seed=100)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and not np.array_equal(a1, a3)
    A0, _ = W.gaussian_system(20, 1, seed=1, zero_leading_pivot=True)
    assert A0[0, 0] == 0.0


def test_real_fourier_matrix_is_orthogonal():
    for n in (7, 8):
        F = W.real_fourier_matrix(n)
        assert np.allclose(F @ F.T, np.eye(n), atol=1e-13)
