"""Seeded synthetic input generators shared by the tests, the benchmark and the oracle checks.

This module holds none of the method's arithmetic (no multiplier application,
no elimination, no solve): it only draws the matrices A, B and the fixed
multipliers G that are passed to both the CUDA library and the CPU oracle as
inputs.  Every generator takes an explicit integer seed and draws from numpy's
counter-based Philox bit generator (or torch's generator for the device-side
variants of the large workloads), so each input is reproducible.

Workload recipes (shapes, value distributions) follow the paper's experiments
(Sec. 7.1: orthogonal-factor matrices built as in Higham's Sec. 28.3, Gaussian
Toeplitz blocks, Gaussian right-hand sides) and the five workload families the
library is measured on.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x5EED0000


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def haar_orthogonal(n: int, r: np.random.Generator) -> np.ndarray:
    """Q factor of the QR factorization of an n x n Gaussian matrix, signs fixed so diag(R) > 0."""
    X = r.standard_normal((n, n))
    Q, R = np.linalg.qr(X)
    return Q * np.sign(np.diag(R))[None, :]


def gaussian_system(n: int, k: int, seed: int, zero_leading_pivot: bool = False):
    """A with i.i.d. N(0,1) entries (optionally A[0,0] = 0, which makes unmultiplied GENP break down at
    step 1), B (n x k) i.i.d. N(0,1)."""
    r = rng(seed)
    A = r.standard_normal((n, n))
    if zero_leading_pivot:
        A[0, 0] = 0.0
    B = r.standard_normal((n, k))
    return A, B


def graded_sigma(n: int, sigma_min: float) -> np.ndarray:
    """Singular values log-spaced from 1 down to sigma_min."""
    if n == 1:
        return np.ones(1)
    return 10.0 ** (np.log10(sigma_min) * np.arange(n) / (n - 1))


def orthogonal_factor_system(n: int, k: int, sigma_min: float, seed: int):
    """A = U diag(sigma) V^T, U and V Haar-orthogonal, sigma log-spaced 1 .. sigma_min; B i.i.d. N(0,1)."""
    r = rng(seed)
    U = haar_orthogonal(n, r)
    V = haar_orthogonal(n, r)
    s = graded_sigma(n, sigma_min)
    A = (U * s[None, :]) @ V.T
    B = r.standard_normal((n, k))
    return A, B


def lowrank_test_matrix(n: int, r: int, seed: int, tail: float = 1e-10):
    """The low-rank test matrices of Sec. 7.2: A = S diag(sigma) T^T with S, T Haar-orthogonal n x n,
    sigma_j = 1/j for j <= r and sigma_j = tail beyond (so ||A|| = 1 and the numerical rank is r).
    Returns (A, S_r): S_r = the first r columns of S, a basis of A's leading r-dimensional left singular
    space."""
    g = rng(seed)
    S = haar_orthogonal(n, g)
    T = haar_orthogonal(n, g)
    sigma = np.full(n, float(tail))
    sigma[:r] = 1.0 / np.arange(1, r + 1)
    A = (S * sigma[None, :]) @ T.T
    return A, np.ascontiguousarray(S[:, :r])


def orthogonal_factor_system_torch(n: int, k: int, sigma_min: float, seed: int, device: str):
    """Same recipe as orthogonal_factor_system, drawn with torch on ``device`` (used for the large
    workloads, whose host-side QR would take minutes).  Returns float64 torch tensors on ``device``."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    s = torch.tensor(graded_sigma(n, sigma_min), dtype=torch.float64, device=device)

    def haar():
        X = torch.randn(n, n, generator=g, dtype=torch.float64, device=device)
        Q, R = torch.linalg.qr(X)
        return Q * torch.sign(torch.diagonal(R))[None, :]

    U = haar()
    V = haar()
    A = (U * s[None, :]) @ V.T
    del U, V
    B = torch.randn(n, k, generator=g, dtype=torch.float64, device=device)
    return A.contiguous(), B.contiguous()


def gaussian_multiplier(n: int, seed: int) -> np.ndarray:
    """A fixed n x n standard Gaussian multiplier (Def. 4.1) drawn by numpy, used where a test passes the
    same G to both sides."""
    return rng(seed).standard_normal((n, n))


def gaussian_column(n: int, seed: int) -> np.ndarray:
    """First column of a Gaussian circulant multiplier."""
    return rng(seed).standard_normal(n)


def toeplitz_from_params(p: np.ndarray, rows: int, cols: int) -> np.ndarray:
    """T[i, j] = p[i - j + cols - 1] (a Toeplitz matrix from its rows + cols - 1 diagonals)."""
    i = np.arange(rows)[:, None]
    j = np.arange(cols)[None, :]
    return p[i - j + cols - 1]


def paper_sec71_matrix(n: int, r: np.random.Generator) -> np.ndarray:
    """The Sec. 7.1 test matrix: A = [[A_k, B], [C, D]], k = n/2, A_k = U Sigma V^T with sigma = 1 (k-4
    times) and 0 (4 times), U, V Haar-orthogonal; B, C, D Gaussian Toeplitz matrices scaled to unit
    spectral norm.  The leading k x k block is singular (nullity 4), so GENP without a multiplier is
    expected to fail numerically."""
    k = n // 2
    U = haar_orthogonal(k, r)
    V = haar_orthogonal(k, r)
    s = np.ones(k)
    s[k - 4:] = 0.0
    Ak = (U * s[None, :]) @ V.T
    blocks = []
    for _ in range(3):
        T = toeplitz_from_params(r.standard_normal(2 * k - 1), k, k)
        blocks.append(T / np.linalg.norm(T, 2))
    Bt, Ct, Dt = blocks
    return np.block([[Ak, Bt], [Ct, Dt]])


def dft_matrix(n: int) -> np.ndarray:
    """Omega = (w^{ij}), w = exp(2 pi sqrt(-1) / n) (Sec. 5)."""
    i = np.arange(n)
    return np.exp(2j * np.pi * np.outer(i, i) / n)


def real_fourier_matrix(n: int) -> np.ndarray:
    """Orthogonal real Fourier matrix (rows: constant, then cos/sin pairs of increasing frequency, and the
    alternating row for even n), each row scaled to unit norm.  A real analogue of the DFT input of
    Theorem 5.2, used on the real GPU path."""
    t = np.arange(n)
    rows = [np.ones(n) / np.sqrt(n)]
    f = 1
    while len(rows) < n:
        if 2 * f == n:
            rows.append(np.cos(np.pi * t) / np.sqrt(n))
            break
        rows.append(np.cos(2 * np.pi * f * t / n) * np.sqrt(2.0 / n))
        if len(rows) < n:
            rows.append(np.sin(2 * np.pi * f * t / n) * np.sqrt(2.0 / n))
        f += 1
    return np.array(rows)


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """System sizes n ~ U{lo..hi} for the uneven batch."""
    return rng(seed).integers(lo, hi + 1, size=count)


def batch_systems(sizes, seed: int, leading_scale: float = 1e-10):
    """Per system: A i.i.d. N(0,1) with A[0,0] scaled by leading_scale, b i.i.d. N(0,1), G i.i.d. N(0,1)."""
    r = rng(seed)
    out = []
    for n in sizes:
        n = int(n)
        A = r.standard_normal((n, n))
        A[0, 0] *= leading_scale
        b = r.standard_normal((n, 1))
        G = r.standard_normal((n, n))
        out.append((A, b, G))
    return out


def grad_system(n: int, k: int, seed: int):
    """A = 4 I + N(0,1)/sqrt(n), B (n x k) N(0,1), W (n x k) N(0,1) (loss = sum(X * W))."""
    r = rng(seed)
    A = 4.0 * np.eye(n) + r.standard_normal((n, n)) / np.sqrt(n)
    B = r.standard_normal((n, k))
    W = r.standard_normal((n, k))
    return A, B, W
