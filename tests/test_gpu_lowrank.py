"""GPU-vs-oracle parity of the randomized low-rank approximation (Sec. 6, Algorithm 6.1) through the C ABI:
the multiplier draw, Q = Q(A H) (unique thin QR factor: equal to the oracle's Householder Q), Z = Q^T A,
the paper's Sec. 7.2 residual levels, exact low rank, rank deficiency and argument checks."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = 2.0**-53
KIND = {"gaussian": 0, "circulant": 1, "circulant_uniform": 2, "circulant_unitary": 3}


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


def oracle_H(kind, H, n):
    h = host(H)
    return h if KIND[kind] == 0 else h[:n]


@pytest.mark.parametrize("kind", list(KIND))
def test_multiplier_matches_oracle(orc, kind):
    n, l = 256, 8
    H = host(rmge.lowrank_multiplier(kind, n, l, 41, 3))
    ref = orc.lowrank_multiplier(KIND[kind], n, l, 41, 3)
    got = H if KIND[kind] == 0 else H[:n]
    if kind == "circulant_uniform":
        assert np.array_equal(got, ref)
    else:
        assert np.max(np.abs(got - ref)) <= 40 * U64 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("kind", list(KIND))
@pytest.mark.parametrize("m,n,l", [(64, 64, 1), (300, 256, 8), (1000, 512, 32), (2048, 1024, 64)])
def test_basis_and_projection_match_oracle(orc, kind, m, n, l):
    g = W.rng(m + n + l + KIND[kind])
    A = g.standard_normal((m, n))
    H = rmge.lowrank_multiplier(kind, n, l, 17, 1)
    Q, Z, info = rmge.lowrank(kind, dev(A), H, l)
    assert int(host(info)[0]) == 0
    Qo, Zo = orc.lowrank(KIND[kind], A, oracle_H(kind, H, n), l)
    Q, Z = host(Q), host(Z)
    B = A @ orc.lowrank_multiplier_dense(KIND[kind], n, l, oracle_H(kind, H, n))
    kappa = np.linalg.cond(B)
    assert np.max(np.abs(Q.T @ Q - np.eye(l))) <= 100 * m * U64
    assert np.max(np.abs(Q - Qo)) <= 100 * kappa * np.sqrt(m) * U64
    assert np.max(np.abs(Z - Zo)) <= 100 * kappa * np.sqrt(m) * U64 * np.max(np.abs(A)) * np.sqrt(m)


@pytest.mark.parametrize("kind", ["gaussian", "circulant_uniform", "circulant_unitary"])
@pytest.mark.parametrize("n,r", [(256, 8), (1024, 32)])
def test_paper_residual_levels(orc, kind, n, r):
    """Sec. 7.2's test matrices (sigma_j = 1/j for j <= r, 1e-10 beyond), l = r: the GPU's rn1 and rn2 equal
    the oracle's for the same H (to the data's conditioning) and stay at the paper's levels (1e-9 .. 1e-4,
    against ||A|| = 1)."""
    A, Sr = W.lowrank_test_matrix(n, r, 77 + n + r)
    H = rmge.lowrank_multiplier(kind, n, r, 5, 1)
    Q, Z, info = rmge.lowrank(kind, dev(A), H, r)
    assert int(host(info)[0]) == 0
    Q, Z = host(Q), host(Z)
    rn1 = np.linalg.norm(Q @ (Q.T @ Sr) - Sr, 2)
    rn2 = np.linalg.norm(A - Q @ Z, 2)
    Qo, Zo = orc.lowrank(KIND[kind], A, oracle_H(kind, H, n), r)
    rn1o = np.linalg.norm(Qo @ (Qo.T @ Sr) - Sr, 2)
    rn2o = np.linalg.norm(A - Qo @ Zo, 2)
    assert rn1 <= 1e-4 and rn2 <= 1e-4
    assert abs(rn1 - rn1o) <= 0.1 * rn1o + 1e-12
    assert abs(rn2 - rn2o) <= 0.1 * rn2o + 1e-12


@pytest.mark.parametrize("kind", list(KIND))
def test_exact_on_exactly_low_rank_input(orc, kind):
    n, r = 2048, 16
    g = W.rng(9 + KIND[kind])
    A = g.standard_normal((n, r)) @ g.standard_normal((r, n))
    H = rmge.lowrank_multiplier(kind, n, r, 3, 1)
    Q, Z, info = rmge.lowrank(kind, dev(A), H, r)
    assert int(host(info)[0]) == 0
    assert np.linalg.norm(A - host(Q) @ host(Z), 2) <= 1e-10 * np.linalg.norm(A, 2)


def test_rank_deficient_basis_is_reported(orc):
    """l above the rank: the Gram matrix of A H is singular and the Cholesky reports the first deficient column."""
    n, r, l = 512, 3, 8
    g = W.rng(4)
    A = g.standard_normal((n, r)) @ g.standard_normal((r, n))
    H = rmge.lowrank_multiplier("gaussian", n, l, 3, 1)
    _, _, info = rmge.lowrank("gaussian", dev(A), H, l)
    assert int(host(info)[0]) == r + 1


def test_invalid_requests_are_refused():
    lib = rmge.load_library()
    assert lib.rmge_lowrank_workspace_size(0, 100, 100, 65) == 0    # l above 64
    assert lib.rmge_lowrank_workspace_size(0, 10, 100, 16) == 0     # l above m
    assert lib.rmge_lowrank_workspace_size(1, 100, 1000, 8) == 0    # circulant n not a power of two
    assert lib.rmge_lowrank_workspace_size(1, 100, 1024, 8) > 0
