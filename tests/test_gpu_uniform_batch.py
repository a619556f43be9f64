"""Uniform batches: many systems of one order factored with one launch per kernel and pivot-block step
(rmge_apply_multiplier_batched, rmge_factor_batched; emulated FP64).  Every system's result must be the one
the single-system calls give, bit for bit (the same kernels and arithmetic, only the system index differs),
a breakdown in one system must leave the others untouched, and the batched autograd path must give the
oracle's solution and gradients."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W
from paper_1406_5802_gb300.autograd import rmge_solve_batched

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


@pytest.mark.parametrize("count,n", [(3, 300), (2, 1000), (5, 64), (4, 129)])
def test_batched_apply_and_factor_equal_single_calls(orc, count, n):
    As = [W.orthogonal_factor_system(n, 1, 1e-4, seed=900 + 7 * i + n)[0] for i in range(count)]
    A = dev(np.stack(As))
    G = torch.stack([rmge.make_multiplier("gaussian", n, seed=40 + i, subsequence=1, prec="f64x")
                     for i in range(count)])
    ws = rmge.uniform_workspace(count, n, "f64x")
    M = rmge.apply_multiplier_batched(A, G, "f64x", ws=ws)
    Mh = host(M).copy()
    info, growth = rmge.factor_batched(M, "f64x", ws=ws)
    LU, info, growth = host(M), host(info), host(growth)
    for i in range(count):
        Mi = rmge.apply_multiplier("gaussian", A[i].contiguous(), G[i].contiguous(), "f64x")
        assert np.array_equal(host(Mi), Mh[i]), i
        inf1, g1 = rmge.factor(Mi, "f64x")
        assert np.array_equal(host(Mi), LU[i]), i
        assert int(host(inf1)[0]) == int(info[i]) == 0
        assert float(host(g1)[0]) == float(growth[i])
    # the factors are those of GENP: reconstruction to FP64 accuracy
    L = np.tril(LU[0], -1) + np.eye(n)
    U = np.triu(LU[0])
    assert np.max(np.abs(L @ U - Mh[0])) <= 1e-13 * np.max(np.abs(L) @ np.abs(U))


def test_breakdown_of_one_system_leaves_the_others(orc):
    """System 1 has a zero pivot at step 70 (Cor. 3.1): info[1] = 70 while the others factor as alone."""
    n, count = 200, 3
    r = W.rng(5)
    Ms = [r.standard_normal((n, n)) + n * np.eye(n) for _ in range(count)]
    Ms[1] = np.eye(n)
    Ms[1][69, 69] = 0.0
    M = dev(np.stack(Ms))
    info, growth = rmge.factor_batched(M, "f64x")
    info = host(info)
    assert list(info) == [0, 70, 0]
    LU = host(M)
    for i in (0, 2):
        Mi = dev(Ms[i])
        rmge.factor(Mi, "f64x")
        assert np.array_equal(host(Mi), LU[i])
    assert np.isnan(host(growth)[1])


def test_batched_factors_solve_to_fp64_target(orc):
    n, k, count = 512, 4, 4
    systems = [W.orthogonal_factor_system(n, k, 1e-6, seed=1200 + i) for i in range(count)]
    A = dev(np.stack([a for a, _ in systems]))
    G = torch.stack([rmge.make_multiplier("gaussian", n, seed=70 + i, subsequence=1, prec="f64x")
                     for i in range(count)])
    M = rmge.apply_multiplier_batched(A, G, "f64x")
    info, _ = rmge.factor_batched(M, "f64x")
    assert np.all(host(info) == 0)
    for i, (a, b) in enumerate(systems):
        X = rmge.solve("gaussian", M[i], G[i], dev(b), "f64x")
        berr, it = rmge.refine("gaussian", A[i], M[i], G[i], dev(b), X, "f64x", 10, 1e-13)
        assert orc.backward_error(a, host(X), b) <= 1e-13


@pytest.mark.parametrize("digits", [(7, 7), (5, 7)])
def test_uniform_autograd_matches_oracle_gradient(orc, digits):
    """The gradient workload's matrices through the uniform batched autograd node (emulated products, all 7
    digits or A G from 5): X and the gradients of sum(X * W) against the oracle's GEPP solution and
    GEPP-based adjoint."""
    n, k, count = 256, 4, 5
    systems = [W.grad_system(n, k, seed=800 + i) for i in range(count)]
    As = [torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=True) for a, _, _ in systems]
    Bs = [torch.tensor(b, dtype=torch.float64, device="cuda", requires_grad=True) for _, b, _ in systems]
    Xs = rmge_solve_batched(As, Bs, seeds=list(range(count)), prec="f64x", streams=3, max_iters=4, digits=digits)
    loss = sum((X * torch.tensor(w, device="cuda")).sum() for X, (_, _, w) in zip(Xs, systems))
    loss.backward()
    torch.cuda.synchronize()
    for i, (a, b, w) in enumerate(systems):
        ref = orc.gepp_solve(*orc.gepp(a)[:2], b)
        assert np.max(np.abs(host(Xs[i]) - ref)) <= 1e-10 * np.max(np.abs(ref))
        rdB, rdA, rinfo = orc.solve_adjoint_gepp(a, ref, w)
        assert rinfo == 0
        assert np.max(np.abs(host(Bs[i].grad) - rdB)) <= 1e-10 * np.max(np.abs(rdB))
        assert np.max(np.abs(host(As[i].grad) - rdA)) <= 1e-10 * np.max(np.abs(rdA))


@pytest.mark.parametrize("count,n,k", [(3, 300, 4), (2, 129, 1), (4, 64, 9)])
def test_batched_solve_refine_adjoint_equal_single_calls(orc, count, n, k):
    """rmge_solve_uniform_batched, rmge_refine_uniform_batched and rmge_solve_backward_uniform_batched give,
    system by system, the bits of rmge_solve, rmge_refine and rmge_solve_backward (the same kernels; only
    the system index differs), including each system's own sweep count."""
    systems = [W.orthogonal_factor_system(n, k, 10.0 ** -(2 + 2 * i), seed=1500 + i + n) for i in range(count)]
    A = dev(np.stack([a for a, _ in systems]))
    B = dev(np.stack([b for _, b in systems]))
    G = torch.stack([rmge.make_multiplier("gaussian", n, seed=90 + i, subsequence=1, prec="f64x")
                     for i in range(count)])
    M = rmge.apply_multiplier_batched(A, G, "f64x")
    info, _ = rmge.factor_batched(M, "f64x")
    assert np.all(host(info) == 0)
    X = rmge.solve_uniform_batched(M, G, B, "f64x")
    X0 = host(X).copy()
    berr, iters = rmge.refine_uniform_batched(A, M, G, B, X, "f64x", 10, 1e-13)
    dX = dev(W.rng(3).standard_normal((count, n, k)))
    dB, dA, berr_b, iters_b = rmge.solve_backward_uniform_batched(A, M, G, X, dX, "f64x", max_iters=6)
    Xh, berr, iters = host(X), host(berr), host(iters)
    dBh, dAh, berr_b, iters_b = host(dB), host(dA), host(berr_b), host(iters_b)
    for i in range(count):
        Xi = rmge.solve("gaussian", M[i], G[i], B[i], "f64x")
        assert np.array_equal(host(Xi), X0[i]), i
        be1, it1 = rmge.refine("gaussian", A[i], M[i], G[i], B[i], Xi, "f64x", 10, 1e-13)
        assert np.array_equal(host(Xi), Xh[i]), i
        assert int(host(it1).reshape(-1)[0]) == int(iters[i])
        assert np.array_equal(host(be1)[: int(iters[i]) + 1], berr[i][: int(iters[i]) + 1])
        assert berr[i][int(iters[i])] <= 1e-13
        dB1, dA1, bb1, ib1 = rmge.solve_backward("gaussian", M[i], G[i], Xi, dX[i], "f64x", want_dA=True, A=A[i],
                                                 max_iters=6)
        assert np.array_equal(host(dB1), dBh[i]), i
        assert np.array_equal(host(dA1), dAh[i]), i
        assert int(host(ib1).reshape(-1)[0]) == int(iters_b[i])
        # the adjoint of the oracle: A^T dB = dX
        a = systems[i][0]
        assert orc.backward_error(a.T.copy(), dBh[i], host(dX[i])) <= 1e-13


def test_batched_solve_rejects_reduced_precision_and_bad_strides():
    count, n, k = 2, 64, 2
    LU = torch.zeros(count, n, n, dtype=torch.float64, device="cuda")
    G = torch.zeros(count, n, n, dtype=torch.float64, device="cuda")
    B = torch.zeros(count, n, k, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        rmge.solve_uniform_batched(LU, G, B, "f32", ws=rmge.uniform_solve_workspace(count, n, k, "f64"))
    with pytest.raises(RuntimeError):
        rmge.solve_uniform_batched(LU[:, :, :32].contiguous(), G, B, "f64")  # ldlu < n
