"""Differentiation through the randomized GENP solve: the autograd Function's gradients (adjoint kernels
reusing the factors of A G) against FP64 central finite differences and the oracle's gradient."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W
from paper_1406_5802_gb300.autograd import rmge_solve, rmge_solve_batched

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


def _grads(A, B, Wt, seed, prec, dtype, kind="gaussian"):
    Ad = torch.tensor(A, dtype=dtype, device="cuda", requires_grad=True)
    Bd = torch.tensor(B, dtype=dtype, device="cuda", requires_grad=True)
    X = rmge_solve(Ad, Bd, seed, kind=kind, prec=prec)
    loss = (X * torch.tensor(Wt, dtype=dtype, device="cuda")).sum()
    loss.backward()
    torch.cuda.synchronize()
    return Ad.grad.double().cpu().numpy(), Bd.grad.double().cpu().numpy(), X.detach().double().cpu().numpy()


@pytest.mark.parametrize("kind", ["gaussian", "circulant"])
def test_gradients_match_central_differences_fp64(orc, kind):
    """FP64, n = 16: dL/dA and dL/dB for L = sum(X * W) against central differences of the oracle's solve."""
    n, k = 16, 4
    A, B, Wt = W.grad_system(n, k, seed=W.SEED_BASE + 5)
    gA, gB, _ = _grads(A, B, Wt, seed=W.SEED_BASE + 5, prec="f64", dtype=torch.float64, kind=kind)

    def loss(A_, B_):
        LU, piv, _ = orc.gepp(A_)
        return float(np.sum(orc.gepp_solve(LU, piv, B_) * Wt))

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
    assert np.max(np.abs(gA - fdA)) <= 1e-6 * np.max(np.abs(fdA))
    assert np.max(np.abs(gB - fdB)) <= 1e-6 * np.max(np.abs(fdB))


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n,k", [(300, 4), (2048, 4)])
def test_gradients_match_oracle_gradient(orc, prec, n, k):
    """The gradient workload's matrices (A = 4I + N(0,1)/sqrt(n)): FP32 or FP64 factors, refined forward and
    adjoint solves, against the oracle's GEPP-based gradient."""
    A, B, Wt = W.grad_system(n, k, seed=W.SEED_BASE + 5 + n)
    dtype = torch.float32 if prec == "f32" else torch.float64
    A_in = A.astype(np.float32).astype(np.float64) if prec == "f32" else A
    B_in = B.astype(np.float32).astype(np.float64) if prec == "f32" else B
    W_in = Wt.astype(np.float32).astype(np.float64) if prec == "f32" else Wt
    gA, gB, X = _grads(A_in, B_in, W_in, seed=11, prec=prec, dtype=dtype)
    orc.set_threads(8)
    rdB, rdA, info = orc.solve_adjoint_gepp(A_in, orc.gepp_solve(*orc.gepp(A_in)[:2], B_in), W_in)
    assert info == 0
    tol = 1e-6 if prec == "f32" else 1e-10  # FP32 outputs: rounding of the FP64-accurate result
    assert np.max(np.abs(gB - rdB)) <= tol * np.max(np.abs(rdB))
    assert np.max(np.abs(gA - rdA)) <= tol * np.max(np.abs(rdA))


def test_batched_streams_match_single_solves(orc):
    n, k, count = 256, 4, 6
    systems = [W.grad_system(n, k, seed=700 + i) for i in range(count)]
    As = [torch.tensor(a, dtype=torch.float32, device="cuda", requires_grad=True) for a, _, _ in systems]
    Bs = [torch.tensor(b, dtype=torch.float32, device="cuda", requires_grad=True) for _, b, _ in systems]
    Xs = rmge_solve_batched(As, Bs, seeds=list(range(count)), prec="f32", streams=3)
    loss = sum((X * torch.tensor(w, dtype=torch.float32, device="cuda")).sum() for X, (_, _, w) in zip(Xs, systems))
    loss.backward()
    torch.cuda.synchronize()
    for i, (a, b, w) in enumerate(systems):
        ref = orc.gepp_solve(*orc.gepp(a.astype(np.float32).astype(np.float64))[:2], b.astype(np.float32))
        assert np.max(np.abs(Xs[i].detach().double().cpu().numpy() - ref)) <= 1e-6 * np.max(np.abs(ref))
        gA, gB, _ = _grads(a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64),
                           w.astype(np.float32).astype(np.float64), seed=i, prec="f32", dtype=torch.float32)
        assert np.max(np.abs(As[i].grad.double().cpu().numpy() - gA)) <= 1e-6 * np.max(np.abs(gA))
        assert np.max(np.abs(Bs[i].grad.double().cpu().numpy() - gB)) <= 1e-6 * np.max(np.abs(gB))
