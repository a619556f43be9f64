"""Parity of the reduced-precision paths (FP32 SIMT, tcgen05 BF16/FP16 tensor cores, plain and
three-pass split) against the FP64 oracle: M = A G, the GENP factors, and the whole solve."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0**-24
# unit roundoff of one product term per precision: plain BF16 / FP16 operands, or the two-term split
TERM_U = {"f32": U32, "bf16": 2.0**-9, "f16": 2.0**-12, "bf16x3": 2.0**-17, "f16x3": 2.0**-22}


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16", "bf16x3", "f16x3"])
@pytest.mark.parametrize("n", [64, 130, 300, 1000])
def test_apply_multiplier_reduced(orc, prec, n):
    A, _ = W.orthogonal_factor_system(n, 1, 1e-4, seed=n)
    Gd = rmge.make_multiplier("gaussian", n, seed=3, subsequence=1, prec=prec)
    G = host(Gd)
    M = host(rmge.apply_multiplier("gaussian", dev(A), Gd, prec))
    ref = orc.matmul(A, G)
    scale = np.abs(A) @ np.abs(G)
    # rounding of each operand to the term precision plus FP32 accumulation over n terms
    tol = (4 * TERM_U[prec] + 2 * n * U32) * scale
    assert np.all(np.abs(M - ref) <= tol), float(np.max(np.abs(M - ref) / scale))


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16", "bf16x3", "f16x3"])
@pytest.mark.parametrize("n", [64, 129, 300, 700])
def test_factor_reduced_matches_oracle(orc, prec, n):
    A, _ = W.gaussian_system(n, 1, seed=70 + n)
    G = W.gaussian_multiplier(n, 71 + n).astype(np.float32).astype(np.float64)
    M = orc.matmul(A, G).astype(np.float32).astype(np.float64)
    Md = dev(M, torch.float32)
    info, growth = rmge.factor(Md, prec)
    LU = host(Md)
    ref, rinfo = orc.genp(M)
    assert int(host(info)[0]) == rinfo == 0
    # the reported growth is max|U| / max|M| of the factors actually produced
    g_own = np.max(np.abs(np.triu(LU))) / np.max(np.abs(M))
    assert abs(float(host(growth)[0]) - g_own) <= 1e-6 * g_own
    # backward error of the factors: ||L U - M|| / (||L|| ||U||) at the working precision (FP32) or the
    # product-term precision, whichever is coarser
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    be = np.max(np.abs(L @ U - M)) / np.max(np.abs(np.abs(L) @ np.abs(U)))
    eps = 8 * max(TERM_U[prec], n * U32 / 8)
    assert be <= eps, be
    # forward error of the factors: to first order L^-1 dM U^-1 = L^-1 dL + dU U^-1 with |dM| <= eps |L||U|,
    # so |dL|, |dU| are bounded by eps || |L^-1||L||U||U^-1| || times the largest factor entry (the
    # conditioning of the leading minors, which GENP does not control)
    Lr = np.tril(ref, -1) + np.eye(n)
    Ur = np.triu(ref)
    kap = np.linalg.norm(np.abs(np.linalg.inv(Lr)) @ np.abs(Lr) @ np.abs(Ur) @ np.abs(np.linalg.inv(Ur)), np.inf)
    assert np.max(np.abs(LU - ref)) <= 10 * eps * kap * max(np.max(np.abs(Lr)), np.max(np.abs(Ur))) + 1e-300


@pytest.mark.parametrize("prec", ["f32", "bf16x3", "f16x3"])
@pytest.mark.parametrize("n,k,smin", [(256, 1, 1e-4), (256, 8, 1e-4), (512, 3, 1e-2)])
def test_mixed_solve_reaches_fp64_accuracy(orc, prec, n, k, smin):
    """Reduced-precision factors of A G, won back to the FP64 target by FP64 residuals and FGMRES sweeps,
    where growth x u_f x kappa(A G) leaves few outlying eigenvalues."""
    A, B = W.orthogonal_factor_system(n, k, smin, seed=900 + n)
    out = rmge.gesv("gaussian", dev(A), dev(B), seed=901, prec=prec, max_iters=40, be_tol=1e-13)
    X = host(out["X"])
    it = int(host(out["iters"])[0])
    berr = host(out["berr"])
    assert int(host(out["info"])[0]) == 0
    be = orc.backward_error(A, X, B)
    assert be <= 1e-13, (be, it, berr[: it + 1])
    assert berr[it] <= 1e-13


def test_reduced_precision_sweeps_start_classical(orc):
    """Where FP32 factors are accurate enough (growth x u_f x kappa(A G) < 1), the sweeps stay classical
    corrections: each at least halves the backward error (here by 20-40x) until the FP64 target, with
    no FGMRES cycle (the schedule switches only after a sweep that fails to halve it)."""
    n, k = 512, 4
    A, B = W.orthogonal_factor_system(n, k, 0.5, seed=55)
    out = rmge.gesv("gaussian", dev(A), dev(B), seed=56, prec="f32", max_iters=40, be_tol=1e-13)
    it = int(host(out["iters"])[0])
    berr = host(out["berr"])
    assert int(host(out["info"])[0]) == 0
    assert 1 <= it <= 12, (it, berr[: it + 1])
    assert np.all(berr[1: it + 1] <= 0.5 * berr[: it]), berr[: it + 1]
    assert orc.backward_error(A, host(out["X"]), B) <= 1e-13


def test_mixed_solve_reports_stagnation(orc):
    """Where FP32 factors are too inexact (GENP growth x u_f x kappa(A G) >> 1) the sweeps stop on the
    stagnation test with the backward error they reached, which the oracle confirms."""
    n, k = 1024, 2
    A, B = W.orthogonal_factor_system(n, k, 1e-4, seed=33)
    out = rmge.gesv("gaussian", dev(A), dev(B), seed=34, prec="f32", max_iters=40, be_tol=1e-13)
    it = int(host(out["iters"])[0])
    berr = host(out["berr"])
    assert 2 <= it < 40 and berr[it] > 1e-13
    assert not (berr[it] <= 0.5 * berr[it - 2])
    assert np.all(berr[it + 1:] == -1.0)
    be = orc.backward_error(A, host(out["X"]), B)
    assert abs(be - berr[it]) <= 0.5 * be


def test_plain_16bit_factors_refine_on_a_well_conditioned_system(orc):
    """Single-term FP16 trailing updates suffice when kappa(A G) u16 growth stays small."""
    n, k = 256, 2
    A, B = W.orthogonal_factor_system(n, k, 0.5, seed=77)
    out = rmge.gesv("gaussian", dev(A), dev(B), seed=78, prec="f16", max_iters=40, be_tol=1e-13)
    be = orc.backward_error(A, host(out["X"]), B)
    assert be <= 1e-13, (be, int(host(out["iters"])[0]))
