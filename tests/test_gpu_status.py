"""Failure detection through the C ABI, with no GPU fault: the status word of the options, the growth gate
(Thm 3.2 bounds the pivots of GENP on a Gaussian-multiplied matrix; Remark 3.2 ties GENP's stability to
pivot growth), non-finite results, refinement that stops above its target, and bounded device waits made to
run out by a spin limit of 0 -- the triangular solves' flag chain and the batched solve's shared fallback
product, neither of which has a tensor-core copy or MMA in flight -- after which the next call on the same
stream and workspace is clean."""
import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W
from paper_1406_5802_gb300.batch import BatchedSolver

pytestmark = pytest.mark.gpu

OK, BREAKDOWN, GROWTH, NOT_CONVERGED, TIMEOUT, NONFINITE = 0, 2, 3, 4, 6, 9


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def status_word():
    return torch.full((1,), -1, dtype=torch.int32, device="cuda")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


def test_growth_gate_unmultiplied_vs_multiplied(orc):
    """The batched workload's reading: A with A[0,0] scaled by 1e-10 is not a breakdown for unmultiplied GENP
    (Cor. 3.1 needs an exact zero), but its growth is about 1e10 and the unrefined solve fails the target;
    with the Gaussian multiplier the same A passes the gate and the target."""
    n, k = 256, 1
    A, B = W.gaussian_system(n, k, seed=W.SEED_BASE + 40)
    A[0, 0] *= 1e-10
    st = status_word()
    M = dev(A)
    info, growth, code = rmge.factor_ex(M, "f64", rmge.options(growth_tol=1e8, status=st))
    assert code == OK  # enqueued; the outcome is in the status word
    assert int(host(info)[0]) == 0
    g = float(host(growth)[0])
    LU_ref, rinfo = orc.genp(A)
    assert rinfo == 0
    g_ref = orc.growth(A, LU_ref)
    assert g > 1e8 and abs(g - g_ref) <= 1e-6 * g_ref
    assert int(host(st)[0]) == GROWTH
    # the synchronising form returns the outcome
    _, _, code = rmge.factor_ex(dev(A), "f64", rmge.options(growth_tol=1e8, sync=True))
    assert code == GROWTH
    # unrefined solve with these factors (G = I): the backward error is far above the target
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    X = rmge.solve("gaussian", M, eye, dev(B), "f64")
    assert orc.backward_error(A, host(X), B) > 1e-9
    # refinement capped at zero sweeps reports that it stopped above be_tol
    st2 = status_word()
    Xr = rmge.solve("gaussian", M, eye, dev(B), "f64")
    _, _, code = rmge.refine_ex("gaussian", dev(A), M, eye, dev(B), Xr, "f64", 0, 1e-13, rmge.options(status=st2))
    assert code == OK and int(host(st2)[0]) == NOT_CONVERGED
    # the multiplied matrix passes the same gate, and the solve meets the target
    G = rmge.make_multiplier("gaussian", n, seed=9, subsequence=1, prec="f64")
    Mg = rmge.apply_multiplier("gaussian", dev(A), G, "f64")
    st3 = status_word()
    info, growth, _ = rmge.factor_ex(Mg, "f64", rmge.options(growth_tol=1e8, status=st3))
    assert int(host(info)[0]) == 0 and float(host(growth)[0]) < 1e8
    assert int(host(st3)[0]) == OK
    Xg = rmge.solve("gaussian", Mg, G, dev(B), "f64")
    st4 = status_word()
    berr, iters, _ = rmge.refine_ex("gaussian", dev(A), Mg, G, dev(B), Xg, "f64", 10, 1e-13, rmge.options(status=st4))
    assert int(host(st4)[0]) == OK
    assert orc.backward_error(A, host(Xg), B) <= 1e-13


def test_breakdown_and_nonfinite_results_are_reported(orc):
    """A zero leading pivot (Cor. 3.1) is a breakdown of the factorization; solving with those factors gives
    a non-finite X, which the solve and the refinement report."""
    n, k = 128, 2
    A, B = W.gaussian_system(n, k, seed=W.SEED_BASE + 41, zero_leading_pivot=True)
    M = dev(A)
    st = status_word()
    info, _, _ = rmge.factor_ex(M, "f64", rmge.options(status=st))
    assert int(host(info)[0]) == 1 and int(host(st)[0]) == BREAKDOWN
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    st2 = status_word()
    X, code = rmge.solve_ex("gaussian", M, eye, dev(B), "f64", rmge.options(status=st2))
    assert code == OK and int(host(st2)[0]) == NONFINITE
    assert not np.all(np.isfinite(host(X)))
    _, _, code = rmge.refine_ex("gaussian", dev(A), M, eye, dev(B), X, "f64", 3, 1e-13, rmge.options(sync=True))
    assert code == NONFINITE
    # a healthy solve through the same entry points reports OK
    out = rmge.gesv("gaussian", dev(A), dev(B), seed=3, prec="f64")
    st3 = status_word()
    X2, _ = rmge.solve_ex("gaussian", out["LU"], out["G"], dev(B), "f64", rmge.options(status=st3))
    assert int(host(st3)[0]) == OK and np.all(np.isfinite(host(X2)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_triangular_solve_wait_runs_out_then_next_call_is_clean(orc, prec):
    """Spin limit 0: a row block whose predecessor has not yet published gives up at its first poll, records
    RMGE_ERR_TIMEOUT and returns without writing; the CTAs behind it see the error and return too.  The
    next call on the same stream and workspace starts from a clean control block and solves correctly."""
    n, k = 4096, 16
    A, B = W.gaussian_system(n, k, seed=W.SEED_BASE + 42)
    out = rmge.gesv("gaussian", dev(A), dev(B), seed=5, prec=prec, max_iters=0, be_tol=0.0)
    LU, G = out["LU"], out["G"]
    Bd = dev(B)
    ws = rmge.workspace(n, k, "gaussian", prec)
    ref = host(rmge.solve("gaussian", LU, G, Bd, prec, ws=ws)).copy()
    st = status_word()
    _, code = rmge.solve_ex("gaussian", LU, G, Bd, prec, rmge.options(spin_limit=0, status=st), ws=ws)
    assert code == OK
    assert int(host(st)[0]) == TIMEOUT
    _, code = rmge.solve_ex("gaussian", LU, G, Bd, prec, rmge.options(spin_limit=0, sync=True), ws=ws)
    assert code == TIMEOUT
    for _ in range(2):
        X = rmge.solve("gaussian", LU, G, Bd, prec, ws=ws)
        assert np.array_equal(host(X), ref)
    st2 = status_word()
    X, _ = rmge.solve_ex("gaussian", LU, G, Bd, prec, rmge.options(status=st2), ws=ws)
    assert int(host(st2)[0]) == OK and np.array_equal(host(X), ref)


def test_batched_shared_product_wait_runs_out_then_next_launch_is_clean(orc):
    """Spin limit 0 in the batched solve.  System 0 (n = 512) holds a NaN, so every FP32 draw breaks down
    at once and it soon reaches the FP64 fallback, whose product it shares out as row blocks while the
    other CTAs are still busy with 20000 small systems and take blocks between two of them.  When the owner
    has done its own block and finds another still in a helper's hands, it gives up at its first poll: that
    system gets info -1 and the status RMGE_ERR_TIMEOUT, while every other system is still solved.  The next
    launch, with the default limit, solves every finite system and reports system 0's breakdown."""
    sizes = np.concatenate([[512], W.batch_sizes(20000, 128, 192, seed=W.SEED_BASE + 43)]).astype(np.int32)
    s = BatchedSolver.synthetic(sizes, seed=W.SEED_BASE + 43, leading_scale=1.0, max_sweeps=40, be_tol=1e-13)
    s.A[5 * 512 + 7] = float("nan")
    timed_out = False
    for _ in range(3):  # the outcome depends on a helper still holding a block at the owner's first poll
        st = status_word()
        s.x.zero_()
        code = s.launch(1, 3 * 152, opts=rmge.options(spin_limit=0, status=st))
        assert code == OK
        info = host(s.info)
        berr = host(s.berr)
        assert info[0] != 0  # the NaN system never succeeds
        assert np.all(berr[info == 0] <= 1e-13)
        if int(host(st)[0]) == TIMEOUT:
            assert np.sum(info == -1) == 1
            assert np.all((info[1:] == 0) | (info[1:] == -1))
            timed_out = True
            break
        assert int(host(st)[0]) == OK and np.all(info[1:] == 0)
    assert timed_out
    st = status_word()
    s.x.zero_()
    s.launch(1, 3 * 152, opts=rmge.options(status=st))
    info = host(s.info)
    assert int(host(st)[0]) == OK
    assert info[0] > 0 and np.all(info[1:] == 0)  # a breakdown for the NaN system, success for the rest
    assert np.all(host(s.berr)[1:] <= 1e-13)
    for i in (1, 9999, 20000):
        n = int(sizes[i])
        off = int(s.offA[i])
        Ai = host(s.A[off:off + n * n]).reshape(n, n)
        bi = host(s.b[int(s.offv[i]):int(s.offv[i]) + n]).reshape(n, 1)
        assert orc.backward_error(Ai, s.solution(i).cpu().numpy().reshape(-1, 1), bi) <= 1e-13
