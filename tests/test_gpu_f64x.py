"""The FP64 products emulated on the BF16 tensor cores (RMGE_F64X_TC): exactness on integer inputs, accuracy
on random FP64 inputs, the GENP factors it produces, and the whole solve at the FP64 target."""
import os

import numpy as np
import pytest
import torch

from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


@pytest.mark.parametrize("n", [5, 128, 200, 1100, 3000, 4096])
def test_emulated_product_is_exact_on_small_integers(orc, n):
    """Entries below 128 in magnitude are a single balanced base-256 digit, and 1024-deep chunks of their
    products stay within 2^24: every step is exact, so the product must equal the integer product bit for bit
    (n = 1100 spans two K chunks; n = 3000 and 4096 span several bands of 12 row blocks of 128, a ragged last
    band, and three and four 1024-deep K super-chunks, as at the bench sizes)."""
    r = W.rng(n)
    A = r.integers(-127, 128, (n, n)).astype(np.float64)
    G = r.integers(-127, 128, (n, n)).astype(np.float64)
    M = host(rmge.apply_multiplier("gaussian", dev(A), dev(G), "f64x"))
    # every partial sum is an integer below 127^2 n < 2^53, so the FP64 product is exact in any order
    ref = A @ G
    assert np.array_equal(M, ref)


@pytest.mark.parametrize("n", [64, 300, 1500, 3000, 4096])
def test_emulated_product_accuracy(orc, n):
    orc.set_threads(os.cpu_count() or 1)  # the oracle's product is the same in any thread count
    A, _ = W.orthogonal_factor_system(n, 1, 1e-6, seed=n)
    G = W.gaussian_multiplier(n, n + 1)
    M = host(rmge.apply_multiplier("gaussian", dev(A), dev(G), "f64x"))
    ref = orc.matmul(A, G)
    # 7 balanced base-256 digits (55 bits) and the 28 pairs of the diagonals p + q <= 6: about 12 2^-56 of
    # the row / column maxima per term (a safety factor of 2^5 on top)
    bound = 8 * n * 2.0**-49 * np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(G), axis=0)[None, :]
    assert np.all(np.abs(M - ref) <= bound), float(np.max(np.abs(M - ref) / bound))


@pytest.mark.parametrize("n", [65, 257, 700, 2048])
def test_emulated_factor_backward_error(orc, n):
    A, _ = W.gaussian_system(n, 1, seed=90 + n)
    G = W.gaussian_multiplier(n, 91 + n)
    M = orc.matmul(A, G)
    Md = dev(M)
    info, growth = rmge.factor(Md, "f64x")
    LU = host(Md)
    assert int(host(info)[0]) == 0
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    be = np.max(np.abs(L @ U - M)) / np.max(np.abs(L) @ np.abs(U))
    assert be <= 1e-13, be
    ref, _ = orc.genp(M)
    g = orc.growth(M, ref)
    # blocked factorizations differ from the unblocked oracle by rounding amplified by growth (Sec. 3: the
    # same Schur complements in exact arithmetic only); the native FP64 blocked factorization of the same
    # M sets that scale
    Md64 = dev(M)
    rmge.factor(Md64, "f64")
    e64 = np.max(np.abs(host(Md64) - ref)) / np.max(np.abs(ref))
    err = np.max(np.abs(LU - ref)) / np.max(np.abs(ref))
    assert err <= 64 * e64 + 1e-15, (err, e64)
    assert abs(float(host(growth)[0]) - g) <= 2 * err * np.max(np.abs(ref)) / np.max(np.abs(M)) + 1e-12 * g


def test_emulated_factor_matches_oracle_at_bench_size(orc):
    """n = 4096, the bench's size: 64 pivot-block steps whose Schur updates run on the emulated path over many
    row bands, against the oracle's unblocked GENP of the same M (Sec. 3: every blocking reaches the same
    Schur complements), entry by entry to rounding x growth, plus the factor backward error."""
    orc.set_threads(os.cpu_count() or 1)
    n = 4096
    A, _ = W.gaussian_system(n, 1, seed=4096 + 90)
    G = W.gaussian_multiplier(n, 4096 + 91)
    M = orc.matmul(A, G)
    Md = dev(M)
    info, growth = rmge.factor(Md, "f64x")
    LU = host(Md)
    ref, rinfo = orc.genp(M.copy())
    assert int(host(info)[0]) == rinfo == 0
    # the native FP64 blocked factorization of the same M sets the scale of rounding-order differences: with
    # growth near 1e5 here, the late Schur complements differ from the unblocked oracle's by far more than u
    Md64 = dev(M)
    info64, growth64 = rmge.factor(Md64, "f64")
    LU64 = host(Md64)
    e64 = np.max(np.abs(LU64 - ref)) / np.max(np.abs(ref))
    err = np.max(np.abs(LU - ref)) / np.max(np.abs(ref))
    assert err <= 64 * e64 + 1e-15, (err, e64)
    g = orc.growth(M, ref)
    for gg, e in ((float(host(growth)[0]), err), (float(host(growth64)[0]), e64)):
        assert abs(gg - g) <= 2 * e * np.max(np.abs(ref)) / np.max(np.abs(M)) + 1e-12 * g
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    be = np.max(np.abs(L @ U - M)) / np.max(np.abs(L) @ np.abs(U))
    assert be <= 1e-13, be


@pytest.mark.parametrize("n", [4352, 4200])
def test_paired_pivot_steps_match_oracle(orc, n):
    """n = 4352: the first pivot steps go in pairs (a thin update of the next block column and row that
    factors the next pivot block, the next panel, then one 128-deep update of the rest by both steps),
    the rest one by one (the trailing matrix falls below 4096 rows).  n = 4200: one pair, whose 128-deep
    update covers a 4072 x 4072 trailing matrix, a ragged edge of 104 rows and 40 columns in its last
    tiles.  Against the oracle's unblocked GENP, on the native FP64 yardstick as at the bench size, and a
    single system of a uniform batch gets the same bits as the system alone."""
    orc.set_threads(os.cpu_count() or 1)
    A, _ = W.gaussian_system(n, 1, seed=n + 90)
    G = W.gaussian_multiplier(n, n + 91)
    M = orc.matmul(A, G)
    Md = dev(M)
    info, growth = rmge.factor(Md, "f64x")
    LU = host(Md)
    ref, rinfo = orc.genp(M.copy())
    assert int(host(info)[0]) == rinfo == 0
    Md64 = dev(M)
    rmge.factor(Md64, "f64")
    e64 = np.max(np.abs(host(Md64) - ref)) / np.max(np.abs(ref))
    err = np.max(np.abs(LU - ref)) / np.max(np.abs(ref))
    assert err <= 64 * e64 + 1e-15, (err, e64)
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    be = np.max(np.abs(L @ U - M)) / np.max(np.abs(L) @ np.abs(U))
    assert be <= 1e-13, be
    Mb = torch.stack([dev(M), dev(M)])
    infob, _ = rmge.factor_batched(Mb, "f64x")
    assert np.all(host(infob) == 0)
    assert np.array_equal(host(Mb)[1], LU)


@pytest.mark.parametrize("n,digits", [(4224, 4), (4224, 7), (4200, 6)])
def test_paired_pivot_steps_exact_on_integer_factors(orc, n, digits):
    """Integer L and U of a few bits at n = 4224 and 4200 (a ragged 4072 x 4072 paired update), so that the
    paired 128-deep updates run: every intermediate is an integer the digits hold exactly, so the factors
    come back bit for bit."""
    r = W.rng(5000 + digits)
    L = np.tril(r.integers(-1, 2, (n, n)), -1).astype(np.float64) + np.eye(n)
    L[:, :] *= (np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]) < 24)  # banded: small integers
    L[np.diag_indices(n)] = 1.0
    U = np.triu(r.integers(-1, 2, (n, n)), 1).astype(np.float64)
    U *= (np.abs(np.arange(n)[:, None] - np.arange(n)[None, :]) < 24)
    U += np.diag(r.choice([-1.0, 1.0], n))
    M0 = L @ U
    assert np.max(np.abs(M0)) < 2.0**20
    M = dev(M0)
    info, _, _ = rmge.factor_ex(M, "f64x", rmge.options(factor_digits=digits))
    LU = host(M)
    assert int(host(info)[0]) == 0
    assert np.array_equal(np.tril(LU, -1), np.tril(L, -1))
    assert np.array_equal(np.triu(LU), U)


def _coupled(n, i):
    """Identity with a 2 x 2 block of ones at rows / columns i, i + 1: pivot i + 1 (1-based) is 1 and the
    Schur update leaves exactly 1 - 1 = 0 at step i + 2."""
    M = np.eye(n)
    M[i:i + 2, i:i + 2] = 1.0
    return M


@pytest.mark.parametrize("n,step", [(200, 70), (130, 64), (130, 65), (300, 300), (512, 200), (1000, 777)])
def test_emulated_breakdown_steps(orc, n, step):
    """Cor. 3.1 on the emulated path, where every pivot block after the first is factored inside the
    previous step's update launch: info is the first zero pivot, also one that the update itself creates
    across a block edge (rows 127 / 128) and inside a block."""
    M = np.eye(n)
    M[step - 1, step - 1] = 0.0
    info, growth = rmge.factor(dev(M), "f64x")
    assert int(host(info)[0]) == step == orc.genp(M)[1]
    assert np.isnan(host(growth)[0])
    for i in (126, 127, 99):
        if i + 2 <= n:
            C = _coupled(n, i)
            info, _ = rmge.factor(dev(C), "f64x")
            assert int(host(info)[0]) == i + 2 == orc.genp(C)[1]


def test_emulated_breakdown_non_finite():
    M = np.eye(150)
    M[100, 100] = np.nan
    info, _ = rmge.factor(dev(M), "f64x")
    assert int(host(info)[0]) == 101


@pytest.mark.parametrize("n,k", [(256, 1), (1000, 16)])
def test_emulated_solve_reaches_fp64_target(orc, n, k):
    A, B = W.orthogonal_factor_system(n, k, 1e-6, seed=300 + n)
    out = rmge.gesv("gaussian", dev(A), dev(B), seed=5, prec="f64x", max_iters=10, be_tol=1e-13)
    assert int(host(out["info"])[0]) == 0
    it = int(host(out["iters"])[0])
    assert it <= 3, it
    assert orc.backward_error(A, host(out["X"]), B) <= 1e-13


@pytest.mark.parametrize("digits", [2, 4, 6])
def test_emulated_product_with_fewer_digits(orc, digits):
    """apply_digits = d keeps d balanced base-256 digits of every entry (8 d - 1 bits) and the d (d + 1) / 2
    digit pairs with p + q < d: each term then errs by at most about (d + 5) 2^(-8 d) of the row and column
    maxima, and the error really is that of d digits (far above the 7-digit product's)."""
    n = 512
    A, _ = W.orthogonal_factor_system(n, 1, 1e-6, seed=n + digits)
    G = W.gaussian_multiplier(n, n + 2)
    M = host(rmge.apply_multiplier_ex("gaussian", dev(A), dev(G), "f64x", rmge.options(apply_digits=digits)))
    ref = orc.matmul(A, G)
    scale = np.max(np.abs(A), axis=1)[:, None] * np.max(np.abs(G), axis=0)[None, :]
    err = np.abs(M - ref) / scale
    assert np.all(err <= 2 * (digits + 5) * n * 2.0**(-8 * digits)), float(np.max(err))
    assert np.max(err) >= 2.0**(-8 * digits - 16)
    # integers below 128 are one digit: exact for every d
    r = W.rng(digits)
    Ai = r.integers(-127, 128, (n, n)).astype(np.float64)
    Gi = r.integers(-127, 128, (n, n)).astype(np.float64)
    Mi = host(rmge.apply_multiplier_ex("gaussian", dev(Ai), dev(Gi), "f64x", rmge.options(apply_digits=digits)))
    assert np.array_equal(Mi, Ai @ Gi)


@pytest.mark.parametrize("digits", [5, 6])
def test_fewer_digit_product_is_won_back_by_refinement(orc, digits):
    """M = A G from 5 or 6 digits (39 or 47 bits), the factorization and the FP64 refinement unchanged: the
    solve still meets the FP64 target (the precision workload's matrices, sigma down to 1e-4)."""
    n, k = 2048, 8
    A, B = W.orthogonal_factor_system(n, k, 1e-4, seed=2048 + digits)
    Ad, Bd = dev(A), dev(B)
    opts = rmge.options(apply_digits=digits)
    ws = rmge.workspace_ex(n, k, "gaussian", "f64x", opts)
    G = rmge.make_multiplier("gaussian", n, seed=31, subsequence=1, prec="f64x")
    M = rmge.apply_multiplier_ex("gaussian", Ad, G, "f64x", opts, ws=ws)
    info, _ = rmge.factor(M, "f64x", ws=ws)
    X = rmge.solve("gaussian", M, G, Bd, "f64x", ws=ws)
    berr, iters, _ = rmge.refine_ex("gaussian", Ad, M, G, Bd, X, "f64x", 10, 1e-13, opts, ws=ws)
    assert int(host(info)[0]) == 0
    it = int(host(iters)[0])
    assert it <= 6, it
    assert orc.backward_error(A, host(X), B) <= 1e-13


@pytest.mark.parametrize("digits", [4, 5, 6, 7])
def test_factor_digits_exact_on_integer_factors(orc, digits):
    """M = L U with small-integer L (unit lower) and U (unit-modulus diagonal): GENP's multipliers, panels and
    Schur complements are all integers of a few bits, which any digit count represents exactly, so the
    factors come back exactly (the fixed-point sums, the per-k balancing and the digit split lose nothing)."""
    n = 320
    r = W.rng(4000 + digits)
    L = np.tril(r.integers(-2, 3, (n, n)), -1).astype(np.float64) + np.eye(n)
    U = np.triu(r.integers(-2, 3, (n, n)), 1).astype(np.float64) + np.diag(r.choice([-1.0, 1.0], n))
    M0 = L @ U
    assert np.max(np.abs(M0)) < 2.0**20
    M = dev(M0)
    info, growth, _ = rmge.factor_ex(M, "f64x", rmge.options(factor_digits=digits))
    LU = host(M)
    assert int(host(info)[0]) == 0
    assert np.array_equal(np.tril(LU, -1), np.tril(L, -1))
    assert np.array_equal(np.triu(LU), U)


@pytest.mark.parametrize("digits", [5, 6])
def test_fewer_factor_digits_are_won_back_by_refinement(orc, digits):
    """Schur updates from 5 or 6 digits (factors of about 39 or 47 bits), A G from the same digits: the FP64
    refinement still takes the precision workload's matrices (sigma down to 1e-4) to the FP64 target."""
    n, k = 2048, 8
    A, B = W.orthogonal_factor_system(n, k, 1e-4, seed=2148 + digits)
    Ad, Bd = dev(A), dev(B)
    opts = rmge.options(apply_digits=digits, factor_digits=digits)
    ws = rmge.workspace_ex(n, k, "gaussian", "f64x", opts)
    G = rmge.make_multiplier("gaussian", n, seed=33, subsequence=1, prec="f64x")
    M7 = rmge.apply_multiplier("gaussian", Ad, G, "f64x")
    _, g7 = rmge.factor(M7, "f64x")
    M = rmge.apply_multiplier_ex("gaussian", Ad, G, "f64x", opts, ws=ws)
    info, growth, _ = rmge.factor_ex(M, "f64x", opts, ws=ws)
    assert int(host(info)[0]) == 0
    g = float(host(growth)[0])
    # the factors really are those of fewer digits (GENP without pivoting amplifies the difference by the
    # conditioning of the leading blocks: the factors move far more than their backward error)
    d = np.max(np.abs(host(M) - host(M7))) / np.max(np.abs(host(M7)))
    assert d >= 2.0**(-8 * digits - 16), (d, g, float(host(g7)[0]))
    X = rmge.solve("gaussian", M, G, Bd, "f64x", ws=ws)
    berr, iters, _ = rmge.refine_ex("gaussian", Ad, M, G, Bd, X, "f64x", 10, 1e-13, opts, ws=ws)
    it = int(host(iters)[0])
    assert it <= 8, it
    assert orc.backward_error(A, host(X), B) <= 1e-13


def _update_launches(n):
    """(M, N, K) of each emulated Schur-update launch of an n x n factorization, by launch class: pivot blocks
    of 64 (Sec. 3), steps paired while the trailing matrix has at least 4096 rows (two thin strips of 64-deep
    updates, then one 128-deep update of the rest), the others one 64-deep update each."""
    u128, u64 = [], []
    k, step = 0, 0
    while k < n:
        b = min(64, n - k)
        rest = n - k - b
        if rest <= 0:
            break
        if step % 2 != 0 or rest < 4096:
            u64.append((rest, rest, b))
            k, step = k + b, step + 1
            continue
        u64 += [(rest, 64, b), (64, rest - 64, b)]
        u128.append((rest - 64, rest - 64, 128))
        k, step = k + 128, step + 2
    return u128, u64


def test_launch_timing_records_the_schur_updates():
    """rmge_launch_timing: one event pair per update launch, with its digit-pair MMA work; nothing once
    stopped, nothing from a launch captured into a CUDA graph."""
    n, d = 4352, 6
    A, _ = W.gaussian_system(n, 1, seed=4352 + 92)
    opts = rmge.options(factor_digits=d)
    rmge.launch_timing(True)
    info, _, _ = rmge.factor_ex(dev(A), "f64x", opts)
    n128, ms128, fl128 = rmge.launch_timing_read(rmge.TIMED_UPDATE128)
    n64, ms64, fl64 = rmge.launch_timing_read(rmge.TIMED_UPDATE)
    assert int(host(info)[0]) == 0
    u128, u64 = _update_launches(n)
    pairs = d * (d + 1) // 2
    assert (n128, n64) == (len(u128), len(u64)) == (2, 67)
    assert fl128 == sum(pairs * 2.0 * m * nn * kk for m, nn, kk in u128)
    assert fl64 == sum(pairs * 2.0 * m * nn * kk for m, nn, kk in u64)
    assert ms128 > 0 and ms64 > 0
    rmge.launch_timing(False)
    rmge.factor_ex(dev(A), "f64x", opts)
    assert rmge.launch_timing_read(rmge.TIMED_UPDATE128) == (n128, ms128, fl128)
    # a launch on a stream under graph capture records nothing
    Mc = dev(A)
    ws = rmge.workspace_ex(n, 1, "gaussian", "f64x", opts)
    rmge.factor_ex(Mc, "f64x", opts, ws=ws)
    torch.cuda.synchronize()
    rmge.launch_timing(True)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rmge.factor_ex(Mc, "f64x", opts, ws=ws)
    g.replay()
    torch.cuda.synchronize()
    assert rmge.launch_timing_read(rmge.TIMED_UPDATE128)[0] == 0
    assert rmge.launch_timing_read(rmge.TIMED_UPDATE)[0] == 0
    rmge.launch_timing(False)
