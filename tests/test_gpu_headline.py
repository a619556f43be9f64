"""The precision workload at its full size, in the launch configuration the benchmark times: n = 16384,
8 right-hand sides, singular values log-spaced from 1 to 1e-4, G drawn on the device with the benchmark's
seeds and options.  The oracle cannot factor or solve a system this large in seconds, so it checks sampled
outputs one by one (entries of G from its own Philox stream, entries of M = A G as its own dot products,
rows and columns of L U against M) and the whole solution through its compensated backward error
(Sec. 7.1's target, 1e-13).  The sampled rows and columns include every tile edge the kernels have: the
128-row tiles, the 64-wide pivot blocks, the last paired pivot step (the trailing matrix falls below 4096
rows at step 12288) and the ragged end."""
import os

import numpy as np
import pytest
import torch

import bench
from paper_1406_5802_gb300 import ranks
from paper_1406_5802_gb300 import rmge
from paper_1406_5802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = 2.0**-53
N, K, SIGMA = bench.N3, bench.K3, bench.SIGMA3
SEED = ranks.system_seed(bench.SEED_BASE + 3, 0)
EDGES = [0, 1, 63, 64, 127, 128, 4095, 4096, 8191, 8192, 12223, 12287, 12288, 12352, N - 129, N - 128, N - 65,
         N - 64, N - 2, N - 1]


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def sample(count, seed):
    r = W.rng(seed)
    return np.unique(np.concatenate([np.array(EDGES), r.integers(0, N, count)]))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1406_5802_gb300 import build as B
    B.build()
    rmge.load_library()


@pytest.fixture(scope="module")
def system():
    A, B = W.orthogonal_factor_system_torch(N, K, SIGMA, seed=SEED, device="cuda")
    return A, B, host(A), host(B)


def staged_step(form, seed):
    """The benchmark's step (bench.Form.step) with its intermediate M and factors copied back."""
    r = rmge
    r.make_multiplier(form.kind, form.n, seed, 1, form.prec, G=form.G)
    G = host(form.G)
    r.apply_multiplier_ex(form.kind, form.A, form.G, form.prec, form.opts, M=form.M, ws=form.ws)
    M = host(form.M)
    info, growth, _ = r.factor_ex(form.M, form.prec, form.opts, ws=form.ws)
    LU = host(form.M)
    r.solve(form.kind, form.M, form.G, form.B, form.prec, X=form.X, ws=form.ws)
    berr, iters, _ = r.refine_ex(form.kind, form.A, form.M, form.G, form.B, form.X, form.prec, form.max_iters,
                                 bench.BE_TOL, form.opts, ws=form.ws)
    it = int(host(iters)[0])
    return dict(G=G, M=M, LU=LU, info=int(host(info)[0]), growth=float(host(growth)[0]), iters=it,
                berr=float(host(berr)[it]), X=host(form.X))


def factor_rows_cols(orc, LU, rows, cols):
    """Sampled rows and columns of L U and of |L| |U| (L unit lower, U upper, both packed in LU), each entry
    the oracle's plain dot product of a row of L with a column of U."""
    n = LU.shape[0]
    U = np.triu(LU)
    Lr = np.zeros((len(rows), n))
    for a, i in enumerate(rows):
        Lr[a, :i] = LU[i, :i]
        Lr[a, i] = 1.0
    LUr, absr = orc.matmul(Lr, U), orc.matmul(np.abs(Lr), np.abs(U))
    del U
    L = np.tril(LU, -1)
    L[np.diag_indices(n)] = 1.0
    Uc = np.zeros((n, len(cols)))
    for b, j in enumerate(cols):
        Uc[:j + 1, b] = LU[:j + 1, j]
    LUc, absc = orc.matmul(L, Uc), orc.matmul(np.abs(L), np.abs(Uc))
    return LUr, absr, LUc, absc


def check_multiplier(orc, G, seed):
    """The first 64 rows of G against the oracle's Philox4x32-10 + Box-Muller stream (Def. 4.1)."""
    ref = orc.gaussian(64 * N, seed, 1).reshape(64, N)
    assert np.max(np.abs(G[:64] - ref)) <= 8 * U64 * max(1.0, np.max(np.abs(ref)))
    # the whole draw: zero mean and unit variance to within a few standard errors of n^2 samples
    assert abs(G.mean()) <= 6.0 / N and abs(G.var() - 1.0) <= 6.0 * np.sqrt(2.0) / N


def test_headline_form_full_size(orc, system):
    """The headline form: A G from 4 balanced base-256 digits, Schur updates from 6, FP64 refinement."""
    orc.set_threads(os.cpu_count() or 1)
    A, B, Ah, Bh = system
    form = bench.Form(rmge, A, B, *bench.HEADLINE, digits=bench.HEADLINE_DIGITS[0],
                      fdigits=bench.HEADLINE_DIGITS[1], max_iters=bench.MAX_ITERS_MIXED)
    seed = SEED + 3  # the first timed step's multiplier after 3 warm-up steps
    out = staged_step(form, seed)
    check_multiplier(orc, out["G"], seed)

    # M = A G on sampled entries: d = 4 digits keep 8 d - 1 bits of every entry and the digit pairs p + q < d;
    # each term errs by at most about (d + 5) 2^(-8 d) of its row and column maxima
    d = bench.HEADLINE_DIGITS[0]
    rows, cols = sample(48, 1), sample(48, 2)
    ref = orc.matmul(Ah[rows], np.ascontiguousarray(out["G"][:, cols]))
    scale = np.max(np.abs(Ah[rows]), axis=1)[:, None] * np.max(np.abs(out["G"][:, cols]), axis=0)[None, :]
    err = np.abs(out["M"][np.ix_(rows, cols)] - ref) / scale
    assert np.max(err) <= 2 * (d + 5) * N * 2.0**(-8 * d), float(np.max(err))
    assert np.max(err) >= 2.0**(-8 * d - 16)  # the product really is one of 4 digits

    # the factors: no breakdown, and the normwise backward error of L U on sampled rows and columns.  Every
    # Schur update keeps 6 digits (47 bits) per product term, so a 64-deep pivot step errs by about 64 2^-47
    # of its share of |L| |U| at most (this draw: 1.05e-13).  One digit pair lost would raise it by 2^8
    assert out["info"] == 0 and np.isfinite(out["growth"])
    frows, fcols = sample(24, 3), sample(24, 4)
    LUr, absr, LUc, absc = factor_rows_cols(orc, out["LU"], frows, fcols)
    M = out["M"]
    be_r = np.max(np.abs(M[frows] - LUr), axis=1) / np.max(absr, axis=1)
    be_c = np.max(np.abs(M[:, fcols] - LUc), axis=0) / np.max(absc, axis=0)
    tol = 64 * 2.0**-47
    assert np.max(be_r) <= tol and np.max(be_c) <= tol, (float(np.max(be_r)), float(np.max(be_c)))

    # the refined solution: the device's gate and the oracle's compensated backward error both at 1e-13
    assert out["iters"] <= bench.MAX_ITERS_MIXED and out["berr"] <= bench.BE_TOL
    be = orc.backward_error(Ah, out["X"], Bh)
    print(f"headline n={N}: M err {np.max(err):.2e} of scale, factor be rows {np.max(be_r):.2e} cols "
          f"{np.max(be_c):.2e}, growth {out['growth']:.3g}, sweeps {out['iters']}, berr {out['berr']:.2e}, "
          f"oracle {be:.2e}")
    assert be <= bench.BE_TOL

    # the benchmark's own step on the same seed gives the same bits
    info, berr, iters, growth = form.step(seed)
    assert np.array_equal(host(form.X), out["X"])


@pytest.mark.parametrize("name", ["f64x_5_6", "unitary_f64x"])
def test_other_mixed_forms_full_size(orc, system, name):
    """The other mixed forms the benchmark times on the same inputs reach the target through the oracle's
    backward error."""
    orc.set_threads(os.cpu_count() or 1)
    A, B, Ah, Bh = system
    _, kind, prec, digits, fdigits, _, _ = next(f for f in bench.FORMS3 if f[0] == name)
    form = bench.Form(rmge, A, B, kind, prec, digits=digits, fdigits=fdigits, max_iters=bench.MAX_ITERS_MIXED)
    info, berr, iters, growth = form.step(SEED + 200)
    it = int(host(iters)[0])
    assert int(host(info)[0]) == 0 and float(host(berr)[it]) <= bench.BE_TOL
    assert orc.backward_error(Ah, host(form.X), Bh) <= bench.BE_TOL


def test_fp64_form_full_size(orc, system):
    """The plain FP64 form (the comparison line): sampled entries of M within the classical dot-product bound
    2 n u (|A| |G|), sampled entries of L U within the blocked-LU bound of a few n u (|L| |U|) entry by entry,
    and the solution at the target."""
    orc.set_threads(os.cpu_count() or 1)
    A, B, Ah, Bh = system
    form = bench.Form(rmge, A, B, "gaussian", "f64")
    seed = SEED + 100
    out = staged_step(form, seed)
    check_multiplier(orc, out["G"], seed)
    rows, cols = sample(32, 5), sample(32, 6)
    Gc = np.ascontiguousarray(out["G"][:, cols])
    ref = orc.matmul(Ah[rows], Gc)
    scale = orc.matmul(np.abs(Ah[rows]), np.abs(Gc))
    assert np.all(np.abs(out["M"][np.ix_(rows, cols)] - ref) <= 2 * N * U64 * scale)
    assert out["info"] == 0
    frows, fcols = sample(16, 7), sample(16, 8)
    LUr, absr, LUc, absc = factor_rows_cols(orc, out["LU"], frows, fcols)
    # the factorization's own error (gamma_n |L| |U|) plus the rounding of the check's dot products (gamma_n)
    assert np.all(np.abs(out["M"][frows] - LUr) <= 4 * N * U64 * absr)
    assert np.all(np.abs(out["M"][:, fcols] - LUc) <= 4 * N * U64 * absc)
    assert out["berr"] <= bench.BE_TOL
    assert orc.backward_error(Ah, out["X"], Bh) <= bench.BE_TOL
