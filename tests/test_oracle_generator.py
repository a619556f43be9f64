"""Pins for the oracle's counter-based generator and multiplier draws (Def. 4.1, Ex. 5.1)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(orc, ctr, key, expect):
    assert [int(x) for x in orc.philox4x32_10(ctr, key)] == expect


def test_gaussian_moments_and_ks(orc):
    z = orc.gaussian(400_000, seed=12345, subseq=1)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.01
    assert abs(stats.skew(z)) < 0.02 and abs(stats.kurtosis(z)) < 0.04
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # even and odd entries are the cos / sin halves of a Box-Muller pair: uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.01


def test_gaussian_streams_are_distinct_and_reproducible(orc):
    a = orc.gaussian(1000, seed=7, subseq=0)
    b = orc.gaussian(1000, seed=7, subseq=1)
    c = orc.gaussian(1000, seed=8, subseq=0)
    assert np.array_equal(a, orc.gaussian(1000, seed=7, subseq=0))
    assert not np.allclose(a, b) and not np.allclose(a, c)
    # prefix property: a shorter draw is the head of a longer one (counter-based addressing)
    assert np.array_equal(orc.gaussian(17, seed=7, subseq=0), a[:17])


def test_uniform_pm1(orc):
    u = orc.uniform_pm1(200_000, seed=99, subseq=3)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3
    # values are exact multiples of 2^-52 (53-bit uniform mapped affinely, exactly)
    assert np.all(np.floor(u * 2.0**52) == u * 2.0**52)


def test_uniform_uses_the_same_words_as_gaussian(orc):
    # entry 0 of the uniform stream is built from Philox words 0,1 of block 0
    x = orc.philox4x32_10([0, 0, 5, 0], [11, 0])
    m = (int(x[0]) << 21) | (int(x[1]) >> 11)
    assert orc.uniform_pm1(2, seed=11, subseq=5)[0] == 2.0 * m / 2.0**53 - 1.0
    u1 = ((int(x[0]) << 21) | (int(x[1]) >> 11)) + 1
    u2 = (int(x[2]) << 21) | (int(x[3]) >> 11)
    r = math.sqrt(-2.0 * math.log(u1 / 2.0**53))
    g = orc.gaussian(2, seed=11, subseq=5)
    assert g[0] == pytest.approx(r * math.cos(2 * math.pi * u2 / 2.0**53), rel=1e-15, abs=1e-15)
    assert g[1] == pytest.approx(r * math.sin(2 * math.pi * u2 / 2.0**53), rel=1e-15, abs=1e-15)


def test_gaussian_matrix_norm_and_condition_bounds(orc):
    """Theorem 4.6 / Appendix A: E||G|| <= 2 sqrt(n); P{||G|| > t + 2 sqrt(n)} <= exp(-t^2/2);
    E log kappa(G) <= log n + 2.258."""
    n, reps = 128, 24
    norms, logk = [], []
    for r in range(reps):
        G = orc.make_multiplier(0, n, seed=1000 + r)
        s = np.linalg.svd(G, compute_uv=False)
        norms.append(s[0])
        logk.append(math.log(s[0] / s[-1]))
    assert np.mean(norms) <= 2 * math.sqrt(n)
    assert max(norms) <= 2 * math.sqrt(n) + 4.0  # t = 4: probability <= e^-8 per draw
    assert np.mean(logk) <= math.log(n) + 2.258


def test_gaussian_f32_stream(orc):
    z = orc.gaussian_f32(200_000, seed=4321, subseq=1).astype(np.float64)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.015
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the 24-bit uniforms are the top bits of the same Philox words as the FP64 stream's
    x = orc.philox4x32_10([0, 0, 1, 0], [4321, 0])
    u1 = ((int(x[0]) >> 8) + 1) / 2.0**24
    u2 = (int(x[2]) >> 8) / 2.0**24
    r = math.sqrt(-2.0 * math.log(u1))
    assert z[0] == pytest.approx(r * math.cos(2 * math.pi * u2), rel=1e-5, abs=1e-5)
