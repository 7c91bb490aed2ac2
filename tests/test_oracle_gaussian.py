"""Pins of the oracle's Gaussian sampler (the Gaussian sketch of Section 1,
second stage of the multisketch): accuracy of the hand-written binary32 ln,
moments and a Kolmogorov-Smirnov test against N(0, 1/p)."""
import math

import numpy as np
import pytest


def test_ln_f32_accuracy(orc):
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(1e-6, 1.0, 4000), rng.uniform(0.5, 1.5, 4000),
                         np.float32(2.0) ** -np.arange(1, 40, dtype=np.float64)])
    xs = xs.astype(np.float32)
    worst = 0.0
    for x in xs:
        got = orc.ln_f32(float(x))
        ref = math.log(float(x))
        # error relative to the result, floored at one binary32 ulp of 1
        worst = max(worst, abs(got - ref) / max(abs(ref), 2.0 ** -23))
    assert worst < 8 * 2.0 ** -24


def test_ln_f32_exact_points(orc):
    assert orc.ln_f32(1.0) == 0.0
    # ln(2^e) = e * fl(ln 2) rounded once
    for e in (-20, -3, -1, 1, 5):
        want = float(np.float32(e) * np.float32(math.log(2)))
        assert orc.ln_f32(2.0 ** e) == want


@pytest.mark.parametrize("p,k", [(256, 4096), (64, 2048)])
def test_gaussian_moments_and_ks(orc, p, k):
    from scipy import stats

    G = orc.gaussian(0x5EED0002, p, k).astype(np.float64)
    assert G.shape == (p, k)
    x = G.ravel() * math.sqrt(p)  # should be N(0,1)
    N = x.size
    assert abs(x.mean()) < 5 / math.sqrt(N)
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / N)
    kurt = float(np.mean(x ** 4))
    assert abs(kurt - 3.0) < 5 * math.sqrt(96.0 / N)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # rows are independent draws: sample correlation of two rows is small
    c = np.corrcoef(G[0], G[1])[0, 1]
    assert abs(c) < 5 / math.sqrt(k)


def test_gaussian_reproducible_and_seeded(orc):
    a = orc.gaussian(11, 8, 100)
    b = orc.gaussian(11, 8, 100)
    c = orc.gaussian(12, 8, 100)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    # the matrix for fewer rows is a prefix of the larger one's standard
    # normal draws (entry (r, c) uses draw number r*k + c), up to the 1/sqrt(p)
    # scaling: compare after undoing the scale in float64 with a tolerance
    small = orc.gaussian(11, 3, 100).astype(np.float64) * math.sqrt(3)
    big = a[:3].astype(np.float64) * math.sqrt(8)
    assert np.allclose(small, big, rtol=1e-6, atol=1e-6)
