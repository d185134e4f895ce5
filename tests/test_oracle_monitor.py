"""Pins of the oracle's min-entropy monitor: exact counts of constructed
sample arrays (every value a known number of times, junk above b ignored),
the estimator's closed forms (uniform data gives b bits, a point mass 0, a
two-point law -log2 of its larger mass), and the plug-in estimate on the
quantised-Gaussian ADC stand-in against its analytic min-entropy."""
import math

import numpy as np
import pytest

import oracle
from paper_2402_14607_gb300 import workloads


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


@pytest.mark.parametrize("b", [1, 4, 8, 12, 16])
def test_constructed_counts(b):
    rng = np.random.Generator(np.random.PCG64(b))
    want = rng.integers(0, 7, size=1 << b).astype(np.uint64)
    vals = np.repeat(np.arange(1 << b, dtype=np.uint32), want.astype(np.int64))
    rng.shuffle(vals)
    junk = rng.integers(0, 1 << 16, size=vals.size).astype(np.uint32) & ~np.uint32((1 << b) - 1)
    got = oracle.sample_histogram(b, (vals | junk).astype(np.uint16))
    assert (got == want).all() and int(got.sum()) == vals.size
    # accumulation over two halves
    h = oracle.sample_histogram(b, (vals[: vals.size // 2] | junk[: vals.size // 2]).astype(np.uint16))
    oracle.sample_histogram(b, (vals[vals.size // 2:] | junk[vals.size // 2:]).astype(np.uint16), h)
    assert (h == want).all()


def test_estimator_closed_forms():
    assert oracle.min_entropy_estimate(8, np.full(256, 5, np.uint64)) == pytest.approx(8.0)
    point = np.zeros(4096, np.uint64)
    point[17] = 1000
    assert oracle.min_entropy_estimate(12, point) == 0.0
    two = np.zeros(16, np.uint64)
    two[3], two[9] = 3, 1
    assert oracle.min_entropy_estimate(4, two) == pytest.approx(-math.log2(0.75))
    assert oracle.min_entropy_estimate(4, np.zeros(16, np.uint64)) == -1.0


@pytest.mark.parametrize("b,sigma", [(8, 1.0), (12, 1.0), (12, 0.95)])
def test_gaussian_adc_estimate_near_analytic(b, sigma):
    """The plug-in estimate of 4M quantised-Gaussian samples lies within a few
    standard errors of -log2 p_max computed from the normal CDF."""
    n = 1 << 22
    s = workloads.adc_samples(5, n, b, sigma=sigma)
    est = oracle.min_entropy_estimate(b, oracle.sample_histogram(b, s))
    ana = workloads.adc_min_entropy(b, sigma=sigma)
    p = 2.0 ** -ana
    # delta method: sd(-log2 p_hat) = sqrt((1-p)/(n p)) / ln 2; the maximum
    # over bins biases the estimate down a little, so allow 6 sd
    sd = math.sqrt((1 - p) / (n * p)) / math.log(2)
    assert abs(est - ana) < 6 * sd + 1e-3, (est, ana, sd)
