"""Pins of the oracle's adaptive resampling (ess_frac > 0).

The filter carries log-weights between cycles and resamples only when the
effective sample size ESS = (sum W)^2 / sum W^2 of the combined quantised
weights falls below ess_frac * n (Kong, Liu & Wong 1994).  Pinned here by:

- the decision against exact rational arithmetic (Python integers), and the
  boundary ESS = n of equal weights;
- ess_frac = 1, which resamples whenever the weights are not all equal: the
  filter must equal the always-resampling filter bit for bit;
- the Kalman filter with known variances, for the adaptive form (both
  branches taken) and for a filter that never resamples (sequential
  importance sampling with the fully adapted proposal), which pins the
  weight accumulation, the weighted summaries and the log marginal
  likelihood's normalisation by the carried weights.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_1212_1639_gb300 import synth


@pytest.fixture(scope="module")
def series():
    x, y = synth.local_level_series(1212, 100, sigma2=1.0, tau2=0.1)
    return x, y


def _exact(W, f):
    T = sum(int(w) for w in W)
    B = sum(int(w) * int(w) for w in W)
    lhs = Fraction(T * T)
    rhs = Fraction(f) * len(W) * B
    return lhs < rhs, float(lhs / rhs) if rhs else np.inf


def test_ess_decision_exact(orc):
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(400):
        n = int(rng.integers(1, 600))
        kind = trial % 4
        k = orc.cdf_shift(n)
        if kind == 0:    # log-normal weights of various spreads
            lw = rng.normal(0, rng.choice([0.1, 1, 3, 8]), n)
            w = np.exp(lw - lw.max())
        elif kind == 1:  # a few heavy particles
            w = np.full(n, 1e-3)
            w[rng.integers(0, n, size=3)] = 1.0
        elif kind == 2:  # many zeros
            w = rng.random(n) * (rng.random(n) < 0.1)
            w[0] = 1.0
        else:            # near-flat
            w = 1.0 - 1e-6 * rng.random(n)
        W = np.floor(w / w.max() * 2.0 ** k).astype(np.uint64)
        for f in (0.05, 0.3, 0.5, 0.9, 1.0):
            want, ratio = _exact(W, f)
            if abs(ratio - 1.0) < 1e-12:
                continue  # a tie within rounding: either answer is the binary64 one
            assert orc.ess_resample(W, f) == want, (trial, n, f, ratio)
            checked += 1
    assert checked > 1500


def test_ess_boundary_equal_weights(orc):
    """Equal weights have ESS = n exactly: no resampling even at ess_frac = 1;
    one particle owning all the weight has ESS = 1."""
    for n in (1, 2, 7, 1000, 1 << 20):
        k = orc.cdf_shift(n)
        W = np.full(n, 1 << k, np.uint64)
        assert not orc.ess_resample(W, 1.0)
        if n > 1:
            W1 = np.zeros(n, np.uint64)
            W1[n // 2] = 1 << k
            assert orc.ess_resample(W1, 1.5 / n)
            assert not orc.ess_resample(W1, 0.5 / n)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 4])
def test_ess_one_equals_always_resampling(orc, series, precision, scheme):
    _, y = series
    kw = dict(seed=51, scheme=scheme, precision=precision)
    a = orc.Filter(orc.make_config(3000, **kw))
    b = orc.Filter(orc.make_config(3000, ess_frac=1.0, **kw))
    for t in range(30):
        a.step(y[t])
        b.step(y[t])
        assert b.resampled()
        assert np.array_equal(a.ancestors(), b.ancestors())
    ra, rb = a.state_raw(), b.state_raw()
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k
    assert a.estimate() == b.estimate()


def _kalman_z(orc, f, y, km, kv, n, T):
    z, kinds = [], []
    for t in range(T):
        f.step(y[t])
        kinds.append(f.resampled())
        if not kinds[-1]:
            assert np.array_equal(f.ancestors(), np.arange(n, dtype=np.uint32))
        e = f.estimate()
        assert e["t"] == t + 1
        z.append((e["x_mean"] - km[t]) / np.sqrt(kv[t] / n))
    return np.array(z), np.array(kinds)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1])
def test_ess_adaptive_matches_kalman(orc, series, precision, scheme):
    _, y = series
    n = 1 << 15
    km, kv, kll = orc.kalman(y, 0.0, 10.0, 1.0, 0.1)
    f = orc.Filter(orc.make_config(n, seed=200 + scheme, scheme=scheme, precision=precision,
                                   known_variances=True, sigma2=1.0, tau2=0.1, ess_frac=0.5))
    z, res = _kalman_z(orc, f, y, km, kv, n, y.size)
    assert 0 < res.sum() < y.size - 10, res.sum()  # both branches taken
    assert np.max(np.abs(z)) < 12, np.max(np.abs(z))
    assert np.sqrt(np.mean(z ** 2)) < 4
    assert abs(f.estimate()["log_marglik"] - kll) < 0.25


@pytest.mark.parametrize("precision", [0, 1])
def test_never_resampling_matches_kalman(orc, series, precision):
    """ess_frac so small that ESS >= 1 never falls below it: importance
    weights accumulate over 15 cycles without resampling."""
    _, y = series
    n, T = 1 << 16, 15
    km, kv, kll = orc.kalman(y[:T], 0.0, 10.0, 1.0, 0.1)
    f = orc.Filter(orc.make_config(n, seed=7, scheme=1, precision=precision,
                                   known_variances=True, sigma2=1.0, tau2=0.1, ess_frac=1e-9))
    z, res = _kalman_z(orc, f, y, km, kv, n, T)
    assert not res.any()
    assert np.max(np.abs(z)) < 15, np.max(np.abs(z))
    assert abs(f.estimate()["log_marglik"] - kll) < 0.25
