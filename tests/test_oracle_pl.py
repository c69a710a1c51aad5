"""Pins of the oracle's particle-learning cycle (paper Sections 2 and 4).

- Known variances: particle learning reduces to a fully adapted particle filter
  whose filtered means, variances and log-likelihood must agree with the Kalman
  filter (the closed form of the Bayes filter for the linear Gaussian model)
  within Monte Carlo error.
- Known states: the sufficient-statistic recursion must reproduce the conjugate
  inverse-gamma posterior IG(a0 + T/2, b0 + sum r^2 / 2) exactly, and the
  parameter draws must follow that law.
- Prior: the paper's priors IG(5, 4) and IG(5, 0.4) have means equal to the
  true sigma^2 = 1 and tau^2 = 0.1, which pins the shape/scale reading.

Tolerances are Monte Carlo bounds calibrated on seeds other than the ones used
here, with a wide margin; any systematic error (a dropped term, the wrong time
index, a transposed variance) is tens of standard errors away.
"""
import numpy as np
import pytest
from scipy import stats

from paper_1212_1639_gb300 import synth


@pytest.fixture(scope="module")
def series():
    x, y = synth.local_level_series(1212, 100, sigma2=1.0, tau2=0.1)
    return x, y


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_known_variances_match_kalman(orc, series, precision, scheme):
    _, y = series
    n = 1 << 15
    km, kv, kll = orc.kalman(y, 0.0, 10.0, 1.0, 0.1)
    cfg = orc.make_config(n, seed=100 + scheme, scheme=scheme, precision=precision,
                          known_variances=True, sigma2=1.0, tau2=0.1)
    f = orc.Filter(cfg)
    z, vr = [], []
    for t in range(y.size):
        f.step(y[t])
        e = f.estimate()
        assert e["t"] == t + 1
        z.append((e["x_mean"] - km[t]) / np.sqrt(kv[t] / n))
        vr.append(e["x_var"] / kv[t])
    z = np.array(z)
    assert np.max(np.abs(z)) < 12, np.max(np.abs(z))
    assert np.sqrt(np.mean(z ** 2)) < 4
    assert np.max(np.abs(np.array(vr[5:]) - 1)) < 0.1
    assert abs(f.estimate()["log_marglik"] - kll) < 0.25
    # known-variance mode leaves the parameters untouched
    s = f.state()
    assert np.all(s["sigma2"] == np.float32(1.0) if precision == 0 else s["sigma2"] == 1.0)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 4])
def test_bootstrap_filter_matches_kalman(orc, series, precision, scheme):
    """Algorithm "Particle Filtering" (the bootstrap filter, known variances):
    blind propagation then weighting by p(y | x) resamples with a noisier
    sample than particle learning's fully adapted step, so its filtered mean
    sits within a larger multiple of sd/sqrt(N) of the Kalman mean; the
    log-likelihood estimate is still within Monte Carlo error."""
    _, y = series
    n = 1 << 15
    km, kv, kll = orc.kalman(y, 0.0, 10.0, 1.0, 0.1)
    cfg = orc.make_config(n, seed=300 + scheme, scheme=scheme, precision=precision,
                          known_variances=True, sigma2=1.0, tau2=0.1, algorithm=orc.BOOTSTRAP)
    f = orc.Filter(cfg)
    z, vr = [], []
    for t in range(y.size):
        f.step(y[t])
        e = f.estimate()
        assert e["t"] == t + 1
        z.append((e["x_mean"] - km[t]) / np.sqrt(kv[t] / n))
        vr.append(e["x_var"] / kv[t])
    z = np.array(z)
    assert np.max(np.abs(z)) < 15, np.max(np.abs(z))
    assert np.sqrt(np.mean(z ** 2)) < 5
    assert np.max(np.abs(np.array(vr[5:]) - 1)) < 0.15
    assert abs(f.estimate()["log_marglik"] - kll) < 0.3
    s = f.state()
    assert np.all(s["sigma2"] == np.float32(1.0) if precision == 0 else s["sigma2"] == 1.0)
    assert np.all(s["tau2"] == np.float32(0.1) if precision == 0 else s["tau2"] == 0.1)


def test_bootstrap_one_step_by_hand(orc):
    """One bootstrap cycle recomputed here step by step in binary64 from the
    oracle's exported primitives (its normals, deterministic log, weight
    quantisation and systematic resampling): propagated particles, weights,
    exact CDF, ancestors, resampled state and log-ML increment."""
    n, y, s2, t2, seed = 37, 0.7, 1.3, 0.4, 11
    cfg = orc.make_config(n, seed=seed, scheme=1, precision=1, known_variances=True,
                          sigma2=s2, tau2=t2, algorithm=orc.BOOTSTRAP)
    f = orc.Filter(cfg)
    x0 = f.state()["x"].copy()
    f.step(y)
    # Step 1: x' = x + sqrt(tau^2) Z, Z Box-Muller from (seed, 0, t=0, i, BOOT_STATE = 10)
    Z = orc.normals(seed, 0, 0, 10, n, np.float64)
    xp = x0 + np.sqrt(t2) * Z
    # Step 2: l = -(log sigma^2 + (y - x')^2 / sigma^2) / 2 (log(2 pi)/2 dropped)
    lg = orc.det_log(np.full(n, s2), np.float64)
    ell = -0.5 * (lg + (y - xp) ** 2 / s2)
    m = ell.max()
    W, e = orc.quant_exp(ell - m, orc.cdf_shift(n), np.float64)
    Q = np.cumsum(W.astype(object)).astype(np.uint64)
    assert np.array_equal(f.cdf(), Q)
    # Step 3: systematic ancestors of that CDF, and the resampled particles
    anc = orc.resample_cdf(Q, orc.SYSTEMATIC, seed, 0, 0)
    assert np.array_equal(f.ancestors(), anc)
    assert np.array_equal(f.state()["x"], xp[anc])
    # log-ML increment: m + log(sum e) - log n - log(2 pi)/2
    ref = m + np.log(np.sum(e)) - np.log(n) - 0.5 * np.log(2 * np.pi)
    assert abs(f.estimate()["log_marglik"] - ref) < 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_known_states_conjugate_inverse_gamma(orc, precision):
    T = 50
    x, y = synth.local_level_series(7, T, sigma2=1.0, tau2=0.1)
    if precision == 0:
        # the FP32 state path works with binary32 states and observations
        x = x.astype(np.float32).astype(np.float64)
        y = y.astype(np.float32).astype(np.float64)
    n = 20_000
    a0s, b0s, a0t, b0t = 3.0, 2.0, 5.0, 0.4
    cfg = orc.make_config(n, seed=3, precision=precision, a_sigma=a0s, b_sigma=b0s,
                          a_tau=a0t, b_tau=b0t)
    out, rc = orc.suffstat_known_states(cfg, x, y)
    assert rc == 0
    bs_ref = b0s + 0.5 * np.sum((y - x[1:]) ** 2)
    bt_ref = b0t + 0.5 * np.sum(np.diff(x) ** 2)
    tol = 1e-12 if precision == 1 else 1e-6
    assert np.allclose(out["b_sigma"], bs_ref, rtol=tol, atol=0)
    assert np.allclose(out["b_tau"], bt_ref, rtol=tol, atol=0)
    a_s, a_t = a0s + T / 2, a0t + T / 2
    for key, a, b in (("sigma2", a_s, bs_ref), ("tau2", a_t, bt_ref)):
        d = out[key]
        mean, sd = b / (a - 1), b / ((a - 1) * np.sqrt(a - 2))
        assert abs(d.mean() - mean) < 5 * sd / np.sqrt(n)
        assert stats.kstest(d, stats.invgamma(a, scale=b).cdf).pvalue > 1e-4


def test_prior_means_pin_shape_scale(orc):
    n = 1 << 16
    cfg = orc.make_config(n, seed=11, precision=1, a_sigma=5.0, b_sigma=4.0, a_tau=5.0,
                          b_tau=0.4, x0_mean=0.0, x0_var=10.0)
    s = orc.Filter(cfg).state()
    # IG(5, 4): mean 4/4 = 1 = sigma^2; IG(5, 0.4): mean 0.1 = tau^2 (paper Section 4)
    for key, mean, a, b in (("sigma2", 1.0, 5.0, 4.0), ("tau2", 0.1, 5.0, 0.4)):
        sd = b / ((a - 1) * np.sqrt(a - 2))
        assert abs(s[key].mean() - mean) < 5 * sd / np.sqrt(n)
        assert stats.kstest(s[key], stats.invgamma(a, scale=b).cdf).pvalue > 1e-4
    assert abs(s["x"].mean()) < 5 * np.sqrt(10 / n)
    assert abs(s["x"].var() / 10 - 1) < 5 * np.sqrt(2 / n)
    assert np.all(s["b_sigma"] == 4.0) and np.all(s["b_tau"] == 0.4)


def test_learning_concentrates_near_truth(orc):
    """Unknown variances, T = 500: the posterior means land near the truth."""
    x, y = synth.local_level_series(1639, 500, sigma2=1.0, tau2=0.1)
    cfg = orc.make_config(1 << 13, seed=5, precision=1)
    f = orc.Filter(cfg)
    f.run(y)
    e = f.estimate()
    assert 0.7 < e["sigma2_mean"] < 1.4
    assert 0.03 < e["tau2_mean"] < 0.3
    assert abs(e["x_mean"] - x[-1]) < 4 * np.sqrt(e["x_var"] + 0.5)
    assert np.isfinite(e["log_marglik"])


def test_fp32_and_fp64_agree_statistically(orc, series):
    _, y = series
    ests = {}
    for prec in (0, 1):
        f = orc.Filter(orc.make_config(1 << 14, seed=21, precision=prec))
        f.run(y[:60])
        ests[prec] = f.estimate()
    for k in ("x_mean", "sigma2_mean", "tau2_mean"):
        assert abs(ests[0][k] - ests[1][k]) < 0.1 * max(1.0, abs(ests[1][k]))
    assert abs(ests[0]["log_marglik"] - ests[1]["log_marglik"]) < 1.0


def test_fp32_state_is_binary32_and_fixed_point(orc):
    f = orc.Filter(orc.make_config(64, seed=1, precision=0))
    f.step(0.3)
    r = f.state_raw()
    assert r["x"].dtype == np.float32 and r["b_sigma"].dtype == np.uint64
    d = f.state()
    assert np.array_equal(d["b_sigma"], r["b_sigma"].astype(np.float64) * 2.0 ** -32)


def _exact_posterior(y, a=3.0, b=2.0, m0=0.0, P0=10.0):
    """log p(y_1..y_T), E[sigma^2 | y] and E[tau^2 | y] for the local-level
    model with IG(a, b) priors on both variances: the Kalman likelihood
    (prediction-error decomposition, written out here) integrated over the
    prior on a 600 x 600 grid in (log sigma^2, log tau^2)."""
    ls = np.linspace(np.log(0.05), np.log(8.0), 600)
    lt = np.linspace(np.log(0.005), np.log(4.0), 600)
    S2, T2 = np.meshgrid(np.exp(ls), np.exp(lt), indexing="ij")
    m = np.full_like(S2, m0)
    P = np.full_like(S2, P0)
    ll = np.zeros_like(S2)
    for v in y:
        R = P + T2
        F = R + S2
        K = R / F
        e = v - m
        ll += -0.5 * (np.log(2 * np.pi * F) + e * e / F)
        m = m + K * e
        P = R - K * R
    prior = (stats.invgamma.pdf(S2, a, scale=b) * stats.invgamma.pdf(T2, a, scale=b)
             * S2 * T2)  # densities in log coordinates
    mx = ll.max()
    w = np.exp(ll - mx) * prior
    dA = (ls[1] - ls[0]) * (lt[1] - lt[0])
    Z = w.sum() * dA
    return mx + np.log(Z), (w * S2).sum() * dA / Z, (w * T2).sum() * dA / Z


@pytest.mark.parametrize("ess_frac", [0.0, 0.5])
def test_learning_matches_exact_posterior(orc, series, ess_frac):
    """Particle learning of sigma^2 and tau^2 (and, with ess_frac = 0.5, its
    adaptive-resampling form) against the exact Bayes posterior by quadrature:
    log marginal likelihood and posterior means of both variances within
    Monte Carlo error (N = 2^14, two seeds averaged).  A state-sufficient-
    statistic variant whose parameter statistics re-draw x_t every cycle
    misses these by 0.6 in log p(y) and 0.04 in E[sigma^2]."""
    _, y = series
    lz, es2, et2 = _exact_posterior(y)
    got = []
    for seed in (900, 901):
        f = orc.Filter(orc.make_config(1 << 14, seed=seed, scheme=1, precision=1,
                                       ess_frac=ess_frac))
        for v in y:
            f.step(v)
        e = f.estimate()
        got.append((e["log_marglik"], e["sigma2_mean"], e["tau2_mean"]))
    g = np.mean(got, axis=0)
    assert abs(g[0] - lz) < 0.25, (g[0], lz)
    assert abs(g[1] - es2) < 0.02, (g[1], es2)
    assert abs(g[2] - et2) < 0.02, (g[2], et2)
