"""GPU parity of the full particle-learning cycle against the CPU oracle.

Both sides take every floating-point decision in the same precision with the
same IEEE operation sequence, so at every step the ancestor indices must match
bit for bit and, at the end, every particle's x, sigma^2, tau^2 and sufficient
statistics must match bit for bit.  Posterior summaries differ only by the
order of the binary64 reductions: they must agree within 1e-12 (FP64 state)
and 1e-5 (FP32 state) relative to max(|oracle|, posterior sd).

Observations are seeded series of the paper's local-level model
(x_0 = 0, sigma^2 = 1, tau^2 = 0.1).
"""
import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _pair(pf, orc, n, scheme, prec, seed=1212, **kw):
    g = pf.Filter(n, seed=seed, scheme=scheme, precision="fp64" if prec else "fp32", **kw)
    o = orc.Filter(orc.make_config(n, seed=seed, scheme=scheme, precision=prec, **kw))
    return g, o


def _compare_states(g, o, prec):
    p = {k: v.cpu().numpy() for k, v in g.particles().items()}
    r = o.state_raw()
    for k in ("x", "sigma2", "tau2"):
        assert np.array_equal(p[k], r[k]), (k, np.flatnonzero(p[k] != r[k])[:5])
    for k in ("b_sigma", "b_tau"):
        got = p[k].view(np.uint64) if prec == 0 else p[k]
        assert np.array_equal(got, r[k]), k


def _compare_estimates(eg, eo, prec):
    tol = TOL[prec]
    assert eg["t"] == eo["t"]
    for k, v in (("x", "x_var"), ("sigma2", "sigma2_var"), ("tau2", "tau2_var")):
        sd = np.sqrt(max(eo[v], 0.0))
        assert abs(eg[k + "_mean"] - eo[k + "_mean"]) <= tol * max(abs(eo[k + "_mean"]), sd), k
        # a variance formed from sums has absolute rounding error ~ eps * mean^2
        eps = np.finfo(np.float64).eps
        floor = 8 * eps * eo[k + "_mean"] ** 2
        assert abs(eg[v] - eo[v]) <= 10 * tol * abs(eo[v]) + floor, v
    assert abs(eg["log_marglik"] - eo["log_marglik"]) <= tol * max(1.0, abs(eo["log_marglik"]))


def _run(pf, orc, n, T, scheme, prec, y=None, every_step=True, **kw):
    if y is None:
        _, y = synth.local_level_series(1212, T)
    g, o = _pair(pf, orc, n, scheme, prec, **kw)
    for t in range(T):
        g.step(y[t])
        o.step(y[t])
        if every_step or t == T - 1:
            anc = g.ancestors().cpu().numpy().view(np.uint32)
            ref = o.ancestors()
            assert np.array_equal(anc, ref), (t, np.flatnonzero(anc != ref)[:5])
    _compare_states(g, o, prec)
    _compare_estimates(g.estimate(), o.estimate(), prec)
    g.close()


def test_fp64_paper_config_multinomial(pf, orc):
    """The plain method in FP64: N = 1024, T = 100, multinomial, IG(3,2) priors."""
    _run(pf, orc, 1024, 100, 0, 1)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_fp32_all_schemes_ragged(pf, orc, scheme):
    _run(pf, orc, 5000, 30, scheme, 0)


@pytest.mark.parametrize("scheme", [0, 1, 4])
def test_fp64_schemes_multi_tile(pf, orc, scheme):
    _run(pf, orc, 3 * 4096 + 17, 15, scheme, 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_known_variances(pf, orc, prec):
    _run(pf, orc, 3000, 20, 1, prec, known_variances=True, sigma2=1.0, tau2=0.1)


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_tiny_filters(pf, orc, n, prec):
    _run(pf, orc, n, 8, 0, prec)
    _run(pf, orc, n, 8, 1, prec)


@pytest.mark.parametrize("scheme", [0, 1])
def test_full_size_2p20_fp32(pf, orc, scheme):
    """The at-scale configuration (N = 2^20, FP32) for a few cycles."""
    _run(pf, orc, 1 << 20, 3, scheme, 0, every_step=False, seed=1639)


@pytest.mark.parametrize("prec", [0, 1])
def test_systematic_cdf_several_tiles_per_cta(pf, orc, prec):
    """Above about 2.5M particles each CTA of the cooperative CDF launch owns
    several tiles and stages them through shared memory by TMA; ragged last
    tile, FP32 and FP64."""
    _run(pf, orc, 3_000_001, 3, 1, prec, every_step=True, seed=77)


def test_systematic_cdf_tile_shapes(pf, orc):
    """Binary32 systematic cycles take 2048-particle CDF tiles (8 per thread)
    while one tile per CTA fits at once and 4096-particle tiles above that:
    both shapes, with ragged last tiles, give the oracle's results."""
    _run(pf, orc, 1_000_003, 3, 1, 0, every_step=True, seed=91)   # 2048-particle tiles
    _run(pf, orc, 2_000_001, 3, 1, 0, every_step=True, seed=92)   # 4096-particle tiles


def test_outlier_observation(pf, orc):
    """y far from every particle: most quantised weights underflow to zero."""
    y = np.array([0.3, 40.0, 40.5, -3.0, 0.0])
    _run(pf, orc, 4096, y.size, 1, 0, y=y)
    _run(pf, orc, 4096, y.size, 0, 1, y=y)


def test_outlier_observation_large(pf, orc):
    """Outlying observations at 300,001 particles (2048-particle CDF tiles,
    one per CTA) and 2,600,003 (several 4096-particle tiles per CTA): a few
    particles own thousands of slots each, so tiles hold far more slots than
    the shared-memory ancestor window and the heavy particles' slots past it
    become runs of the CTA."""
    y = np.array([0.3, 40.0, 0.1])
    _run(pf, orc, 300_001, y.size, 1, 0, y=y)
    _run(pf, orc, 300_001, y.size, 4, 0, y=y)  # stratified: the warp stores long ranges
    _run(pf, orc, 2_600_003, 2, 1, 0, y=np.array([0.3, -35.0]), every_step=True, seed=3)


@pytest.mark.parametrize("scheme,prec", [(1, 0), (0, 0), (4, 0), (3, 0), (1, 1), (0, 1)])
def test_bootstrap_filter_matches_oracle(pf, orc, scheme, prec):
    """Algorithm "Particle Filtering" with known variances: blind propagation,
    weights p(y | x), resampling; ancestors every step and the final state bit
    for bit, summaries within the oracle tolerance."""
    kw = dict(known_variances=True, sigma2=0.8, tau2=0.15, algorithm=1)
    _run(pf, orc, 5000, 20, scheme, prec, seed=41, **kw)


def test_bootstrap_filter_at_scale(pf, orc):
    """The bootstrap cycle at 2^20 (one 2048-particle CDF tile per CTA) and at
    2,600,003 particles (several tiles per CTA), systematic, FP32."""
    kw = dict(known_variances=True, sigma2=1.0, tau2=0.1, algorithm=1)
    _run(pf, orc, 1 << 20, 3, 1, 0, seed=42, **kw)
    _run(pf, orc, 2_600_003, 2, 1, 0, seed=43, **kw)


def test_bootstrap_needs_known_variances(pf):
    with pytest.raises(pf.PfError) as e:
        pf.Filter(1000, algorithm="bootstrap")
    assert e.value.status == pf.PF_ERR_INVALID
    with pytest.raises(pf.PfError):
        pf.Filter(1000, algorithm=7, known_variances=True)


def test_run_matches_step(pf, orc):
    _, y = synth.local_level_series(5, 40)
    a = pf.Filter(2048, seed=5, scheme="multinomial")
    b = pf.Filter(2048, seed=5, scheme="multinomial")
    for v in y:
        a.step(v)
    b.run(torch.from_numpy(y).cuda())
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert torch.equal(pa[k], pb[k]), k
    assert a.estimate() == b.estimate()
    c = pf.Filter(2048, seed=5, scheme="multinomial")
    c.run(y)  # host observations
    assert c.estimate() == a.estimate()


def test_many_steps_wrap_observation_ring(pf):
    """More cycles than the 8192-slot observation ring holds."""
    _, y = synth.local_level_series(6, 9000)
    f = pf.Filter(256, seed=6, scheme="systematic")
    f.run(y)
    e = f.estimate()
    assert e["t"] == 9000 and np.isfinite(e["log_marglik"])


def test_nan_observation_is_sticky_error(pf):
    f = pf.Filter(1000, seed=1)
    f.step(0.1)
    f.step(float("nan"))
    with pytest.raises(pf.PfError) as e:
        f.sync()
    assert e.value.status == pf.PF_ERR_NUMERIC
    with pytest.raises(pf.PfError):
        f.step(0.2)
    f.close()
    g = pf.Filter(100, seed=1)  # a new handle works
    g.step(0.0)
    g.sync()


def test_invalid_config(pf):
    with pytest.raises(pf.PfError) as e:
        pf.Filter(0)
    assert e.value.status == pf.PF_ERR_INVALID
    with pytest.raises(pf.PfError):
        pf.Filter(10, a_sigma=0.5)
    with pytest.raises(pf.PfError):
        pf.Filter(pf.MAX_PARTICLES + 1)
