"""GPU parity of adaptive resampling (pf_config.ess_frac > 0) against the CPU
oracle.

Both sides take the resampling decision from the same exact integer sums in
the same binary64 operations, carry the same log-weights and draw the same
Philox counters, so at every cycle the ancestors (the identity when the cycle
does not resample) must match bit for bit, and at the end every particle must
match; the summaries (weighted by the carried weights, so a wrong weight shows
there and in the next cycle's ancestors) and the log marginal likelihood
within 1e-5 (FP32 state) and 1e-12 (FP64 state) relative to
max(|oracle|, posterior sd).
"""
import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _run(pf, orc, n, T, scheme, prec, ess, seed=61, y=None, every_step=True, **kw):
    if y is None:
        _, y = synth.local_level_series(seed, T)
    g = pf.Filter(n, seed=seed, scheme=scheme, precision="fp64" if prec else "fp32",
                  ess_frac=ess, **kw)
    o = orc.Filter(orc.make_config(n, seed=seed, scheme=scheme, precision=prec, ess_frac=ess,
                                   **kw))
    kinds = []
    for t in range(T):
        g.step(y[t])
        o.step(y[t])
        kinds.append(o.resampled())
        if every_step or t == T - 1:
            anc = g.ancestors().cpu().numpy().view(np.uint32)
            ref = o.ancestors()
            assert np.array_equal(anc, ref), (t, kinds[-1], np.flatnonzero(anc != ref)[:5])
    p = {k: v.cpu().numpy() for k, v in g.particles().items()}
    r = o.state_raw()
    for k in ("x", "sigma2", "tau2"):
        assert np.array_equal(p[k], r[k]), (k, np.flatnonzero(p[k] != r[k])[:5])
    for k in ("b_sigma", "b_tau"):
        got = p[k].view(np.uint64) if prec == 0 else p[k]
        assert np.array_equal(got, r[k]), k
    eg, eo = g.estimate(), o.estimate()
    tol = TOL[prec]
    assert eg["t"] == eo["t"]
    for k, v in (("x", "x_var"), ("sigma2", "sigma2_var"), ("tau2", "tau2_var")):
        sd = np.sqrt(max(eo[v], 0.0))
        assert abs(eg[k + "_mean"] - eo[k + "_mean"]) <= tol * max(abs(eo[k + "_mean"]), sd), k
        eps = np.finfo(np.float64).eps
        assert abs(eg[v] - eo[v]) <= 10 * tol * abs(eo[v]) + 8 * eps * eo[k + "_mean"] ** 2, v
    assert abs(eg["log_marglik"] - eo["log_marglik"]) <= tol * max(1.0, abs(eo["log_marglik"]))
    g.close()
    return np.array(kinds)


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_all_schemes(pf, orc, scheme, prec):
    """ess_frac = 0.5 over 30 cycles: both branches are taken."""
    kinds = _run(pf, orc, 3 * 4096 + 17, 30, scheme, prec, 0.5)
    assert 0 < kinds.sum() < kinds.size


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_known_variances(pf, orc, prec):
    kinds = _run(pf, orc, 5000, 40, 1, prec, 0.5, known_variances=True, sigma2=1.0, tau2=0.1)
    assert 0 < kinds.sum() < kinds.size


@pytest.mark.parametrize("prec", [0, 1])
def test_never_and_always(pf, orc, prec):
    """ess_frac far below 1/n never resamples; ess_frac = 1 always does."""
    assert not _run(pf, orc, 4000, 12, 1, prec, 1e-9).any()
    assert _run(pf, orc, 4000, 12, 0, prec, 1.0).all()


@pytest.mark.parametrize("n", [1, 2, 3, 37])
def test_adaptive_tiny(pf, orc, n):
    _run(pf, orc, n, 10, 0, 0, 0.7)
    _run(pf, orc, n, 10, 1, 1, 0.7)


def test_adaptive_at_scale(pf, orc):
    """2^20 particles, FP32, systematic; and 2,600,003 with outlying
    observations (heavy weights)."""
    _run(pf, orc, 1 << 20, 4, 1, 0, 0.5, seed=1639, every_step=False)
    y = np.array([0.3, 9.0, 9.2, 0.1])
    _run(pf, orc, 2_600_003, 4, 1, 0, 0.3, y=y, seed=5)


def test_adaptive_ticketed_propagation(pf, orc):
    """4,194,305 particles, FP32: the adaptive propagation hands its slots
    out by ticket (and carries the log-weights of the cycles that do not
    resample); systematic through the staged cooperative kernel, and
    stratified through the general path."""
    y = np.array([0.3, 0.5, 7.5, 7.9, 0.2])
    kinds = _run(pf, orc, 4_194_305, 5, 1, 0, 0.6, y=y, seed=17)
    assert kinds.any() and not kinds.all()
    _run(pf, orc, 4_194_305, 3, 4, 0, 0.6, seed=18, every_step=False)


def test_ess_one_equals_always_resampling_filter(pf):
    """At ess_frac = 1 every cycle resamples: the adaptive filter's particles
    and log marginal likelihood equal those of the plain filter (the
    cooperative systematic kernel) bit for bit; its weighted summaries (all
    weights 1) agree within the binary32 rounding of the unweighted sums."""
    _, y = synth.local_level_series(62, 20)
    a = pf.Filter(1 << 16, seed=62)
    b = pf.Filter(1 << 16, seed=62, ess_frac=1.0)
    a.run(y)
    b.run(y)
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert torch.equal(pa[k], pb[k]), k
    ea, eb = a.estimate(), b.estimate()
    assert ea["log_marglik"] == eb["log_marglik"]
    for k in ("x_mean", "sigma2_mean", "tau2_mean"):
        assert abs(ea[k] - eb[k]) <= 1e-5 * max(1.0, abs(ea[k])), k


def test_adaptive_checkpoint_resume(pf):
    """The carried weights and their sum travel in the checkpoint."""
    _, y = synth.local_level_series(63, 16)
    a = pf.Filter(6000, seed=63, ess_frac=0.6, precision="fp64")
    a.run(y[:9])
    b = pf.Filter.restore(a.checkpoint())
    assert b.estimate() == a.estimate()
    a.run(y[9:])
    b.run(y[9:])
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert torch.equal(pa[k], pb[k]), k
    assert a.estimate() == b.estimate()


def test_adaptive_config_errors(pf):
    with pytest.raises(pf.PfError) as e:
        pf.Filter(100, ess_frac=1.5)
    assert e.value.status == pf.PF_ERR_INVALID
    with pytest.raises(pf.PfError):
        pf.Filter(100, ess_frac=-0.1)
    with pytest.raises(pf.PfError):
        pf.Filter(100, ess_frac=0.5, algorithm="bootstrap", known_variances=True)
    f = pf.Filter(1000, ess_frac=0.5)
    f.step_ahead(0.1, 0.2)  # adaptive filters do not fuse: a plain cycle
    f.step(0.2)
    assert f.estimate()["t"] == 2
