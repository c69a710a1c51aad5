"""GPU parity of the fused cross-cycle weights against the CPU oracle.

When the next observation is known (pf_step_ahead), the propagation of cycle
t also computes the predictive weights of cycle t + 1 and their maximum, and
cycle t + 1 skips the weights kernel.  The
weights are the same IEEE operations on the same values, so every ancestor,
every particle and every summary must equal the oracle's exactly as for the
unfused cycle: ancestors and states bit for bit, summaries within 1e-5 (FP32
state) and 1e-12 (FP64 state) relative to max(|oracle|, posterior sd).
"""
import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}


def _pair(pf, orc, n, scheme, prec, seed, **kw):
    g = pf.Filter(n, seed=seed, scheme=scheme, precision="fp64" if prec else "fp32", **kw)
    o = orc.Filter(orc.make_config(n, seed=seed, scheme=scheme, precision=prec, **kw))
    return g, o


def _check_final(g, o, prec):
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
    assert abs(eg["log_marglik"] - eo["log_marglik"]) <= tol * max(1.0, abs(eo["log_marglik"]))


def _run_ahead(pf, orc, n, T, scheme, prec, seed=1212, y=None, every_step=True, **kw):
    """pf_step_ahead for every observation but the last, ancestors checked."""
    if y is None:
        _, y = synth.local_level_series(seed, T)
    g, o = _pair(pf, orc, n, scheme, prec, seed, **kw)
    for t in range(T):
        if t + 1 < T:
            g.step_ahead(y[t], y[t + 1])
        else:
            g.step(y[t])
        o.step(y[t])
        if every_step or t == T - 1:
            anc = g.ancestors().cpu().numpy().view(np.uint32)
            ref = o.ancestors()
            assert np.array_equal(anc, ref), (t, np.flatnonzero(anc != ref)[:5])
    _check_final(g, o, prec)
    g.close()


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("prec", [0, 1])
def test_step_ahead_all_schemes(pf, orc, scheme, prec):
    """Ragged size over several scan tiles, every scheme, both precisions."""
    _run_ahead(pf, orc, 3 * 4096 + 17, 12, scheme, prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_step_ahead_known_variances(pf, orc, prec):
    _run_ahead(pf, orc, 3000, 15, 1, prec, known_variances=True, sigma2=1.0, tau2=0.1)


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_step_ahead_tiny(pf, orc, n):
    _run_ahead(pf, orc, n, 8, 0, 0)
    _run_ahead(pf, orc, n, 8, 1, 1)


def test_step_ahead_outliers(pf, orc):
    """Outlying next observations: most of the weights computed ahead
    underflow in the next cycle's CDF."""
    y = np.array([0.3, 40.0, 40.5, -3.0, 0.0, 25.0])
    _run_ahead(pf, orc, 4096, y.size, 1, 0, y=y)
    _run_ahead(pf, orc, 4096, y.size, 0, 1, y=y)


def test_step_ahead_at_scale(pf, orc):
    """2^20 particles (one 2048-particle CDF tile per CTA) and 2,600,003
    (several tiles per CTA, TMA-staged), FP32 systematic."""
    _run_ahead(pf, orc, 1 << 20, 3, 1, 0, seed=1639, every_step=False)
    _run_ahead(pf, orc, 2_600_003, 3, 1, 0, seed=7, every_step=True)


def test_step_ahead_ticketed_propagation(pf, orc):
    """4,194,305 particles: at least 16 units of 64 slots per warp, so the
    binary32 propagation (fused and not) hands its slots out by ticket; the
    CDF kernel is TMA-staged.  Systematic (an outlying observation for heavy
    particles), multinomial, and known variances."""
    n = 4_194_305
    y = np.array([0.2, 6.5, 6.8, 0.4])
    _run_ahead(pf, orc, n, 4, 1, 0, y=y, seed=11, every_step=True)
    _run_ahead(pf, orc, n, 3, 0, 0, seed=12, every_step=False)
    _run_ahead(pf, orc, n, 3, 1, 0, seed=13, every_step=False, known_variances=True, sigma2=0.9,
               tau2=0.2)


def test_step_ahead_equals_unfused_cycles(pf):
    """A chain of fused cycles equals the unfused cycles (pf_step, and pf_run
    over host or device-resident observations) bit for bit, every scheme and
    both precisions, summaries included."""
    _, y = synth.local_level_series(8, 25)
    for scheme in ("systematic", "multinomial", "stratified", "multinomial_cutpoint"):
        for prec in ("fp32", "fp64"):
            a = pf.Filter(5000, seed=8, scheme=scheme, precision=prec)
            for t in range(y.size):
                if t + 1 < y.size:
                    a.step_ahead(y[t], y[t + 1])
                else:
                    a.step(y[t])
            b = pf.Filter(5000, seed=8, scheme=scheme, precision=prec)
            b.run(y)
            c = pf.Filter(5000, seed=8, scheme=scheme, precision=prec)
            c.run(torch.from_numpy(y).cuda())
            pa = a.particles()
            for f in (b, c):
                pb = f.particles()
                for k in pa:
                    assert torch.equal(pa[k], pb[k]), (scheme, prec, k)
                assert f.estimate() == a.estimate()


def test_step_ahead_then_profiled_and_estimate(pf, orc):
    """An announced cycle may be run by pf_step_profiled (without weights) or
    pf_step_ahead_profiled (fusing again); estimates in between see the same
    state."""
    _, y = synth.local_level_series(9, 6)
    g, o = _pair(pf, orc, 10_000, 1, 0, 9)
    g.step_ahead(y[0], y[1])
    o.step(y[0])
    ms = g.step_profiled(y[1], y_next=y[2])
    assert "propagate_weights_next" in ms and "weights" not in ms
    o.step(y[1])
    e = g.estimate()
    assert e["t"] == 2
    ms = g.step_profiled(y[2])
    assert "weights" not in ms and "propagate" in ms
    o.step(y[2])
    ms = g.step_profiled(y[3])
    assert "weights" in ms
    o.step(y[3])
    g.step_ahead(y[4], y[5])
    g.step(y[5])
    o.step(y[4])
    o.step(y[5])
    _check_final(g, o, 0)


def test_announced_observation_must_match(pf, orc):
    """After pf_step_ahead(y, y_next) any other observation is refused with
    PF_ERR_INVALID, nothing enqueued and the handle usable."""
    _, y = synth.local_level_series(10, 4)
    g, o = _pair(pf, orc, 4096, 1, 0, 10)
    g.step_ahead(y[0], y[1])
    o.step(y[0])
    with pytest.raises(pf.PfError) as e:
        g.step(y[1] + 1e-9)
    assert e.value.status == pf.PF_ERR_INVALID
    with pytest.raises(pf.PfError):
        g.step_ahead(y[2], y[3])
    with pytest.raises(pf.PfError):
        g.run(torch.from_numpy(y[1:]).cuda())  # device series: cannot be compared
    g.run(y[1:])  # host series starting with the announced value
    for v in y[1:]:
        o.step(v)
    _check_final(g, o, 0)


def test_nan_next_observation_is_sticky_error(pf):
    """A non-finite next observation makes the fused weights non-finite: the
    handle fails with PF_ERR_NUMERIC, as the weights kernel would."""
    f = pf.Filter(1000, seed=1)
    f.step_ahead(0.1, float("nan"))
    with pytest.raises(pf.PfError) as e:
        f.sync()
    assert e.value.status == pf.PF_ERR_NUMERIC
    f.close()


def test_bootstrap_step_ahead_is_step(pf, orc):
    """The bootstrap filter weighs after its own blind propagation: for it
    pf_step_ahead is pf_step."""
    kw = dict(known_variances=True, sigma2=0.8, tau2=0.15, algorithm=1)
    _, y = synth.local_level_series(11, 6)
    g, o = _pair(pf, orc, 3000, 1, 0, 11, **kw)
    for t in range(6):
        if t + 1 < 6:
            g.step_ahead(y[t], y[t + 1])
        else:
            g.step(y[t])
        o.step(y[t])
    _check_final(g, o, 0)
