"""The cycle at the single-filter target size (2^24 particles, the launch
configuration the benchmark times) against the oracle, and at the maximum
size PF_MAX_PARTICLES = 2^26 through properties that hold at any size.

At 2^26 the oracle's cycle would take minutes, so the checks are exact
properties of the returned CDF Q and ancestors a: the CDF is the inclusive
sum of nonnegative quantised weights; ancestors are nondecreasing and in
range; systematic resampling gives every particle c_i = #{j : a_j = i} in
{floor(n W_i / T), ceil(n W_i / T)} (with sum n); multinomial ancestors only
land on particles of nonzero weight.  The state must stay finite with
positive variances, and the summaries finite.
"""
import numpy as np
import pytest

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu


def test_cycle_2p24_matches_oracle(pf, orc):
    """Two cycles at 2^24 (FP32, systematic: the cooperative CDF kernel with
    several TMA-staged tiles per CTA): ancestors and every particle bit for
    bit."""
    n = 1 << 24
    _, y = synth.local_level_series(1639, 2)
    g = pf.Filter(n, seed=24)
    o = orc.Filter(orc.make_config(n, seed=24, scheme=1, precision=0))
    for v in y:
        g.step(v)
        o.step(v)
        assert np.array_equal(g.ancestors().cpu().numpy().view(np.uint32), o.ancestors())
    p = {k: v.cpu().numpy() for k, v in g.particles().items()}
    r = o.state_raw()
    for k in ("x", "sigma2", "tau2"):
        assert np.array_equal(p[k], r[k]), k
    for k in ("b_sigma", "b_tau"):
        assert np.array_equal(p[k].view(np.uint64), r[k]), k
    eo = o.estimate()
    assert abs(g.estimate()["log_marglik"] - eo["log_marglik"]) <= 1e-5 * abs(eo["log_marglik"])
    g.close()


def _check_cycle(g, n, scheme):
    anc, Q = g.ancestors(with_cdf=True)
    a = anc.cpu().numpy().view(np.uint32)
    q = Q.cpu().numpy().view(np.uint64)
    W = np.diff(q, prepend=np.uint64(0))
    assert np.all(q[1:] >= q[:-1])  # nonnegative weights, no wrap-around
    T = int(q[-1])
    assert T > 0 and T <= (1 << 61)
    assert np.all(np.diff(a.astype(np.int64)) >= 0) and int(a[-1]) < n
    c = np.bincount(a, minlength=n)
    assert c.sum() == n
    if scheme == "systematic":
        nw = W * np.uint64(n)  # n W_i <= 2^26 * 2^35
        lo = nw // np.uint64(T)
        hi = lo + (nw % np.uint64(T) != 0)
        assert np.all((c >= lo) & (c <= hi))
    else:
        assert np.all(W[c > 0] > 0)


@pytest.mark.parametrize("scheme", ["systematic", "multinomial"])
def test_cycle_at_maximum_size(pf, scheme):
    n = pf.MAX_PARTICLES
    _, y = synth.local_level_series(26, 3)
    g = pf.Filter(n, seed=26, scheme=scheme)
    for v in y:
        g.step(v)
        _check_cycle(g, n, scheme)
    p = g.particles()
    for k in ("x", "sigma2", "tau2"):
        assert bool(p[k].isfinite().all()), k
    assert bool((p["sigma2"] > 0).all()) and bool((p["tau2"] > 0).all())
    e = g.estimate()
    assert e["t"] == 3
    assert all(np.isfinite(v) for v in e.values())
    g.close()
