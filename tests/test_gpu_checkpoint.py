"""Checkpoint and resume (pf_checkpoint / pf_restore).

A filter restored from a checkpoint taken after t cycles draws the same
Philox counters from cycle t on, so it must continue bit for bit as the
original filter does: ancestors, every particle and every summary equal.  One
case also checks the resumed filter against the CPU oracle run without a
break.
"""
import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu


def _same(a, b):
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert torch.equal(pa[k], pb[k]), k
    assert torch.equal(a.ancestors(), b.ancestors())
    assert a.estimate() == b.estimate()


@pytest.mark.parametrize("scheme,prec,kw", [
    ("systematic", "fp32", {}),
    ("multinomial", "fp64", {}),
    ("stratified", "fp32", {}),
    ("multinomial_cutpoint", "fp32", {}),
    ("systematic", "fp64", dict(known_variances=True, sigma2=1.0, tau2=0.1)),
    ("systematic", "fp32", dict(known_variances=True, sigma2=0.8, tau2=0.15, algorithm="bootstrap")),
])
@pytest.mark.parametrize("device", [False, True])
def test_resume_continues_bit_for_bit(pf, scheme, prec, kw, device):
    _, y = synth.local_level_series(21, 17)
    a = pf.Filter(6001, seed=21, scheme=scheme, precision=prec, **kw)
    a.run(y[:10])
    ck = a.checkpoint(device=device)
    b = pf.Filter.restore(ck)
    assert b.estimate()["t"] == 10
    assert b.estimate() == a.estimate()
    for v in y[10:]:
        a.step(v)
        b.step(v)
    _same(a, b)
    # a second restore from the same blob is independent of the first
    c = pf.Filter.restore(ck)
    c.run(y[10:])
    _same(a, c)


def test_resumed_filter_matches_uninterrupted_oracle(pf, orc):
    """Checkpoint at t = 12 of 20 (2^20 particles, FP32, systematic, several
    CDF tiles); the restored filter ends on the oracle's particles bit for bit."""
    n, T = 1 << 20, 20
    _, y = synth.local_level_series(1639, T)
    a = pf.Filter(n, seed=1639)
    a.run(y[:12])
    ck = a.checkpoint()
    a.close()
    b = pf.Filter.restore(ck)
    b.run(y[12:])
    o = orc.Filter(orc.make_config(n, seed=1639, scheme=1, precision=0))
    for v in y:
        o.step(v)
    p = {k: v.cpu().numpy() for k, v in b.particles().items()}
    r = o.state_raw()
    for k in ("x", "sigma2", "tau2"):
        assert np.array_equal(p[k], r[k]), k
    for k in ("b_sigma", "b_tau"):
        assert np.array_equal(p[k].view(np.uint64), r[k]), k
    assert np.array_equal(b.ancestors().cpu().numpy().view(np.uint32), o.ancestors())
    eo = o.estimate()
    assert abs(b.estimate()["log_marglik"] - eo["log_marglik"]) <= 1e-5 * abs(eo["log_marglik"])


def test_checkpoint_at_start_equals_fresh_filter(pf):
    _, y = synth.local_level_series(22, 5)
    a = pf.Filter(3000, seed=22)
    b = pf.Filter.restore(a.checkpoint())
    a.run(y)
    b.run(y)
    _same(a, b)


def test_bad_checkpoints_are_refused(pf):
    a = pf.Filter(1000, seed=23)
    a.step(0.2)
    ck = a.checkpoint()
    bad = ck.copy()
    bad[0] ^= 0xFF  # magic
    with pytest.raises(pf.PfError) as e:
        pf.Filter.restore(bad)
    assert e.value.status == pf.PF_ERR_INVALID
    bad = ck.copy()
    bad[8] = 99  # format version
    with pytest.raises(pf.PfError):
        pf.Filter.restore(bad)
    with pytest.raises(pf.PfError):
        pf.Filter.restore(ck[:-1])  # truncated
    with pytest.raises(pf.PfError):
        pf.Filter.restore(ck[:100])  # shorter than the header
    b = pf.Filter.restore(ck)  # the original still works
    assert b.estimate() == a.estimate()


def test_checkpoint_refused_while_announcement_pending(pf):
    f = pf.Filter(2000, seed=24)
    f.step_ahead(0.1, 0.3)
    with pytest.raises(pf.PfError) as e:
        f.checkpoint()
    assert e.value.status == pf.PF_ERR_INVALID
    f.step(0.3)
    g = pf.Filter.restore(f.checkpoint())
    assert g.estimate() == f.estimate()


def test_checkpoint_of_failed_filter_reports_its_error(pf):
    f = pf.Filter(1000, seed=25)
    f.step(float("nan"))
    with pytest.raises(pf.PfError) as e:
        f.checkpoint()
    assert e.value.status == pf.PF_ERR_NUMERIC
