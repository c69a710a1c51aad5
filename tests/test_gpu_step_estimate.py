"""pf_step_estimate: one cycle and its summaries as one captured graph must
give exactly what pf_step followed by pf_estimate gives, step by step, for
every filter form; an announced observation (pf_step_ahead) and a failing
cycle are handled as the two calls would."""
import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu

FORMS = [
    dict(scheme="systematic", precision="fp32"),
    dict(scheme="multinomial", precision="fp64"),
    dict(scheme="stratified", precision="fp32", ess_frac=0.5),
    dict(scheme="systematic", precision="fp32", known_variances=True, sigma2=0.8, tau2=0.15,
         algorithm="bootstrap"),
    dict(scheme="systematic_cutpoint", precision="fp64", known_variances=True),
]


@pytest.mark.parametrize("kw", FORMS)
def test_step_estimate_equals_step_then_estimate(pf, kw):
    _, y = synth.local_level_series(81, 12)
    a = pf.Filter(20_001, seed=81, **kw)
    b = pf.Filter(20_001, seed=81, **kw)
    for v in y:
        a.step(v)
        ea = a.estimate()
        eb = b.step_estimate(v)
        assert ea == eb
    pa, pb = a.particles(), b.particles()
    for k in pa:
        assert torch.equal(pa[k], pb[k]), k


def test_step_estimate_after_announcement(pf):
    _, y = synth.local_level_series(82, 4)
    a = pf.Filter(5000, seed=82)
    b = pf.Filter(5000, seed=82)
    a.step_ahead(y[0], y[1])
    b.step(y[0])
    ea = a.step_estimate(y[1])  # the announced cycle, then the summaries
    b.step(y[1])
    assert ea == b.estimate()
    assert a.step_estimate(y[2]) == b.step_estimate(y[2])


def test_step_estimate_reports_failure(pf):
    f = pf.Filter(1000, seed=83)
    f.step_estimate(0.2)
    with pytest.raises(pf.PfError) as e:
        f.step_estimate(float("nan"))
    assert e.value.status == pf.PF_ERR_NUMERIC
    with pytest.raises(pf.PfError):
        f.step(0.1)  # sticky
