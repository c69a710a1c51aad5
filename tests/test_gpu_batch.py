"""Batched filters (pf_batch_*): parity with the CPU oracle and with standalone
filters.

A filter stepped inside a batch must give exactly what the oracle gives
(ancestors at every step and the final particles bit for bit; summaries within
the oracle tolerance) and exactly what a standalone pf_create filter of the
same configuration gives (everything bit for bit, summaries and log-ML
included), whatever the other filters of the batch are doing: different
sizes, seeds, observation series, masks, admission and removal.
"""
import numpy as np
import pytest

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-12}
PREC = {0: "fp32", 1: "fp64"}


def _spec(i, n, **kw):
    d = dict(n=n, seed=100 + 17 * i, filter_id=3 + 7 * i)
    d.update(kw)
    return d


def _series(i, T):
    return synth.local_level_series(500 + i, T, filter_id=i)[1]


def _oracle(orc, spec, scheme, prec):
    kw = {k: v for k, v in spec.items() if k not in ("n", "seed", "filter_id")}
    return orc.Filter(orc.make_config(spec["n"], seed=spec["seed"], filter_id=spec["filter_id"],
                                      scheme=scheme, precision=prec, **kw))


def _standalone(pf, spec, scheme, prec):
    kw = {k: v for k, v in spec.items() if k != "n"}
    return pf.Filter(spec["n"], scheme=scheme, precision=PREC[prec], **kw)


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _raw(p, prec):
    out = {k: v.cpu().numpy() for k, v in p.items()}
    if prec == 0:
        for k in ("b_sigma", "b_tau"):
            out[k] = out[k].view(np.uint64)
    return out


def _same_particles(a, b):
    for k in ("x", "sigma2", "tau2", "b_sigma", "b_tau"):
        assert np.array_equal(a[k], b[k]), (k, np.flatnonzero(a[k] != b[k])[:5])


def _close_to_oracle(eg, eo, prec):
    tol = TOL[prec]
    assert eg["t"] == eo["t"]
    eps = np.finfo(np.float64).eps
    for k, v in (("x", "x_var"), ("sigma2", "sigma2_var"), ("tau2", "tau2_var")):
        sd = np.sqrt(max(eo[v], 0.0))
        assert abs(eg[k + "_mean"] - eo[k + "_mean"]) <= tol * max(abs(eo[k + "_mean"]), sd), k
        assert abs(eg[v] - eo[v]) <= 10 * tol * abs(eo[v]) + 8 * eps * eo[k + "_mean"] ** 2, v
    assert abs(eg["log_marglik"] - eo["log_marglik"]) <= tol * max(1.0, abs(eo["log_marglik"]))


SIZES = [1, 5, 257, 4096, 4099, 9000, 140001]  # one particle .. 35 scan tiles, ragged tails


@pytest.mark.parametrize("scheme,prec", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_batch_matches_oracle_and_standalone(pf, orc, scheme, prec):
    T = 6
    specs = [_spec(i, n) for i, n in enumerate(SIZES)]
    ys = [_series(i, T) for i in range(len(specs))]
    b = pf.Batch(specs, scheme=scheme, precision=PREC[prec])
    alone = [_standalone(pf, s, scheme, prec) for s in specs]
    orcs = [_oracle(orc, s, scheme, prec) for s in specs]
    y = np.zeros(b.max_filters)
    for t in range(T):
        for i in range(len(specs)):
            y[i] = ys[i][t]
            alone[i].step(ys[i][t])
            orcs[i].step(ys[i][t])
        b.step(y)
        for i in range(len(specs)):
            got = _u32(b.ancestors(i))
            assert np.array_equal(got, orcs[i].ancestors()), (t, i)
            assert np.array_equal(got, _u32(alone[i].ancestors())), (t, i)
    est = b.estimates()
    for i, s in enumerate(specs):
        pb = _raw(b.particles(i), prec)
        _same_particles(pb, _raw(alone[i].particles(), prec))
        _same_particles(pb, orcs[i].state_raw())
        assert est[i] == alone[i].estimate(), i       # bit for bit, log-ML included
        _close_to_oracle(est[i], orcs[i].estimate(), prec)
        alone[i].close()
        orcs[i].close()
    b.close()


def test_batch_masks_known_variances_and_outliers(pf):
    """Filters step on their own schedules (masks), some with known
    variances; an outlying observation concentrates the weights on a few
    particles (long runs of equal ancestors).  Each filter must equal a
    standalone filter that saw only its own steps."""
    T = 10
    sizes = [3000, 70000, 33, 4096, 12345, 2]
    specs = [_spec(i, n, known_variances=(i % 3 == 1), sigma2=0.7, tau2=0.2)
             for i, n in enumerate(sizes)]
    b = pf.Batch(specs, scheme="systematic", precision="fp32", max_filters=8)
    alone = [_standalone(pf, s, 1, 0) for s in specs]
    rng = np.random.default_rng(7)
    ys = [_series(i, T) for i in range(len(specs))]
    pos = [0] * len(specs)
    for t in range(T):
        mask = np.zeros(b.max_filters, np.uint8)
        mask[:len(specs)] = rng.integers(0, 2, len(specs))
        if t == 0:
            mask[:len(specs)] = 1
        y = np.zeros(b.max_filters)
        for i in range(len(specs)):
            if mask[i]:
                v = ys[i][pos[i]] + (25.0 if (t == 3 and i == 1) else 0.0)
                y[i] = v
                alone[i].step(v)
                pos[i] += 1
        b.step(y, mask)
    est = b.estimates()
    for i in range(len(specs)):
        assert est[i]["t"] == pos[i]
        assert est[i] == alone[i].estimate(), i
        _same_particles(_raw(b.particles(i), 0), _raw(alone[i].particles(), 0))
        assert np.array_equal(_u32(b.ancestors(i)), _u32(alone[i].ancestors()))
        alone[i].close()
    b.close()


def test_batch_admission_by_budget_and_slot_reuse(pf):
    """Admission under an HBM budget: filters are refused (PF_ERR_BUSY) when
    the pool or the slots are full, admitted again once a filter leaves, and
    a filter admitted into a reused range equals a fresh standalone one."""
    per = pf.Batch([_spec(0, 32)], max_filters=1).info()["bytes_per_particle"]
    budget = per * 20000
    b = pf.Batch([], max_filters=3, hbm_budget_bytes=budget)
    info = b.info()
    assert info["pool_particles"] == 20000 // 32 * 32 and info["resident"] == 0
    s0 = b.add(**_spec(0, 9000))
    s1 = b.add(**_spec(1, 9000))
    assert (s0, s1) == (0, 1)
    assert b.try_add(**_spec(2, 9000)) is None          # pool full
    s2 = b.add(**_spec(3, 1000))
    assert s2 == 2
    with pytest.raises(pf.PfError) as e:
        b.add(**_spec(4, 32))                            # slots full
    assert e.value.status == pf.PF_ERR_BUSY
    y = np.zeros(3)
    for t in range(3):
        y[:] = [0.1 * t, -0.2 * t, 0.3]
        b.step(y)
    b.remove(s0)
    s3 = b.add(**_spec(5, 8000))                         # into the freed range
    assert s3 == 0 and b.info()["resident"] == 3
    ref = _standalone(pf, _spec(5, 8000), 1, 0)
    for t in range(4):
        y[:] = [0.5 - t, 0.0, 0.0]
        ref.step(y[0])
        b.step(y, np.array([1, 0, 1], np.uint8))
    assert b.estimates()[0] == ref.estimate()
    _same_particles(_raw(b.particles(0), 0), _raw(ref.particles(), 0))
    ref.close()
    b.close()


def test_batch_rejects_bad_configs(pf):
    with pytest.raises(pf.PfError) as e:
        pf.Batch([_spec(0, 100), _spec(1, 0)])
    assert e.value.status == pf.PF_ERR_INVALID
    with pytest.raises(pf.PfError) as e:
        pf.Batch([_spec(0, 100)], hbm_budget_bytes=1000)
    assert e.value.status == pf.PF_ERR_BUSY
    b = pf.Batch([_spec(0, 100)], max_filters=2)
    with pytest.raises(pf.PfError) as e:
        b.remove(1)
    assert e.value.status == pf.PF_ERR_INVALID
    b.close()


@pytest.mark.parametrize("scheme", ["systematic", "multinomial"])
def test_batch_launch_shapes_change_no_result(pf, scheme):
    """The autotuner's trial cycles commit nothing, and every candidate launch
    shape (256 or 512 threads, 1 .. max CTAs) gives the same bits."""
    sizes = [70000, 9000, 4099, 300, 1, 20000, 5000, 140001]
    specs = [_spec(i, n) for i, n in enumerate(sizes)]
    T = 3
    ys = [_series(i, T) for i in range(len(specs))]
    tuned = pf.Batch(specs, scheme=scheme, autotune=True)
    ref = pf.Batch(specs, scheme=scheme)
    shapes, chosen = ref.tune(np.array([y[0] for y in ys]))
    assert len(shapes) >= 2 and 0 <= chosen < len(shapes)
    assert {sh["block"] for sh in shapes} == {256, 512}
    assert {sh["cluster"] for sh in shapes} >= {1, 2, 4, 8}
    assert all(sh["ms"] > 0 for sh in shapes)
    others = []
    for sh in shapes:
        o = pf.Batch(specs, scheme=scheme)
        cl = sh["cluster"]
        grid = max(cl, sh["grid"] // 7 // cl * cl)  # fewer CTAs than filters, too
        o.set_shape(sh["block"], grid, cl, sh["big_min"])
        others.append(o)
    # clusters taking every filter of 1 or more particles, and filters of
    # fewer tiles than CTAs in the cluster
    for cl in (2, 8):
        o = pf.Batch(specs, scheme=scheme)
        o.set_shape(256, cl * 3, cl, 1)
        others.append(o)
    for t in range(T):
        y = np.array([ys[i][t] for i in range(len(specs))])
        for b in [tuned, ref] + others:
            b.step(y)
    assert tuned.info()["tuned"] == 1
    est = ref.estimates()
    for b in [tuned] + others:
        assert b.estimates() == est
        for i in range(len(specs)):
            _same_particles(_raw(b.particles(i), 0), _raw(ref.particles(i), 0))
        b.close()
    ref.close()


ESS = [0.5, 0.0, 0.9, 0.3, 1e-9, 0.5, 0.7]  # per filter of SIZES: adaptive next to plain


@pytest.mark.parametrize("scheme,prec", [(1, 0), (0, 0), (1, 1)])
def test_batch_adaptive_matches_oracle_and_standalone(pf, orc, scheme, prec):
    """Adaptive resampling per filter (ess_frac > 0) in an adaptive batch,
    beside plain filters: each filter's ancestors at every cycle (the
    identity when it does not resample) equal the oracle's and a standalone
    filter's, its particles equal both bit for bit, its summaries and log-ML
    equal the standalone filter's bit for bit and the oracle's within the
    tolerance.  An outlying observation at cycle 4 makes every adaptive filter
    resample there; both branches occur."""
    T = 12
    specs = [_spec(i, n, ess_frac=e) for i, (n, e) in enumerate(zip(SIZES, ESS))]
    ys = [_series(i, T) for i in range(len(specs))]
    for y in ys:
        y[4] += 12.0
    b = pf.Batch(specs, scheme=scheme, precision=PREC[prec], adaptive=True)
    alone = [_standalone(pf, s, scheme, prec) for s in specs]
    orcs = [_oracle(orc, s, scheme, prec) for s in specs]
    kinds = np.zeros((T, len(specs)), bool)
    y = np.zeros(b.max_filters)
    for t in range(T):
        for i in range(len(specs)):
            y[i] = ys[i][t]
            alone[i].step(ys[i][t])
            orcs[i].step(ys[i][t])
            kinds[t, i] = orcs[i].resampled()
        b.step(y)
        for i in range(len(specs)):
            got = _u32(b.ancestors(i))
            assert np.array_equal(got, orcs[i].ancestors()), (t, i, kinds[t, i])
            assert np.array_equal(got, _u32(alone[i].ancestors())), (t, i)
        if t % 4 == 3:
            est = b.estimates()
            for i in range(len(specs)):
                assert est[i] == alone[i].estimate(), (t, i)
    both = [i for i, e in enumerate(ESS) if 0 < kinds[:, i].sum() < T]
    assert len(both) >= 3, kinds.sum(axis=0)   # adaptive filters that took both branches
    est = b.estimates()
    for i, s in enumerate(specs):
        pb = _raw(b.particles(i), prec)
        _same_particles(pb, _raw(alone[i].particles(), prec))
        _same_particles(pb, orcs[i].state_raw())
        assert est[i] == alone[i].estimate(), i
        _close_to_oracle(est[i], orcs[i].estimate(), prec)
        alone[i].close()
        orcs[i].close()
    b.close()


def test_batch_adaptive_shapes_trials_and_admission(pf):
    """Adaptive filters under clusters (the ESS sums exchanged between the
    CTAs of a cluster), autotuner trial cycles (which must leave the carried
    log-weights alone) and admission into a reused pool range: all equal
    standalone adaptive filters bit for bit.  A plain batch refuses
    ess_frac > 0 and an adaptive batch reports the larger per-particle size."""
    sizes = [140001, 70000, 9000, 4099, 300, 20000]
    specs = [_spec(i, n, ess_frac=0.6 if i % 2 == 0 else 0.4) for i, n in enumerate(sizes)]
    T = 8
    ys = [_series(i, T) for i in range(len(specs))]
    for y in ys:
        y[5] -= 10.0
    plain = pf.Batch([_spec(0, 32)], max_filters=1)
    with pytest.raises(pf.PfError) as e:
        plain.add(**_spec(1, 100, ess_frac=0.5))
    assert e.value.status == pf.PF_ERR_INVALID
    per = plain.info()["bytes_per_particle"]
    plain.close()
    tuned = pf.Batch(specs, adaptive=True, autotune=True)
    assert tuned.info()["bytes_per_particle"] == per + 4
    shaped = []
    for cl in (2, 8):
        o = pf.Batch(specs, adaptive=True)
        o.set_shape(256, cl * 3, cl, 1)
        shaped.append(o)
    alone = [_standalone(pf, s, 1, 0) for s in specs]
    for t in range(T):
        y = np.array([ys[i][t] for i in range(len(specs))])
        for i in range(len(specs)):
            alone[i].step(y[i])
        for bb in [tuned] + shaped:
            bb.step(y)
    assert tuned.info()["tuned"] == 1
    for bb in [tuned] + shaped:
        est = bb.estimates()
        for i in range(len(specs)):
            assert est[i] == alone[i].estimate(), i
            _same_particles(_raw(bb.particles(i), 0), _raw(alone[i].particles(), 0))
        bb.close()
    for a in alone:
        a.close()
    # a filter admitted into a freed range starts from equal weights
    b = pf.Batch([_spec(0, 9000, ess_frac=0.5), _spec(1, 5000)], adaptive=True, max_filters=2)
    y = np.array([0.2, -0.1])
    for t in range(5):
        b.step(y + t)
    b.remove(0)
    s = b.add(**_spec(2, 8000, ess_frac=0.5))
    ref = _standalone(pf, _spec(2, 8000, ess_frac=0.5), 1, 0)
    for t in range(6):
        v = 0.3 * t - (9.0 if t == 2 else 0.0)
        ref.step(v)
        b.step(np.array([v, 0.0]), np.array([1, 0], np.uint8))
    assert b.estimates()[s] == ref.estimate()
    _same_particles(_raw(b.particles(s), 0), _raw(ref.particles(), 0))
    ref.close()
    b.close()


def test_batch_at_full_size_matches_oracle_on_sampled_filters(pf, orc):
    """The benchmark's batch: 4096 filters, N log-uniform in [256, 65536]
    (about 4.7e7 particles), each with its own series from prior-drawn
    variances, FP32, systematic, the autotuned launch shape.  After three
    cycles, sampled filters (the smallest, the largest and six others) equal
    the oracle bit for bit: ancestors of the last cycle and every particle."""
    nf, seed, T = 4096, 4096, 3
    ns, s2, t2 = synth.batch_specs(nf, seed)
    ys = np.stack([synth.local_level_series(seed + i, T + 1, sigma2=s2[i], tau2=t2[i],
                                            filter_id=i)[1] for i in range(nf)], axis=1)
    specs = [dict(n=int(ns[i]), seed=seed + i, filter_id=i) for i in range(nf)]
    b = pf.Batch(specs, scheme="systematic", precision="fp32")
    b.tune(ys[0])  # trial cycles choose the launch shape and change no result
    for t in range(T):
        b.step(ys[t])
    rng = np.random.default_rng(7)
    pick = sorted({int(np.argmin(ns)), int(np.argmax(ns))} |
                  set(int(i) for i in rng.choice(nf, 6, replace=False)))
    for i in pick:
        o = orc.Filter(orc.make_config(int(ns[i]), seed=seed + i, filter_id=i, scheme=1,
                                       precision=0))
        for t in range(T):
            o.step(ys[t, i])
        assert np.array_equal(_u32(b.ancestors(i)), o.ancestors()), i
        _same_particles(_raw(b.particles(i), 0), o.state_raw())
        o.close()
    b.close()
