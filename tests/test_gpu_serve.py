"""Serving (pf_server_*): continuous batching of filter streams.

Every observation's result (the stream's posterior summaries after it) must
be exactly what a standalone filter of the stream's configuration gives
after the same observations, whatever the interleaving with other streams,
the composition of the batched cycles, the number of cycles in flight, or
the time a stream waited for admission under the HBM budget.
"""
import time

import numpy as np
import pytest

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu


def _cfg(i, n):
    return dict(n=n, seed=9000 + 31 * i, filter_id=100 + i)


def _alone(pf, cfg, ys):
    f = pf.Filter(cfg["n"], seed=cfg["seed"], filter_id=cfg["filter_id"], scheme="systematic",
                  precision="fp32", ess_frac=cfg.get("ess_frac", 0.0))
    out = []
    for y in ys:
        f.step(y)
        out.append(f.estimate())
    f.close()
    return out


def _check_against_alone(pf, results, cfgs, series):
    by = {}
    for sid, seq, est, lat, status in results:
        assert status == pf.PF_OK
        assert lat > 0
        by.setdefault(sid, {})[seq] = est
    for sid, cfg in cfgs.items():
        ys = series[sid]
        got = by.get(sid, {})
        assert sorted(got) == list(range(len(ys))), sid
        ref = _alone(pf, cfg, ys)
        for k in range(len(ys)):
            assert got[k] == ref[k], (sid, k)


def _bytes_per_particle(pf):
    b = pf.Batch([dict(n=32, seed=1, filter_id=0)], max_filters=1)
    v = b.info()["bytes_per_particle"]
    b.close()
    return v


@pytest.mark.parametrize("inflight", [1, 3])
def test_served_results_equal_alone_results(pf, inflight):
    sizes = {11: 1, 22: 300, 33: 4099, 44: 20000, 55: 140001, 66: 7000, 77: 2}
    cfgs = {sid: _cfg(k, n) for k, (sid, n) in enumerate(sizes.items())}
    rng = np.random.default_rng(inflight)
    series = {sid: synth.local_level_series(sid, int(rng.integers(3, 9)), filter_id=sid)[1]
              for sid in sizes}
    srv = pf.Server(max_streams=16, hbm_budget_bytes=1 << 30, max_inflight=inflight,
                    keep_results=True)
    for sid, c in cfgs.items():
        srv.open(sid, **c)
    todo = [(sid, k) for sid, ys in series.items() for k in range(len(ys))]
    # interleave the streams randomly, each stream's observations in order
    nxt = {sid: 0 for sid in series}
    order = rng.permutation(len(todo))
    for i in order:
        sid = todo[i][0]
        srv.submit(sid, series[sid][nxt[sid]])
        nxt[sid] += 1
        if rng.random() < 0.3:
            time.sleep(0.002)  # let cycles of different compositions form
    for sid in series:
        srv.close_stream(sid)
    srv.drain(120)
    st = srv.stats()
    n_obs = sum(len(v) for v in series.values())
    assert st["submitted"] == st["completed"] == n_obs
    assert st["streams_closed"] == len(series) and st["resident"] == 0
    assert st["cycles"] >= max(len(v) for v in series.values())
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    _check_against_alone(pf, srv.poll(), cfgs, series)
    srv.close()


def test_served_results_match_the_oracle(pf, orc):
    """Served results against the CPU oracle directly (not through a
    standalone GPU filter): each observation's summaries within the parity
    tolerance (1e-5 relative, or of the posterior sd near zero) of the
    oracle's after the same observations, streams interleaved in the server."""
    sizes = {5: 1, 6: 777, 7: 4099, 8: 70001}
    cfgs = {sid: _cfg(sid, n) for sid, n in sizes.items()}
    series = {sid: synth.local_level_series(200 + sid, 5, filter_id=sid)[1] for sid in sizes}
    srv = pf.Server(max_streams=8, hbm_budget_bytes=1 << 30, max_inflight=2, keep_results=True)
    for sid, c in cfgs.items():
        srv.open(sid, **c)
    for k in range(5):
        for sid in sizes:
            srv.submit(sid, series[sid][k])
    for sid in sizes:
        srv.close_stream(sid)
    srv.drain(120)
    by = {}
    for sid, seq, est, lat, status in srv.poll():
        assert status == pf.PF_OK
        by.setdefault(sid, {})[seq] = est
    srv.close()
    tol = 1e-5
    for sid, c in cfgs.items():
        o = orc.Filter(orc.make_config(c["n"], seed=c["seed"], filter_id=c["filter_id"],
                                       scheme=orc.SYSTEMATIC, precision=orc.FP32))
        for k, y in enumerate(series[sid]):
            o.step(y)
            eo, eg = o.estimate(), by[sid][k]
            assert eg["t"] == eo["t"] == k + 1
            for m, v in (("x", "x_var"), ("sigma2", "sigma2_var"), ("tau2", "tau2_var")):
                sd = np.sqrt(max(eo[v], 0.0))
                assert abs(eg[m + "_mean"] - eo[m + "_mean"]) <= tol * max(abs(eo[m + "_mean"]), sd), (sid, k, m)
                assert abs(eg[v] - eo[v]) <= 10 * tol * abs(eo[v]) + 8e-16 * eo[m + "_mean"] ** 2, (sid, k, v)
            assert abs(eg["log_marglik"] - eo["log_marglik"]) <= tol * max(1.0, abs(eo["log_marglik"]))
        o.close()


def test_served_adaptive_streams(pf):
    """A server created for adaptive resampling: streams with ess_frac > 0
    beside plain ones, interleaved, two cycles in flight; every result equals
    a standalone filter's of the same configuration."""
    sizes = {1: 3000, 2: 70001, 3: 512, 4: 20000, 5: 9}
    cfgs = {sid: dict(_cfg(sid, n), ess_frac=(0.5 if sid % 2 else 0.0)) for sid, n in sizes.items()}
    series = {sid: synth.local_level_series(90 + sid, 8, filter_id=sid)[1] for sid in sizes}
    for sid in sizes:
        series[sid][3] += 10.0
    srv = pf.Server(max_streams=8, hbm_budget_bytes=1 << 30, max_inflight=2, keep_results=True,
                    adaptive=True)
    for sid, c in cfgs.items():
        srv.open(sid, **c)
    for k in range(8):
        for sid in sizes:
            srv.submit(sid, series[sid][k])
    for sid in sizes:
        srv.close_stream(sid)
    srv.drain(120)
    _check_against_alone(pf, srv.poll(), cfgs, series)
    srv.close()
    plain = pf.Server(max_streams=2, hbm_budget_bytes=1 << 26)
    with pytest.raises(pf.PfError) as e:
        plain.open(1, **dict(_cfg(1, 100), ess_frac=0.5))
    assert e.value.status == pf.PF_ERR_INVALID
    plain.close()


def test_admission_waits_for_budget_and_results_stay_exact(pf):
    """A budget of 25,000 particles: streams that do not fit wait in FIFO
    order and enter as earlier streams close."""
    per = _bytes_per_particle(pf)
    sizes = {1: 20000, 2: 9000, 3: 9000, 4: 15000, 5: 3000, 6: 20000}
    cfgs = {sid: _cfg(sid, n) for sid, n in sizes.items()}
    series = {sid: synth.local_level_series(50 + sid, 4, filter_id=sid)[1] for sid in sizes}
    srv = pf.Server(max_streams=4, hbm_budget_bytes=per * 25000, keep_results=True)
    with pytest.raises(pf.PfError) as e:
        srv.open(99, **_cfg(99, 40000))          # can never fit
    assert e.value.status == pf.PF_ERR_BUSY
    for sid, c in cfgs.items():
        srv.open(sid, **c)
        for y in series[sid]:
            srv.submit(sid, y)
        srv.close_stream(sid)
    srv.drain(120)
    st = srv.stats()
    assert st["admitted"] == len(sizes) and st["streams_closed"] == len(sizes)
    assert st["completed"] == sum(len(v) for v in series.values())
    assert st["used_particles"] == 0 and st["waiting"] == 0
    _check_against_alone(pf, srv.poll(), cfgs, series)
    srv.close()


def test_replayed_poisson_load(pf):
    """The library's replay thread drives Poisson arrivals (open, observations,
    close); every observation completes and the latency percentiles are
    ordered."""
    n_streams, dur, rate = 6, 0.5, 40.0
    sizes = [512, 3000, 131072, 700, 20000, 5000]
    cfgs = [_cfg(i, n) for i, n in enumerate(sizes)]
    arr = synth.poisson_arrivals(rate, n_streams, dur, seed=3)
    series = {i: synth.local_level_series(700 + i, len(a), filter_id=i)[1] for i, a in enumerate(arr)}
    ev = [(0.0, pf.EVENT_OPEN, i, 0.0) for i in range(n_streams)]
    for i, a in enumerate(arr):
        ev += [(float(t), pf.EVENT_OBS, i, float(series[i][k])) for k, t in enumerate(a)]
        ev.append((dur + 0.01, pf.EVENT_CLOSE, i, 0.0))
    ev.sort(key=lambda e: (e[0], e[1] != pf.EVENT_OPEN))
    t, kind, ids, y = (np.array(c) for c in zip(*ev))
    srv = pf.Server(max_streams=8, hbm_budget_bytes=1 << 30, keep_results=True)
    srv.replay(t, kind, ids, y, cfgs)
    srv.drain(120)
    st = srv.stats()
    assert st["submitted"] == st["completed"] == sum(len(a) for a in arr)
    assert 0 < st["p50_us"] <= st["p90_us"] <= st["p99_us"] <= st["max_us"]
    assert st["obs_per_s"] > 0 and st["particle_steps"] == sum(
        len(a) * n for a, n in zip(arr, sizes))
    _check_against_alone(pf, srv.poll(), {i: c for i, c in enumerate(cfgs)}, series)
    srv.close()


def test_served_at_full_size_sampled_streams_equal_alone(pf):
    """The served workload's streams: 10,000 of them, N log-uniform in
    [512, 131072] (about 2.35e8 particles), in the benchmark's launch
    configuration (120 GB budget, clusters of 8 for streams of at least
    16,384 particles, two cycles in flight).  Three observations each,
    submitted round-robin; sampled streams (the smallest, the largest and six
    others) give exactly a standalone filter's summaries after each."""
    n_streams, seed, T = 10000, 10000, 3
    ns, s2, t2 = synth.batch_specs(n_streams, seed, 512, 131072)
    series = [synth.local_level_series(seed + i, T, sigma2=s2[i], tau2=t2[i], filter_id=i)[1]
              for i in range(n_streams)]
    srv = pf.Server(max_streams=n_streams, hbm_budget_bytes=int(120e9), scheme="systematic",
                    precision="fp32", max_inflight=2, cluster=8, big_min=16384,
                    keep_results=True)
    cfgs = {i: dict(n=int(ns[i]), seed=seed + i, filter_id=i) for i in range(n_streams)}
    for i, c in cfgs.items():
        srv.open(i, **c)
    for k in range(T):
        for i in range(n_streams):
            srv.submit(i, series[i][k])
    for i in range(n_streams):
        srv.close_stream(i)
    srv.drain(600)
    st = srv.stats()
    assert st["completed"] == n_streams * T
    rng = np.random.default_rng(3)
    pick = sorted({int(np.argmin(ns)), int(np.argmax(ns))} |
                  set(int(i) for i in rng.choice(n_streams, 6, replace=False)))
    results = []
    while True:
        r = srv.poll()
        if not r:
            break
        results.extend(r)
    res = [r for r in results if r[0] in set(pick)]
    _check_against_alone(pf, res, {i: cfgs[i] for i in pick}, {i: series[i] for i in pick})
    srv.close()
