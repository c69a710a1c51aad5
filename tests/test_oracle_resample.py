"""Pins of the oracle's fixed-point CDF and resampling (paper Section 3).

- Table 1 of the paper (the N = 10 worked example of the parallelized cut-point
  search and cut-point method), from tests/golden/table1_cutpoint.txt.
- The cut-point definition I_j = min{i : q(i) > (j-1)/N} and the properties of
  L_j listed in Section 3.2, by brute force.
- Agreement of the sequential walk, the naive O(N^2) search and the cut-point
  method on the same positions.
- Systematic resampling: offspring counts in {floor(N w_i), ceil(N w_i)} and an
  exact expectation E[c_i] = N W_i / T by enumerating every breakpoint of the
  offset.
- Multinomial resampling: the offspring vector follows Multinomial(N, W/T)
  (G-test against the exactly enumerated pmf), and the sorted positions from
  exponential spacings follow the uniform order-statistic laws Beta(j+1, N-j).
- Stratified resampling: each slot's position stays in its own stratum and
  picks particle i with probability |stratum j intersect interval i| (G-test per
  slot against those exact overlaps); offspring within floor(N W_i / T) - 1 and
  ceil(N W_i / T) + 1; mean offspring N W_i / T.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_cutpoint.txt")


def _table1():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append(dict(j=int(f[0]), q=f[1], L=int(f[2]), cut=int(f[3]), I=int(f[4]),
                         u=f[5], ceilNu=int(f[6]), Iceil=int(f[7]), res=int(f[8]),
                         I_printed=int(f[9])))
    return rows


def test_table1_cutpoint_search_and_method(orc):
    rows = _table1()
    n = len(rows)
    assert n == 10
    # q and u are printed with 4 decimals: scale by 10^4 to exact integers, T = 10^4.
    Q = np.array([round(float(r["q"]) * 10_000) for r in rows], np.uint64)
    U = np.array([round(float(r["u"]) * 10_000) for r in rows], np.uint64)
    L, I = orc.cutpoint_search(Q)
    assert L.tolist() == [r["L"] for r in rows]
    cut = [int(L[0] > 0)] + [int(L[i] > L[i - 1]) for i in range(1, n)]
    assert cut == [r["cut"] for r in rows]
    assert (I + 1).tolist() == [r["I"] for r in rows]
    # exactly one printed entry differs: the typo I_2 = 2
    diff = [r["j"] for r in rows if r["I"] != r["I_printed"]]
    assert diff == [2]
    anc, bucket = orc.cutpoint_method_int(Q, I, U)
    assert (bucket + 1).tolist() == [r["ceilNu"] for r in rows]
    assert (I[bucket] + 1).tolist() == [r["Iceil"] for r in rows]
    assert (anc + 1).tolist() == [r["res"] for r in rows]


def _random_cdf(rng, n, zero_frac=0.3, k=None):
    k = k if k is not None else 61 - math.ceil(math.log2(max(n, 1)))
    W = rng.integers(0, 1 << k, size=n, dtype=np.uint64)
    W[rng.random(n) < zero_frac] = 0
    if W.sum() == 0:
        W[rng.integers(n)] = 1 << k
    return W


def test_cdf_scan_exact(orc):
    rng = np.random.default_rng(3)
    for n in [1, 2, 3, 17, 1000, 4099]:
        W = _random_cdf(rng, n)
        Q = orc.cdf_scan(W)
        ref = list(itertools.accumulate(int(w) for w in W))
        assert [int(q) for q in Q] == ref


def test_cutpoint_definition_and_L_properties(orc):
    rng = np.random.default_rng(4)
    for n in [1, 2, 5, 10, 33, 200]:
        for zero_frac in (0.0, 0.5, 0.95):
            W = _random_cdf(rng, n, zero_frac)
            Q = orc.cdf_scan(W)
            T = int(Q[-1])
            L, I = orc.cutpoint_search(Q)
            Li = [int(v) for v in L]
            assert Li[-1] == n and all(b >= a for a, b in zip([0] + Li, Li))
            if zero_frac == 0.0:
                assert Li[0] > 0  # 0 = L_0 < L_1 when every weight is positive
            for k in range(n):  # I_k = min{i : Q_i / T > k / n}
                ref = next(i for i in range(n) if int(Q[i]) * n > k * T)
                assert I[k] == ref


@pytest.mark.parametrize("positions", ["systematic", "multinomial", "stratified"])
def test_walk_naive_cutpoint_agree(orc, positions):
    rng = np.random.default_rng(5)
    for trial in range(60):
        n = int(rng.integers(1, 65))
        W = _random_cdf(rng, n, zero_frac=float(rng.choice([0.0, 0.3, 0.9])))
        Q = orc.cdf_scan(W)
        a = orc.resample_method(Q, positions, "walk", 99, 2, trial)
        b = orc.resample_method(Q, positions, "naive", 99, 2, trial)
        c = orc.resample_method(Q, positions, "cutpoint", 99, 2, trial)
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert np.all(np.diff(a.astype(np.int64)) >= 0) and a.max() < n
        assert np.all(W[a] > 0)  # a zero-weight particle is never drawn


def test_systematic_offspring_floor_ceil(orc):
    rng = np.random.default_rng(6)
    for trial in range(200):
        n = int(rng.integers(1, 300))
        W = _random_cdf(rng, n, zero_frac=0.2)
        Q = orc.cdf_scan(W)
        T = int(Q[-1])
        anc = orc.resample_method(Q, "systematic", "walk", 1, 0, trial)
        c = np.bincount(anc, minlength=n)
        for i in range(n):
            lo, rem = divmod(n * int(W[i]), T)
            assert c[i] in ((lo,) if rem == 0 else (lo, lo + 1))


def test_systematic_exact_expectation_by_breakpoints(orc):
    """E_r[c_i] over a uniform offset r in [0, T) equals N W_i / T exactly."""
    rng = np.random.default_rng(7)
    for n in [1, 2, 3, 5, 6]:
        W = _random_cdf(rng, n, zero_frac=0.2, k=20)
        Q = orc.cdf_scan(W)
        T = int(Q[-1])
        # c(r) is constant between offsets r = Q_b * n - j T (slot j crosses Q_b)
        bps = {0, T}
        for b in range(n):
            for j in range(n):
                r = int(Q[b]) * n - j * T
                if 0 < r < T:
                    bps.add(r)
                if 0 < r + 1 < T:
                    bps.add(r + 1)
        bps = sorted(bps)
        expect = [Fraction(0)] * n
        for lo, hi in zip(bps[:-1], bps[1:]):
            c = np.bincount(orc.systematic_with_offset(Q, lo), minlength=n)
            c_hi = np.bincount(orc.systematic_with_offset(Q, hi - 1), minlength=n)
            assert np.array_equal(c, c_hi)  # constant on [lo, hi)
            for i in range(n):
                expect[i] += Fraction(hi - lo, T) * int(c[i])
        assert expect == [Fraction(n * int(W[i]), T) for i in range(n)]


def _compositions(n, parts):
    if parts == 1:
        yield (n,)
        return
    for k in range(n + 1):
        for rest in _compositions(n - k, parts - 1):
            yield (k,) + rest


@pytest.mark.parametrize("n", [3, 5])
def test_multinomial_offspring_pmf_gtest(orc, n):
    rng = np.random.default_rng(8 + n)
    W = rng.integers(1, 1 << 20, size=n, dtype=np.uint64)
    W[1] = 0 if n == 5 else W[1]
    Q = orc.cdf_scan(W)
    T = int(Q[-1])
    p = [int(w) / T for w in W]
    comps = list(_compositions(n, n))
    idx = {c: i for i, c in enumerate(comps)}
    draws = 40_000
    counts = np.zeros(len(comps))
    for t in range(draws):
        anc = orc.resample_cdf(Q, orc.MULTINOMIAL, 1234, 0, t)
        counts[idx[tuple(np.bincount(anc, minlength=n).tolist())]] += 1
    pmf = np.array([math.factorial(n) * np.prod([pi ** ci / math.factorial(ci) for pi, ci in zip(p, c)])
                    for c in comps])
    assert abs(pmf.sum() - 1) < 1e-12
    keep = pmf > 0
    assert counts[~keep].sum() == 0
    exp = pmf[keep] * draws
    obs = counts[keep]
    pos = obs > 0
    g = 2 * np.sum(obs[pos] * np.log(obs[pos] / exp[pos]))
    dof = keep.sum() - 1
    assert stats.chi2.sf(g, dof) > 1e-4


def test_multinomial_mean_offspring(orc):
    rng = np.random.default_rng(9)
    n = 40
    W = _random_cdf(rng, n, zero_frac=0.25)
    Q = orc.cdf_scan(W)
    T = int(Q[-1])
    reps = 4000
    c = np.zeros((reps, n))
    for t in range(reps):
        c[t] = np.bincount(orc.resample_cdf(Q, orc.MULTINOMIAL, 77, 3, t), minlength=n)
    p = W.astype(np.float64) / T
    z = (c.mean(0) - n * p) / np.sqrt(np.maximum(n * p * (1 - p), 1e-300) / reps)
    assert np.all(np.abs(z[p > 0]) < 5)
    assert np.all(c[:, p == 0] == 0)


def test_spacings_are_uniform_order_statistics(orc):
    n = 4
    reps = 20_000
    U = np.zeros((reps, n))
    for t in range(reps):
        S = orc.spacing_prefix(n, 31, 0, t).astype(np.float64)
        U[t] = S[:n] / S[n]
    for j in range(n):
        assert stats.kstest(U[:, j], stats.beta(j + 1, n - j).cdf).pvalue > 1e-4
    # n = 1: a single uniform
    u1 = np.array([(lambda S: S[0] / S[1])(orc.spacing_prefix(1, 5, 0, t).astype(np.float64))
                   for t in range(reps)])
    assert stats.kstest(u1, "uniform").pvalue > 1e-4


def test_quantize_weights_exact(orc):
    rng = np.random.default_rng(10)
    for n in [1, 7, 1000]:
        for s in (0.1, 1.0, 5.0):
            lw = rng.standard_normal(n) * s
            w = np.exp(lw - lw.max())
            w = (w / w.sum()).astype(np.float32)
            W = orc.quantize_weights(w)
            k = orc.cdf_shift(n)
            e = math.frexp(float(w.max()))[1]
            ref = [math.floor(Fraction(float(x)) * Fraction(2) ** (k - e)) for x in w]
            assert [int(v) for v in W] == ref
            assert int(W.sum()) < 2 ** 61 and int(W.max()) >= 2 ** (k - 1)
    with pytest.raises(ValueError):
        orc.quantize_weights(np.array([0.5, -0.1], np.float32))
    with pytest.raises(ValueError):
        orc.quantize_weights(np.zeros(3, np.float32))


@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
def test_edge_cases(orc, scheme):
    # single particle
    assert orc.resample_weights(np.array([0.3], np.float32), scheme, 1, 0, 0).tolist() == [0]
    # one particle carries all the weight
    w = np.zeros(100, np.float32)
    w[37] = 1.0
    assert np.all(orc.resample_weights(w, scheme, 1, 0, 0) == 37)
    # flat weights, systematic: every particle exactly once
    if scheme in (1, 3):
        w = np.full(256, 1 / 256, np.float32)
        assert np.array_equal(orc.resample_weights(w, scheme, 5, 0, 3), np.arange(256))


def test_systematic_offset_uniform_and_unbiased(orc):
    """r = floor(R T / 2^64) is uniform on [0, T), so E[c_i] = N W_i / T over t."""
    T = (1 << 61) - 12345
    r = np.array([orc.systematic_offset(T, 17, 2, t) for t in range(20_000)], np.float64)
    assert r.max() < T
    assert stats.kstest(r / T, "uniform").pvalue > 1e-4
    rng = np.random.default_rng(12)
    n = 30
    W = _random_cdf(rng, n, zero_frac=0.2)
    Q = orc.cdf_scan(W)
    reps = 3000
    c = np.zeros(n)
    for t in range(reps):
        c += np.bincount(orc.resample_cdf(Q, orc.SYSTEMATIC, 4, 0, t), minlength=n)
    p = W.astype(np.float64) / float(Q[-1])
    # systematic counts are floor or ceil of N p_i: per-draw variance <= 1/4
    assert np.all(np.abs(c / reps - n * p) < 5 * 0.5 / np.sqrt(reps))


def test_stratified_offsets_in_range_and_uniform(orc):
    """r_j = floor(R_j T / 2^64) lies in [0, T) and is uniform, for even and odd j
    (the two word pairs of one draw)."""
    T = (1 << 61) - 999
    for j in (0, 1, 6, 7):
        r = np.array([orc.stratified_offset(T, 23, 1, t, j) for t in range(10_000)], np.float64)
        assert r.max() < T
        assert stats.kstest(r / T, "uniform").pvalue > 1e-4
    # independent across slots: the two words of one draw, and different draws
    # (one offset for every slot would be systematic resampling)
    for j0, j1 in ((4, 5), (0, 2), (3, 9)):
        a = np.array([orc.stratified_offset(T, 23, 1, t, j0) for t in range(5000)], np.float64) / T
        b = np.array([orc.stratified_offset(T, 23, 1, t, j1) for t in range(5000)], np.float64) / T
        assert abs(np.corrcoef(a, b)[0, 1]) < 0.06, (j0, j1)


def test_stratified_offspring_bounds(orc):
    """Particle i covers L = N W_i / T strata: at least floor(L) - 1 of its
    strata lie wholly inside its interval and at most two more touch it."""
    rng = np.random.default_rng(16)
    for trial in range(200):
        n = int(rng.integers(1, 300))
        W = _random_cdf(rng, n, zero_frac=0.2)
        Q = orc.cdf_scan(W)
        T = int(Q[-1])
        anc = orc.resample_cdf(Q, orc.STRATIFIED, 3, 1, trial)
        assert np.all(np.diff(anc.astype(np.int64)) >= 0)
        c = np.bincount(anc, minlength=n)
        assert c.sum() == n
        for i in range(n):
            lo, rem = divmod(n * int(W[i]), T)
            hi = lo if rem == 0 else lo + 1
            assert max(0, lo - 1) <= c[i] <= hi + 1, (trial, i, c[i], lo, rem)
            if W[i] == 0:
                assert c[i] == 0


def test_stratified_per_slot_law(orc):
    """Slot j's position is uniform on its stratum [j T, (j+1) T) (in units of
    n Q): it picks particle i with probability |[jT, (j+1)T) intersect
    [n Q_{i-1}, n Q_i)| / T.  G-test of every slot's ancestor over seeds."""
    W = np.array([3, 0, 7, 1, 5], np.uint64) * np.uint64(1 << 40)
    n = W.size
    Q = orc.cdf_scan(W)
    T = int(Q[-1])
    reps = 20_000
    anc = np.array([orc.resample_cdf(Q, orc.STRATIFIED, 5, 2, t) for t in range(reps)])
    edges = [0] + [n * int(q) for q in Q]
    for j in range(n):
        p = np.array([max(0, min((j + 1) * T, edges[i + 1]) - max(j * T, edges[i])) / T
                      for i in range(n)])
        assert abs(p.sum() - 1) < 1e-12
        obs = np.bincount(anc[:, j], minlength=n)
        assert np.all(obs[p == 0] == 0)
        keep = p > 0
        exp = reps * p[keep]
        g = 2 * np.sum(np.where(obs[keep] > 0, obs[keep] * np.log(np.maximum(obs[keep], 1) / exp), 0))
        dof = keep.sum() - 1
        if dof > 0:
            assert stats.chi2.sf(g, dof) > 1e-4, (j, obs, exp)


def test_stratified_mean_offspring(orc):
    rng = np.random.default_rng(19)
    n = 40
    W = _random_cdf(rng, n, zero_frac=0.25)
    Q = orc.cdf_scan(W)
    T = int(Q[-1])
    reps = 4000
    c = np.array([np.bincount(orc.resample_cdf(Q, orc.STRATIFIED, 7, 4, t), minlength=n)
                  for t in range(reps)], np.float64)
    L = n * W.astype(np.float64) / T
    sd = c.std(0, ddof=1)
    ok = sd > 0
    z = (c.mean(0) - L)[ok] / (sd[ok] / np.sqrt(reps))
    assert np.all(np.abs(z) < 5)
    assert np.allclose(c.mean(0)[~ok], L[~ok], atol=1e-9)  # degenerate counts are exact
