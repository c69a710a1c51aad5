"""Pins of the oracle's counter-based RNG and its uniform / normal / gamma draws.

Philox4x32-10 and Philox4x64-10 (Salmon et al. 2011) are checked against two
independent implementations: triton's (run by its CPU interpreter) for 4x32 and
numpy's Philox bit generator for 4x64.  The derived draws are checked against
their distributions.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy import stats


def test_philox4x64_matches_numpy(orc):
    rng = np.random.default_rng(7)
    ctr = rng.integers(1, 2**63, size=(64, 4), dtype=np.uint64)
    key = rng.integers(0, 2**63, size=(64, 2), dtype=np.uint64)
    ours = orc.philox4x64(ctr, key)
    for i in range(64):
        prev = ctr[i].copy()
        prev[0] -= np.uint64(1)  # numpy increments the counter before each block
        g = np.random.Philox(counter=prev, key=key[i])
        assert np.array_equal(g.random_raw(4).astype(np.uint64), ours[i]), i


_TRITON_SCRIPT = textwrap.dedent("""
    import os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, seed_ptr, out_ptr, n: tl.constexpr):
        i = tl.arange(0, n)
        c0 = tl.load(c_ptr + 4 * i + 0)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        s = tl.load(seed_ptr + i)
        a, b, c, d = tl.philox(s, c0, c1, c2, c3)
        tl.store(out_ptr + 4 * i + 0, a)
        tl.store(out_ptr + 4 * i + 1, b)
        tl.store(out_ptr + 4 * i + 2, c)
        tl.store(out_ptr + 4 * i + 3, d)

    data = np.load(sys.argv[1])
    ctr = torch.from_numpy(data["ctr"].astype(np.int64).astype(np.int32))
    seed = torch.from_numpy(data["seed"].astype(np.int64))
    out = torch.zeros_like(ctr)
    k[(1,)](ctr, seed, out, ctr.shape[0] // 4)
    np.save(sys.argv[2], out.numpy().view(np.uint32))
""")


def test_philox4x32_matches_triton_interpreter(orc, tmp_path):
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    n = 64
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    seed = rng.integers(0, 2**63, size=n, dtype=np.int64)
    key = np.stack([(seed & 0xFFFFFFFF).astype(np.uint32),
                    (seed >> 32).astype(np.uint32)], axis=1)
    ours = orc.philox4x32(ctr, key)
    inp = tmp_path / "in.npz"
    outp = tmp_path / "out.npy"
    np.savez(inp, ctr=ctr.reshape(-1), seed=seed)
    script = tmp_path / "tri.py"
    script.write_text(_TRITON_SCRIPT)
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, str(script), str(inp), str(outp)], env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-300:])
    theirs = np.load(outp).reshape(n, 4)
    assert np.array_equal(ours, theirs)


def test_draw_counter_layout(orc):
    # draw(seed, filter, t, j, purpose, attempt) = Philox4x32-10 with
    # counter (j, t, filter, purpose | attempt << 8) and key (seed lo, seed hi).
    seed = 0x123456789ABCDEF0
    d = orc.draws(seed, 7, 5, 100, 3, orc.P_GAMMA_TAU, attempt=2)
    ctr = np.array([[100 + i, 5, 7, orc.P_GAMMA_TAU | (2 << 8)] for i in range(3)], np.uint32)
    key = np.array([[seed & 0xFFFFFFFF, seed >> 32]] * 3, np.uint32)
    assert np.array_equal(d, orc.philox4x32(ctr, key))


def test_uniform_f32_exact_grid_and_chisq(orc):
    w = orc.draws(1, 0, 0, 0, 1 << 16, orc.P_STATE).reshape(-1)
    u = orc.unif_f32(w)
    assert u.min() > 0 and u.max() < 1
    m = u.astype(np.float64) * 2**24
    assert np.all(np.mod(m, 2) == 1)  # odd multiples of 2^-24: (2*(w>>9)+1) * 2^-24
    assert np.array_equal(m, 2.0 * (w >> 9).astype(np.float64) + 1.0)
    counts = np.bincount((u * 64).astype(int), minlength=64)
    assert stats.chisquare(counts).pvalue > 1e-4


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_box_muller_normal(orc, dtype):
    z = orc.normals(3, 0, 9, orc.P_STATE, 200_000, dtype).astype(np.float64)
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("a", [1.0, 3.0, 5.0, 50.5])
def test_gamma_marsaglia_tsang(orc, dtype, a):
    g, fail = orc.gammas(a, 5, 1, 3, orc.P_GAMMA_SIGMA, 100_000, dtype)
    assert fail == 0
    assert stats.kstest(g.astype(np.float64), stats.gamma(a).cdf).pvalue > 1e-4
    assert abs(g.mean() - a) < 5 * np.sqrt(a / g.size)


def _g_minus(d, u):
    """1 - exp(g) for Z = 3 sqrt(d) u: g = d h(u), h(u) = 3 log(1+u) - 3u + 3u^2/2 - u^3 is the
    log acceptance ratio of Marsaglia-Tsang with v = (1 + u)^3 (u = c Z, c = 1/sqrt(9d))."""
    h = 3 * np.log1p(u) - 3 * u + 1.5 * u * u - u ** 3
    return -np.expm1(d * h)


def test_gamma_squeeze_is_a_lower_bound(orc):
    """The squeeze U < 1 - K Z^4 may only accept what the full test accepts:
    1 - K Z^4 <= exp(g(Z)) for every Z with v > 0, at every shape.  K = 0.0331 (2/3) / d is
    Marsaglia & Tsang's 0.0331 at d = 2/3, and the supremum of (1 - e^g) d / Z^4 over Z is
    largest there (0.022049) and falls toward 1/108 as d grows."""
    u = np.concatenate([np.linspace(-1 + 1e-9, -1e-3, 400_001), np.linspace(1e-3, 30, 200_001)])
    worst = 0.0
    for a in np.concatenate([[1.0, 1.1, 1.5, 2.0, 3.0, 3.5, 5.0], np.geomspace(5.5, 1e6, 60)]):
        d, c, K = orc.mt_constants(a)
        assert d == a - float.fromhex("0x1.5555555555555p-2")
        assert K == float.fromhex("0x1.698a4eea9073cp-6") / d
        Z4 = (u / c) ** 4
        ratio = _g_minus(d, u) / (K * Z4)
        worst = max(worst, ratio.max())
        assert ratio.max() <= 1.0 - 1e-4, (a, ratio.max())
    assert worst > 0.99  # the bound is tight at a = 1 (Marsaglia-Tsang's own constant)


def test_gamma_accepts_exactly_the_full_test(orc):
    """Attempt 0 of the sampler (binary64) against the plain Marsaglia-Tsang full test written
    out here with exact rationals for the fused steps: a draw the full test accepts returns
    d v^3 of that attempt, one it rejects returns something else (a later attempt)."""
    from fractions import Fraction as F
    import math
    n = 20_000
    for a in (1.0, 1.3, 3.5, 53.5):
        d, c, K = orc.mt_constants(a)
        g, fail = orc.gammas(a, 11, 2, 7, orc.P_GAMMA_TAU, n, np.float64)
        assert fail == 0
        Z = orc.normals(11, 2, 7, orc.P_GAMMA_TAU, n, np.float64)
        w = orc.draws(11, 2, 7, 0, n, orc.P_GAMMA_TAU)
        U = (2.0 * w[:, 3].astype(np.float64) + 1.0) * 2.0**-33
        acc = 0
        for j in range(n):
            v = float(F(c) * F(float(Z[j])) + 1)          # fma(c, Z, 1)
            if not v > 0:
                continue
            v3 = (v * v) * v
            full = math.log(U[j]) < Z[j] * Z[j] / 2 + d * (1 - v3 + math.log(v3))
            if full:
                acc += 1
                assert g[j] == d * v3, (a, j)
            else:
                assert g[j] != d * v3, (a, j)
        assert acc > 0.9 * n


def test_streams_differ_by_purpose_and_time(orc):
    a = orc.draws(9, 0, 0, 0, 1024, orc.P_STATE)
    b = orc.draws(9, 0, 0, 0, 1024, orc.P_GAMMA_SIGMA)
    c = orc.draws(9, 0, 1, 0, 1024, orc.P_STATE)
    d = orc.draws(9, 1, 0, 0, 1024, orc.P_STATE)
    e = orc.draws(9, 0, 0, 0, 1024, orc.P_STATE, attempt=1)
    words = [x.tobytes() for x in (a, b, c, d, e)]
    assert len(set(words)) == 5


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_theta_draws_law(orc, dtype):
    """The propagation draws of a cycle: Zx, Zs, Zt standard normal and Us, Ut uniform,
    all mutually uncorrelated within a slot and between the two slots of a pair (in
    binary32 the pair 2i, 2i + 1 takes its tau^2 normals from one Box-Muller transform
    and its two uniforms from one draw), and the pair's tau^2 normals jointly standard
    bivariate normal: angle uniform, squared radius chi-square with 2 degrees of freedom."""
    n = 200_000
    d = orc.theta_draws(77, 3, 12, n, dtype).astype(np.float64)
    for c in (0, 1, 3):
        assert stats.kstest(d[:, c], "norm").pvalue > 1e-4, c
    for c in (2, 4):
        assert d[:, c].min() > 0 and d[:, c].max() < 1
        counts = np.bincount((d[:, c] * 50).astype(int), minlength=50)
        assert stats.chisquare(counts).pvalue > 1e-4, c
    lim = 5 / np.sqrt(n)
    r = np.corrcoef(d.T)
    assert np.all(np.abs(r[np.triu_indices(5, 1)]) < lim), r
    ev, od = d[0::2], d[1::2]
    rp = np.corrcoef(np.hstack([ev, od]).T)[:5, 5:]
    assert np.all(np.abs(rp) < 5 / np.sqrt(n // 2)), rp
    zt0, zt1 = ev[:, 3], od[:, 3]
    ang = (np.arctan2(zt1, zt0) / (2 * np.pi)) % 1.0
    assert stats.kstest(ang, "uniform").pvalue > 1e-4
    assert stats.kstest(zt0 ** 2 + zt1 ** 2, stats.chi2(2).cdf).pvalue > 1e-4
    assert not np.any(ev[:, 4] == od[:, 4])
