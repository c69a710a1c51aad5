"""Pins of the oracle's deterministic elementary functions against libm.

The functions are the methods named in the oracle (log after reduction to
[sqrt(1/2), sqrt(2)): in binary64 by the atanh series, in binary32 by a fitted
polynomial in f - 1 without division; exp by Cody-Waite reduction and a Taylor
polynomial; cos(2 pi u) by octant reduction and Taylor polynomials).  They are
checked against an extended-precision reference within a few units in the last
place (the binary32 log within one), which any dropped term, wrong coefficient
or sign breaks.
"""
import numpy as np
import pytest

LD = np.longdouble
HAVE_EXT = np.finfo(LD).eps < np.finfo(np.float64).eps


def _ulp_err(got, ref, dtype):
    got = got.astype(LD)
    ulp = np.spacing(np.abs(ref).astype(dtype)).astype(LD)
    return np.abs(got - ref) / ulp


def _samples_pos(dtype, n=400_000):
    rng = np.random.default_rng(1)
    lo, hi = (-37, 38) if dtype == np.float32 else (-300, 300)
    e = rng.uniform(lo, hi, n)
    x = (10.0 ** e).astype(dtype)
    near1 = (1 + rng.uniform(-0.3, 0.3, n // 4)).astype(dtype)
    grid = np.arange(1, 1 << 23, 97, dtype=np.float64) * 2.0**-24  # the uniform grid
    return np.concatenate([x, near1, grid.astype(dtype), np.array([1.0, 2.0, 0.5], dtype)])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_det_log_accuracy(orc, dtype):
    if dtype == np.float64 and not HAVE_EXT:
        pytest.skip("no extended precision reference on this platform")
    x = _samples_pos(dtype)
    got = orc.det_log(x, dtype)
    ref = np.log(x.astype(LD))
    err = _ulp_err(got, ref, dtype)
    # absolute error near log(x) = 0 is bounded instead (x within 2^-20 of 1)
    small = np.abs(ref) < 1e-6
    # binary32: the division-free polynomial log is within 0.93 ulp everywhere
    bound = 1.0 if dtype == np.float32 else 3.0
    assert err[~small].max() <= bound, err[~small].max()
    assert np.all(np.abs(got[small].astype(LD) - ref[small]) <= 4 * np.finfo(dtype).eps * np.abs(ref[small]) + np.finfo(dtype).tiny)
    assert got[np.where(x == 1)[0][0]] == 0


def test_det_log_f32_subnormal_and_special(orc):
    if not HAVE_EXT:
        pytest.skip("no extended precision reference on this platform")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.integers(1, 1 << 23, 100_000).astype(np.uint32).view(np.float32),
                        np.array([np.float32(2.0**-149), np.float32(2.0**-126)])])
    got = orc.det_log(x, np.float32)
    err = _ulp_err(got, np.log(x.astype(LD)), np.float32)
    assert err.max() <= 1.0, err.max()
    sp = orc.det_log(np.array([np.inf, np.nan], np.float32), np.float32)
    assert sp[0] == np.inf and np.isnan(sp[1])


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_det_exp_core_accuracy(orc, dtype):
    if dtype == np.float64 and not HAVE_EXT:
        pytest.skip("no extended precision reference on this platform")
    r = np.linspace(-0.36, 0.36, 200_001).astype(dtype)
    got = orc.det_exp_core(r, dtype)
    err = _ulp_err(got, np.exp(r.astype(LD)), dtype)
    assert err.max() <= 2.0, err.max()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_quant_exp_accuracy_and_exactness(orc, dtype):
    if dtype == np.float64 and not HAVE_EXT:
        pytest.skip("no extended precision reference on this platform")
    rng = np.random.default_rng(2)
    dl = np.concatenate([-rng.uniform(0, 50, 300_000), -rng.uniform(0, 1e-3, 10_000),
                         [0.0, -50.0, -50.0001, -1e9, -np.inf]]).astype(dtype)
    k = 37
    W, e = orc.quant_exp(dl, k, dtype)
    ok = dl >= -50
    err = _ulp_err(e[ok], np.exp(dl[ok].astype(LD)), dtype)
    assert err.max() <= 3.0, err.max()
    assert np.all(e[~ok] == 0) and np.all(W[~ok] == 0)
    # W = floor(e * 2^k) exactly, and the maximum particle maps to 2^k
    ref = np.floor(e[ok].astype(LD) * LD(2.0) ** k).astype(np.uint64)
    assert np.array_equal(W[ok], np.minimum(ref, np.uint64(1) << np.uint64(k)))
    assert W[np.where(dl == 0)[0][0]] == 1 << k
    # monotone in dl
    order = np.argsort(dl[ok], kind="stable")
    assert np.all(np.diff(W[ok][order].astype(np.int64)) >= 0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_det_cos2pi_accuracy(orc, dtype):
    if dtype == np.float64 and not HAVE_EXT:
        pytest.skip("no extended precision reference on this platform")
    u = np.concatenate([np.linspace(0, 1, 400_001), [0.125, 0.375, 0.625, 0.875, 0.25, 0.5]]).astype(dtype)
    got = orc.det_cos2pi(u, dtype).astype(LD)
    ref = np.cos(LD(2) * np.pi * u.astype(LD))
    # absolute error in units of eps (cos has zeros, where relative error is meaningless)
    assert np.max(np.abs(got - ref)) <= 2 * np.finfo(dtype).eps
    assert got[0] == 1 and got[-1] == -1


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_det_sincos2pi_accuracy_and_consistency(orc, dtype):
    if dtype == np.float64 and not HAVE_EXT:
        pytest.skip("no extended precision reference on this platform")
    u = np.concatenate([np.linspace(0, 1, 400_001), [0.125, 0.375, 0.625, 0.875]]).astype(dtype)
    s, c = orc.det_sincos2pi(u, dtype)
    ang = LD(2) * np.pi * u.astype(LD)
    assert np.max(np.abs(s.astype(LD) - np.sin(ang))) <= 2 * np.finfo(dtype).eps
    assert np.max(np.abs(c.astype(LD) - np.cos(ang))) <= 2 * np.finfo(dtype).eps
    # the cos output is the same function as det_cos2pi
    assert np.array_equal(c, orc.det_cos2pi(u, dtype))
