"""Precision: FP32 state against FP64 state, each result's error measured
against the FP64 oracle.

FP64 filters follow the FP64 oracle operation for operation, so every
posterior summary must agree within 1e-12 relative (to max(|value|, posterior
sd)) at every step.  FP32 filters use the same draws but round the state to
binary32: at first they pick the FP64 ancestors, then the paths drift apart
and the estimates differ by Monte Carlo error, which is what FP32 costs.  The
scale of that error is measured, not assumed: the spread of the FP64
oracle's estimates over independent seeds (for the static parameters it is
several times posterior sd / sqrt(N), as particle-learning estimates of
static parameters degenerate).  An FP32 estimate and the FP64 estimate with
the same seed differ by at most about sqrt(2) such spreads; the test allows
7 (5 sigma of the difference, at each of the 400 step-summary pairs).
"""
import numpy as np
import pytest

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu

Q = ("x", "sigma2", "tau2")
KEYS = [q + "_mean" for q in Q] + ["log_marglik"]


def _path(f, y):
    out = []
    for v in y:
        f.step(v)
        out.append(f.estimate())
    return out


def _oracle_path(orc, n, seed, scheme, y):
    o = orc.Filter(orc.make_config(n, seed=seed, scheme=scheme, precision=1))
    out = []
    for v in y:
        o.step(v)
        out.append(o.estimate())
    o.close()
    return out


@pytest.mark.parametrize("scheme", ["multinomial", "systematic"])
def test_fp32_and_fp64_against_the_fp64_oracle(pf, orc, scheme):
    n, T, reps = 1024, 100, 16
    _, y = synth.local_level_series(1212, T)
    sc = pf.SCHEMES[scheme]
    g64 = pf.Filter(n, seed=1212, scheme=scheme, precision="fp64")
    g32 = pf.Filter(n, seed=1212, scheme=scheme, precision="fp32")
    e64, e32 = _path(g64, y), _path(g32, y)
    eo = _oracle_path(orc, n, 1212, sc, y)
    # Monte Carlo spread of the FP64 oracle's estimates over independent seeds
    rep = np.array([[[e[k] for k in KEYS] for e in _oracle_path(orc, n, 5000 + r, sc, y)]
                    for r in range(reps)])             # [reps, T, keys]
    mc_sd = rep.std(axis=0, ddof=1)                    # [T, keys]
    worst64 = 0.0
    worst32 = np.zeros(len(KEYS))
    for t in range(T):
        for i, k in enumerate(KEYS):
            ref = eo[t][k]
            if k == "log_marglik":
                scale = max(1.0, abs(ref))
            else:
                scale = max(abs(ref), np.sqrt(max(eo[t][k.replace("_mean", "_var")], 0.0)))
            r64 = abs(e64[t][k] - ref) / scale
            assert r64 <= 1e-12, (t, k, r64)
            worst64 = max(worst64, r64)
            z32 = abs(e32[t][k] - ref) / mc_sd[t, i]
            assert z32 <= 7.0, (t, k, z32, mc_sd[t, i])
            worst32[i] = max(worst32[i], z32)
    print("\nprecision %s N=%d T=%d: FP64 vs FP64 oracle max rel err %.1e; FP32 vs FP64 oracle "
          "max |err| in Monte Carlo sd: %s; MC sd at T: %s" % (
              scheme, n, T, worst64, dict(zip(KEYS, np.round(worst32, 2))),
              dict(zip(KEYS, np.round(mc_sd[-1], 4)))))
    g64.close()
    g32.close()


def test_fp32_and_fp64_against_kalman_with_known_variances(pf, orc):
    """With sigma^2, tau^2 known the exact filter is the Kalman filter: both
    precisions must sit within Monte Carlo error of its filtered mean (the
    bounds the oracle's own Kalman pin uses) and of its log-likelihood, and
    FP32 must not be measurably worse than FP64."""
    n, T = 1 << 16, 60
    _, y = synth.local_level_series(77, T)
    km, kv, kll = orc.kalman(y, 0.0, 10.0, 1.0, 0.1)
    rms = {}
    for prec in ("fp64", "fp32"):
        f = pf.Filter(n, seed=5, precision=prec, known_variances=True, sigma2=1.0, tau2=0.1)
        z = []
        for t in range(T):
            f.step(y[t])
            z.append((f.estimate()["x_mean"] - km[t]) / np.sqrt(kv[t] / n))
        z = np.array(z)
        assert np.max(np.abs(z)) < 12, (prec, np.max(np.abs(z)))
        rms[prec] = float(np.sqrt(np.mean(z ** 2)))
        assert rms[prec] < 4, (prec, rms[prec])
        assert abs(f.estimate()["log_marglik"] - kll) < 0.25, prec
        f.close()
    print("\nKalman check N=%d T=%d: rms z FP64 %.2f, FP32 %.2f" % (n, T, rms["fp64"], rms["fp32"]))
    assert rms["fp32"] <= 2.0 * rms["fp64"] + 1.0
