"""Seeded synthetic inputs for the particle-learning workloads.

This module generates *inputs only* (observation series, weight vectors,
per-filter sizes and true parameters) with numpy's PCG64 generator.  It holds
none of the method's arithmetic: no weights, CDF, resampling or propagation.
Both the CUDA path and the CPU oracle consume exactly these arrays.

Workload shapes follow the paper's Section 4 experiment (the local-level
"stochastic trend with noise" model with x_0 = 0, sigma^2 = 1, tau^2 = 0.1) and
the scaled configurations built on it (one filter at 2^20..2^24 particles, a
weight sweep from flat to degenerate, thousands of uneven filters).
"""
import numpy as np


def local_level_series(seed, T, sigma2=1.0, tau2=0.1, x0=0.0, filter_id=0):
    """Simulate y_1..y_T from y_t = x_t + v_t, x_t = x_{t-1} + w_t (paper Section 4).

    Returns (x, y) with x of length T+1 (x[0] = x0) and y of length T, float64.
    """
    rng = np.random.default_rng([int(seed), int(filter_id), 0x5EED])
    w = rng.standard_normal(T) * np.sqrt(tau2)
    v = rng.standard_normal(T) * np.sqrt(sigma2)
    x = np.empty(T + 1)
    x[0] = x0
    x[1:] = x0 + np.cumsum(w)
    y = x[1:] + v
    return x, y


def sweep_weights(n, s, seed):
    """Normalised FP32 weights with log-weights ~ N(0, s^2).

    s = 0.1 is nearly flat, s = 1 moderate, s = 5 degenerate (a few particles
    carry almost all the mass, the worst case of the cut-point search).
    Normalisation is done in float64, then the weights are cast to float32.
    """
    rng = np.random.default_rng([int(seed), int(n), int(round(s * 1000)), 0xC3])
    lw = rng.standard_normal(n) * s
    w = np.exp(lw - lw.max())
    w /= w.sum()
    return w.astype(np.float32)


def batch_specs(n_filters, seed, n_lo=256, n_hi=65536, a=3.0, b=2.0):
    """Per-filter particle counts (log-uniform in [n_lo, n_hi]) and true
    variances (sigma^2, tau^2) drawn from the IG(a, b) prior."""
    rng = np.random.default_rng([int(seed), int(n_filters), 0xB4])
    u = rng.random(n_filters)
    lo, hi = np.log2(n_lo), np.log2(n_hi)
    n = np.round(2.0 ** (lo + (hi - lo) * u)).astype(np.int64)
    sigma2 = b / rng.gamma(a, 1.0, n_filters)
    tau2 = b / rng.gamma(a, 1.0, n_filters)
    return n, sigma2, tau2


def poisson_arrivals(rate_per_stream, n_streams, duration_s, seed):
    """Arrival times (seconds) of observations for each stream: independent
    Poisson processes.  Returns a list of sorted float64 arrays."""
    rng = np.random.default_rng([int(seed), int(n_streams), 0xA7])
    out = []
    for _ in range(n_streams):
        k = rng.poisson(rate_per_stream * duration_s)
        out.append(np.sort(rng.random(k) * duration_s))
    return out
