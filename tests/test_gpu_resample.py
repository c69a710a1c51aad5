"""GPU parity of resampling (pf_resample, pf_cdf, the cut-point primitives)
against the CPU oracle: ancestor indices and CDF values are compared bit for
bit on the same seeded FP32 weight vectors.

Weight vectors follow the resampling sweep workload: log-weights ~ N(0, s^2)
with s = 0.1 (flat), 1 and 5 (degenerate), normalised in float64 and cast to
float32; sizes span single elements, one scan tile (4096), ragged tails and the
full 2^24 particles.
"""
import os

import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu

SMALL = [1, 2, 3, 5, 64, 1000, 4095, 4096, 4097, 12345, 16383, 16384, 16385, (1 << 16) + 3]
SCHEMES = [0, 1, 2, 3, 4]


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("s", [0.1, 1.0, 5.0])
def test_resample_small_sizes_bit_exact(pf, orc, scheme, s):
    for n in SMALL:
        w = synth.sweep_weights(n, s, seed=3)
        anc = _u32(pf.resample(torch.from_numpy(w).cuda(), seed=77, filter_id=3, t=5, scheme=scheme))
        ref = orc.resample_weights(w, scheme, 77, 3, 5)
        assert np.array_equal(anc, ref), (n, s, scheme, np.flatnonzero(anc != ref)[:5])


@pytest.mark.parametrize("scheme", SCHEMES)
def test_resample_2p20_bit_exact(pf, orc, scheme):
    n = 1 << 20
    for s in (0.1, 1.0, 5.0):
        w = synth.sweep_weights(n, s, seed=4)
        anc = _u32(pf.resample(torch.from_numpy(w).cuda(), seed=1639, filter_id=0, t=0, scheme=scheme))
        ref = orc.resample_weights(w, scheme, 1639, 0, 0)
        assert np.array_equal(anc, ref), (s, scheme)


@pytest.mark.parametrize("scheme", [0, 1, 4])
@pytest.mark.parametrize("s", [1.0, 5.0])
def test_resample_2p24_bit_exact(pf, orc, scheme, s):
    """Full size of the resampling sweep, in the configuration the bench times."""
    n = 1 << 24
    w = synth.sweep_weights(n, s, seed=5)
    anc = _u32(pf.resample(torch.from_numpy(w).cuda(), seed=24, filter_id=1, t=9, scheme=scheme))
    ref = orc.resample_weights(w, scheme, 24, 1, 9)
    assert np.array_equal(anc, ref)


def test_resample_unaligned_input(pf, orc):
    n = 10_001
    w = synth.sweep_weights(n + 1, 1.0, seed=6)
    wd = torch.from_numpy(w).cuda()[1:]  # 4-byte offset: scalar load path
    assert wd.data_ptr() % 16 != 0
    for scheme in SCHEMES:
        anc = _u32(pf.resample(wd, seed=8, scheme=scheme))
        assert np.array_equal(anc, orc.resample_weights(w[1:], scheme, 8, 0, 0))


def test_cdf_bit_exact(pf, orc):
    for n in (1, 7, 4096, 4097, 100_003, 1 << 20):
        w = synth.sweep_weights(n, 1.0, seed=7)
        Q = pf.cdf(torch.from_numpy(w).cuda()).cpu().numpy().view(np.uint64)
        ref = orc.cdf_scan(orc.quantize_weights(w))
        assert np.array_equal(Q, ref), n


def test_unnormalised_and_degenerate_weights(pf, orc):
    rng = np.random.default_rng(9)
    cases = [
        (rng.random(5000) * 1e30).astype(np.float32),       # large scale
        (rng.random(5000) * 1e-30).astype(np.float32),      # tiny scale
        np.where(rng.random(5000) < 0.999, 0, 1).astype(np.float32),  # mostly zero
        np.eye(1, 9000, 4321, dtype=np.float32)[0],          # one particle
    ]
    for w in cases:
        if w.sum() == 0:
            w[0] = 1
        for scheme in SCHEMES:
            anc = _u32(pf.resample(torch.from_numpy(w).cuda(), seed=2, scheme=scheme))
            assert np.array_equal(anc, orc.resample_weights(w, scheme, 2, 0, 0))


def test_table1_cutpoint_on_gpu(pf):
    """The paper's Table 1 (N = 10) through pf_cutpoint_search / pf_cutpoint_method."""
    rows = []
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_cutpoint.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows.append((float(f[1]), int(f[4]), float(f[5]), int(f[8])))
    Q = torch.tensor([round(q * 10_000) for q, _, _, _ in rows], dtype=torch.int64, device="cuda")
    U = torch.tensor([round(u * 10_000) for _, _, u, _ in rows], dtype=torch.int64, device="cuda")
    I = pf.cutpoint_search(Q)
    assert (I.cpu() + 1).tolist() == [r[1] for r in rows]
    anc = pf.cutpoint_method(Q, I, U)
    assert (anc.cpu() + 1).tolist() == [r[3] for r in rows]


def test_cutpoint_search_matches_oracle(pf, orc):
    rng = np.random.default_rng(11)
    for n in (1, 13, 5000, 300_001):
        W = rng.integers(0, 1 << 30, size=n, dtype=np.uint64)
        W[rng.random(n) < 0.5] = 0
        W[0] += 1
        Q = orc.cdf_scan(W)
        _, I_ref = orc.cutpoint_search(Q)
        I = pf.cutpoint_search(torch.from_numpy(Q.view(np.int64)).cuda())
        assert np.array_equal(_u32(I), I_ref), n


def test_resample_errors(pf):
    w = torch.rand(1000, device="cuda")
    w[17] = -1.0
    with pytest.raises(pf.PfError) as e:
        pf.resample(w, seed=1)
    assert e.value.status == pf.PF_ERR_NUMERIC
    with pytest.raises(pf.PfError) as e:
        pf.resample(torch.zeros(100, device="cuda"), seed=1)
    assert e.value.status == pf.PF_ERR_NUMERIC
    w = torch.rand(100, device="cuda")
    w[3] = float("nan")
    with pytest.raises(pf.PfError) as e:
        pf.resample(w, seed=1)
    assert e.value.status == pf.PF_ERR_NUMERIC
    # the device is still usable afterwards
    anc = pf.resample(torch.ones(64, device="cuda"), seed=1, scheme="systematic")
    assert anc.cpu().tolist() == list(range(64))
