"""pf_resample_noalloc: resampling for callers that cannot allocate device memory.

The entry point keeps its scratch in a fixed device array inside the library
instead of allocating, so code that must not allocate at that point
(latency-critical loops, processes with all device memory reserved up front)
can still resample.  Its ancestors must equal
pf_resample's exactly (integer output), on consecutive calls that reuse the
same scratch, and sizes above the array's limit must be refused.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_noalloc_matches_resample_on_two_calls_in_a_row(pf):
    cases = [(1, 1.0), (5000, 0.1), (4097, 5.0), (300_001, 1.0), (pf.NOALLOC_MAX_PARTICLES, 1.0)]
    for call in range(2):  # the second round reuses the scratch the first left behind
        for n, s in cases:
            w = torch.from_numpy(synth.sweep_weights(n, s, seed=40 + call)).cuda()
            for scheme in (0, 1, 2, 3, 4):  # every scheme the entry point accepts
                ref = _u32(pf.resample(w, seed=11 + call, filter_id=2, t=call, scheme=scheme))
                got = _u32(pf.resample_noalloc(w, seed=11 + call, filter_id=2, t=call,
                                               scheme=scheme))
                assert np.array_equal(got, ref), (call, n, s, scheme)


def test_noalloc_refuses_sizes_above_its_array(pf):
    n = pf.NOALLOC_MAX_PARTICLES + 1
    w = torch.ones(n, device="cuda")
    with pytest.raises(pf.PfError) as e:
        pf.resample_noalloc(w, seed=1)
    assert e.value.status == pf.PF_ERR_INVALID
    assert "n must be in" in str(e.value)
