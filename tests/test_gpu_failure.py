"""Failure detection without faulting a GPU.

- A bounded device wait that runs out: the look-back of the single-pass CDF
  scan polls a predecessor tile's status word a bounded number of times.  A
  diagnostic call makes one tile withhold its status, so its successor's wait
  gives up; the call must report PF_ERR_TIMEOUT, return, and leave the context
  usable (the next scan on the same stream is exact).
- Device allocation failure: an allocator callback that returns NULL on its
  k-th call.  Creation must report PF_ERR_OOM and give back every allocation
  it had made, for every k, for single filters and for batches.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1212_1639_gb300 import synth

pytestmark = pytest.mark.gpu


def _quantised_cdf(orc, w):
    W = np.zeros(w.size, np.uint64)
    assert orc.lib().or_quantize_weights_f32(np.ascontiguousarray(w, np.float32), w.size, W) == 0
    Q = np.zeros(w.size, np.uint64)
    orc.lib().or_cdf_scan(W, w.size, Q)
    return Q


def test_lookback_wait_runs_out_and_the_next_scan_is_exact(pf, orc):
    n = 3 * 4096 + 17  # four tiles
    w_np = synth.sweep_weights(n, 1.0, seed=3)
    w = torch.from_numpy(w_np).cuda()
    ref = _quantised_cdf(orc, w_np)
    # tile 1 publishes nothing: tile 2's wait gives up after 64 polls
    st, _ = pf.diag_cdf_wait(w, withhold_tile=1, spin_limit=64)
    assert st == pf.PF_ERR_TIMEOUT, pf.STATUS_NAMES.get(st, st)
    assert "timed out" in pf.last_error()
    # the context is usable: a plain scan on the same stream is exact, twice
    for _ in range(2):
        Q = pf.cdf(w).cpu().numpy().view(np.uint64)
        assert np.array_equal(Q, ref)
    # nothing withheld: the same call with a short (but sufficient) wait is exact
    st, Q = pf.diag_cdf_wait(w, withhold_tile=0xFFFFFFFF, spin_limit=1 << 20)
    assert st == pf.PF_OK
    assert np.array_equal(Q.cpu().numpy().view(np.uint64), ref)


class FailingAllocator:
    """Device allocations through torch's caching allocator, except that call
    number `fail_at` (1-based; 0 = never) returns NULL.  Tracks the pointers
    handed out and not yet freed."""

    def __init__(self, fail_at=0):
        self.fail_at = fail_at
        self.calls = 0
        self.live = set()
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            self.live.add(p)
            return p

        def _free(ptr, stream, ctx):
            self.live.discard(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        from paper_1212_1639_gb300 import pf as _pf
        self.alloc = _pf.ALLOC_FN(_alloc)
        self.free = _pf.FREE_FN(_free)


@pytest.mark.parametrize("scheme,precision", [("systematic", "fp32"), ("multinomial", "fp64"),
                                              ("systematic", "fp32-ess")])
def test_create_reports_oom_and_frees_everything(pf, scheme, precision):
    kw = {}
    if precision == "fp32-ess":
        precision, kw = "fp32", {"ess_frac": 0.5}
    n = 70_001
    ok = FailingAllocator()
    f = pf.Filter(n, seed=5, scheme=scheme, precision=precision, torch_alloc=ok, **kw)
    calls = ok.calls
    assert calls >= 3 and ok.live
    f.close()
    assert not ok.live
    for k in range(1, calls + 1):
        bad = FailingAllocator(fail_at=k)
        with pytest.raises(pf.PfError) as e:
            pf.Filter(n, seed=5, scheme=scheme, precision=precision, torch_alloc=bad, **kw)
        assert e.value.status == pf.PF_ERR_OOM, (k, e.value)
        assert not bad.live, (k, len(bad.live))
    # and a filter created afterwards works
    g = pf.Filter(n, seed=5, scheme=scheme, precision=precision, **kw)
    g.step(0.1)
    assert g.estimate()["t"] == 1
    g.close()


def test_batch_create_reports_oom_and_frees_everything(pf):
    specs = [dict(n=1000 + 37 * i, seed=i, filter_id=i) for i in range(5)]
    ok = FailingAllocator()
    b = pf.Batch(specs, scheme="systematic", precision="fp32", torch_alloc=ok)
    calls = ok.calls
    assert calls >= 2
    b.close()
    assert not ok.live
    for k in range(1, calls + 1):
        bad = FailingAllocator(fail_at=k)
        with pytest.raises(pf.PfError) as e:
            pf.Batch(specs, scheme="systematic", precision="fp32", torch_alloc=bad)
        assert e.value.status == pf.PF_ERR_OOM, (k, e.value)
        assert not bad.live, (k, len(bad.live))
