"""The C-ABI library builds, loads and exports every function include/*.h declares
(no compute: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for path in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        src = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names.update(re.findall(r"^\s*(?:pf_status|const char\*)\s+(pf_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pf_create", "pf_step", "pf_resample", "pf_estimate", "pf_destroy",
                     "pf_last_error", "pf_cutpoint_search", "pf_cutpoint_method",
                     "pf_diag_cdf_wait"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1212_1639_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_rejects_bad_arguments_without_gpu():
    from paper_1212_1639_gb300 import build
    build.build()
    from paper_1212_1639_gb300 import pf
    # argument checks happen on the host before any CUDA call
    cfg = pf.PfConfig(n_particles=0, seed=1, scheme=1, precision=0, a_sigma=3, b_sigma=2,
                      a_tau=3, b_tau=2, x0_var=10)
    h = ctypes.c_void_p()
    assert pf._lib.pf_create(ctypes.byref(cfg), ctypes.byref(h)) == pf.PF_ERR_INVALID
    assert "n_particles" in pf.last_error()
    cfg.n_particles = 16
    cfg.scheme = 9
    assert pf._lib.pf_create(ctypes.byref(cfg), ctypes.byref(h)) == pf.PF_ERR_INVALID
    cfg.scheme = 1
    cfg.a_sigma = 0.5
    assert pf._lib.pf_create(ctypes.byref(cfg), ctypes.byref(h)) == pf.PF_ERR_INVALID
    assert pf._lib.pf_resample(None, 10, 0, 0, 0, 1, None, None) == pf.PF_ERR_INVALID
    assert pf._lib.pf_destroy(None) == pf.PF_OK


def test_product_path_has_no_oracle_dependency():
    """The CUDA path never imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_1212_1639_gb300")
    pat = re.compile(r"(^\s*(from|import)\s+oracle\b)|liboracle|oracle/", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not pat.search(text), f
