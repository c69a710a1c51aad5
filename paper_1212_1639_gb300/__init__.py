"""GB300-native particle learning (arXiv 1212.1639): a C-ABI CUDA library
(libpf.so, built from csrc/) and a thin ctypes binding (pf.py).

Importing the package loads nothing; `from paper_1212_1639_gb300 import pf`
loads the CUDA library and raises if it has not been built.
"""
