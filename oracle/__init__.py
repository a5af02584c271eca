"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Written from the paper (Kumari & Donzis, arXiv 2003.10561), it is the plain,
slow definition of what the CUDA path computes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library and its Python binding never do, and the two share no code.

Modules:
  philox     Philox4x32-10 (Salmon et al. SC'11), pinned by the published
             known-answer vectors.
  stencils   4th-order central / one-sided stencils and the Table B AT weights.
  ns         vectorised RHS, delay map, forcing, AB2, statistics.
  pointwise  brute-force one-point RHS (explicit Table B term lists).

Every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
against closed forms, polynomial exactness, convergence orders, conservation,
published test vectors or a symbolic (sympy) evaluation of the PDE; none is
"parity unpinned".
"""
