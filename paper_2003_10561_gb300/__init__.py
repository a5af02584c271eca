"""GB300-native AT-DNS: one time step of compressible Navier-Stokes with
Asynchrony-Tolerant stencils (arXiv 2003.10561), as a C-ABI CUDA library.

``synth`` (seeded inputs) imports nothing else; the CUDA binding is loaded on
first use of ``paper_2003_10561_gb300.at_dns``.
"""
