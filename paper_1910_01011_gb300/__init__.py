"""GB300-native multiple-domain Galerkin BEM for the Helmholtz transmission
problem (arXiv 1910.01011): C ABI over hand-written sm_103a CUDA kernels,
with a thin Python binding.  `from paper_1910_01011_gb300.api import Context`.
"""
