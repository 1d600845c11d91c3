"""gfp: exact matrix multiplication over small prime fields on GB300.

Implements Dumas, Fousse, Salvy, "Compressed Modular Matrix Multiplication"
(arXiv 0803.1975) as CUDA kernels for sm_103a behind the C ABI of
include/gfp.h.  `paper_0803_1975_gb300.gfp` is the Python binding (argument
marshalling only); `paper_0803_1975_gb300.inputs` draws seeded synthetic
inputs.  Importing the package does not load the CUDA library; the first
binding call does, and fails loudly if it has not been built.
"""
