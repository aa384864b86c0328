"""GB300-native spectral clustering: LOBPCG on graph Laplacians + k-means (sm_103a).

The compute path is the C-ABI library ``libsc_gb300.so`` (hand-written CUDA for sm_103a);
``paper_1708_07481_gb300.sc`` is its thin ctypes binding.  ``workload`` holds the seeded
synthetic inputs.  Importing this package loads nothing; ``sc`` loads the library on first
use and fails loudly when it has not been built.
"""
__all__ = ["sc", "workload"]
