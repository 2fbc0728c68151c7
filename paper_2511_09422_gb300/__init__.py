"""GB300-native fused diffuse-interface lattice Boltzmann step for binary freezing.

The compute path is the C-ABI library ``liblbfreeze.so`` (hand-written sm_103a
CUDA kernels) built from ``csrc/``; ``lbfreeze`` is its thin ctypes binding and
``workloads`` builds seeded synthetic inputs.  Importing the package does not
load the library; ``lbfreeze.load()`` does, and fails loudly if it is missing.
"""
__all__ = ["lbfreeze", "workloads"]
