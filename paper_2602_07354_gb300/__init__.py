"""GB300-native matrix-free voxel finite-element elasticity PCG (ELAS3D-Xtal, arXiv 2602.07354).

The compute path is the C-ABI library ``libelas.so`` (hand-written sm_103a CUDA kernels); the
``binding`` module exposes its entry points under the same names.  ``synth`` generates seeded
synthetic microstructures.  Importing this package loads nothing native.
"""
__all__ = ["binding", "synth"]
