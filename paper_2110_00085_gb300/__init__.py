"""GB300-native Monte-Carlo scattering tomography with path recycling.

The compute path is the C-ABI library ``libpathrecycle.so`` (hand-written
sm_103a CUDA kernels) reached through :mod:`paper_2110_00085_gb300.native`.
Importing this package does not load the library; the first call does, and
fails loudly if it has not been built.
"""
__all__ = ["synth"]
