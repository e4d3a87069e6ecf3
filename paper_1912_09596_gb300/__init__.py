"""GB300-native empty-space-skipping volume renderer (arXiv 1912.09596).

The compute path is the C-ABI library ``libess.so`` (CUDA for sm_103a plus host
C++), reached through :mod:`paper_1912_09596_gb300.ess`.  Importing this package
does not load the library; ``ess`` does, and fails loudly if it is missing.
"""
__all__ = ["ess", "synth"]
