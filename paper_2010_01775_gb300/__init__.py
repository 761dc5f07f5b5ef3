"""GB300-native guiding-distribution hot path of Photon-Driven Neural Path Guiding.

The compute path lives in the C-ABI library ``libpg.so`` (hand-written sm_103a
CUDA kernels, ``csrc/``); ``paper_2010_01775_gb300.pg`` is its thin ctypes
binding. ``paper_2010_01775_gb300.synth`` holds the seeded input generators.
Nothing is imported eagerly so that the generators can be used without the
CUDA library.
"""
__all__ = ["pg", "synth", "build"]
