"""GB300-native constrained-GR elliptic solver (fully constrained ADM, CMC
slicing, minimal-distortion shift, conformal flatness): CIC deposit and the
multigrid solve of the ten constraint and gauge equations on a periodic grid,
as hand-written sm_103a CUDA kernels behind a C ABI (``include/gr.h``).

The CUDA library is loaded lazily by :mod:`paper_1905_08890_gb300.gr`; importing
this package (or :mod:`.synth`) does not touch the GPU.
"""

__all__ = ["gr", "synth"]
