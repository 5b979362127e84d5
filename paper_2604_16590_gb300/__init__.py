"""GB300-native STORM global propagation attention (STORM-GPA, arXiv 2604.16590).

The compute path is the CUDA library ``libgattn.so`` built from ``csrc/``
(hand-written sm_103a kernels behind a C ABI, declared in ``include/gattn.h``);
``gattn`` is its thin ctypes binding and ``inputs`` the seeded synthetic input
generators.  Import ``paper_2604_16590_gb300.gattn`` for the operator.
"""

__all__ = ["gattn", "inputs"]
