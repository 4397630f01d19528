"""GB300-native frequent-episode counting and mining (Cao et al., arXiv 0905.2200).

The compute path lives in ``libfem.so`` (CUDA C++ for sm_103a, C ABI declared in
``include/fem.h``); :mod:`paper_0905_2200_gb300.fem` is the thin ctypes binding
with the same names.  :mod:`paper_0905_2200_gb300.synth` builds seeded synthetic
spike-train workloads.  Submodules are imported on demand so that the input
generators work on machines without the CUDA library.
"""

__all__ = ["fem", "synth"]
