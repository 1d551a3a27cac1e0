"""HOTRG for the 2D generalized XY model (q = 2) on NVIDIA B300 (sm_103a).

The compute path is the C-ABI library ``libhotrg.so`` (CUDA, built from
``csrc/`` by :mod:`paper_2609_20536_b300.build`); :mod:`.hotrg` is a thin
ctypes binding with the same entry-point names.  Importing this package does
not load the library; ``from paper_2609_20536_b300 import hotrg`` does, and
fails loudly when it is missing.

Modules: :mod:`.hotrg` (binding: points, batches, observables, phase-boundary
scans, surrogate), :mod:`.cli` (command line), :mod:`.replicas` (sharding of
independent points over ranks), :mod:`.workloads` (synthetic inputs),
:mod:`.build` (nvcc build).
"""

__all__ = ["hotrg", "build", "cli", "replicas", "workloads"]
