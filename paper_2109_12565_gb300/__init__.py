"""GB300-native thermal two-component lattice Boltzmann step (TLBfind, arXiv 2109.12565).

Submodules: ``inputs`` builds seeded synthetic workloads; ``lb`` is the thin
ctypes binding of the CUDA C-ABI library ``libtlbgb300.so`` (``include/tlb.h``);
``build`` compiles that library for sm_103a.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "lb", "build"]
