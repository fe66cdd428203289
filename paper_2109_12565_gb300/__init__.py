"""GB300-native thermal two-component lattice Boltzmann step (TLBfind, arXiv 2109.12565).

``inputs`` builds seeded synthetic workloads; ``lb`` is the thin ctypes
binding of the CUDA C-ABI library ``libtlbgb300.so`` (see ``include/tlb.h``).
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "lb"]


def __getattr__(name):
    if name == "lb":
        from . import lb
        return lb
    raise AttributeError(name)
