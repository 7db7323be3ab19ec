"""GB300 (sm_103a) implementation of the D3Q27 KBC entropic multi-relaxation lattice
Boltzmann step (Boesch, Chikatamarla, Karlin, arXiv:1507.02518).

``lb`` binds the C ABI of ``libkbc.so`` (include/kbc_lb.h); ``workloads`` generates seeded
synthetic initial fields; ``build`` compiles the CUDA library in-tree.
"""
from . import lb, workloads  # noqa: F401

__all__ = ["lb", "workloads"]
