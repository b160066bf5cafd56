"""GB300 solver for the deflated Schur-complement method of Joshi & Diamessis
(arXiv 1601.03432): SMPM discretisation of the 2-D Poisson-Neumann problem,
GMRES on the deflated, block-Jacobi preconditioned Schur complement system.

The computation lives in the CUDA library ``libsmpm.so`` behind the C ABI of
``include/smpm.h``; ``Grid`` is its Python binding.  ``inputs`` holds the
seeded synthetic workloads.
"""
from ._binding import Batch, Grid, SmpmError, default_opts, factor_many, lib  # noqa: F401

__all__ = ["Batch", "Grid", "SmpmError", "default_opts", "factor_many", "lib"]
