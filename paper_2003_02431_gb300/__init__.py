"""GB300-native multigrid solve of agglomerated XDG (cut-cell DG) systems.

Kummer, Smuda, Weber, "BoSSS: a package for multigrid extended discontinuous Galerkin
methods", arXiv 2003.02431. The solve (operator apply, block-Jacobi smoothing, fused
residual-restriction and prolongation, Galerkin coarse operators, coarsest direct solve,
multigrid-preconditioned CG) runs in the CUDA library libxdg.so behind the C ABI of
include/xdg.h; this package holds its sources (csrc/) and the ctypes binding (xdg.py).
"""
from . import xdg  # noqa: F401
from .xdg import Hierarchy, XdgError, build, create_hierarchy, load  # noqa: F401
