"""GB300-native diagonally oriented multigrid for Poisson's equation.

A.J. Roberts, "Fast and accurate multigrid solution of Poisson's equation
using diagonally oriented grids".  The compute path is the CUDA library
``libdiagmg.so`` (C ABI in include/diagmg.h); this package is its Python
binding.  Importing the package does not load the library; the first call
that needs it does, and fails loudly if it is not built.
"""

from .api import (  # noqa: F401
    Batch, Context, PoissonSolve, default_omega, solve,
)

__all__ = ["Batch", "Context", "PoissonSolve", "default_omega", "solve"]
