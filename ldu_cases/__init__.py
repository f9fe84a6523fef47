"""Seeded synthetic LDU systems shaped like the paper's laplacianFoam and
icoFoam cases.  Shared by the oracle tests and the CUDA path as *inputs*
only: this package contains no solver arithmetic."""
from .mesh import LduSystem, BoxGeometry, graded_widths, uniform_widths  # noqa: F401
from .configs import (config1, config2, config3, config4, config4_sides, config5,  # noqa: F401
                      poisson_box, X_WALLS, ALL_WALLS)
from .reorder import renumber, random_order, rcm_order, bandwidth  # noqa: F401
from . import rng  # noqa: F401
