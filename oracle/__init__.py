"""CPU oracle for the PS quadrature (test infrastructure; see psq_oracle's docstring)."""
from .psq_oracle import *  # noqa: F401,F403
from .psq_oracle import compute, contractions, grid_key, build_grid, rmse  # noqa: F401
