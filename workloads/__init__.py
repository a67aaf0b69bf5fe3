"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *describes* inputs: cell geometry, ion charges, ion positions,
grid size and temperature.  It holds none of the functional's arithmetic, so the
CPU oracle and the CUDA path can both take their inputs from here without
sharing any part of the method.
"""
from .cells import (Cell, fcc_cell, random_cell, small_fcc_cell, config_cell,
                    batch_cells, serving_requests, smooth_grid, SEED_BASE,
                    PROTON_MASS, md_velocities, hydrogen_md_cells)

__all__ = ["Cell", "fcc_cell", "random_cell", "small_fcc_cell", "config_cell",
           "batch_cells", "serving_requests", "smooth_grid", "SEED_BASE",
           "PROTON_MASS", "md_velocities", "hydrogen_md_cells"]
