"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package draws random numbers and lays out geometries, velocities and
cavity-mode lists. It holds none of the method's arithmetic: no Slater-Koster
evaluation, no charges, no forces, no coupling contraction and no time
stepping. Both sides of every parity test read their inputs from here.
"""
from .units import AMU, FS, KB, C_LIGHT, EV, ANGSTROM, WATER_DENSITY  # noqa: F401
from .params import (ELEM_O, ELEM_H, N_ELEM, N_ORB, ZVAL, MASS_AMU, SKParams,  # noqa: F401
                     draw_sk_params, load_water_params, water_reference_geometry)
from .systems import (System, Modes, water_batch, cluster_batch, periodic_water_cells,  # noqa: F401
                      mb_momenta,
                      standing_modes, line_modes, grid_modes, make_workload, WORKLOADS)
