"""Physical constants and unit conversions (atomic units: hbar = m_e = e = 1).

Conversion factors only; no part of the dynamics is computed here.
"""

AMU = 1822.888486          # electron masses per unified atomic mass unit
FS = 41.341373335          # atomic time units per femtosecond
KB = 3.166811563e-6        # Boltzmann constant, Hartree per Kelvin
C_LIGHT = 137.035999       # speed of light in vacuum, atomic units
EV = 0.0367493             # Hartree per electron-volt
ANGSTROM = 1.8897261       # bohr per Angstrom

DT_HALF_FS = 0.5 * FS      # the 0.5 fs time step of the workloads, 20.670687 a.u.

# liquid-water number density: 33 molecules per (10 Angstrom)^3 cell
WATER_DENSITY = 33.0 / (10.0 * ANGSTROM) ** 3   # molecules per bohr^3 (4.95e-3)
