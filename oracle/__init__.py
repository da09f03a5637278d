"""Plain FP64 CPU oracle of the cavity-MD hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this package: only
the tests, the smoke check and the CPU-baseline leg of the benchmark do. It
shares no code with the CUDA path; both read their inputs from cavmd_synth.

Modules:
  dftb.py          second-order SCC-DFTB of isolated molecules / clusters
  cavity.py        k-space light-matter coupling, photon rotation, time step
  paper_scheme.py  the paper's real-space Steps 1-4 (flat-dispersion pin)
  harmonic.py      closed forms of the harmonic test model (Rabi splitting)
  fit_water_params.py  writes the stored synthetic water parameter set
"""
