"""GB300-native hot path of on-the-fly cavity molecular dynamics (arXiv:2512.03277).

The compute path is the CUDA library libcavmd.so (include/cavmd.h); cavmd.py is its thin
ctypes binding. Build with python -m paper_2512_03277_gb300.build.
"""
from .cavmd import (Context, CavmdError, default_options, load_library, sk_tables,  # noqa: F401
                    PREC_FP64, CHARGE_MULLIKEN, SPLIT_PHOTON_EXACT, PHOTON_RELAXED, PHOTON_ZERO)
