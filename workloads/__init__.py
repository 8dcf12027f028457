"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This package holds only input construction (material cells, Bloch paths,
random vectors).  It contains none of the method's arithmetic: no shift,
difference, strain, stiffness product or eigen-solve lives here.
"""

from .materials import (  # noqa: F401
    TwoPhaseCell,
    isotropic_voigt,
    random_spd_voigt,
    two_phase_sphere,
    config_cell,
    quartz_silicon_constants,
    fcc_lattice,
    fcc_quartz_silicon_cell,
)
from .kpath import FCC_POINTS, fcc_kappa, fcc_path, sc_path, sc_eight_points, sc_uniform_path  # noqa: F401
from .vectors import complex_gaussian  # noqa: F401
