"""Seeded random complex vectors."""

from __future__ import annotations

import numpy as np


def complex_gaussian(shape, seed: int) -> np.ndarray:
    """complex128 array with i.i.d. standard complex Gaussian entries (real and imaginary N(0,1))."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return re + 1j * im
