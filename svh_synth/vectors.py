"""Seeded random coefficient vectors (no arithmetic of the method)."""
from __future__ import annotations

import numpy as np


def random_state(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_complex(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Complex128 array with independent N(0, scale^2/2) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) * (scale / np.sqrt(2.0))
